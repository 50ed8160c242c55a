"""permx: Gray-code Ryser permanents on one B300 — Python binding.

A thin ctypes layer over ``libpermx.so`` (the C-ABI in ``include/permx.h``):
the functions below carry the C names and only marshal arguments.  Device
tensors come from PyTorch (device memory and streams only); every step of the
computation runs in the library's CUDA kernels.  There is no CPU fallback:
if the library is missing or fails to load, importing this package raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpermx.so")

PERMX_OK = 0
PERMX_EINVAL = -1
PERMX_ENOMEM = -2
PERMX_EBUSY = -3
PERMX_ECUDA = -4
PERMX_ETIMEOUT = -5
PERMX_ENOTFOUND = -6
PERMX_EIO = -7
PERMX_EAGAIN = -8
MAX_N_FP = 32
MAX_N_MODP = 48
MAX_PRIMES = 64
FIELD_C128, FIELD_F64, FIELD_MODP = 0, 1, 2
FP_ARITH_FP64, FP_ARITH_INT = 0, 1


class PermxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"permx error {code}: {msg}")
        self.code = code


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2602_10141_b300/build.py`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
    P = ctypes.POINTER
    sig = {
        "perm_last_error": ([], ctypes.c_char_p),
        "permx_version": ([], ctypes.c_char_p),
        # host arrays of the batched calls travel as raw addresses (numpy .ctypes.data):
        # these run once per matrix in one-call-per-matrix use, where ctypes pointer
        # objects cost more than the launch
        "perm_c128": ([vp, vp, vp, i64, vp, vp], ctypes.c_int),
        "perm_f64": ([vp, vp, vp, i64, vp, vp], ctypes.c_int),
        "perm_modp": ([vp, vp, vp, vp, i64, vp, vp], ctypes.c_int),
        "perm_c128_host": ([vp, P(i32), P(i64), i64, vp, vp], ctypes.c_int),
        "perm_f64_host": ([vp, P(i32), P(i64), i64, vp, vp], ctypes.c_int),
        "perm_modp_host": ([vp, P(i32), P(i64), P(u32), i64, vp, vp], ctypes.c_int),
        "perm_modp_noalloc": ([vp, vp, vp, vp, i64, vp, vp], ctypes.c_int),
        "perm_modp_gray_range": ([vp, i32, u32, u64, u64, P(u32), vp], ctypes.c_int),
        "perm_schur_crt": ([i32, i32, ctypes.c_char_p, P(i64), ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
        "perm_schur_crt_ex": ([i32, i32, ctypes.c_char_p, u64, i64, P(i64), ctypes.c_char_p, ctypes.c_size_t,
                               P(u32), P(u32)], ctypes.c_int),
        "perm_schur_crt_primes": ([i32, P(u32), i32, ctypes.c_char_p, u64, i64, P(i64), ctypes.c_char_p,
                                   ctypes.c_size_t, P(u32)], ctypes.c_int),
        "perm_primes_1_mod_n": ([i32, i32, i32, P(u32)], ctypes.c_int),
        "perm_primitive_root": ([u32, i32, P(u32)], ctypes.c_int),
        "perm_schur_residues": ([i32, u32, u32, P(u32)], ctypes.c_int),
        "perm_crt": ([P(u32), P(u32), i32, P(i64)], ctypes.c_int),
        "perm_schur_prime_count": ([i32], ctypes.c_int),
        "perm_schur_shard": ([i32, P(u32), i32, i32, i32, i32, P(u32)], ctypes.c_int),
        "permx_set_fp_arith": ([ctypes.c_int], ctypes.c_int),
        "perm_plan_create": ([ctypes.c_int, P(i32), P(i64), P(u32), i64, vp, P(vp)], ctypes.c_int),
        "perm_plan_execute": ([vp, vp, vp, vp], ctypes.c_int),
        "perm_plan_graph_launch": ([vp, vp, vp, vp], ctypes.c_int),
        "perm_plan_destroy": ([vp], ctypes.c_int),
        "perm_tune_set": ([ctypes.c_int, i32, i32], ctypes.c_int),
        "perm_tune_get": ([ctypes.c_int, i32], ctypes.c_int),
        "perm_autotune": ([ctypes.c_int, i32, i64, i32, P(i32)], ctypes.c_int),
        "perm_tune_save": ([ctypes.c_char_p], ctypes.c_int),
        "perm_tune_load": ([ctypes.c_char_p], ctypes.c_int),
        "permx_get_fp_arith": ([], ctypes.c_int),
        "perm_c128_gather": ([vp, i32, i64, P(i32), P(i32), i32, i64, vp, vp], ctypes.c_int),
        "perm_f64_gather": ([vp, i32, i64, P(i32), P(i32), i32, i64, vp, vp], ctypes.c_int),
        "perm_sample_histogram": ([ctypes.c_int, vp, i64, ctypes.c_int, P(ctypes.c_double), i32, vp, vp],
                                  ctypes.c_int),
        "perm_sample_stats": ([ctypes.c_int, vp, i64, ctypes.c_double, ctypes.c_double, vp, vp], ctypes.c_int),
        "permx_peak_probe": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_double),
                              P(ctypes.c_double)], ctypes.c_int),
        "perm_graph_create": ([P(vp), P(vp), P(vp), i32, P(vp)], ctypes.c_int),
        "perm_graph_launch": ([vp, vp], ctypes.c_int),
        "perm_graph_destroy": ([vp], ctypes.c_int),
        "serve_create": ([vp, P(vp)], ctypes.c_int),
        "serve_submit": ([vp, ctypes.c_int, i32, vp, u32, P(u64)], ctypes.c_int),
        "serve_poll": ([vp, u64, vp, P(ctypes.c_int)], ctypes.c_int),
        "serve_poll_timed": ([vp, u64, vp, P(ctypes.c_int), P(i64), P(i64)], ctypes.c_int),
        "serve_drain": ([vp, i64], ctypes.c_int),
        "serve_stats": ([vp, P(i64)], ctypes.c_int),
        "serve_stats2": ([vp, vp], ctypes.c_int),
        "serve_destroy": ([vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def last_error() -> str:
    return _lib.perm_last_error().decode()


def _check(rc: int) -> int:
    if rc < 0:
        raise PermxError(rc, last_error())
    return rc


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _current_device() -> int:
    """Index of the calling thread's current CUDA device (the library launches there)."""
    import torch
    return torch.cuda.current_device()


def _stream(stream) -> int | None:
    """Raw cudaStream_t of `stream` (None: torch's current stream; an int is
    taken as a raw handle).  A torch stream must belong to the current device."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    dev = getattr(stream, "device", None)
    idx = getattr(dev, "index", None)
    if idx is not None and idx != _current_device():
        raise ValueError(f"the stream is on cuda:{idx}, the current device is cuda:{_current_device()}")
    return stream.cuda_stream


def version() -> str:
    return _lib.permx_version().decode()


# ---------------------------------------------------------------------------
# tensor checks: the C-ABI takes bare device pointers and cannot see sizes or
# dtypes, so the binding rejects a tensor that would make a kernel read or
# write outside it before the pointer reaches the library
# ---------------------------------------------------------------------------

def _need(n: np.ndarray, offset: np.ndarray, max_n: int) -> int:
    """Elements a batch reads: max over b of offset[b] + n[b]^2, over the sizes
    the library accepts (it rejects the others itself, with PERMX_EINVAL)."""
    if len(n) != len(offset):
        raise ValueError(f"n has {len(n)} entries, offset {len(offset)}")
    if len(n) <= 8:                  # a handful of matrices: plain Python beats numpy's per-call cost
        need = 0
        for k, o in zip(n.tolist(), offset.tolist()):
            if 1 <= k <= max_n:
                need = max(need, o + k * k)
        return need
    ok = (n >= 1) & (n <= max_n)
    if not ok.any():
        return 0
    return int(np.max(offset[ok].astype(np.int64) + n[ok].astype(np.int64) ** 2))


_DTYPES: dict = {}


def _dtypes(kind: str):
    if not _DTYPES:
        import torch
        _DTYPES.update({"c128": (torch.complex128,), "f64": (torch.float64,),
                        "modp": tuple(d for d in (torch.int32, getattr(torch, "uint32", None)) if d is not None)})
    return _DTYPES[kind]


def _tensors(*specs) -> None:
    """specs: (tensor, name, kind, elements needed).  Type, dtype, layout and
    size of every tensor first, then that all of them are on a CUDA device."""
    import torch
    for t, what, kind, need in specs:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{what} must be a torch tensor")
        dts = _dtypes(kind)
        if t.dtype not in dts:
            raise TypeError(f"{what} must be {' or '.join(str(d) for d in dts)}, not {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
        if t.numel() < need:
            raise ValueError(f"{what} holds {t.numel()} elements; the call needs {need}")
    _on_current_device(*[(t, what) for t, what, _, _ in specs])


def _on_current_device(*named) -> None:
    """Every (tensor, name) must be a CUDA tensor on the current device: the
    library launches on the current device and would otherwise be handed
    another GPU's pointers."""
    for t, what in named:
        if not t.is_cuda:
            raise ValueError(f"{what} must be on a CUDA device")
    cur = _current_device()
    for t, what in named:
        idx = t.get_device()
        if idx != cur:
            raise ValueError(f"{what} is on cuda:{idx}, the current device is cuda:{cur}; "
                             "all tensors of a call must be on the current device")


# ---------------------------------------------------------------------------
# batched device calls (arguments: device tensors + host index arrays)
# ---------------------------------------------------------------------------

def perm_c128(A, n: Sequence[int], offset: Sequence[int], out, stream=None):
    """out[b] = perm of the n[b] x n[b] complex128 matrix at A.view(-1)[offset[b]:]."""
    n, offset = _i32(n), _i64(offset)
    _tensors((A, "A", "c128", _need(n, offset, MAX_N_FP)), (out, "out", "c128", len(n)))
    _check(_lib.perm_c128(A.data_ptr(), n.ctypes.data, offset.ctypes.data, len(n), out.data_ptr(), _stream(stream)))
    return out


def perm_f64(A, n: Sequence[int], offset: Sequence[int], out, stream=None):
    """out[b] = perm of the n[b] x n[b] float64 matrix at A.view(-1)[offset[b]:]."""
    n, offset = _i32(n), _i64(offset)
    _tensors((A, "A", "f64", _need(n, offset, MAX_N_FP)), (out, "out", "f64", len(n)))
    _check(_lib.perm_f64(A.data_ptr(), n.ctypes.data, offset.ctypes.data, len(n), out.data_ptr(), _stream(stream)))
    return out


def perm_modp(A, n: Sequence[int], offset: Sequence[int], p: Sequence[int], out, stream=None):
    """A: device int32/uint32 residues (< p[b]); out: device int32 tensor of residues."""
    n, offset, p = _i32(n), _i64(offset), _u32(p)
    _tensors((A, "A", "modp", _need(n, offset, MAX_N_MODP)), (out, "out", "modp", len(n)))
    _check(_lib.perm_modp(A.data_ptr(), n.ctypes.data, offset.ctypes.data, p.ctypes.data, len(n), out.data_ptr(),
                          _stream(stream)))
    return out


def perm_gather(U, rows, cols, out, stream=None):
    """out[b] = perm(U[rows[b], :][:, cols[b]]) for a device matrix U (complex128 or
    float64, 2-D, unit column stride) and host index arrays rows, cols of shape (batch, n)."""
    import torch
    rows, cols = _i32(rows), _i32(cols)
    if rows.ndim != 2 or rows.shape != cols.shape:
        raise ValueError("rows and cols must both have shape (batch, n)")
    if U.dim() != 2 or U.shape[0] != U.shape[1] or U.stride(1) != 1:
        raise ValueError("U must be a square 2-D tensor with unit column stride")
    f = _lib.perm_c128_gather if U.dtype == torch.complex128 else _lib.perm_f64_gather
    if U.dtype not in (torch.complex128, torch.float64):
        raise TypeError("U must be complex128 or float64")
    _tensors((out, "out", "c128" if U.dtype == torch.complex128 else "f64", rows.shape[0]))
    _on_current_device((U, "U"), (out, "out"))
    _check(f(U.data_ptr(), U.shape[0], U.stride(0), _p(rows, ctypes.c_int32), _p(cols, ctypes.c_int32),
             rows.shape[1], rows.shape[0], out.data_ptr(), _stream(stream)))
    return out


HIST_ABS2, HIST_RE, HIST_IM = 0, 1, 2


def _values_field(values) -> int:
    """Field code of a device tensor of permanents (complex128 or float64)."""
    import torch
    if not isinstance(values, torch.Tensor):
        raise TypeError("values must be a torch tensor")
    if values.dtype == torch.complex128:
        field = FIELD_C128
    elif values.dtype == torch.float64:
        field = FIELD_F64
    else:
        raise TypeError("values must be complex128 or float64")
    if not values.is_contiguous():
        raise ValueError("values must be contiguous")
    _on_current_device((values, "values"))
    return field


def perm_sample_histogram(values, edges, kind: int = 0, stream=None):
    """Counts of |z|^2 (kind 0), Re z (1) or Im z (2) over sorted host `edges`:
    a numpy int64 array of len(edges) + 1 (below, bins, at-or-above).  Synchronises."""
    import torch
    field = _values_field(values)
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.float64))
    counts = torch.empty(len(e) + 1, dtype=torch.int64, device=values.device)
    _check(_lib.perm_sample_histogram(field, values.data_ptr(), values.numel(), kind, _p(e, ctypes.c_double),
                                      len(e), counts.data_ptr(), _stream(stream)))
    torch.cuda.synchronize(values.device)
    return counts.cpu().numpy()


class PermStats(ctypes.Structure):
    """perm_stats_t: sample statistics of a batch of permanents."""
    _fields_ = [(k, ctypes.c_int64) for k in ("count", "count_nonzero", "count_above", "count_real")] + \
        [(k, ctypes.c_double) for k in ("mean_re", "mean_im", "var_re", "var_im", "cov_re_im", "skew_re",
                                        "exkurt_re", "mean_abs2", "mean_abs4", "mean_z2_re", "mean_z2_im",
                                        "min_abs2", "max_abs2", "log_mean", "log_var", "log_skew",
                                        "log_exkurt")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def perm_sample_stats_async(values, out, threshold: float = float("inf"), real_tol: float = 0.0, stream=None):
    """Enqueue perm_sample_stats on `stream`: values is a device complex128 or
    float64 tensor, out a device uint8 tensor of at least sizeof(perm_stats_t)."""
    field = _values_field(values)
    if out.numel() * out.element_size() < ctypes.sizeof(PermStats):
        raise ValueError("output buffer too small for perm_stats_t")
    if not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA tensor")
    _on_current_device((values, "values"), (out, "out"))
    _check(_lib.perm_sample_stats(field, values.data_ptr(), values.numel(), threshold, real_tol,
                                  out.data_ptr(), _stream(stream)))
    return out


def perm_sample_stats(values, threshold: float = float("inf"), real_tol: float = 0.0, stream=None) -> dict:
    """Statistics of the device tensor `values` (see perm_sample_stats in permx.h), as a dict.
    Synchronises the stream."""
    import torch
    _values_field(values)                      # type, layout and device before anything is allocated
    out = torch.empty(ctypes.sizeof(PermStats), dtype=torch.uint8, device=values.device)
    perm_sample_stats_async(values, out, threshold, real_tol, stream)
    torch.cuda.synchronize(values.device)
    raw = out.cpu().numpy().tobytes()
    return PermStats.from_buffer_copy(raw).as_dict()


class Plan:
    """A planned batch (perm_plan_*): sizes, offsets and primes fixed once;
    ``execute`` enqueues only kernels, ``graph_launch`` replays a captured CUDA graph."""

    def __init__(self, field: int, n, offset, p=None, stream=None):
        n, offset = _i32(n), _i64(offset)
        pp = _u32(p) if p is not None else None
        self._keep = (n, offset, pp)
        self._kind = {FIELD_C128: "c128", FIELD_F64: "f64", FIELD_MODP: "modp"}.get(field)
        self._need = _need(n, offset, MAX_N_MODP if field == FIELD_MODP else MAX_N_FP)
        h = ctypes.c_void_p()
        _check(_lib.perm_plan_create(field, _p(n, ctypes.c_int32), _p(offset, ctypes.c_int64),
                                     _p(pp, ctypes.c_uint32) if pp is not None else None, len(n), _stream(stream),
                                     ctypes.byref(h)))
        self.h = h

    def _args(self, A, out):
        _tensors((A, "A", self._kind, self._need), (out, "out", self._kind, len(self._keep[0])))

    def execute(self, A, out, stream=None):
        self._args(A, out)
        _check(_lib.perm_plan_execute(self.h, A.data_ptr(), out.data_ptr(), _stream(stream)))
        return out

    def graph_launch(self, A, out, stream=None):
        self._args(A, out)
        _check(_lib.perm_plan_graph_launch(self.h, A.data_ptr(), out.data_ptr(), _stream(stream)))
        return out

    def close(self):
        if self.h:
            _lib.perm_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """Several plans captured into one CUDA graph (perm_graph_*): plans[i] runs
    on A[i] -> out[i]; ``launch`` replays all of them with one graph launch."""

    def __init__(self, plans, A, out):
        if not (len(plans) == len(A) == len(out)) or not plans:
            raise ValueError("need one A and one out per plan")
        for pl, a, o in zip(plans, A, out):
            pl._args(a, o)
        n = len(plans)
        self._keep = (list(plans), list(A), list(out))
        hp = (ctypes.c_void_p * n)(*[pl.h.value for pl in plans])
        ha = (ctypes.c_void_p * n)(*[a.data_ptr() for a in A])
        ho = (ctypes.c_void_p * n)(*[o.data_ptr() for o in out])
        h = ctypes.c_void_p()
        _check(_lib.perm_graph_create(hp, ha, ho, n, ctypes.byref(h)))
        self.h = h

    def launch(self, stream=None):
        _check(_lib.perm_graph_launch(self.h, _stream(stream)))

    def close(self):
        if self.h:
            _lib.perm_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ServeCfg(ctypes.Structure):
    """perm_serve_cfg (include/permx.h): the serving loop's limits."""
    _fields_ = [("max_requests", ctypes.c_int32), ("max_resident", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("chunks_per_step", ctypes.c_int64),
                ("device", ctypes.c_int32), ("plain_fifo", ctypes.c_int32),
                ("work_budget", ctypes.c_int64)]


class ServeStats(ctypes.Structure):
    """perm_serve_stats (include/permx.h): counters of a server."""
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "resident", "steps", "launches",
                                              "pending", "resident_work")] + \
        [("gpu_busy_ms", ctypes.c_double), ("uptime_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_RESULT_BYTES = {FIELD_C128: 16, FIELD_F64: 8, FIELD_MODP: 4}


class Server:
    """Continuous-batching server (serve_*): ``submit`` copies a host matrix and
    returns a ticket, ``poll`` returns None until the result is ready, then
    (value, latency_s) with the latency measured inside the library."""

    def __init__(self, max_requests: int = 0, max_resident: int = 0, device_bytes: int = 0,
                 chunks_per_step: int = 0, device: int | None = None, plain_fifo: bool = False,
                 work_budget: int = 0):
        self.cfg = ServeCfg(max_requests, max_resident, device_bytes, chunks_per_step,
                            _current_device() if device is None else device, int(bool(plain_fifo)), work_budget)
        h = ctypes.c_void_p()
        _check(_lib.serve_create(ctypes.byref(self.cfg), ctypes.byref(h)))
        self.h = h
        self._res = (ctypes.c_char * 16)()
        self._done = ctypes.c_int(0)
        self._ts, self._td = ctypes.c_int64(0), ctypes.c_int64(0)
        self._field = {}

    def submit(self, A: np.ndarray, field: int, p: int = 0) -> int:
        """A: square host matrix (complex128, float64 or uint32 residues < p)."""
        dt = {FIELD_C128: np.complex128, FIELD_F64: np.float64, FIELD_MODP: np.uint32}.get(field)
        if dt is None:
            raise ValueError("unknown field")
        A = np.ascontiguousarray(A, dtype=dt)
        if A.ndim != 2 or A.shape[0] != A.shape[1]:
            raise ValueError("A must be a square matrix")
        t = ctypes.c_uint64()
        _check(_lib.serve_submit(self.h, field, A.shape[0], A.ctypes.data, p, ctypes.byref(t)))
        self._field[t.value] = field
        return t.value

    def poll(self, ticket: int):
        _check(_lib.serve_poll_timed(self.h, ticket, self._res, ctypes.byref(self._done), ctypes.byref(self._ts),
                                     ctypes.byref(self._td)))
        if not self._done.value:
            return None
        field = self._field.pop(ticket)
        raw = bytes(self._res)[:_RESULT_BYTES[field]]
        if field == FIELD_C128:
            v = complex(*np.frombuffer(raw, np.float64))
        elif field == FIELD_F64:
            v = float(np.frombuffer(raw, np.float64)[0])
        else:
            v = int(np.frombuffer(raw, np.uint32)[0])
        return v, (self._td.value - self._ts.value) * 1e-9

    def drain(self, timeout_ms: int = 60000) -> None:
        _check(_lib.serve_drain(self.h, timeout_ms))

    def stats(self) -> dict:
        st = ServeStats()
        _check(_lib.serve_stats2(self.h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self.h:
            _lib.serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def perm_tune_set(field: int, n: int, ell: int) -> None:
    _check(_lib.perm_tune_set(field, n, ell))


def perm_tune_get(field: int, n: int) -> int:
    return _check(_lib.perm_tune_get(field, n))


def _tune_path(path) -> bytes:
    path = path if path is not None else os.environ.get("PERMX_TUNE_CACHE")
    if not path:
        raise ValueError("no tuning-file path given and PERMX_TUNE_CACHE is not set")
    return os.fsencode(path)


def perm_tune_save(path=None) -> None:
    """Write the pinned chunk lengths to ``path`` (default: $PERMX_TUNE_CACHE)."""
    _check(_lib.perm_tune_save(_tune_path(path)))


def perm_tune_load(path=None) -> None:
    """Replace the tuning table by the file at ``path`` (default: $PERMX_TUNE_CACHE)."""
    _check(_lib.perm_tune_load(_tune_path(path)))


def perm_autotune(field: int, n: int, batch: int, reps: int = 3) -> int:
    best = ctypes.c_int32(0)
    _check(_lib.perm_autotune(field, n, batch, reps, ctypes.byref(best)))
    return int(best.value)


def perm_modp_noalloc(A, n: Sequence[int], offset: Sequence[int], p: Sequence[int], out, stream=None):
    """perm_modp for callers that cannot allocate: at most 64 matrices per call,
    intermediates in the library's fixed device array (see include/permx.h)."""
    n, offset, p = _i32(n), _i64(offset), _u32(p)
    _tensors((A, "A", "modp", _need(n, offset, MAX_N_MODP)), (out, "out", "modp", len(n)))
    _check(_lib.perm_modp_noalloc(A.data_ptr(), n.ctypes.data, offset.ctypes.data, p.ctypes.data, len(n),
                                  out.data_ptr(), _stream(stream)))
    return out


# ---------------------------------------------------------------------------
# host-buffer calls (numpy in, numpy out; copies and sync inside the library)
# ---------------------------------------------------------------------------

def perm_c128_host(A: np.ndarray, n, offset, out: np.ndarray | None = None, stream=None) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n, offset = _i32(n), _i64(offset)
    out = np.empty(len(n), np.complex128) if out is None else out
    _check(_lib.perm_c128_host(A.ctypes.data, _p(n, ctypes.c_int32), _p(offset, ctypes.c_int64), len(n),
                               out.ctypes.data, _stream(stream)))
    return out


def perm_f64_host(A: np.ndarray, n, offset, out: np.ndarray | None = None, stream=None) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    n, offset = _i32(n), _i64(offset)
    out = np.empty(len(n), np.float64) if out is None else out
    _check(_lib.perm_f64_host(A.ctypes.data, _p(n, ctypes.c_int32), _p(offset, ctypes.c_int64), len(n),
                              out.ctypes.data, _stream(stream)))
    return out


def perm_modp_host(A: np.ndarray, n, offset, p, out: np.ndarray | None = None, stream=None) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.uint32)
    n, offset, p = _i32(n), _i64(offset), _u32(p)
    out = np.empty(len(n), np.uint32) if out is None else out
    _check(_lib.perm_modp_host(A.ctypes.data, _p(n, ctypes.c_int32), _p(offset, ctypes.c_int64),
                               _p(p, ctypes.c_uint32), len(n), out.ctypes.data, _stream(stream)))
    return out


def perm_modp_gray_range(A, n: int, p: int, k0: int, k1: int, stream=None) -> int:
    """Signed Ryser sum over Gray indices [k0, k1) of one device matrix, mod p (no (-1)^n)."""
    _tensors((A, "A", "modp", int(n) * int(n) if 1 <= n <= MAX_N_MODP else 0))
    r = ctypes.c_uint32(0)
    _check(_lib.perm_modp_gray_range(A.data_ptr(), n, p, k0, k1, ctypes.byref(r), _stream(stream)))
    return int(r.value)


# ---------------------------------------------------------------------------
# Schur permanent and field helpers
# ---------------------------------------------------------------------------

def _i128(v: np.ndarray) -> int:
    m = (1 << 64) - 1
    x = ((int(v[1]) & m) << 64) | (int(v[0]) & m)
    return x - (1 << 128) if x >> 127 else x


def perm_schur_crt(n: int, nprimes: int = 0, ckpt_path: str | None = None) -> int:
    """Exact perm(S_n) as a Python int (via the decimal output)."""
    buf = ctypes.create_string_buffer(512)
    _check(_lib.perm_schur_crt(n, nprimes, ckpt_path.encode() if ckpt_path else None, None, buf, len(buf)))
    return int(buf.value.decode())


def perm_schur_crt_ex(n: int, nprimes: int = 0, ckpt_path: str | None = None, slice_subsets: int = 0,
                      max_slices: int = 0):
    """Returns (value, primes, residues); raises PermxError with code PERMX_EAGAIN when stopped early."""
    buf = ctypes.create_string_buffer(512)
    res = np.zeros(MAX_PRIMES, np.uint32)
    pr = np.zeros(MAX_PRIMES, np.uint32)
    rc = _lib.perm_schur_crt_ex(n, nprimes, ckpt_path.encode() if ckpt_path else None, slice_subsets, max_slices,
                                None, buf, len(buf), _p(res, ctypes.c_uint32), _p(pr, ctypes.c_uint32))
    _check(rc)
    k = int(np.count_nonzero(pr))
    return int(buf.value.decode()), [int(x) for x in pr[:k]], [int(x) for x in res[:k]]


def perm_schur_crt_primes(n: int, primes, ckpt_path: str | None = None, slice_subsets: int = 0,
                          max_slices: int = 0):
    """perm(S_n) with the given primes (the last one checks); returns (value, residues)."""
    pp = _u32(primes)
    buf = ctypes.create_string_buffer(512)
    res = np.zeros(len(pp), np.uint32)
    _check(_lib.perm_schur_crt_primes(n, _p(pp, ctypes.c_uint32), len(pp),
                                      ckpt_path.encode() if ckpt_path else None, slice_subsets, max_slices, None,
                                      buf, len(buf), _p(res, ctypes.c_uint32)))
    return int(buf.value.decode()), [int(x) for x in res]


def perm_schur_shard(n: int, primes, slices: int, shard: int, nshards: int) -> list[int]:
    """One shard's partial sums of perm(S_n) on the current GPU (see
    perm_schur_shard in include/permx.h and sharding.py)."""
    pp = _u32(primes)
    out = np.zeros(len(pp), np.uint32)
    _check(_lib.perm_schur_shard(n, _p(pp, ctypes.c_uint32), len(pp), slices, shard, nshards,
                                 _p(out, ctypes.c_uint32)))
    return [int(x) for x in out]


def perm_primes_1_mod_n(n: int, count: int, skip: int = 0) -> list[int]:
    out = np.zeros(max(count, 1), np.uint32)
    _check(_lib.perm_primes_1_mod_n(n, count, skip, _p(out, ctypes.c_uint32)))
    return [int(x) for x in out[:count]]


def perm_primitive_root(p: int, n: int) -> int:
    g = ctypes.c_uint32(0)
    _check(_lib.perm_primitive_root(p, n, ctypes.byref(g)))
    return int(g.value)


def perm_schur_residues(n: int, p: int, g: int) -> np.ndarray:
    out = np.zeros((n, n), np.uint32)
    _check(_lib.perm_schur_residues(n, p, g, _p(out, ctypes.c_uint32)))
    return out


def perm_crt(residues: Sequence[int], primes: Sequence[int]) -> int:
    r, p = _u32(residues), _u32(primes)
    out = np.zeros(2, np.int64)
    _check(_lib.perm_crt(_p(r, ctypes.c_uint32), _p(p, ctypes.c_uint32), len(r), _p(out, ctypes.c_int64)))
    return _i128(out)


def permx_set_fp_arith(mode: int) -> int:
    """Select the float64/complex128 arithmetic (FP_ARITH_INT or FP_ARITH_FP64); returns the previous mode."""
    return _check(_lib.permx_set_fp_arith(mode))


def permx_get_fp_arith() -> int:
    return int(_lib.permx_get_fp_arith())


def perm_schur_prime_count(n: int) -> int:
    return _check(_lib.perm_schur_prime_count(n))


def permx_peak_probe(kind: int, blocks: int, threads: int, iters: int) -> tuple[float, float]:
    """(operations per second, milliseconds) of one issue-rate probe kernel."""
    ops, ms = ctypes.c_double(0), ctypes.c_double(0)
    _check(_lib.permx_peak_probe(kind, blocks, threads, iters, ctypes.byref(ops), ctypes.byref(ms)))
    return ops.value, ms.value
