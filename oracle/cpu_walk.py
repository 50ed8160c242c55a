"""Plain CPU Gray-code Ryser walks — BENCHMARK / TEST INFRASTRUCTURE ONLY.

The paper's §2.2 algorithm as a plain one-core program (``cpu_walk.c``): row
sums kept and updated by one column per Gray step, uint64 ``%`` for F_p,
uncompensated double for R and C.  It is the comparator for the paper's
GPU-over-single-threaded-CPU speed-ups, not a correctness reference: the
oracle proper (``oracle.c``) recomputes every row sum, and the tests pin these
walks to it (F_p bit for bit, floating point within the drift of an
uncompensated walk).  Only ``tests/`` and ``bench.py``'s ``cpu_baseline`` leg
use it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_walk.c")
_LIB = os.path.join(_HERE, "libcpuwalk.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``cpu_walk.c`` into ``libcpuwalk.so`` (gcc -O2; OpenMP only for the block-split F_p walk)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall",
               "-o", _LIB + ".tmp", _SRC]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i, u64 = ctypes.c_int, ctypes.c_uint64
        dp = ctypes.POINTER(ctypes.c_double)
        lib.cpuwalk_modp_gray_range.argtypes = [i, ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32, u64, u64,
                                                ctypes.POINTER(ctypes.c_uint32)]
        lib.cpuwalk_modp_gray_range_mt.argtypes = lib.cpuwalk_modp_gray_range.argtypes
        lib.cpuwalk_f64_gray_range.argtypes = [i, dp, u64, u64, dp]
        lib.cpuwalk_c128_gray_range.argtypes = [i, dp, u64, u64, dp]
        for f in (lib.cpuwalk_modp_gray_range, lib.cpuwalk_modp_gray_range_mt, lib.cpuwalk_f64_gray_range,
                  lib.cpuwalk_c128_gray_range):
            f.restype = i
        _lib = lib
    return _lib


def _square(A) -> int:
    n = A.shape[0]
    if A.ndim != 2 or A.shape[1] != n:
        raise ValueError("square matrix expected")
    return n


def modp_gray_range(A, p: int, k0: int, k1: int) -> int:
    """sum_{k0<=k<k1} (-1)^{|g(k)|} prod_i sum_{j in g(k)} a_ij mod p by the
    incremental walk (the same quantity as ``oracle.ryser_modp_gray_range``)."""
    a = np.ascontiguousarray(np.asarray(A, dtype=np.uint32))
    n = _square(a)
    out = np.zeros(1, np.uint32)
    rc = _load().cpuwalk_modp_gray_range(n, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), int(p), int(k0),
                                         int(k1), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    if rc != 0:
        raise ValueError(f"cpuwalk_modp_gray_range: bad arguments (rc {rc})")
    return int(out[0])


def modp_gray_range_mt(A, p: int, k0: int, k1: int) -> tuple[int, int]:
    """modp_gray_range with one contiguous Gray block per OpenMP thread:
    (the same residue, the number of threads used)."""
    a = np.ascontiguousarray(np.asarray(A, dtype=np.uint32))
    n = _square(a)
    out = np.zeros(1, np.uint32)
    rc = _load().cpuwalk_modp_gray_range_mt(n, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), int(p), int(k0),
                                            int(k1), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    if rc < 1:
        raise ValueError(f"cpuwalk_modp_gray_range_mt: bad arguments (rc {rc})")
    return int(out[0]), int(rc)


def fp_gray_range(A, k0: int, k1: int):
    """The same signed sum over a float64 or complex128 matrix in plain double
    arithmetic (float or complex result, no (-1)^n factor)."""
    A = np.asarray(A)
    cplx = np.iscomplexobj(A)
    a = np.ascontiguousarray(A, dtype=np.complex128 if cplx else np.float64)
    n = _square(a)
    out = np.zeros(2, np.float64)
    f = _load().cpuwalk_c128_gray_range if cplx else _load().cpuwalk_f64_gray_range
    dp = ctypes.POINTER(ctypes.c_double)
    rc = f(n, a.ctypes.data_as(dp), int(k0), int(k1), out.ctypes.data_as(dp))
    if rc != 0:
        raise ValueError(f"cpu walk: bad arguments (rc {rc})")
    return complex(out[0], out[1]) if cplx else float(out[0])


def perm(A):
    """perm(A) = (-1)^n x the walk over all 2^n subsets (float or complex)."""
    n = np.asarray(A).shape[0]
    s = fp_gray_range(A, 0, 1 << n)
    return -s if n & 1 else s
