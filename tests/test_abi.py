"""The C-ABI library loads without a GPU, exports every function the public
header declares, and its host-side helpers (primes, roots, Schur residues,
CRT; paper §2.1) agree with the oracle's independent Python versions."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "permx.h")
LIB = os.path.join(ROOT, "paper_2602_10141_b300", "libpermx.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s+(\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def px():
    if not os.path.exists(LIB):
        import importlib.util
        spec = importlib.util.spec_from_file_location("_b", os.path.join(ROOT, "paper_2602_10141_b300", "build.py"))
        b = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(b)
        b.build()
    import paper_2602_10141_b300 as px
    return px


def test_header_symbols_exported(px):
    names = declared_functions()
    assert len(names) >= 20
    lib = ctypes.CDLL(LIB)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string(px):
    assert "sm_103a" in px.version()
    with pytest.raises(px.PermxError) as e:
        px.perm_primes_1_mod_n(0, 3)
    assert e.value.code == px.PERMX_EINVAL and px.last_error()


@pytest.mark.parametrize("n", [1, 2, 7, 12, 33, 43, 48])
def test_primes_match_oracle(px, n):
    assert px.perm_primes_1_mod_n(n, 7) == O.primes_1_mod_n(n, 7)
    assert px.perm_primes_1_mod_n(n, 3, skip=4) == O.primes_1_mod_n(n, 3, skip=4)


@pytest.mark.parametrize("n", [3, 9, 16, 33, 43])
def test_roots_and_residues_match_oracle(px, n):
    for p in O.primes_1_mod_n(n, 3):
        g = px.perm_primitive_root(p, n)
        assert g == O.primitive_nth_root(p, n)
        assert np.array_equal(px.perm_schur_residues(n, p, g), O.schur_residue_matrix(n, p, g))


def test_crt_matches_oracle(px):
    g = np.random.default_rng(5)
    ps = O.primes_1_mod_n(43, 4)
    M = int(np.prod([int(p) for p in ps], dtype=object))
    for _ in range(200):
        x = int(g.integers(-2 ** 62, 2 ** 62)) * int(g.integers(1, 2 ** 62))
        x = ((x + M // 2) % M) - M // 2
        if x > M // 2 or abs(x) >= 2 ** 127:
            continue
        res = [x % p for p in ps]
        assert px.perm_crt(res, ps) == O.crt(res, ps) == x


def test_prime_count_matches_bound(px):
    for n in range(1, 49):
        k = px.perm_schur_prime_count(n)
        ps = O.primes_1_mod_n(n, k)
        assert O.crt_modulus_suffices(n, ps)
        if n >= 36 and n <= 43:
            assert k == O.prime_count_for(n) == 5


def test_invalid_helper_arguments(px):
    for args in ((7, 4), (9, 2)):   # 7 != 1 (mod 4); 9 is not prime
        with pytest.raises(px.PermxError):
            px.perm_primitive_root(*args)
    with pytest.raises(px.PermxError):
        px.perm_crt([1, 2], [7, 7])
    with pytest.raises(px.PermxError):
        px.perm_schur_residues(0, 7, 2)
    # the issue-rate probe checks its kind and sizes before any CUDA call
    for args in ((18, 1, 256, 1), (-1, 1, 256, 1), (0, 0, 256, 1), (0, 1, 16, 1), (0, 1, 256, 0)):
        with pytest.raises(px.PermxError) as e:
            px.permx_peak_probe(*args)
        assert e.value.code == px.PERMX_EINVAL


def test_chunk_tuning_table_host_logic(px):
    """perm_tune_* is host logic: set / get / restore, and the limits (the F_p
    chunk sums need ell <= 30, the float 128-bit chunk accumulator ell <= 16)."""
    try:
        default = px.perm_tune_get(px.FIELD_C128, 20)
        assert 3 <= default <= 10
        px.perm_tune_set(px.FIELD_C128, 20, 7)
        assert px.perm_tune_get(px.FIELD_C128, 20) == 7
        px.perm_tune_set(px.FIELD_C128, 20, 16)
        with pytest.raises(px.PermxError):
            px.perm_tune_set(px.FIELD_C128, 20, 17)
        px.perm_tune_set(px.FIELD_MODP, 40, 30)
        assert px.perm_tune_get(px.FIELD_MODP, 40) == 30
        with pytest.raises(px.PermxError):
            px.perm_tune_set(px.FIELD_MODP, 40, 31)
        with pytest.raises(px.PermxError):
            px.perm_tune_set(px.FIELD_F64, 49, 5)     # n above the table
        with pytest.raises(px.PermxError):
            px.perm_tune_set(7, 10, 3)                # unknown field
    finally:
        px.perm_tune_set(px.FIELD_C128, 20, 0)
        px.perm_tune_set(px.FIELD_MODP, 40, 0)
    assert px.perm_tune_get(px.FIELD_C128, 20) == default


def test_schur_crt_primes_argument_checks(px):
    """perm_schur_crt_primes rejects bad prime lists on the host, before any GPU work."""
    n = 23
    good = O.primes_1_mod_n(n, 6)
    for bad, what in (([good[0]], "need 2"), ([good[0], good[0], good[1]], "repeated"),
                      ([good[0], 2147483647], "not an odd prime"), ([4] + good[:2], "not an odd prime"),
                      (good[:2], "does not exceed")):
        with pytest.raises(px.PermxError):
            px.perm_schur_crt_primes(n, bad)
        assert what in px.last_error(), (bad, px.last_error())


def test_tuning_table_save_and_load(px, tmp_path, monkeypatch):
    """perm_tune_save / perm_tune_load round-trip the pinned entries, replace
    the whole table, reject malformed files without touching the table, and
    take $PERMX_TUNE_CACHE as the default path."""
    f = tmp_path / "tune.txt"
    d_c = px.perm_tune_get(px.FIELD_C128, 20)
    d_m = px.perm_tune_get(px.FIELD_MODP, 40)
    d_r = px.perm_tune_get(px.FIELD_F64, 9)
    try:
        px.perm_tune_set(px.FIELD_C128, 20, 7)
        px.perm_tune_set(px.FIELD_MODP, 40, 25)
        px.perm_tune_save(str(f))
        lines = f.read_text().splitlines()
        assert lines[0] == "permx-tune 1"
        assert sorted(lines[1:]) == sorted([f"{px.FIELD_C128} 20 7", f"{px.FIELD_MODP} 40 25"])
        assert not (tmp_path / "tune.txt.tmp").exists()
        # loading replaces the table: entries not in the file return to the rule
        px.perm_tune_set(px.FIELD_C128, 20, 0)
        px.perm_tune_set(px.FIELD_MODP, 40, 0)
        px.perm_tune_set(px.FIELD_F64, 9, 5)
        px.perm_tune_load(str(f))
        assert px.perm_tune_get(px.FIELD_C128, 20) == 7
        assert px.perm_tune_get(px.FIELD_MODP, 40) == 25
        assert px.perm_tune_get(px.FIELD_F64, 9) == d_r
        # malformed files change nothing
        for text in ("", "permx-tune 2\n", "permx-tune 1\n0 20 17\n", "permx-tune 1\n2 40 31\n",
                     "permx-tune 1\n0 49 5\n", "permx-tune 1\n3 10 3\n", "permx-tune 1\n0 20 7\n0 20 8\n",
                     "permx-tune 1\n0 20 7 9\n", "permx-tune 1\n0 20\n", "permx-tune 1\n0 20 0\n"):
            bad = tmp_path / "bad.txt"
            bad.write_text(text)
            with pytest.raises(px.PermxError):
                px.perm_tune_load(str(bad))
            assert px.perm_tune_get(px.FIELD_C128, 20) == 7
        with pytest.raises(px.PermxError):
            px.perm_tune_load(str(tmp_path / "missing.txt"))
        with pytest.raises(px.PermxError):
            px.perm_tune_save(str(tmp_path / "no_such_dir" / "t.txt"))
        # the environment variable supplies the default path
        monkeypatch.setenv("PERMX_TUNE_CACHE", str(tmp_path / "env.txt"))
        px.perm_tune_save()
        px.perm_tune_set(px.FIELD_C128, 20, 0)
        px.perm_tune_load()
        assert px.perm_tune_get(px.FIELD_C128, 20) == 7
        monkeypatch.delenv("PERMX_TUNE_CACHE")
        with pytest.raises(ValueError):
            px.perm_tune_save()
    finally:
        px.perm_tune_set(px.FIELD_C128, 20, 0)
        px.perm_tune_set(px.FIELD_MODP, 40, 0)
        px.perm_tune_set(px.FIELD_F64, 9, 0)
    assert px.perm_tune_get(px.FIELD_C128, 20) == d_c
    assert px.perm_tune_get(px.FIELD_MODP, 40) == d_m


def test_binding_rejects_tensors_that_do_not_fit(px):
    """The binding checks dtype, contiguity, size (against n and offset) and
    device before a pointer reaches the library, whose C-ABI cannot see them."""
    import torch
    n, off = [3, 4], [0, 9]                      # needs 9 + 16 = 25 elements
    c = torch.zeros(25, dtype=torch.complex128)  # CPU tensors: every check before the device one
    out_c = torch.zeros(2, dtype=torch.complex128)
    with pytest.raises(TypeError):
        px.perm_c128(c.real.contiguous(), n, off, out_c)            # float64 where complex128 is due
    with pytest.raises(ValueError, match="needs 25"):
        px.perm_c128(c[:24], n, off, out_c)
    with pytest.raises(ValueError, match="contiguous"):
        px.perm_c128(torch.zeros(50, dtype=torch.complex128)[::2], n, off, out_c)
    with pytest.raises(ValueError, match="needs 2"):
        px.perm_c128(c, n, off, out_c[:1])
    with pytest.raises(ValueError, match="entries"):
        px.perm_c128(c, n, [0], out_c)
    with pytest.raises(ValueError, match="CUDA"):
        px.perm_c128(c, n, off, out_c)
    with pytest.raises(TypeError):
        px.perm_f64(c, n, off, torch.zeros(2, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA"):
        px.perm_f64(torch.zeros(25, dtype=torch.float64), n, off, torch.zeros(2, dtype=torch.float64))
    r = torch.zeros(25, dtype=torch.int32)
    with pytest.raises(ValueError, match="needs 25"):
        px.perm_modp(r[:20], n, off, [7, 7], torch.zeros(2, dtype=torch.int32))
    with pytest.raises(TypeError):
        px.perm_modp(r.to(torch.int64), n, off, [7, 7], torch.zeros(2, dtype=torch.int32))
    with pytest.raises(ValueError, match="CUDA"):
        px.perm_modp_noalloc(r, n, off, [7, 7], torch.zeros(2, dtype=torch.int32))
    with pytest.raises(ValueError, match="needs 36"):
        px.perm_modp_gray_range(r, 6, 7, 0, 4)
    with pytest.raises(TypeError):
        px.perm_c128([0j] * 25, n, off, out_c)                     # not a tensor
    with pytest.raises(ValueError, match="CUDA"):
        px.perm_gather(torch.zeros((4, 4), dtype=torch.complex128), [[0, 1]], [[1, 2]], out_c)
    with pytest.raises(TypeError):
        px.perm_sample_stats(torch.zeros(4, dtype=torch.float32))
    with pytest.raises(ValueError, match="CUDA"):
        px.perm_sample_stats(torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError, match="contiguous"):
        px.perm_sample_histogram(torch.zeros(8, dtype=torch.complex128)[::2], [0.0, 1.0])


def test_binding_rejects_tensors_on_another_device(px, monkeypatch):
    """Every tensor of a call, and a torch stream given to it, must be on the
    current device (where the library launches): a tensor on another GPU is
    refused before its pointer reaches the C-ABI.  CPU-only: tensors that
    report a CUDA device stand in for real ones."""
    import torch

    class FakeCuda(torch.Tensor):
        @property
        def is_cuda(self):
            return True

        @property
        def device(self):
            return torch.device("cuda", self._dev)

        def get_device(self):
            return self._dev

    def on(t, dev):
        f = t.as_subclass(FakeCuda)
        f._dev = dev
        return f

    class FakeStream:
        def __init__(self, dev):
            self.device = torch.device("cuda", dev)
            self.cuda_stream = 0

    monkeypatch.setattr(px, "_current_device", lambda: 0)
    n, off = [3], [0]
    c = torch.zeros(9, dtype=torch.complex128)
    o = torch.zeros(1, dtype=torch.complex128)
    with pytest.raises(ValueError, match="A is on cuda:1"):
        px.perm_c128(on(c, 1), n, off, on(o, 0))
    with pytest.raises(ValueError, match="out is on cuda:1"):
        px.perm_c128(on(c, 0), n, off, on(o, 1))
    with pytest.raises(ValueError, match="current device is cuda:0"):
        px.perm_f64(on(torch.zeros(9, dtype=torch.float64), 2), n, off, on(torch.zeros(1, dtype=torch.float64), 2))
    with pytest.raises(ValueError, match="cuda:1"):
        px.perm_modp(on(torch.zeros(9, dtype=torch.int32), 0), n, off, [7], on(torch.zeros(1, dtype=torch.int32), 1))
    with pytest.raises(ValueError, match="stream is on cuda:1"):
        px._stream(FakeStream(1))
    assert px._stream(FakeStream(0)) == 0
    with pytest.raises(ValueError, match="U is on cuda:3"):
        px.perm_gather(on(torch.zeros((4, 4), dtype=torch.complex128), 3), [[0, 1]], [[1, 2]],
                       on(torch.zeros(1, dtype=torch.complex128), 0))
    with pytest.raises(ValueError, match="values is on cuda:1"):
        px.perm_sample_stats(on(torch.zeros(4, dtype=torch.complex128), 1))
