"""Pins of the single-threaded CPU Gray-code walks (oracle/cpu_walk.c) to the
recomputing oracle: the F_p walk bit for bit on arbitrary Gray ranges (empty,
one step, ragged, whole), the float walks within the drift an uncompensated
walk of 2^n steps can reach."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import cpu_walk as W
from workloads import rng

U = 2.0 ** -53


@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 14])
def test_modp_walk_equals_recomputing_oracle(n):
    g = rng(900 + n)
    for p in (2147483647, 65537, 7):
        A = g.integers(0, p, size=(n, n), dtype=np.uint64).astype(np.uint32)
        full = 1 << n
        cuts = sorted({0, full, 1, full - 1, int(g.integers(0, full + 1)), int(g.integers(0, full + 1))})
        for k0 in cuts:
            for k1 in cuts:
                if k1 < k0:
                    continue
                assert W.modp_gray_range(A, p, k0, k1) == O.ryser_modp_gray_range(A, p, k0, k1), (p, k0, k1)
        whole = W.modp_gray_range(A, p, 0, full)
        ref = O.perm_modp_brute(A, p) if n <= 8 else O.perm_modp(A, p)
        assert (p - whole) % p == ref if n & 1 else whole == ref


def test_modp_walk_schur_range_matches_oracle():
    """A Gray range deep inside S_33 mod p (the bench's sample), against the oracle."""
    n, p = 33, 2147483647
    S = O.schur_residue_matrix(n, p, O.primitive_nth_root(p, n))
    k0 = (1 << 31) + 12345
    assert W.modp_gray_range(S, p, k0, k0 + 3000) == O.ryser_modp_gray_range(S, p, k0, k0 + 3000)


def test_walk_arguments():
    A = np.zeros((3, 3), np.uint32)
    with pytest.raises(ValueError):
        W.modp_gray_range(A, 7, 5, 4)           # k1 < k0
    with pytest.raises(ValueError):
        W.modp_gray_range(A, 7, 0, 9)           # beyond 2^n
    with pytest.raises(ValueError):
        W.fp_gray_range(np.zeros((2, 3)), 0, 1)


@pytest.mark.parametrize("n", [1, 2, 4, 7, 10, 12])
@pytest.mark.parametrize("cplx", [False, True])
def test_float_walk_within_drift_of_oracle(n, cplx):
    g = rng(950 + n + 100 * cplx)
    A = g.normal(size=(n, n))
    if cplx:
        A = A + 1j * g.normal(size=(n, n))
    ref, terms = O.perm_ryser(A, with_abs=True)
    got = W.perm(A)
    # every row sum is updated once per step: drift <= 2^n u max|r|, n factors, complex x4
    bound = 4 * n * (1 << n) * U * terms + 1e-300
    assert abs(got - ref) <= bound, (got, ref, bound)


def test_float_walk_closed_forms():
    """perm(J_n) = n!, perm(I) = 1, and a permutation matrix gives 1, exactly
    representable at every step for these small integer matrices."""
    for n in (3, 6, 9):
        assert W.perm(np.ones((n, n))) == math.factorial(n)
        assert W.perm(np.eye(n)) == 1.0
        P = np.eye(n)[::-1].copy()
        assert W.perm(P.astype(np.complex128)) == 1.0


@pytest.mark.parametrize("cplx", [False, True])
def test_float_walk_ranges_add_up(cplx):
    """Splitting the Gray range anywhere gives the same total (each piece
    starts its row sums from scratch at its own first subset)."""
    n = 9
    g = rng(970 + cplx)
    A = g.normal(size=(n, n)) + (1j * g.normal(size=(n, n)) if cplx else 0)
    whole = W.fp_gray_range(A, 0, 1 << n)
    _, terms = O.perm_ryser(A, with_abs=True)
    for k in (1, 5, 77, 300, (1 << n) - 1):
        parts = W.fp_gray_range(A, 0, k) + W.fp_gray_range(A, k, 1 << n)
        assert abs(parts - whole) <= 8 * n * (1 << n) * U * terms


def _walk_pins():
    g = rng(5)
    for n in (3, 6):
        p = 2147483629
        A = g.integers(0, p, size=(n, n), dtype=np.uint64).astype(np.uint32)
        yield "modp_range", W.modp_gray_range(A, p, 3, (1 << n) - 2) == O.ryser_modp_gray_range(A, p, 3, (1 << n) - 2)
        for cplx in (False, True):
            B = g.normal(size=(n, n)) + (1j * g.normal(size=(n, n)) if cplx else 0)
            ref, terms = O.perm_ryser(B, with_abs=True)
            yield "fp_whole", abs(W.perm(B) - ref) <= 4 * n * (1 << n) * U * terms
            k = 5
            yield "fp_split", abs(W.fp_gray_range(B, 0, k) + W.fp_gray_range(B, k, 1 << n)
                                  - W.fp_gray_range(B, 0, 1 << n)) <= 8 * n * (1 << n) * U * terms


WALK_PLANTS = [
    ("modp walk adds where it should subtract",
     "for (int i = 0; i < n; ++i) r[i] = (r[i] + pp - A[i * n + j]) % pp;",
     "for (int i = 0; i < n; ++i) r[i] = (r[i] + A[i * n + j]) % pp;"),
    ("modp walk keeps the sign of the first subset",
     "odd ^= 1;\n            if (S & (1ull << j)) {\n                for (int i = 0; i < n; ++i) r[i] = (r[i] + A",
     "if (S & (1ull << j)) {\n                for (int i = 0; i < n; ++i) r[i] = (r[i] + A"),
    ("complex walk product cross term sign", "pi = pr * ri[i] + pi * rr[i];", "pi = pr * ri[i] - pi * rr[i];"),
    ("real walk starts from k0 instead of its Gray subset",
     "uint64_t S = k0 ^ (k0 >> 1);\n    for (int i = 0; i < n; ++i) {\n        r[i] = 0.0;",
     "uint64_t S = k0;\n    for (int i = 0; i < n; ++i) {\n        r[i] = 0.0;"),
]


def test_walk_pins_pass():
    assert not [name for name, ok in _walk_pins() if not ok]


@pytest.mark.parametrize("desc,old,new", WALK_PLANTS, ids=[p[0] for p in WALK_PLANTS])
def test_walk_planted_mistake_is_caught(tmp_path, desc, old, new):
    import ctypes
    import subprocess
    src = open(W._SRC).read()
    assert src.count(old) == 1, f"plant site not unique: {desc}"
    mutated = tmp_path / "cpu_walk_planted.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libcpuwalk_planted.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-w", "-o", str(so),
                           str(mutated)])
    saved = W._load()
    lib = ctypes.CDLL(str(so))
    for name in ("cpuwalk_modp_gray_range", "cpuwalk_modp_gray_range_mt", "cpuwalk_f64_gray_range",
                 "cpuwalk_c128_gray_range"):
        getattr(lib, name).argtypes = getattr(saved, name).argtypes
        getattr(lib, name).restype = getattr(saved, name).restype
    W._lib = lib
    try:
        failed = [name for name, ok in _walk_pins() if not ok]
    finally:
        W._lib = saved
    assert failed, f"planted mistake not caught: {desc}"


@pytest.mark.parametrize("span", [0, 1, 3, 7, 8, 9, 1000, 40000])
def test_block_split_walk_equals_one_thread_walk(span):
    """One contiguous Gray block per OpenMP thread (paper §2.2) gives the
    one-thread walk's residue, also when the range is shorter than the
    thread count (empty blocks)."""
    n, p = 16, 2147483629
    g = rng(990 + span)
    A = g.integers(0, p, size=(n, n), dtype=np.uint64).astype(np.uint32)
    k0 = int(g.integers(0, (1 << n) - span + 1))
    got, threads = W.modp_gray_range_mt(A, p, k0, k0 + span)
    assert threads >= 1
    assert got == W.modp_gray_range(A, p, k0, k0 + span) == O.ryser_modp_gray_range(A, p, k0, k0 + span)
