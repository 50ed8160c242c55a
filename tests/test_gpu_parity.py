"""CUDA path vs the oracle, element by element on seeded inputs (the C-ABI
through the Python binding).  F_p and CRT results must be bit-exact; float64
and complex128 results must meet the floating-point tolerance below."""
import math

import numpy as np
import pytest

import oracle as O
from workloads import ENSEMBLES, ensemble, geodesic_cycle, random_residues, rng

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def fp_tolerance(ref, abs_terms, n):
    """Pass bound for a float64 / complex128 result.

    1e-9 relative, or the forward error bound of the Gray-code walk: every
    term prod_i r_i carries at most ~n roundings in its product plus the
    row-sum drift of a walk of <= 2^12 steps (a few dozen ulps), so
    |error| <= 64 n u sum_S |prod_i r_i(S)|.  The second clause only matters
    when the alternating sum cancels by many orders of magnitude."""
    return max(1e-9 * abs(ref), 64 * n * U * abs_terms)


@pytest.fixture(scope="module")
def px():
    import torch
    assert torch.cuda.is_available()
    import paper_2602_10141_b300 as px
    return px


@pytest.fixture(params=[1, 0], ids=["int_mantissa", "fp64"])
def arith(request, px):
    """Run a float64/complex128 test under both walk arithmetics."""
    old = px.permx_set_fp_arith(request.param)
    yield request.param
    px.permx_set_fp_arith(old)


def _dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda()


def _pack(mats):
    n = [m.shape[0] for m in mats]
    off = np.concatenate([[0], np.cumsum([k * k for k in n])[:-1]]).astype(np.int64)
    flat = np.concatenate([m.reshape(-1) for m in mats])
    return flat, n, off


def run_modp(px, mats, primes):
    import torch
    flat, n, off = _pack(mats)
    A = _dev(flat.astype(np.int32))
    out = torch.empty(len(mats), dtype=torch.int32, device="cuda")
    px.perm_modp(A, n, off, primes, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.int64) & 0xFFFFFFFF


def run_fp(px, mats):
    import torch
    flat, n, off = _pack(mats)
    cplx = np.iscomplexobj(flat)
    A = _dev(flat)
    out = torch.empty(len(mats), dtype=torch.complex128 if cplx else torch.float64, device="cuda")
    (px.perm_c128 if cplx else px.perm_f64)(A, n, off, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


# ---------------------------------------------------------------------------
# F_p: bit-exact
# ---------------------------------------------------------------------------

def test_modp_ragged_batch_bit_exact(px):
    g = rng(1000)
    primes = [2147483629, 2147483647, 65537, 3, 1000003]
    mats, ps = [], []
    for n in list(range(1, 25)) + [7, 13, 22, 24]:
        p = primes[n % len(primes)]
        mats.append(random_residues(n, p, g))
        ps.append(p)
    got = run_modp(px, mats, ps)
    for A, p, v in zip(mats, ps, got):
        n = A.shape[0]
        ref = O.perm_modp_dp(A, p) if n > 10 else O.perm_modp_brute(A, p)
        assert int(v) == ref, (n, p)


def test_modp_edge_values(px):
    # all zeros, all p-1, identity, the largest admissible prime
    p = 2147483647
    mats = [np.zeros((5, 5), np.uint32), np.full((9, 9), p - 1, np.uint32), np.eye(17, dtype=np.uint32),
            np.full((1, 1), p - 1, np.uint32)]
    got = run_modp(px, mats, [p] * len(mats))
    for A, v in zip(mats, got):
        assert int(v) == O.perm_modp_dp(A, p)


@pytest.mark.parametrize("ell", [1, 2, 3])
def test_modp_short_tuned_chunks(px, ell):
    # chunks of 2^ell steps: most chunk indices are odd, and the last toggle of
    # every chunk takes its sign from bit ell of k, i.e. from the chunk index
    g = rng(1050 + ell)
    primes = [2147483629, 65537, 2147483647, 1000003]
    ns = [9, 13, 17, 20]
    old = {n: px.perm_tune_get(px.FIELD_MODP, n) for n in ns}
    try:
        for n in ns:
            px.perm_tune_set(px.FIELD_MODP, n, ell)
        mats = [random_residues(n, primes[i], g) for i, n in enumerate(ns)]
        got = run_modp(px, mats, primes)
    finally:
        for n in ns:
            px.perm_tune_set(px.FIELD_MODP, n, old[n])
    for A, p, v in zip(mats, primes, got):
        assert int(v) == O.perm_modp_dp(A, p), (A.shape[0], p, ell)


@pytest.mark.parametrize("n", [25, 26])
def test_modp_larger_sizes(px, n):
    g = rng(1100 + n)
    p = 2147483629
    A = random_residues(n, p, g)
    assert int(run_modp(px, [A], [p])[0]) == O.perm_modp_dp(A, p)


def test_gray_range_partial_sums(px):
    import torch
    g = rng(1200)
    p = 2147483629
    n = 30
    A = random_residues(n, p, g)
    dA = _dev(A.astype(np.int32))
    for k0, k1 in ((0, 1 << 20), (123457, 123457 + 999983), ((1 << 29) - 77777, (1 << 29) + 1234567),
                   ((1 << 30) - 4096, 1 << 30), (5, 5)):
        assert px.perm_modp_gray_range(dA, n, p, k0, k1) == O.ryser_modp_gray_range(A, p, k0, k1)
    torch.cuda.synchronize()


@pytest.mark.parametrize("n", [3, 5, 8, 12, 16, 19])
def test_schur_residues_and_crt_small(px, n):
    exact = O.schur_exact(n)
    assert px.perm_schur_crt(n) == exact
    for p in O.primes_1_mod_n(n, 2):
        gr = O.primitive_nth_root(p, n)
        S = O.schur_residue_matrix(n, p, gr)
        assert int(run_modp(px, [S], [p])[0]) == exact % p


def test_schur_n33_disjoint_prime_sets(px):
    # 5 primes just below 2^31 (plus a check prime inside the library); a second,
    # disjoint set of 5 primes must reconstruct the same integer
    n = 33
    v, primes, res = px.perm_schur_crt_ex(n, 5)
    assert primes == O.primes_1_mod_n(n, 6)
    assert O.crt(res[:5], primes[:5]) == v
    assert v * v <= n ** n
    other = O.primes_1_mod_n(n, 5, skip=6)
    gs = [O.primitive_nth_root(p, n) for p in other]
    got = run_modp(px, [O.schur_residue_matrix(n, p, gg) for p, gg in zip(other, gs)], other)
    assert O.crt([int(x) for x in got], other) == v
    # Galois invariance: another primitive root gives the same residue
    p = other[0]
    g2 = pow(gs[0], 2, p)
    assert int(run_modp(px, [O.schur_residue_matrix(n, p, g2)], [p])[0]) == int(got[0])


def test_modp_invalid_arguments(px):
    import torch
    A = torch.zeros(16, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    for n, p in ((0, 7), (49, 2147483629), (4, 2147483648 - 1 + 2), (4, 9), (4, 2)):
        with pytest.raises(px.PermxError) as e:
            px.perm_modp(A, [n], [0], [p], out)
        assert e.value.code == px.PERMX_EINVAL
    with pytest.raises(px.PermxError):
        px.perm_modp_host(np.full((2, 2), 11, np.uint32), [2], [0], [11])


# ---------------------------------------------------------------------------
# float64 / complex128
# ---------------------------------------------------------------------------

def _check_fp(mats, got):
    worst = 0.0
    for A, v in zip(mats, got):
        n = A.shape[0]
        ref = O.perm_dp(A)
        _, abs_terms = O.perm_ryser(A, with_abs=True) if n <= 18 else (None, None)
        if abs_terms is None:
            abs_terms = 0.0
        err = abs(v - ref)
        assert err <= fp_tolerance(ref, abs_terms, n), (n, v, ref, err)
        if ref != 0:
            worst = max(worst, err / abs(ref))
    return worst


@pytest.mark.parametrize("name", list(ENSEMBLES))
def test_fp_ensembles_ragged(px, arith, name):
    mats = []
    for n in list(range(1, 19)) + [9, 14]:
        mats.append(ensemble(name, n, 1, seed=2000 + n)[0])
    worst = _check_fp(mats, run_fp(px, mats))
    assert worst < 1e-9


@pytest.mark.parametrize("cplx", [True, False])
def test_fp_larger_sizes(px, arith, cplx):
    # n = 20, 21: relative error against the error bound of float64 products; at
    # these sizes the Haar permanent's terms cancel by ~1e8-1e9, so 1e-9 relative
    # is at the edge of what float64 products can deliver
    name = "haar_u" if cplx else "haar_o"
    mats = [ensemble(name, n, 1, seed=2100 + n)[0] for n in (20, 21)]
    got = run_fp(px, mats)
    for A, v in zip(mats, got):
        ref = O.perm_dp(A)
        _, abs_terms = O.perm_ryser(A, with_abs=True)
        assert abs(v - ref) <= fp_tolerance(ref, abs_terms, A.shape[0]), (A.shape[0], v, ref)
        if arith == 1:
            # exact row sums and 62-bit products: 1e-9 relative holds here too
            assert abs(v - ref) <= 1e-9 * abs(ref), (A.shape[0], v, ref)


def test_int_mantissa_relative_at_n22(px):
    # Haar U(22): float64 products miss 1e-9 relative (measured 1.2e-9); the
    # integer-mantissa walk must meet it
    old = px.permx_set_fp_arith(1)
    try:
        A = ensemble("haar_u", 22, 1, seed=2100 + 22)[0]
        v = run_fp(px, [A])[0]
        ref = O.perm_dp(A)
        assert abs(v - ref) <= 1e-9 * abs(ref), (v, ref)
    finally:
        px.permx_set_fp_arith(old)


def test_haar_unitary_n14_one_per_launch(px, arith):
    # 256 Haar-random U(14), seed 0, one matrix per launch
    mats = ensemble("haar_u", 14, 256, seed=0)
    for A in mats[::16]:
        v = run_fp(px, [A])[0]
        ref = O.perm_dp(A)
        assert abs(v - ref) <= 1e-9 * abs(ref)


def test_geodesic_midpoints(px, arith):
    # paper §4.1 table: midpoint of the cycle geodesic; even n -> 0
    ns = [5, 7, 9, 11, 13, 15, 17]
    mats = [geodesic_cycle(n, 0.5, "circulant") for n in ns] + [geodesic_cycle(n, 0.5, "principal") for n in ns]
    got = run_fp(px, mats)
    for A, v in zip(mats, got):
        n = A.shape[0]
        ref = O.perm_dp(A)
        _, abs_terms = O.perm_ryser(A, with_abs=True)
        assert abs(v - ref) <= fp_tolerance(ref, abs_terms, n)
        pred = 2 * math.exp(-n) * (1 + 1 / (3 * n))
        assert abs(abs(v) / pred - 1) <= 1.0 / n ** 2
    even = run_fp(px, [geodesic_cycle(n, 0.5, "circulant") for n in (6, 10, 14)])
    assert np.all(np.abs(even) <= 1e-13)


def test_fp_identity_ones_and_hermitian(px, arith):
    mats = [np.eye(12, dtype=complex), np.ones((10, 10), complex), np.ones((12, 12))]
    got = run_fp(px, mats[:2])
    assert got[0] == 1.0
    assert got[1] == math.factorial(10)
    assert run_fp(px, mats[2:])[0] == math.factorial(12)
    # Hermitian => real permanent (paper §6.1, Proposition); the computed imaginary part is
    # rounding error and must stay within the float64 error bound of the walk
    H = ensemble("gue", 15, 4, seed=5)
    for A, v in zip(H, run_fp(px, list(H))):
        _, abs_terms = O.perm_ryser(A, with_abs=True)
        assert abs(v.imag) <= fp_tolerance(0.0, abs_terms, 15)


def test_fp_alone_equals_in_mix(px, arith):
    # the same matrix alone and inside a ragged batch gives bit-identical results
    A = ensemble("haar_u", 16, 1, seed=77)[0]
    B = ensemble("ginibre_r", 15, 1, seed=78)[0]
    alone = run_fp(px, [A])[0]
    mix = run_fp(px, [ensemble("haar_u", 9, 1, seed=1)[0], A] + list(ensemble("haar_u", 16, 5, seed=2)) + [A])
    assert mix[1] == alone and mix[-1] == alone
    alone_r = run_fp(px, [B])[0]
    mix_r = run_fp(px, list(ensemble("goe", 12, 3, seed=3)) + [B])
    assert mix_r[-1] == alone_r


@pytest.mark.parametrize("cplx", [True, False])
def test_nonfinite_entries_give_nan(px, cplx):
    """Integer mode: a matrix with a NaN or infinite entry gives NaN and leaves
    the other matrices of the batch bit-identical."""
    old = px.permx_set_fp_arith(px.FP_ARITH_INT)
    try:
        name = "haar_u" if cplx else "goe"
        good = [ensemble(name, n, 1, seed=60 + n)[0] for n in (7, 18, 23)]
        bad_nan = ensemble(name, 18, 1, seed=70)[0].copy()
        bad_nan[3, 5] = np.nan
        bad_inf = ensemble(name, 7, 1, seed=71)[0].copy()
        bad_inf[6, 0] = -np.inf
        bad_big = ensemble(name, 23, 1, seed=72)[0].copy()
        bad_big[0, 0] = np.inf if not cplx else complex(0.0, np.inf)
        clean = run_fp(px, good)
        mixed = run_fp(px, [good[0], bad_nan, good[1], bad_inf, bad_big, good[2]])
        assert np.array_equal(mixed[[0, 2, 5]], clean)
        for v in mixed[[1, 3, 4]]:
            assert np.isnan(v.real) and (not cplx or np.isnan(v.imag))
    finally:
        px.permx_set_fp_arith(old)


def test_host_variants_match_device(px, arith):
    mats = [ensemble("haar_u", n, 1, seed=3000 + n)[0] for n in (4, 11, 15)]
    flat, n, off = _pack(mats)
    host = px.perm_c128_host(flat, n, off)
    dev = run_fp(px, mats)
    assert np.array_equal(host, dev)
    p = 2147483629
    g = rng(9)
    rm = [random_residues(k, p, g) for k in (3, 12, 20)]
    flat, n, off = _pack(rm)
    host = px.perm_modp_host(flat, n, off, [p] * 3)
    assert [int(x) for x in host] == [O.perm_modp_dp(A, p) for A in rm]


def test_fp_invalid_arguments(px):
    import torch
    A = torch.zeros(33 * 33, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in (0, 33, -1):
        with pytest.raises(px.PermxError) as e:
            px.perm_f64(A, [n], [0], out)
        assert e.value.code == px.PERMX_EINVAL


# ---------------------------------------------------------------------------
# maximum sizes: closed forms the oracle can evaluate block by block
# ---------------------------------------------------------------------------

def _block_diag(blocks):
    n = sum(b.shape[0] for b in blocks)
    M = np.zeros((n, n), dtype=np.result_type(*blocks))
    i = 0
    for b in blocks:
        k = b.shape[0]
        M[i:i + k, i:i + k] = b
        i += k
    return M


def test_fp_max_size_block_diagonal(px, arith):
    # n = 32 (the float maximum): perm of a block-diagonal matrix is the product of the
    # blocks' permanents; rows and columns permuted so the blocks interleave
    g = rng(4000)
    for cplx in (True, False):
        blocks = [ensemble("haar_u" if cplx else "haar_o", 8, 1, seed=4000 + 10 * k + cplx)[0] for k in range(4)]
        M = _block_diag(blocks)
        P, Q = g.permutation(32), g.permutation(32)
        M = np.ascontiguousarray(M[P][:, Q])
        ref = np.prod([O.perm_dp(b) for b in blocks])
        v = run_fp(px, [M])[0]
        assert abs(v - ref) <= 1e-9 * abs(ref), (cplx, v, ref)


def test_modp_large_block_diagonal(px):
    # n = 36: product of four 9 x 9 blocks' permanents mod p
    g = rng(4100)
    p = 2147483629
    blocks = [random_residues(9, p, g) for _ in range(4)]
    M = _block_diag(blocks).astype(np.uint32)
    P, Q = g.permutation(36), g.permutation(36)
    M = np.ascontiguousarray(M[P][:, Q])
    ref = 1
    for b in blocks:
        ref = ref * O.perm_modp_brute(b, p) % p
    assert int(run_modp(px, [M], [p])[0]) == ref


def test_modp_n48_gray_window(px):
    # the F_p maximum n = 48: a sampled window of Gray indices against the oracle
    g = rng(4200)
    p = 2147483647
    A = random_residues(48, p, g)
    dA = _dev(A.astype(np.int32))
    for k0 in ((1 << 47) - 300000, (1 << 46) + 12345):
        assert px.perm_modp_gray_range(dA, 48, p, k0, k0 + 600000) == O.ryser_modp_gray_range(A, p, k0, k0 + 600000)


@pytest.mark.parametrize("n", [41, 44, 46])
def test_modp_paired_large_n_gray_window(px, n):
    # n = 41..46 take the paired steps with a few registers spilled: sampled Gray
    # windows (one starting on an odd index) against the oracle
    g = rng(4300 + n)
    p = 2147483629
    A = random_residues(n, p, g)
    dA = _dev(A.astype(np.int32))
    for k0 in ((1 << (n - 1)) - 200000, (1 << (n - 2)) + 4321):
        assert px.perm_modp_gray_range(dA, n, p, k0, k0 + 400000) == O.ryser_modp_gray_range(A, p, k0, k0 + 400000)


def test_n1_all_fields(px, arith):
    assert run_fp(px, [np.array([[2.5 - 1j]])])[0] == 2.5 - 1j
    assert run_fp(px, [np.array([[-3.25]])])[0] == -3.25
    assert int(run_modp(px, [np.array([[12345]], np.uint32)], [2147483629])[0]) == 12345


def test_schur_crt_matches_oracle_fixture(px):
    """Exact perm(S_n) for every n of tests/golden/schur_crt_oracle.txt (written
    by make_schur_crt.py from the oracle alone; n = 21..31), through
    the GPU F_p walk and the library's CRT, equals the oracle's value."""
    from conftest import read_golden
    rows = read_golden("schur_crt_oracle.txt")
    assert set(range(21, 32)) <= {int(r[0]) for r in rows}
    for r in rows:
        n, value = int(r[0]), int(r[1])
        assert px.perm_schur_crt(n) == value, n


def test_schur_crt_disjoint_primes_match_fixture(px):
    """perm_schur_crt_primes with primes disjoint from the default set (the
    next ones down) gives the oracle's perm(S_n) for n = 23, 25, 27."""
    from conftest import read_golden
    rows = {int(r[0]): (int(r[1]), [int(x) for x in r[2:]]) for r in read_golden("schur_crt_oracle.txt")}
    for n in (23, 25, 27):
        value, used = rows[n]
        k = len(used) - 1
        disjoint = O.primes_1_mod_n(n, k + 1, below=min(used))
        assert not set(disjoint) & set(used)
        got, residues = px.perm_schur_crt_primes(n, disjoint)
        assert got == value, n
        assert residues[-1] == value % disjoint[-1]


def test_schur33_benchmark_launch_matches_oracle_residue(px):
    """Full-size parity in the benchmark's launch configuration: the five S_33
    residue matrices in one batched perm_modp call (the Nijenhuis-Wilf walk the
    benchmark times) give, for the first prime, the residue the oracle computed
    over all 2^33 subsets (tests/golden/schur33_residue.txt, written by
    make_schur33_residue.py from the oracle alone).  perm(S_33) mod p does not
    depend on the primitive root chosen."""
    from conftest import read_golden
    n, p, _, r = (int(x) for x in read_golden("schur33_residue.txt")[0])
    primes = O.primes_1_mod_n(n, 5)
    assert primes[0] == p
    mats = [O.schur_residue_matrix(n, q, O.primitive_nth_root(q, n)) for q in primes]
    got = run_modp(px, mats, primes)
    assert int(got[0]) == r


@pytest.mark.parametrize("n", [8, 9, 12, 14, 15, 16])
def test_lone_complex_walk_equals_batched_bits(px, n):
    """Integer mode: a lone complex matrix runs four lanes per chunk, the same
    matrix in a batch large enough for the one-lane walk runs one; the bits
    agree, with the built-in chunking (lane groups of 16 or 32 chunks, merged
    across warps) and with a pinned chunk length that leaves groups of 4."""
    import torch
    old = px.permx_set_fp_arith(px.FP_ARITH_INT)
    saved = px.perm_tune_get(px.FIELD_C128, n)
    try:
        A = ensemble("haar_u", n, 1, seed=8000 + n)[0]
        for ell in (0, n - 3):                    # 0: the built-in rule
            px.perm_tune_set(px.FIELD_C128, n, ell)
            chunks = 2 ** (n - 1 - px.perm_tune_get(px.FIELD_C128, n))
            others = list(ensemble("ginibre_c", n, -(-20000 // chunks) + 1, seed=8100 + n))
            lone = run_fp(px, [A])[0]
            both = run_fp(px, others[:3] + [A] + others[3:])
            assert both[3] == lone, (n, ell)
            ref = O.perm_dp(A)
            assert abs(lone - ref) <= 1e-9 * abs(ref)
        torch.cuda.synchronize()
    finally:
        px.perm_tune_set(px.FIELD_C128, n, 0)
        assert px.perm_tune_get(px.FIELD_C128, n) == saved
        px.permx_set_fp_arith(old)
