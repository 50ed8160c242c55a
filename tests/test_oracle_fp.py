"""Pins for the real/complex oracle: each function is tied to something other
than itself — brute force over all permutations, pure-Python enumeration,
closed forms, invariants, and the paper's printed midpoint table (§4.1)."""
import math
import os

import numpy as np
import pytest

import oracle as O
from workloads import geodesic_cycle, ginibre_c, ginibre_r, goe, gue, haar_orthogonal, haar_unitary, rng


def _absperm(A):
    """perm(|A|) by brute force: the sum of |terms| of the definition."""
    return O.perm_brute(np.abs(A))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_brute_matches_pure_python(n):
    g = rng(100 + n)
    for A in (ginibre_r(n, g), ginibre_c(n, g), g.integers(-3, 4, (n, n)).astype(float)):
        py = O.perm_python(A)
        assert abs(O.perm_brute(A) - py) <= 1e-15 * max(1.0, _absperm(A))


def test_brute_integer_exact():
    # small-integer matrices: every partial product is an exact integer in long double
    g = rng(7)
    for n in range(1, 8):
        A = g.integers(-4, 5, (n, n))
        assert O.perm_brute(A.astype(float)) == O.perm_python(A)


@pytest.mark.parametrize("n", list(range(1, 10)))
def test_dp_and_ryser_match_brute(n):
    g = rng(200 + n)
    for A in (ginibre_r(n, g), ginibre_c(n, g), haar_unitary(n, g), goe(n, g)):
        ref = O.perm_brute(A)
        scale = _absperm(A)
        assert abs(O.perm_dp(A) - ref) <= 4e-18 * n * scale
        assert abs(O.perm_ryser(A) - ref) <= 4e-18 * n * scale * 2 ** n


@pytest.mark.parametrize("n", [12, 14, 16])
def test_dp_matches_ryser_at_larger_n(n):
    # two different algorithms (row-expansion DP vs inclusion-exclusion)
    g = rng(300 + n)
    for A in (ginibre_c(n, g), haar_orthogonal(n, g)):
        r, abs_terms = O.perm_ryser(A, with_abs=True)
        d = O.perm_dp(A)
        assert abs(r - d) <= 1e-28 * n * abs_terms + 1e-15 * abs(d)


@pytest.mark.parametrize("n", [1, 2, 5, 10, 16, 20])
def test_identity_and_all_ones(n):
    assert O.perm_dp(np.eye(n)) == 1.0
    assert O.perm_dp(np.ones((n, n))) == float(math.factorial(n))
    if n <= 16:
        assert O.perm_ryser(np.eye(n)) == 1.0
        assert O.perm_ryser(np.ones((n, n))) == float(math.factorial(n))


def test_permutation_matrices():
    g = rng(11)
    for n in (3, 6, 9, 13):
        P = np.eye(n)[g.permutation(n)]
        assert O.perm_dp(P) == 1.0
        assert O.perm_ryser(P) == 1.0


def _derangements(n):
    d = [1, 0]
    for k in range(2, n + 1):
        d.append((k - 1) * (d[k - 1] + d[k - 2]))
    return d[n]


@pytest.mark.parametrize("n", [2, 3, 7, 12, 15])
def test_derangements(n):
    # perm(J - I) counts fixed-point-free permutations: D_n = (n-1)(D_{n-1} + D_{n-2})
    A = np.ones((n, n)) - np.eye(n)
    assert O.perm_dp(A) == float(_derangements(n))
    assert O.perm_ryser(A) == float(_derangements(n))


def test_rank_one_closed_form():
    # perm(u v^T) = n! prod u_i prod v_j
    g = rng(12)
    for n in (4, 9, 13):
        u = g.normal(size=n) + 1j * g.normal(size=n)
        v = g.normal(size=n) + 1j * g.normal(size=n)
        ref = math.factorial(n) * np.prod(u) * np.prod(v)
        A = np.outer(u, v)
        for val in (O.perm_dp(A), O.perm_ryser(A)):
            assert abs(val - ref) <= 1e-13 * abs(ref)


def test_two_by_two_and_diagonal():
    a, b, c, d = 1.5, -2.25, 0.75, 3.0
    assert O.perm_ryser(np.array([[a, b], [c, d]])) == a * d + b * c
    assert O.perm_dp(np.array([[a, b], [c, d]])) == a * d + b * c
    g = rng(13)
    dg = g.normal(size=11)
    assert abs(O.perm_ryser(np.diag(dg)) - np.prod(dg)) <= 1e-15 * abs(np.prod(dg))


def test_block_diagonal_product():
    g = rng(14)
    A, B = ginibre_c(5, g), ginibre_c(7, g)
    M = np.zeros((12, 12), complex)
    M[:5, :5] = A
    M[5:, 5:] = B
    ref = O.perm_dp(A) * O.perm_dp(B)
    assert abs(O.perm_dp(M) - ref) <= 1e-13 * abs(ref)
    assert abs(O.perm_ryser(M) - ref) <= 1e-12 * abs(ref)


def test_invariances_and_linearity():
    g = rng(15)
    n = 11
    A = ginibre_c(n, g)
    ref = O.perm_dp(A)
    tol = 1e-12 * abs(ref)
    P, Q = g.permutation(n), g.permutation(n)
    assert abs(O.perm_dp(A[P][:, Q]) - ref) <= tol
    assert abs(O.perm_ryser(A[P][:, Q]) - ref) <= tol
    assert abs(O.perm_dp(A.T) - ref) <= tol
    assert abs(O.perm_ryser(A.T) - ref) <= tol
    d = g.normal(size=n) + 1j * g.normal(size=n)
    assert abs(O.perm_ryser(d[:, None] * A) - np.prod(d) * ref) <= 1e-12 * abs(np.prod(d) * ref)
    # multilinearity in one row
    B = A.copy()
    B[3] = g.normal(size=n)
    C = A.copy()
    C[3] = A[3] + B[3]
    assert abs(O.perm_ryser(C) - (ref + O.perm_dp(B))) <= 1e-12 * (abs(ref) + abs(O.perm_dp(B)))


def test_unitary_bound():
    # |perm(U)| <= 1 for unitary U (paper §2.1, Minc)
    g = rng(16)
    for n in (5, 9, 13):
        for _ in range(5):
            assert abs(O.perm_dp(haar_unitary(n, g))) <= 1.0
            assert abs(O.perm_dp(haar_orthogonal(n, g))) <= 1.0


def test_hermitian_is_real():
    # paper §6.1, Proposition: Hermitian H => perm(H) real
    g = rng(17)
    for n in (5, 8, 12):
        H = gue(n, g)
        for v in (O.perm_ryser(H), O.perm_dp(H)):
            assert abs(v.imag) <= 1e-14 * abs(v.real)


def _midpoint_rows(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "midpoint_table.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n, v, ratio, corr = line.split()
            rows.append((int(n), float(v), float(ratio), float(corr)))
    return rows


def test_midpoint_table(golden_dir):
    # paper §4.1, Table "midpoint": perm(gamma(1/2)) to 4 significant digits
    for n, v, ratio, corr in _midpoint_rows(golden_dir):
        if n > 19:
            continue   # n = 23 is covered by the slow test below
        val = O.perm_dp(geodesic_cycle(n, 0.5, "circulant"))
        assert abs(val.imag) <= 1e-12 * abs(val.real)
        assert float(f"{val.real:.3e}") == v, (n, val, v)
        r = abs(val.real) / (2 * math.exp(-n))
        assert round(r, 4) == ratio
        assert abs(n * (r - 1) - corr) <= 1.5e-3
        # same magnitude on the principal branch (the branch the serving workload uses)
        pr = O.perm_dp(geodesic_cycle(n, 0.5, "principal"))
        assert abs(abs(pr) - abs(val)) <= 1e-12 * abs(val)


@pytest.mark.slow
def test_midpoint_table_n23(golden_dir):
    n, v, ratio, corr = [r for r in _midpoint_rows(golden_dir) if r[0] == 23][0]
    val = O.perm_dp(geodesic_cycle(n, 0.5, "circulant"))
    assert float(f"{val.real:.3e}") == v
    assert round(abs(val.real) / (2 * math.exp(-n)), 4) == ratio


def test_midpoint_asymptotic_and_even_zero():
    # paper §4.1, Observation "Midpoint asymptotic": odd n -> (-1)^((n-1)/2) 2 e^{-n} (1 + 1/(3n) + O(n^-2)),
    # even n -> 0
    for n in (9, 15):
        val = O.perm_dp(geodesic_cycle(n, 0.5, "circulant")).real
        pred = (-1) ** ((n - 1) // 2) * 2 * math.exp(-n) * (1 + 1 / (3 * n))
        assert np.sign(val) == np.sign(pred)
        assert abs(val / pred - 1) <= 0.5 / n ** 2
    for n in (4, 6, 8, 10, 12):
        val = O.perm_dp(geodesic_cycle(n, 0.5, "circulant"))
        assert abs(val) <= 1e-15


def test_geodesic_endpoints_and_realness():
    # gamma(0) = I -> 1; gamma(1) = C_n (a permutation matrix) -> 1.  The cycle geodesic
    # is real-valued (paper §4.1 remark): on the principal branch gamma(t) itself is a real
    # matrix; eq. (circulant) differs from it only by a phase of perm, so |perm| agrees.
    for n in (5, 9):
        assert abs(O.perm_dp(geodesic_cycle(n, 0.0)) - 1) <= 1e-14
        assert abs(O.perm_dp(geodesic_cycle(n, 1.0, "circulant")) - 1) <= 1e-12
        for t in (0.1, 0.37, 0.8):
            v = O.perm_dp(geodesic_cycle(n, t, "principal"))
            assert abs(v.imag) <= 1e-14 * abs(v.real)
            w = O.perm_dp(geodesic_cycle(n, t, "circulant"))
            assert abs(abs(w) - abs(v)) <= 1e-13 * abs(v)
