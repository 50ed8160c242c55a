"""DFT inputs and the oracle on them (paper §3.3 Table "dft", §4.2): the
geodesic towards F_n is a one-parameter unitary group with the right end
points, and the oracle's perm(F_n) times n^{n/2} is the exact integer
perm(S_n) that the oracle's cyclotomic count reduction gives; the
composite/prime percentile values of Table "dft" follow from |perm(F_n)| and
the exponential law of |perm U|^2 with mean n!(n-1)!/(2n-1)!."""
import math

import numpy as np
import pytest

import oracle as O
from workloads import dft_matrix, geodesic_dft


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9, 12])
@pytest.mark.parametrize("branch", ["principal", "minus"])
def test_dft_geodesic_group(n, branch):
    F = dft_matrix(n)
    assert np.allclose(F @ F.conj().T, np.eye(n), atol=1e-13)
    assert np.allclose(geodesic_dft(n, 0.0, branch), np.eye(n), atol=1e-13)
    assert np.allclose(geodesic_dft(n, 1.0, branch), F, atol=1e-13)
    a, b = 0.31, 0.42
    G = geodesic_dft(n, a, branch) @ geodesic_dft(n, b, branch)
    assert np.allclose(G, geodesic_dft(n, a + b, branch), atol=1e-12)
    H = geodesic_dft(n, 0.37, branch)
    assert np.allclose(H @ H.conj().T, np.eye(n), atol=1e-13)


def test_branches_differ_only_on_minus_one():
    # the branches differ exactly when -1 is an eigenvalue of F_n
    for n in (2, 3, 4, 5, 9):
        F = dft_matrix(n)
        has_m1 = np.linalg.matrix_rank(F + np.eye(n), tol=1e-8) < n
        same = np.allclose(geodesic_dft(n, 0.5, "principal"), geodesic_dft(n, 0.5, "minus"), atol=1e-12)
        assert same == (not has_m1), n


@pytest.mark.parametrize("n", [3, 5, 7, 9, 11, 13])
def test_perm_dft_is_exact_schur_over_root(n):
    exact = O.schur_exact(n)
    v = O.perm_dp(dft_matrix(n))
    assert abs(v * n ** (n / 2) - exact) <= 1e-9 * max(abs(exact), 1.0)


@pytest.mark.parametrize("n,pct", [(9, 0.34), (15, 0.14)])
def test_table_dft_composite_percentiles_from_exponential_law(n, pct):
    """Paper §3.3 Table "dft": the DFT permanent's percentile among Haar
    samples for composite n.  Under |perm U|^2 ~ Exp(mean mu),
    mu = n!(n-1)!/(2n-1)!, the percentile is 1 - exp(-|perm F_n|^2 / mu)."""
    pf = abs(O.perm_dp(dft_matrix(n)))
    mu = math.factorial(n) * math.factorial(n - 1) / math.factorial(2 * n - 1)
    assert abs((1.0 - math.exp(-pf * pf / mu)) - pct) <= 0.015
