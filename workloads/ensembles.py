"""Random-matrix ensembles and geodesic points (inputs only).

Every generator takes a ``numpy.random.Generator`` (PCG64 from
``rng(seed)``) so that a seed fixes the input exactly.

* Haar unitary: QR of a complex Ginibre matrix with N(0,1/2)+iN(0,1/2)
  entries, with the phases of R's diagonal folded into Q (paper §3.1,
  Mezzadri's recipe).
* Haar orthogonal: the same with real N(0,1) entries and the signs of R's
  diagonal folded into Q (paper §5.1, "same pipeline").
* GUE (A+A^*)/2 with A complex Ginibre CN(0,1); GOE (A+A^T)/2 with A real
  Ginibre N(0,1); complex Ginibre CN(0,1) (Re, Im ~ N(0,1/2)); real
  Ginibre N(0,1) (paper §6, list of ensembles).
* Cycle geodesic gamma(t) = Q diag(e^{i t theta_k}) Q^* towards the n-cycle
  permutation matrix (paper §4, §4.1): ``branch="principal"`` takes the
  eigenphases in (-pi, pi]; ``branch="circulant"`` takes 2 pi k / n,
  k = 0..n-1, which is the closed form of paper eq. (circulant).
* DFT matrix F_n = (e^{2 pi i jk/n})_{j,k} / sqrt(n) (paper §1, §3.3) and the
  geodesic gamma(t) = exp(t log F_n) towards it (paper §4.2).  F_n^4 = I, so
  its eigenvalues lie in {1, i, -1, -i} and the spectral projectors are
  P_lambda = (1/4) sum_{m<4} (F_n / lambda)^m; gamma(t) = sum_lambda
  e^{i t theta_lambda} P_lambda with theta = 0, pi/2, -pi/2 for 1, i, -i and,
  for -1, +pi (``branch="principal"``, phases in (-pi, pi]) or -pi
  (``branch="minus"``).  No eigen-solver: the projectors are exact
  polynomials in F_n.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def _cn(n: int, g: np.random.Generator, var: float = 1.0) -> np.ndarray:
    s = np.sqrt(var / 2.0)
    return g.normal(0.0, s, (n, n)) + 1j * g.normal(0.0, s, (n, n))


def haar_unitary(n: int, g: np.random.Generator) -> np.ndarray:
    Z = _cn(n, g, 1.0)
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    ph = d / np.abs(d)
    return np.ascontiguousarray(Q * ph[None, :])


def haar_orthogonal(n: int, g: np.random.Generator) -> np.ndarray:
    Z = g.normal(0.0, 1.0, (n, n))
    Q, R = np.linalg.qr(Z)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return np.ascontiguousarray(Q * s[None, :])


def gue(n: int, g: np.random.Generator) -> np.ndarray:
    A = _cn(n, g, 1.0)
    return np.ascontiguousarray((A + A.conj().T) / 2.0)


def goe(n: int, g: np.random.Generator) -> np.ndarray:
    A = g.normal(0.0, 1.0, (n, n))
    return np.ascontiguousarray((A + A.T) / 2.0)


def ginibre_c(n: int, g: np.random.Generator) -> np.ndarray:
    return np.ascontiguousarray(_cn(n, g, 1.0))


def ginibre_r(n: int, g: np.random.Generator) -> np.ndarray:
    return np.ascontiguousarray(g.normal(0.0, 1.0, (n, n)))


ENSEMBLES = {
    # name: (generator, is_complex)
    "haar_u": (haar_unitary, True),
    "haar_o": (haar_orthogonal, False),
    "gue": (gue, True),
    "goe": (goe, False),
    "ginibre_c": (ginibre_c, True),
    "ginibre_r": (ginibre_r, False),
}


def ensemble(name: str, n: int, count: int, seed: int) -> np.ndarray:
    """``count`` matrices of one ensemble, shape (count, n, n)."""
    fn, cplx = ENSEMBLES[name]
    g = rng(seed)
    out = np.empty((count, n, n), dtype=np.complex128 if cplx else np.float64)
    for i in range(count):
        out[i] = fn(n, g)
    return out


def geodesic_cycle(n: int, t: float, branch: str = "principal") -> np.ndarray:
    """gamma(t) on the geodesic from I to the n-cycle C_n, (C_n)_{ij} = delta_{i, j+1 mod n}.

    C_n v_k = e^{-2 pi i k/n} v_k with v_k = (e^{2 pi i k j / n})_j / sqrt(n), so
    gamma(t)_{jl} = (1/n) sum_k e^{i t phi_k} e^{2 pi i k (j - l)/n}, phi_k the
    chosen phase of e^{-2 pi i k / n}.
    """
    k = np.arange(n)
    if branch == "principal":
        phi = -2.0 * np.pi * k / n
        phi = np.where(phi <= -np.pi, phi + 2.0 * np.pi, phi)   # into (-pi, pi]
    elif branch == "circulant":
        phi = (2.0 * np.pi * ((-k) % n)) / n                     # into [0, 2 pi)
    else:
        raise ValueError(branch)
    j = np.arange(n)
    V = np.exp(2j * np.pi * np.outer(j, k) / n) / np.sqrt(n)     # columns v_k
    return np.ascontiguousarray((V * np.exp(1j * t * phi)[None, :]) @ V.conj().T)


def dft_matrix(n: int) -> np.ndarray:
    """F_n = S_n / sqrt(n), S_n = (e^{2 pi i jk/n})_{j,k=0}^{n-1}."""
    j = np.arange(n)
    return np.ascontiguousarray(np.exp(2j * np.pi * np.outer(j, j) / n) / np.sqrt(n))


def geodesic_dft(n: int, t: float, branch: str = "principal") -> np.ndarray:
    """gamma(t) = exp(t log F_n) on the geodesic from I to the DFT matrix."""
    if branch not in ("principal", "minus"):
        raise ValueError(branch)
    F = dft_matrix(n)
    eye = np.eye(n, dtype=np.complex128)
    out = np.zeros((n, n), dtype=np.complex128)
    theta_m1 = np.pi if branch == "principal" else -np.pi
    for lam, th in ((1.0, 0.0), (1j, np.pi / 2), (-1.0, theta_m1), (-1j, -np.pi / 2)):
        B = F / lam
        B2 = B @ B
        P = (eye + B + B2 + B2 @ B) / 4.0
        out += np.exp(1j * t * th) * P
    return np.ascontiguousarray(out)


def random_residues(n: int, p: int, g: np.random.Generator) -> np.ndarray:
    """Uniform entries in [0, p) as uint32."""
    return g.integers(0, p, (n, n), dtype=np.uint64).astype(np.uint32)
