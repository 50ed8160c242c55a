"""Plain CPU oracle for matrix permanents — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product (``paper_2602_10141_b300``) never imports it, and it imports nothing
from the product: the two share no code.  The one module both sides use is
``workloads`` (seeded input generators, none of the method's arithmetic).

What it computes, and where the paper defines it:

* ``perm_*`` — the permanent ``perm(A) = sum_sigma prod_i a_{i,sigma(i)}``
  (paper §1, definition) by brute force, by a row-expansion DP of the same
  sum, and by Ryser's inclusion–exclusion formula
  ``(-1)^n sum_S (-1)^|S| prod_i sum_{j in S} a_ij`` (paper §1, cited; §2.2)
  with row sums recomputed from scratch — all in ``oracle.c``.
* F_p versions with ``uint64`` and ``%`` (paper §2.1).
* Field set-up for the Schur matrix (paper §2.1): primes ``p = 1 (mod n)``
  below ``2**31`` by trial division, a primitive n-th root of unity ``g``,
  and the residue matrix ``(g^{jk} mod p)``.
* Chinese remaindering to the symmetric range (paper §2.1) in Python ints,
  with the prime count driven by ``|perm(S_n)| <= n^{n/2}`` (paper §2.1).
* The exact integer ``perm(S_n)`` from the counts
  ``c_m = #{sigma : sum_i i*sigma(i) = m (mod n)}`` reduced modulo the
  cyclotomic polynomial ``Phi_n`` (definition of ``S_n``, paper §1).

* ``cpu_walk`` — the paper's Gray-code walk as a plain single-threaded CPU
  program (incremental row sums), the comparator for GPU-over-one-core
  speed-ups; pinned to the recomputing Ryser above.
* ``sample_histogram`` — counts of |z|^2, Re z or Im z between given edges
  (the distributions behind the paper's Q-Q plots and tail probabilities).
* ``sample_stats`` — the sample moments, counts and extremes the paper
  reports over batches of permanents (§3.2 second moment and circularity, §5.1
  Table "orthogonal", §6.1 real-valuedness, §7.2 Table "lognormal", the
  anti-concentration probabilities), from their textbook definitions with
  exactly rounded sums (``math.fsum``) in two passes.

Pins (tests/test_oracle_*.py) tie each function to something other than
itself: brute force, closed forms, invariants and the paper's printed
midpoint table (Table "midpoint", §4.1).
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
from typing import Iterable, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, OpenMP), and the
    single-core CPU walks of ``cpu_walk.c`` beside it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-Wall", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    from . import cpu_walk
    cpu_walk.build(force)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i = ctypes.c_int
        for name in ("oracle_perm_brute_r", "oracle_perm_brute_c", "oracle_perm_dp_r", "oracle_perm_dp_c"):
            getattr(lib, name).argtypes = [i, dp, dp]
            getattr(lib, name).restype = i
        for name in ("oracle_perm_ryser_r", "oracle_perm_ryser_c"):
            getattr(lib, name).argtypes = [i, dp, dp, dp]
            getattr(lib, name).restype = i
        for name in ("oracle_perm_brute_modp", "oracle_perm_dp_modp", "oracle_perm_ryser_modp"):
            getattr(lib, name).argtypes = [i, u32p, ctypes.c_uint32, u32p]
            getattr(lib, name).restype = i
        lib.oracle_perm_ryser_modp_gray_range.argtypes = [i, u32p, ctypes.c_uint32, ctypes.c_uint64,
                                                          ctypes.c_uint64, u32p]
        lib.oracle_perm_ryser_modp_gray_range.restype = i
        lib.oracle_schur_counts.argtypes = [i, u64p]
        lib.oracle_schur_counts.restype = i
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = i
        lib.oracle_set_num_threads.argtypes = [i]
        lib.oracle_set_num_threads.restype = None
        _lib = lib
    return _lib


class use_library:
    """Context manager that makes every oracle function call a different build
    of ``oracle.c`` (used by the planted-mistake tests)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        lib = ctypes.CDLL(self.path)
        for name in dir(self._saved):
            if name.startswith("oracle_"):
                src, dst = getattr(self._saved, name), getattr(lib, name)
                dst.argtypes, dst.restype = src.argtypes, src.restype
        _lib = lib
        return lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().oracle_num_threads())


def set_num_threads(k: int) -> None:
    """Use k OpenMP threads in the following calls (timing on one core or on all)."""
    _load().oracle_set_num_threads(int(k))


def _real(A) -> tuple[np.ndarray, int]:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    return A, A.shape[0]


def _cplx(A) -> tuple[np.ndarray, int]:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    return A.view(np.float64), A.shape[0]


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"{what} failed with code {rc}")


# ----------------------------------------------------------------------------
# real / complex permanents
# ----------------------------------------------------------------------------

def perm_brute(A, pair: bool = False):
    """Definition by brute force over all n! permutations (n <= 11), long double."""
    A = np.asarray(A)
    out = np.zeros(4)
    if np.iscomplexobj(A):
        a, n = _cplx(A)
        _check(_load().oracle_perm_brute_c(n, _ptr(a, ctypes.c_double), _ptr(out, ctypes.c_double)), "brute_c")
        v = complex(out[0] + out[1], out[2] + out[3])
        return ((out[0], out[1]), (out[2], out[3])) if pair else v
    a, n = _real(A)
    _check(_load().oracle_perm_brute_r(n, _ptr(a, ctypes.c_double), _ptr(out, ctypes.c_double)), "brute_r")
    return (out[0], out[1]) if pair else float(out[0] + out[1])


def perm_dp(A, pair: bool = False):
    """Definition organised as a row-expansion DP over column sets, double-double.

    Real n <= 26, complex n <= 25 (memory 2^n double-double values).
    """
    A = np.asarray(A)
    out = np.zeros(4)
    if np.iscomplexobj(A):
        a, n = _cplx(A)
        _check(_load().oracle_perm_dp_c(n, _ptr(a, ctypes.c_double), _ptr(out, ctypes.c_double)), "dp_c")
        return ((out[0], out[1]), (out[2], out[3])) if pair else complex(out[0] + out[1], out[2] + out[3])
    a, n = _real(A)
    _check(_load().oracle_perm_dp_r(n, _ptr(a, ctypes.c_double), _ptr(out, ctypes.c_double)), "dp_r")
    return (out[0], out[1]) if pair else float(out[0] + out[1])


def perm_ryser(A, with_abs: bool = False):
    """Ryser's formula by direct subset enumeration, double-double (n <= 30).

    With ``with_abs`` also returns ``sum_S |prod_i r_i(S)|``: the total size
    of the terms that cancel, which scales floating-point error bounds.
    """
    A = np.asarray(A)
    out = np.zeros(4)
    ab = np.zeros(1)
    if np.iscomplexobj(A):
        a, n = _cplx(A)
        _check(_load().oracle_perm_ryser_c(n, _ptr(a, ctypes.c_double), _ptr(out, ctypes.c_double),
                                           _ptr(ab, ctypes.c_double)), "ryser_c")
        v = complex(out[0] + out[1], out[2] + out[3])
    else:
        a, n = _real(A)
        _check(_load().oracle_perm_ryser_r(n, _ptr(a, ctypes.c_double), _ptr(out, ctypes.c_double),
                                           _ptr(ab, ctypes.c_double)), "ryser_r")
        v = float(out[0] + out[1])
    return (v, float(ab[0])) if with_abs else v


def perm_python(A):
    """Definition in pure Python (itertools.permutations), for tiny n only."""
    A = np.asarray(A)
    n = A.shape[0]
    if n > 8:
        raise ValueError("pure-Python brute force is for n <= 8")
    total = 0
    for sigma in itertools.permutations(range(n)):
        t = 1
        for i in range(n):
            t = t * A[i, sigma[i]].item()
        total += t
    return total


# ----------------------------------------------------------------------------
# F_p
# ----------------------------------------------------------------------------

def _u32(A, p) -> tuple[np.ndarray, int]:
    A = np.asarray(A)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    if A.size and (int(A.min()) < 0 or int(A.max()) >= p):
        raise ValueError("entries must lie in [0, p)")
    return np.ascontiguousarray(A.astype(np.uint32)), A.shape[0]


def perm_modp_brute(A, p: int) -> int:
    """perm(A) mod p by brute force (n <= 11)."""
    a, n = _u32(A, p)
    out = np.zeros(1, np.uint32)
    _check(_load().oracle_perm_brute_modp(n, _ptr(a, ctypes.c_uint32), p, _ptr(out, ctypes.c_uint32)), "brute_modp")
    return int(out[0])


def perm_modp_dp(A, p: int) -> int:
    """perm(A) mod p by the row-expansion DP (n <= 28)."""
    a, n = _u32(A, p)
    out = np.zeros(1, np.uint32)
    _check(_load().oracle_perm_dp_modp(n, _ptr(a, ctypes.c_uint32), p, _ptr(out, ctypes.c_uint32)), "dp_modp")
    return int(out[0])


def perm_modp(A, p: int) -> int:
    """perm(A) mod p by Ryser's formula, subsets in binary order (n <= 48)."""
    a, n = _u32(A, p)
    out = np.zeros(1, np.uint32)
    _check(_load().oracle_perm_ryser_modp(n, _ptr(a, ctypes.c_uint32), p, _ptr(out, ctypes.c_uint32)), "ryser_modp")
    return int(out[0])


def ryser_modp_gray_range(A, p: int, k0: int, k1: int) -> int:
    """sum_{k0<=k<k1} (-1)^{|g(k)|} prod_i sum_{j in g(k)} a_ij mod p, g(k) = k ^ (k >> 1).

    No ``(-1)^n`` factor: over the whole range [0, 2^n) this equals
    ``(-1)^n perm(A) mod p``.
    """
    a, n = _u32(A, p)
    out = np.zeros(1, np.uint32)
    _check(_load().oracle_perm_ryser_modp_gray_range(n, _ptr(a, ctypes.c_uint32), p, k0, k1,
                                                     _ptr(out, ctypes.c_uint32)), "gray_range")
    return int(out[0])


# ----------------------------------------------------------------------------
# Field set-up for the Schur matrix (paper §2.1)
# ----------------------------------------------------------------------------

def is_prime(m: int) -> bool:
    """Trial division by every integer up to sqrt(m)."""
    if m < 2:
        return False
    if m % 2 == 0:
        return m == 2
    d = 3
    while d * d <= m:
        if m % d == 0:
            return False
        d += 2
    return True


def ryser_nw_modp_gray_range(A, p: int, k0: int, k1: int) -> int:
    """The Nijenhuis-Wilf form of Ryser's sum over Gray indices [k0, k1) of its
    2^(n-1)-subset walk, mod p (pure Python, small n):

        sum_{k0<=k<k1} (-1)^{|g(k)|} prod_i (x_i + sum_{j in g(k)} a_ij),
        x_i = a_{i,n-1} - (1/2) sum_j a_ij,  1/2 = (p+1)/2 mod p,

    with g(k) = k ^ (k >> 1) a subset of the columns 0..n-2 and every row sum
    recomputed for every subset.  No (-1)^(n-1) 2 factor: over the whole range
    [0, 2^(n-1)) it equals (-1)^(n-1) perm(A) / 2 mod p (p odd).
    """
    a = [[int(v) % p for v in row] for row in np.asarray(A)]
    n = len(a)
    if n < 1 or not 0 <= k0 <= k1 <= 1 << (n - 1):
        raise ValueError("need n >= 1 and 0 <= k0 <= k1 <= 2^(n-1)")
    half = (p + 1) // 2
    x = [(a[i][n - 1] - half * sum(a[i])) % p for i in range(n)]
    total = 0
    for k in range(k0, k1):
        S = k ^ (k >> 1)
        cols = [j for j in range(n - 1) if S >> j & 1]
        prod = 1
        for i in range(n):
            prod = prod * ((x[i] + sum(a[i][j] for j in cols)) % p) % p
        total = (total - prod) % p if len(cols) & 1 else (total + prod) % p
    return total


def primes_1_mod_n(n: int, count: int, below: int = 2 ** 31, skip: int = 0) -> list[int]:
    """The largest primes p < ``below`` with p = 1 (mod n), in descending order.

    ``skip`` drops that many of the largest ones first (to build a second,
    disjoint prime set).
    """
    out = []
    k = (below - 2) // n
    while len(out) < count + skip and k > 0:
        p = k * n + 1
        if p < below and is_prime(p):
            out.append(p)
        k -= 1
    return out[skip:]


def prime_count_for(n: int) -> int:
    """⌈((n/2)·log2 n + 2)/30⌉ + 1 primes below 2^31 (the configured count).

    ``crt_modulus_suffices`` checks the exact requirement separately.
    """
    return math.ceil(((n / 2) * math.log2(n) + 2) / 30) + 1


def _prime_factors(m: int) -> list[int]:
    fs, d = [], 2
    while d * d <= m:
        if m % d == 0:
            fs.append(d)
            while m % d == 0:
                m //= d
        d += 1
    if m > 1:
        fs.append(m)
    return fs


def primitive_nth_root(p: int, n: int) -> int:
    """Smallest-h choice: g = h^((p-1)/n) mod p for the smallest h >= 2 whose g
    has multiplicative order exactly n (g^n = 1 and g^(n/q) != 1 for every
    prime q | n)."""
    if (p - 1) % n:
        raise ValueError("p != 1 (mod n)")
    qs = _prime_factors(n)
    for h in range(2, p):
        g = pow(h, (p - 1) // n, p)
        if pow(g, n, p) != 1:
            continue
        if all(pow(g, n // q, p) != 1 for q in qs):
            return g
    raise ValueError("no primitive root found")


def schur_residue_matrix(n: int, p: int, g: int) -> np.ndarray:
    """(g^{jk} mod p)_{j,k=0..n-1} as uint32 (paper §2.1)."""
    M = np.zeros((n, n), dtype=np.uint32)
    for j in range(n):
        for k in range(n):
            M[j, k] = pow(g, j * k, p)
    return M


def schur_complex_matrix(n: int) -> np.ndarray:
    """S_n = (exp(2 pi i jk / n)) (paper §1)."""
    j = np.arange(n)
    return np.exp(2j * np.pi * np.outer(j, j) / n)


# ----------------------------------------------------------------------------
# Chinese remaindering (paper §2.1)
# ----------------------------------------------------------------------------

def crt(residues: Sequence[int], primes: Sequence[int]) -> int:
    """The unique x in (-M/2, M/2] with x = r_k (mod p_k), M = prod p_k.

    Textbook construction x = sum_k r_k * M_k * (M_k^{-1} mod p_k) mod M.
    """
    if len(residues) != len(primes) or not primes:
        raise ValueError("one residue per prime")
    M = 1
    for p in primes:
        M *= p
    x = 0
    for r, p in zip(residues, primes):
        Mk = M // p
        x += r * Mk * pow(Mk, -1, p)
    x %= M
    if x > M // 2:
        x -= M
    return x


def crt_modulus_suffices(n: int, primes: Iterable[int]) -> bool:
    """True iff M = prod p > 2 * n^{n/2}, so (-M/2, M/2] holds every
    integer of absolute value <= n^{n/2} (the bound of paper §2.1).
    Compared exactly: M^2 > 4 n^n."""
    M = 1
    for p in primes:
        M *= p
    return M * M > 4 * n ** n


# ----------------------------------------------------------------------------
# Exact perm(S_n) from the permutation counts
# ----------------------------------------------------------------------------

def schur_counts(n: int) -> list[int]:
    """c_m = #{sigma in S_n : sum_i i*sigma(i) = m (mod n)}, m = 0..n-1 (n <= 20)."""
    out = np.zeros(n, dtype=np.uint64)
    _check(_load().oracle_schur_counts(n, _ptr(out, ctypes.c_uint64)), "schur_counts")
    return [int(v) for v in out]


def _poly_divmod(num: list[int], den: list[int]) -> tuple[list[int], list[int]]:
    """Integer polynomial long division by a monic ``den``; coefficients low to high."""
    num = list(num)
    dn = len(den) - 1
    if den[-1] != 1:
        raise ValueError("monic divisor expected")
    q = [0] * max(len(num) - dn, 1)
    for k in range(len(num) - 1, dn - 1, -1):
        c = num[k]
        if c:
            q[k - dn] = c
            for i in range(dn + 1):
                num[k - dn + i] -= c * den[i]
    rem = num[:dn] if dn > 0 else [0]
    return q, rem


def cyclotomic(n: int) -> list[int]:
    """Phi_n with integer coefficients (low to high), from x^n - 1 = prod_{d | n} Phi_d."""
    num = [-1] + [0] * (n - 1) + [1]
    for d in range(1, n):
        if n % d == 0:
            num, rem = _poly_divmod(num, cyclotomic(d))
            if any(rem):
                raise ArithmeticError("non-exact cyclotomic division")
    return num


def schur_exact(n: int) -> int:
    """perm(S_n) as an exact integer: sum_m c_m x^m reduced modulo Phi_n(x).

    The remainder must be a constant (perm(S_n) is a rational integer); a
    non-constant remainder raises.
    """
    c = schur_counts(n)
    _, rem = _poly_divmod(c, cyclotomic(n))
    if any(rem[1:]):
        raise ArithmeticError("perm(S_n) did not reduce to an integer")
    return rem[0]


def schur_modp_from_counts(n: int, p: int, g: int) -> int:
    """perm((g^{jk}) mod p) = sum_m c_m g^m mod p."""
    return sum(c * pow(g, m, p) for m, c in enumerate(schur_counts(n))) % p


def sample_stats(values, threshold: float = math.inf, real_tol: float = 0.0) -> dict:
    """Sample statistics of a list of permanents (paper §3-§7).

    Plain (biased, divide-by-N) moments: means, central second moments of
    Re and Im and their covariance, skewness m3/m2^1.5 and excess kurtosis
    m4/m2^2 - 3 of Re z, E|z|^2, E|z|^4, E[z^2], min and max |z|^2, and the
    mean, variance, skewness and excess kurtosis of log|z| over the samples
    with |z|^2 > 0.  Counts: |z|^2 > 0, |z|^2 >= threshold, and
    |Im z| <= real_tol |z|, where |z|^2 = re*re + im*im with each product and
    the sum rounded to double (numpy float64, no fused multiply-add) and
    |z| = sqrt(|z|^2).  Central moments are taken about the means (second
    pass); every sum is math.fsum.
    """
    z = np.asarray(values)
    re = np.ascontiguousarray(z.real, dtype=np.float64).reshape(-1)
    im = (np.ascontiguousarray(z.imag, dtype=np.float64).reshape(-1) if np.iscomplexobj(z)
          else np.zeros_like(re))
    N = re.size
    if N < 1:
        raise ValueError("need at least one sample")
    a2 = re * re + im * im                       # elementwise: two roundings, no fma
    nz = a2 > 0.0
    logs = 0.5 * np.log(a2[nz])
    fs = math.fsum
    mean_re, mean_im = fs(re) / N, fs(im) / N
    dr, di = re - mean_re, im - mean_im
    m2r = fs(dr * dr) / N
    out = {
        "count": N,
        "count_nonzero": int(nz.sum()),
        "count_above": int((a2 >= threshold).sum()),
        "count_real": int((np.abs(im) <= real_tol * np.sqrt(a2)).sum()),
        "mean_re": mean_re, "mean_im": mean_im,
        "var_re": m2r, "var_im": fs(di * di) / N, "cov_re_im": fs(dr * di) / N,
        "mean_abs2": fs(a2) / N, "mean_abs4": fs(a2 * a2) / N,
        "mean_z2_re": fs(re * re - im * im) / N, "mean_z2_im": fs(2.0 * re * im) / N,
        "min_abs2": float(a2.min()), "max_abs2": float(a2.max()),
    }
    with np.errstate(divide="ignore", invalid="ignore"):
        out["skew_re"] = float(np.float64(fs(dr ** 3) / N) / np.float64(m2r) ** 1.5)
        out["exkurt_re"] = float(np.float64(fs(dr ** 4) / N) / np.float64(m2r) ** 2 - 3.0)
        M = logs.size
        if M:
            lm = fs(logs) / M
            dl = logs - lm
            lv = fs(dl * dl) / M
            out["log_mean"], out["log_var"] = lm, lv
            out["log_skew"] = float(np.float64(fs(dl ** 3) / M) / np.float64(lv) ** 1.5)
            out["log_exkurt"] = float(np.float64(fs(dl ** 4) / M) / np.float64(lv) ** 2 - 3.0)
        else:
            out.update(log_mean=math.nan, log_var=math.nan, log_skew=math.nan, log_exkurt=math.nan)
    return out


def sample_histogram(values, edges, kind: int = 0) -> np.ndarray:
    """Counts of x = |z|^2 (kind 0; re*re + im*im, each product and the sum
    rounded to double), Re z (1) or Im z (2) against sorted edges: element 0
    counts x < edges[0], element b counts edges[b-1] <= x < edges[b], the last
    x >= edges[-1]; NaN is not counted."""
    z = np.asarray(values)
    re = np.asarray(z.real, dtype=np.float64).reshape(-1)
    im = np.asarray(z.imag, dtype=np.float64).reshape(-1) if np.iscomplexobj(z) else np.zeros_like(re)
    x = re * re + im * im if kind == 0 else (re if kind == 1 else im)
    x = x[~np.isnan(x)]
    e = np.asarray(edges, dtype=np.float64)
    out = np.zeros(len(e) + 1, np.int64)
    for v in x:                                    # plain definition: count the edges at or below v
        out[int(np.sum(e <= v))] += 1
    return out
