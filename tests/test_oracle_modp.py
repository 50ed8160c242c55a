"""Pins for the F_p / exact-integer oracle (paper §2.1): brute force,
pure-Python enumeration, two independent algorithms, the exact integer
permanent reduced mod p, the Schur-matrix count identity, Galois invariance,
library primality, and Chinese remaindering of known integers."""
import itertools
import math

import numpy as np
import pytest
import sympy

import oracle as O
from workloads import random_residues, rng

PRIMES = [2, 3, 5, 13, 65537, 2147483629, 2147483647, 4294967291]


def _py_perm_int(A):
    n = A.shape[0]
    return sum(math.prod(int(A[i, s[i]]) for i in range(n)) for s in itertools.permutations(range(n)))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_brute_modp_matches_python(n):
    g = rng(400 + n)
    for p in PRIMES:
        A = random_residues(n, p, g)
        assert O.perm_modp_brute(A, p) == _py_perm_int(A) % p


@pytest.mark.parametrize("n", list(range(1, 10)))
def test_three_algorithms_agree_small(n):
    g = rng(500 + n)
    for p in PRIMES:
        A = random_residues(n, p, g)
        b = O.perm_modp_brute(A, p)
        assert O.perm_modp_dp(A, p) == b
        assert O.perm_modp(A, p) == b


@pytest.mark.parametrize("n", [12, 15, 18, 20])
def test_dp_matches_ryser_modp(n):
    g = rng(600 + n)
    for p in (2147483629, 65537):
        A = random_residues(n, p, g)
        assert O.perm_modp_dp(A, p) == O.perm_modp(A, p)


def test_integer_matrices_reduce_mod_p():
    # an integer matrix's exact permanent (pure Python) reduced mod p
    g = rng(7)
    for n in (4, 6, 7):
        A = g.integers(0, 50, (n, n))
        exact = _py_perm_int(A)
        for p in (101, 2147483629):
            assert O.perm_modp(A.astype(np.uint32), p) == exact % p


def test_gray_range_python_and_bijection():
    # the Gray-range partial sum against pure-Python subset enumeration, and the full
    # range against the binary-order Ryser sum (the Gray map is a bijection of [0, 2^n))
    g = rng(8)
    p = 2147483629
    n = 6
    A = random_residues(n, p, g)
    for k0, k1 in ((0, 64), (5, 17), (32, 64), (13, 14), (20, 20)):
        ref = 0
        for k in range(k0, k1):
            S = k ^ (k >> 1)
            t = 1
            for i in range(n):
                t *= sum(int(A[i, j]) for j in range(n) if S >> j & 1)
            ref += (-1) ** bin(S).count("1") * t
        assert O.ryser_modp_gray_range(A, p, k0, k1) == ref % p
    for n in (7, 12):
        A = random_residues(n, p, g)
        full = O.ryser_modp_gray_range(A, p, 0, 1 << n)
        assert full == ((-1) ** n * O.perm_modp_dp(A, p)) % p


def test_primes_and_roots():
    for n in (7, 12, 33, 43):
        ps = O.primes_1_mod_n(n, 6)
        assert all(sympy.isprime(p) and p % n == 1 and p < 2 ** 31 for p in ps)
        assert ps == sorted(ps, reverse=True) and len(set(ps)) == 6
        # nothing skipped: no prime = 1 (mod n) between consecutive entries
        for hi, lo in zip([2 ** 31] + ps[:-1], ps):
            assert not any(sympy.isprime(q) for q in range(lo + n, hi, n))
        for p in ps[:2]:
            gr = O.primitive_nth_root(p, n)
            assert sympy.n_order(gr, p) == n
    for m in range(1, 2000):
        assert O.is_prime(m) == sympy.isprime(m)


def test_prime_count_formula():
    # configured count: 5 primes for every n in 36..43 (with the n^{n/2} bound satisfied)
    for n in range(36, 44):
        k = O.prime_count_for(n)
        assert k == 5
        assert O.crt_modulus_suffices(n, O.primes_1_mod_n(n, k))
    assert O.prime_count_for(33) == 4
    assert O.crt_modulus_suffices(33, O.primes_1_mod_n(33, 4))


def test_crt_roundtrip():
    g = rng(9)
    ps = O.primes_1_mod_n(43, 5)
    M = math.prod(ps)
    for _ in range(50):
        x = int(g.integers(-2 ** 62, 2 ** 62)) * int(g.integers(1, 2 ** 60)) * int(g.integers(1, 2 ** 30))
        x %= M
        if x > M // 2:
            x -= M
        assert O.crt([x % p for p in ps], ps) == x
    assert O.crt([0] * 5, ps) == 0
    assert O.crt([p - 1 for p in ps], ps) == -1


def test_cyclotomic():
    for n in range(1, 40):
        phi = O.cyclotomic(n)
        assert len(phi) - 1 == sympy.totient(n)
        assert phi == [int(c) for c in reversed(sympy.Poly(sympy.cyclotomic_poly(n, sympy.Symbol("x"))).all_coeffs())]
    assert O.cyclotomic(7) == [1] * 7


@pytest.mark.parametrize("n", list(range(1, 15)))
def test_schur_counts_and_exact(n):
    c = O.schur_counts(n)
    assert sum(c) == math.factorial(n)
    x = O.schur_exact(n)
    assert x * x <= n ** n   # |perm(S_n)| <= n^{n/2} (paper §2.1)
    # the complex permanent of S_n, computed independently in double-double, rounds to x
    v = O.perm_dp(O.schur_complex_matrix(n))
    assert abs(v.real - x) < 1e-6 * max(1, abs(x)) and abs(v.imag) < 1e-6 * max(1, abs(x))
    if n % 2 == 0:
        assert x == 0


def test_schur_counts_brute():
    for n in range(1, 8):
        c = [0] * n
        for s in itertools.permutations(range(n)):
            c[sum(i * s[i] for i in range(n)) % n] += 1
        assert O.schur_counts(n) == c


@pytest.mark.parametrize("n", [5, 9, 12, 16])
def test_schur_modp_three_ways(n):
    for p in O.primes_1_mod_n(n, 2):
        g = O.primitive_nth_root(p, n)
        S = O.schur_residue_matrix(n, p, g)
        r = O.perm_modp(S, p)
        assert r == O.schur_modp_from_counts(n, p, g)
        assert r == O.schur_exact(n) % p
        # Galois invariance: any other primitive n-th root gives the same residue
        for k in range(2, n):
            if math.gcd(k, n) == 1:
                assert O.perm_modp(O.schur_residue_matrix(n, p, pow(g, k, p)), p) == r
                break


def test_crt_recovers_schur_with_disjoint_prime_sets():
    for n in (11, 13, 14):
        x = O.schur_exact(n)
        for skip in (0, 3):
            ps = O.primes_1_mod_n(n, 3, skip=skip)
            assert O.crt_modulus_suffices(n, ps)
            res = [O.perm_modp(O.schur_residue_matrix(n, p, O.primitive_nth_root(p, n)), p) for p in ps]
            assert O.crt(res, ps) == x


def test_schur_crt_fixture_consistent():
    """The stored oracle values of perm(S_n) (n = 21..31) agree with the oracle's
    F_p Ryser modulo a prime that the generator did not use (n = 21, 22, 23)
    and respect |perm(S_n)|^2 <= n^n."""
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "schur_crt_oracle.txt")
    rows = [ln.split() for ln in open(here) if ln.strip() and not ln.startswith("#")]
    for r in rows:
        n, value, used = int(r[0]), int(r[1]), [int(x) for x in r[2:]]
        assert value * value <= n ** n
        if n <= 23:
            q = O.primes_1_mod_n(n, 1, below=min(used))[0]     # the next prime down, unused
            S = O.schur_residue_matrix(n, q, O.primitive_nth_root(q, n))
            assert value % q == O.perm_modp(S, q), n


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_nw_range_sum_gives_perm_by_brute_force(n):
    """Nijenhuis-Wilf form: (-1)^(n-1) 2 times the sum over all 2^(n-1) Gray
    indices is perm(A) mod p (brute force over the n! permutations); sums over
    the pieces of a partition of the range add up to the whole."""
    g = rng(6000 + n)
    for p in (3, 7, 2147483629):
        A = random_residues(n, p, g)
        full = O.ryser_nw_modp_gray_range(A, p, 0, 1 << (n - 1))
        v = full * 2 % p
        if (n - 1) % 2:
            v = (p - v) % p
        assert v == O.perm_modp_brute(A, p), (n, p)
        cuts = sorted({0, 1 << (n - 1)} | {int(c) for c in g.integers(0, (1 << (n - 1)) + 1, size=3)})
        parts = sum(O.ryser_nw_modp_gray_range(A, p, a, b) for a, b in zip(cuts, cuts[1:])) % p
        assert parts == full
