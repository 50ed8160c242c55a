"""Planted mistakes: each plausible slip in the oracle (a dropped term, a
wrong sign, a wrong index, a missing reduction) is planted into a copy of
``oracle.c`` on the CPU, and at least one pin must then fail.  This checks
that the pins are sharp enough to have caught it."""
import itertools
import math
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from workloads import geodesic_cycle, ginibre_c, ginibre_r, random_residues, rng

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.c")

PLANTS = [
    ("ryser drops the (-1)^n factor (real)", "if (n & 1) s = dd_neg(s);", ";"),
    ("ryser sign of |S| flipped (complex)", "if (popcount64((uint64_t)S) & 1) acc = cdd_sub(acc, prod);",
     "if (!(popcount64((uint64_t)S) & 1)) acc = cdd_sub(acc, prod);"),
    ("ryser row sum drops the last column (real)",
     "for (int j = 0; j < n; ++j)\n                    if ((uint64_t)S & (1ull << j)) r = dd_add(r, dd_from(A[i * n + j]));",
     "for (int j = 0; j < n - 1; ++j)\n                    if ((uint64_t)S & (1ull << j)) r = dd_add(r, dd_from(A[i * n + j]));"),
    ("dp reads row 0 for every layer (real)", "const double* arow = A + (size_t)(k - 1) * n;",
     "const double* arow = A;"),
    ("complex product drops a cross term", "dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))", "dd_mul(a.re, b.im)"),
    ("complex product wrong sign", "dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im))",
     "dd_add(dd_mul(a.re, b.re), dd_mul(a.im, b.im))"),
    ("twoprod loses its error term", "dd r = { p, fma(a, b, -p) };", "dd r = { p, 0.0 };"),
    ("modp product not reduced",
     "if (S & (1ull << j)) r = (r + A[i * n + j]) % pp;\n            prod = (prod * r) % pp;\n        }\n        if (popcount64(S) & 1) neg = (neg + prod) % pp; else pos = (pos + prod) % pp;\n    }\n    uint64_t s",
     "if (S & (1ull << j)) r = (r + A[i * n + j]) % pp;\n            prod = (prod * r);\n        }\n        if (popcount64(S) & 1) neg = (neg + prod) % pp; else pos = (pos + prod) % pp;\n    }\n    uint64_t s"),
    ("modp ryser sign not applied for odd n", "if (n & 1) s = (pp - s) % pp;", ";"),
    ("gray map uses k >> 2", "uint64_t S = k ^ (k >> 1);", "uint64_t S = k ^ (k >> 2);"),
    ("schur counts add row + column", "int shift = (row * j) % n;", "int shift = (row + j) % n;"),
    ("dp modp drops the last column", "for (int j = 0; j < n; ++j)\n                if ((uint64_t)T & (1ull << j))\n                    s = (s + (uint64_t)f",
     "for (int j = 0; j < n - 1; ++j)\n                if ((uint64_t)T & (1ull << j))\n                    s = (s + (uint64_t)f"),
]


def _pins():
    """A compact battery of the pins; yields (name, ok)."""
    g = rng(1)
    ok = True
    for n in (1, 2, 3, 5, 7):
        for A in (ginibre_r(n, g), ginibre_c(n, g)):
            py = O.perm_python(A) if n <= 6 else O.perm_brute(A)
            scale = O.perm_brute(np.abs(A))
            yield "brute", abs(O.perm_brute(A) - py) <= 1e-14 * scale
            yield "dp", abs(O.perm_dp(A) - py) <= 1e-14 * scale
            yield "ryser", abs(O.perm_ryser(A) - py) <= 1e-14 * scale * 2 ** n
    # cancellation-heavy input that needs the double-double accuracy
    v = O.perm_ryser(geodesic_cycle(15, 0.5, "circulant"))
    yield "midpoint15", abs(v.real / O.perm_dp(geodesic_cycle(15, 0.5, "circulant")).real - 1) <= 1e-12
    Asym = np.random.default_rng(3).normal(size=(6, 6))
    yield "asym", abs(O.perm_dp(Asym) - O.perm_python(Asym)) <= 1e-13 * O.perm_brute(np.abs(Asym))
    p = 2147483629
    for n in (3, 5, 6):
        A = random_residues(n, p, g)
        ref = sum(math.prod(int(A[i, s[i]]) for i in range(n)) for s in itertools.permutations(range(n))) % p
        yield "modp_brute", O.perm_modp_brute(A, p) == ref
        yield "modp_dp", O.perm_modp_dp(A, p) == ref
        yield "modp_ryser", O.perm_modp(A, p) == ref
        yield "gray", O.ryser_modp_gray_range(A, p, 0, 1 << n) == ((-1) ** n * ref) % p
        k0, k1 = 3, (1 << n) - 5
        part = 0
        for k in range(k0, k1):
            S = k ^ (k >> 1)
            part += (-1) ** bin(S).count("1") * math.prod(
                sum(int(A[i, j]) for j in range(n) if S >> j & 1) for i in range(n))
        yield "gray_part", O.ryser_modp_gray_range(A, p, k0, k1) == part % p
    for n in (4, 5, 6):
        c = [0] * n
        for s in itertools.permutations(range(n)):
            c[sum(i * s[i] for i in range(n)) % n] += 1
        yield "schur_counts", O.schur_counts(n) == c


def test_pins_pass_on_the_real_oracle():
    bad = [name for name, ok in _pins() if not ok]
    assert not bad


@pytest.mark.parametrize("desc,old,new", PLANTS, ids=[p[0] for p in PLANTS])
def test_planted_mistake_is_caught(tmp_path, desc, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"plant site not unique: {desc}"
    mutated = tmp_path / "oracle_planted.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_planted.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-w",
                           "-o", str(so), str(mutated), "-lm"])
    with O.use_library(str(so)):
        failed = [name for name, ok in _pins() if not ok]
    assert failed, f"planted mistake not caught: {desc}"
