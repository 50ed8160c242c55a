"""The integer-mantissa arithmetic of the float64 / complex128 walks, run on
the CPU through the library's self-test hooks (the same inline functions the
kernels use) and checked against exact Python integers and fractions."""
import ctypes
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2602_10141_b300 as px
    L = px._lib
    L.permx_x64_mulhi62.argtypes = [ctypes.c_int64, ctypes.c_int64]
    L.permx_x64_mulhi62.restype = ctypes.c_int64
    L.permx_x64_mulhi64.argtypes = [ctypes.c_int64, ctypes.c_int64]
    L.permx_x64_mulhi64.restype = ctypes.c_int64
    L.permx_x64c_mulhi.argtypes = [ctypes.c_int64] * 4 + [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                                          ctypes.POINTER(ctypes.c_int64)]
    P = ctypes.POINTER
    L.permx_x64_product.argtypes = [P(ctypes.c_int64), ctypes.c_int32, P(ctypes.c_int64), P(ctypes.c_int32)]
    L.permx_x64c_product.argtypes = [P(ctypes.c_int64), P(ctypes.c_int64), ctypes.c_int32, P(ctypes.c_int64),
                                     P(ctypes.c_int64), P(ctypes.c_int32)]
    L.permx_x64_accumulate.argtypes = [P(ctypes.c_int64), P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int32,
                                       ctypes.c_int32, P(ctypes.c_double), P(ctypes.c_double)]
    return L


def _arr(v, t=np.int64):
    a = np.ascontiguousarray(np.array(v, dtype=t))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64 if t == np.int64 else ctypes.c_int32))


def test_mulhi62_truncation_bound(lib):
    """Combining operands: mantissas up to 2^62 + 2^20 in size."""
    rnd = random.Random(1)
    top = 2 ** 62 + 2 ** 20
    edge = [0, 1, -1, top, -top, 2 ** 62, -2 ** 62, 2 ** 61, -(2 ** 61), 2 ** 62 - 1, -(2 ** 62) + 1, 2 ** 31,
            -(2 ** 31), 12345]
    cases = [(a, b) for a in edge for b in edge]
    cases += [(rnd.randint(-top, top), rnd.randint(-top, top)) for _ in range(20000)]
    cases += [(rnd.randint(-top, top), rnd.randint(-2 ** 40, 2 ** 40)) for _ in range(5000)]
    for a, b in cases:
        got = lib.permx_x64_mulhi62(a, b)
        exact = (a * b) >> 62            # floor
        assert -2 <= got - exact <= 1, (a, b, got, exact)


def test_mulhi64_truncation_bound(lib):
    """The chain factor's product: |a| <= 2^62 + 2^32 (a mantissa, or an
    un-normalised first row sum; the stated bound is 2^62 + 2^20), |b| < 2^63 - 2^32
    (a row sum, or the Karatsuba sum/difference of two row-sum components)."""
    rnd = random.Random(2)
    amax, bmax = 2 ** 62 + 2 ** 32, 2 ** 63 - 2 ** 32 - 1
    edge_a = [0, 1, -1, amax, -amax, 2 ** 62, -(2 ** 62), 2 ** 61, -(2 ** 61), 2 ** 31, -(2 ** 31), 2 ** 31 - 1]
    edge_b = [0, 1, -1, bmax, -bmax, 2 ** 62 + 64, -(2 ** 62) - 64, 2 ** 31, -(2 ** 31), 2 ** 32 - 1, 777]
    cases = [(a, b) for a in edge_a for b in edge_b]
    cases += [(rnd.randint(-amax, amax), rnd.randint(-bmax, bmax)) for _ in range(20000)]
    cases += [(rnd.randint(-amax, amax), rnd.randint(-2 ** 40, 2 ** 40)) for _ in range(5000)]
    for a, b in cases:
        got = lib.permx_x64_mulhi64(a, b)
        exact = (a * b) >> 64
        assert -2 <= got - exact <= 1, (a, b, got, exact)


def _cplx_operand(rnd, top):
    """A complex operand with |re| + |im| <= top, its size drawn from the full range."""
    mag = rnd.choice((top, rnd.randint(0, top), rnd.randint(0, top) >> rnd.randint(0, 60)))
    x = rnd.randint(0, mag)
    return x * rnd.choice((-1, 1)), (mag - x) * rnd.choice((-1, 1))


def test_complex_mulhi_components_bound(lib):
    """(ar + i ai)(br + i bi) >> 64 (chain factor) and >> 62 (combining factor):
    each component within 4 of the exact value's floor (Karatsuba: three
    truncated products, each within [-2, +1] of its floor)."""
    rnd = random.Random(3)
    top = 2 ** 62 + 2 ** 20
    re, im = ctypes.c_int64(), ctypes.c_int64()
    edges = [(top, 0), (-top, 0), (0, top), (0, -top), (top // 2, -(top - top // 2)), (2 ** 31, -(2 ** 31)), (0, 0)]
    cases = [(a, b) for a in edges for b in edges]
    cases += [(_cplx_operand(rnd, top), _cplx_operand(rnd, top)) for _ in range(20000)]
    for (ar, ai), (br, bi) in cases:
        er, ei = ar * br - ai * bi, ar * bi + ai * br
        assert lib.permx_x64c_mulhi(ar, ai, br, bi, 64, ctypes.byref(re), ctypes.byref(im)) == 0
        assert -4 <= re.value - (er >> 64) <= 4 and -4 <= im.value - (ei >> 64) <= 4, (ar, ai, br, bi)
        assert lib.permx_x64c_mulhi(ar, ai, br, bi, 62, ctypes.byref(re), ctypes.byref(im)) == 0
        assert -4 <= re.value - (er >> 62) <= 4 and -4 <= im.value - (ei >> 62) <= 4, (ar, ai, br, bi)
    assert lib.permx_x64c_mulhi(1, 2, 3, 4, 63, ctypes.byref(re), ctypes.byref(im)) != 0


def _error_scale(R):
    """sum_i 2^61 prod_{k != i} max(|R_k|, 2^32): the size one truncation per factor
    can reach.  Normalisation looks at the high 32-bit word only, so a factor below
    2^32 (a row sum cancelling to 2^-29 of its row's scale) counts as 2^32; such a
    term is itself that much below typical terms.  A chain's head row sum enters
    its first chain factor un-normalised (factor i = q + 4 for head q), which
    truncates as if the head were 2^62 in size: that factor's share counts the
    head as max(|R_q|, 2^62)."""
    n = len(R)
    tot = 0
    for i in range(n):
        p = 2 ** 61
        for k, r in enumerate(R):
            if k == i:
                continue
            if 4 <= i < 8 and k == i - 4:
                p *= max(abs(r), 2 ** 62)
            else:
                p *= max(abs(r), 2 ** 32)
        tot += p
    return tot


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 12, 23, 32])
def test_real_product(lib, n):
    rnd = random.Random(n)
    for trial in range(300):
        # staged row sums: |R| < 2^62 + 2^17 (row scale 2^sigma with the float64 row sum
        # times 2^sigma below 2^63, which may undercount the exact sum by 64 ulps)
        top = 2 ** 62 + 2 ** 17
        if trial % 10 == 0:
            R = [rnd.randint(-top, top) >> rnd.randint(0, 40) for _ in range(n)]
        elif trial % 10 == 1:
            R = [rnd.choice((-top, top)) for _ in range(n)]
        else:
            R = [rnd.randint(-top, top) for _ in range(n)]
        if trial == 5:
            R[n // 2] = 0
        a, pa = _arr(R)
        m, e = ctypes.c_int64(), ctypes.c_int32()
        assert lib.permx_x64_product(pa, n, ctypes.byref(m), ctypes.byref(e)) == 0
        exact = 1
        for r in R:
            exact *= r
        got = Fraction(m.value) * Fraction(2) ** e.value
        assert abs(got - exact) <= Fraction(4 * n, 2 ** 59) * _error_scale(R) + 0, (R, m.value, e.value)
        if exact == 0:
            assert m.value == 0
        # mantissas: |m| <= 2^62 + 2^20 (a chain that is a lone staged row sum enters the
        # combining products un-normalised, up to 2^62 + 2^17)
        elif min(abs(r) for r in R) >= 2 ** 40:
            assert 2 ** 61 <= abs(m.value) <= 2 ** 62 + 2 ** 20
        else:                      # tiny row sums may leave the mantissa partly normalised
            assert abs(m.value) <= 2 ** 62 + 2 ** 20


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 11, 26])
def test_complex_product(lib, n):
    rnd = random.Random(100 + n)
    for trial in range(200):
        # staged complex row sums: |Re R| + |Im R| < 2^62 + 2^17
        top = 2 ** 62 + 2 ** 17
        Rr, Ri = [], []
        for _ in range(n):
            mag = top if trial % 5 == 1 else rnd.randint(0, top)
            x = rnd.randint(0, mag)
            Rr.append(x * rnd.choice((-1, 1)))
            Ri.append((mag - x) * rnd.choice((-1, 1)))
        if trial % 7 == 0:
            Rr[0] >>= 30
            Ri[0] >>= 30
        ar, pr = _arr(Rr)
        ai, pi = _arr(Ri)
        re, im, e = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        assert lib.permx_x64c_product(pr, pi, n, ctypes.byref(re), ctypes.byref(im), ctypes.byref(e)) == 0
        exact = complex(1, 0)
        er, ei = 1, 0
        for x, y in zip(Rr, Ri):
            er, ei = er * x - ei * y, er * y + ei * x
        scale = Fraction(2) ** e.value
        mags = [max(abs(x), abs(y)) * 2 for x, y in zip(Rr, Ri)]   # bound on |R_k|
        bound = Fraction(16 * n, 2 ** 59) * _error_scale(mags)
        assert abs(Fraction(re.value) * scale - er) <= bound
        assert abs(Fraction(im.value) * scale - ei) <= bound
        assert abs(re.value) + abs(im.value) <= 2 ** 62 + 2 ** 20


def test_accumulator_exact_sum(lib):
    rnd = random.Random(7)
    for trial in range(60):
        count = rnd.choice([1, 2, 17, 4096])
        base = rnd.randint(-3000, 3000)
        m = [rnd.choice([-1, 1]) * rnd.randint(2 ** 61, 2 ** 62) for _ in range(count)]
        e = [base + rnd.randint(-30, 12) for _ in range(count)]
        if trial % 5 == 0:                     # a far larger term late in the chunk (rescale path)
            e[-1] = base + 200
        neg = [rnd.randint(0, 1) for _ in range(count)]
        am, pm = _arr(m)
        ae, pe = _arr(e, np.int32)
        an, pn = _arr(neg, np.int32)
        scale = -base
        hi, lo = ctypes.c_double(), ctypes.c_double()
        assert lib.permx_x64_accumulate(pm, pe, pn, count, scale, ctypes.byref(hi), ctypes.byref(lo)) == 0
        exact = sum(Fraction((-1) ** s * mm) * Fraction(2) ** (ee + scale) for mm, ee, s in zip(m, e, neg))
        tot = sum(Fraction(abs(mm)) * Fraction(2) ** (ee + scale) for mm, ee in zip(m, e))
        got = Fraction(hi.value) + Fraction(lo.value)
        # terms may be truncated to the accumulator's grid (2^-24 of the first term's
        # lowest bit) or, after a rescale, to the larger term's grid
        assert abs(got - exact) <= tot * Fraction(1, 2 ** 80) + abs(exact) * Fraction(1, 2 ** 100)


def test_accumulator_zero_and_tiny(lib):
    m, pm = _arr([2 ** 61, -(2 ** 61)])
    e, pe = _arr([0, 0], np.int32)
    s, ps = _arr([0, 0], np.int32)
    hi, lo = ctypes.c_double(), ctypes.c_double()
    lib.permx_x64_accumulate(pm, pe, ps, 2, 0, ctypes.byref(hi), ctypes.byref(lo))
    assert hi.value == 0.0 and lo.value == 0.0


@pytest.mark.parametrize("parts", [1, 2, 4, 32])
def test_accumulator_merge_exact_and_symmetric(lib, parts):
    """Lane accumulators merged by the group butterfly: every lane ends with
    the same bits, the operand order of a merge does not matter, and the
    result is the exact sum up to the larger grid's truncation."""
    f = lib.permx_x64_accumulate_merged
    P = ctypes.POINTER
    f.argtypes = [P(ctypes.c_int64), P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int32, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_int32, P(ctypes.c_double), P(ctypes.c_double)]
    rnd = random.Random(40 + parts)
    for trial in range(40):
        count = rnd.choice([parts, 3 * parts + 1, 1024])
        base = rnd.randint(-2000, 2000)
        m = [rnd.choice([-1, 1]) * rnd.randint(2 ** 61, 2 ** 62) for _ in range(count)]
        e = [base + rnd.randint(-60, 60) for _ in range(count)]   # lanes start at very different grids
        neg = [rnd.randint(0, 1) for _ in range(count)]
        am, pm = _arr(m)
        ae, pe = _arr(e, np.int32)
        an, pn = _arr(neg, np.int32)
        outs = []
        for swap in (0, 1):
            hi, lo = ctypes.c_double(), ctypes.c_double()
            assert f(pm, pe, pn, count, parts, swap, -base, ctypes.byref(hi), ctypes.byref(lo)) == 0
            outs.append((hi.value, lo.value))
        assert outs[0] == outs[1]
        exact = sum(Fraction((-1) ** s * mm) * Fraction(2) ** (ee - base) for mm, ee, s in zip(m, e, neg))
        tot = sum(Fraction(abs(mm)) * Fraction(2) ** (ee - base) for mm, ee in zip(m, e))
        got = Fraction(outs[0][0]) + Fraction(outs[0][1])
        assert abs(got - exact) <= tot * Fraction(1, 2 ** 70) + abs(exact) * Fraction(1, 2 ** 100)


def test_scaled_round_is_exact_round_half_even(lib):
    """Staging's float -> integer conversion rounds a 2^k once, to nearest with
    ties to even, for normal and subnormal a and both signs, checked against
    exact rational arithmetic."""
    import math
    from fractions import Fraction
    f = lib.permx_x64_scaled_round
    f.argtypes = [ctypes.c_double, ctypes.c_int32]
    f.restype = ctypes.c_int64
    rnd = random.Random(11)
    vals = [0.0, -0.0, 1.0, -1.0, 0.5, 1.5, 2.5, -2.5, 3.5, 5e-324, -5e-324, 2.2250738585072014e-308,
            1.7976931348623157e308, math.ldexp(1.0, -1074) * 3]
    vals += [rnd.uniform(-1, 1) * 10 ** rnd.uniform(-300, 300) for _ in range(3000)]
    vals += [math.ldexp(rnd.randint(1, 2 ** 53) + 0.5, rnd.randint(-60, 0)) for _ in range(500)]   # exact ties
    for a in vals:
        e = math.frexp(a)[1] if a else 0
        for k in (60 - e, 59 - e, 40 - e, 1 - e, -e, -e - 1, -e - 60, 61 - e):
            x = Fraction(a) * Fraction(2) ** k
            if abs(x) >= 2 ** 62:
                continue
            fl = math.floor(x)
            d = x - fl
            want = fl + 1 if d > Fraction(1, 2) or (d == Fraction(1, 2) and fl % 2) else fl
            assert f(a, k) == want, (a, k)


def test_integer_rounding_to_double_is_correctly_rounded(lib):
    """The finalisation's single rounding: (hi:lo) * 2^e to the nearest double,
    ties to even, against Python's correctly rounded Fraction -> float, over
    normal, subnormal and overflowing results and exact ties."""
    lib.permx_x64_to_double.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32]
    lib.permx_x64_to_double.restype = ctypes.c_double
    rnd = random.Random(11)

    def expect(v, e):
        try:
            return float(Fraction(v) * Fraction(2) ** e)
        except OverflowError:
            return math.inf if v > 0 else -math.inf

    cases = []
    for _ in range(4000):
        bits = rnd.randint(1, 126)
        v = rnd.getrandbits(bits) * rnd.choice((-1, 1))
        e = rnd.choice((rnd.randint(-200, 200), rnd.randint(-1300, -1000), rnd.randint(900, 1100)))
        cases.append((v, e))
    # exact ties at the 53-bit boundary, odd and even significands, and the carry to 2^53
    for sig in (2 ** 52, 2 ** 52 + 1, 2 ** 53 - 1):
        for sh in (1, 2, 11, 70):
            cases.append(((2 * sig + 1) << (sh - 1), -sh))
    cases += [((2 ** 53 - 1) * 2 + 1, 0), (1, -1074), (1, -1075), (3, -1076), (1, -1076), (2 ** 127 - 1, 1000),
              (-(2 ** 127), -1200), (1, 1023), (2 ** 53 - 1, 971), (2 ** 53 - 1, 972)]
    for v, e in cases:
        if v == 0:
            continue
        hi, lo = (v >> 64), v & (2 ** 64 - 1)
        got = lib.permx_x64_to_double(hi, lo, e)
        want = expect(v, e)
        assert got == want and math.copysign(1.0, got) == math.copysign(1.0, want), (v, e, got, want)
