"""The integer-mantissa products as the GPU computes them (inline-PTX
multiply-adds) against the host forms of the same functions (bit for bit) and
against exact integers (the truncation bound), over the operand ranges the
float walks use."""
import ctypes
import math
import random

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2602_10141_b300 as px
    L = px._lib
    i64 = ctypes.c_int64
    L.permx_x64_mulhi62.argtypes = [i64, i64]
    L.permx_x64_mulhi62.restype = i64
    L.permx_x64_mulhi64.argtypes = [i64, i64]
    L.permx_x64_mulhi64.restype = i64
    P = ctypes.POINTER(i64)
    L.permx_x64_mulhi_device.argtypes = [P, P, i64, P, P]
    L.permx_x64c_mulhi.argtypes = [i64] * 4 + [ctypes.c_int32, P, P]
    L.permx_x64c_mulhi_device.argtypes = [P, i64, P]
    return L


def _device(lib, a, b):
    a = np.ascontiguousarray(a, dtype=np.int64)
    b = np.ascontiguousarray(b, dtype=np.int64)
    h62 = np.zeros_like(a)
    h64 = np.zeros_like(a)
    P = ctypes.POINTER(ctypes.c_int64)
    rc = lib.permx_x64_mulhi_device(a.ctypes.data_as(P), b.ctypes.data_as(P), len(a), h62.ctypes.data_as(P),
                                    h64.ctypes.data_as(P))
    assert rc == 0
    return h62, h64


def _operands(rnd, count, amax, bmax):
    edge_a = [0, 1, -1, amax, -amax, 2 ** 62, -(2 ** 62), 2 ** 61, -(2 ** 61), 2 ** 31, -(2 ** 31), 2 ** 31 - 1,
              2 ** 32 - 1, -(2 ** 32) + 1]
    edge_b = [0, 1, -1, bmax, -bmax, 2 ** 62, -(2 ** 62), 2 ** 31, -(2 ** 31), 2 ** 32 - 1, 2 ** 32, 777]
    pairs = [(x, y) for x in edge_a for y in edge_b]
    pairs += [(rnd.randint(-amax, amax), rnd.randint(-bmax, bmax)) for _ in range(count)]
    pairs += [(rnd.randint(-amax, amax) >> rnd.randint(0, 60), rnd.randint(-bmax, bmax) >> rnd.randint(0, 60))
              for _ in range(count // 4)]
    return [p[0] for p in pairs], [p[1] for p in pairs]


def test_combining_and_chain_products_match_host_and_bound(lib):
    rnd = random.Random(5)
    lim = 2 ** 62 + 2 ** 20                     # combining operands: both mantissas
    a, b = _operands(rnd, 40000, lim, lim)
    h62, h64 = _device(lib, a, b)
    for i, (x, y) in enumerate(zip(a, b)):
        assert h62[i] == lib.permx_x64_mulhi62(x, y), (x, y)
        assert h64[i] == lib.permx_x64_mulhi64(x, y), (x, y)
        assert -2 <= int(h62[i]) - ((x * y) >> 62) <= 1, (x, y)
        assert -2 <= int(h64[i]) - ((x * y) >> 64) <= 1, (x, y)


def test_chain_product_full_row_sum_range(lib):
    """Chain factors: the second operand is a staged row sum or a Karatsuba
    sum / difference of two row-sum components (|b| < 2^63 - 2^32)."""
    rnd = random.Random(6)
    a, b = _operands(rnd, 40000, 2 ** 62 + 2 ** 20, 2 ** 63 - 2 ** 32 - 1)
    _, h64 = _device(lib, a, b)
    for i, (x, y) in enumerate(zip(a, b)):
        assert h64[i] == lib.permx_x64_mulhi64(x, y), (x, y)
        assert -2 <= int(h64[i]) - ((x * y) >> 64) <= 1, (x, y)


def test_argument_errors(lib):
    import paper_2602_10141_b300 as px
    P = ctypes.POINTER(ctypes.c_int64)
    buf = np.zeros(4, dtype=np.int64)
    p = buf.ctypes.data_as(P)
    assert lib.permx_x64_mulhi_device(p, p, 0, p, p) == px.PERMX_EINVAL
    assert lib.permx_x64_mulhi_device(p, p, (1 << 20) + 1, p, p) == px.PERMX_EINVAL
    assert lib.permx_x64_mulhi_device(None, p, 4, p, p) == px.PERMX_EINVAL


def test_complex_products_match_host_and_bound(lib):
    """Chain (>> 64) and combining (>> 62) complex factors on the GPU equal the
    host's bit for bit and stay within their truncation bounds."""
    rnd = random.Random(7)
    top = 2 ** 62 + 2 ** 20

    def operand():
        mag = rnd.choice((top, rnd.randint(0, top), rnd.randint(0, top) >> rnd.randint(0, 60)))
        x = rnd.randint(0, mag)
        return x * rnd.choice((-1, 1)), (mag - x) * rnd.choice((-1, 1))

    quads = [operand() + operand() for _ in range(30000)]
    quads += [(top, 0, -top, 0), (0, top, 0, top), (-top, 0, 0, -top), (2 ** 31, -(2 ** 31), -(2 ** 31), 2 ** 31)]
    inp = np.ascontiguousarray(np.array(quads, dtype=np.int64).reshape(-1))
    out = np.zeros_like(inp)
    P = ctypes.POINTER(ctypes.c_int64)
    assert lib.permx_x64c_mulhi_device(inp.ctypes.data_as(P), len(quads), out.ctypes.data_as(P)) == 0
    out = out.reshape(-1, 4)
    re, im = ctypes.c_int64(), ctypes.c_int64()
    for k, (ar, ai, br, bi) in enumerate(quads):
        er, ei = ar * br - ai * bi, ar * bi + ai * br
        assert lib.permx_x64c_mulhi(ar, ai, br, bi, 64, ctypes.byref(re), ctypes.byref(im)) == 0
        assert (out[k, 0], out[k, 1]) == (re.value, im.value)
        assert -4 <= re.value - (er >> 64) <= 4 and -4 <= im.value - (ei >> 64) <= 4
        assert lib.permx_x64c_mulhi(ar, ai, br, bi, 62, ctypes.byref(re), ctypes.byref(im)) == 0
        assert (out[k, 2], out[k, 3]) == (re.value, im.value)
        assert -4 <= re.value - (er >> 62) <= 4 and -4 <= im.value - (ei >> 62) <= 4


def _perm_batch(mats):
    """Integer-mode permanents of a list of equal-size matrices (one call)."""
    import torch
    import paper_2602_10141_b300 as px
    n = mats[0].shape[0]
    flat = np.ascontiguousarray(np.stack(mats)).reshape(-1)
    cplx = np.iscomplexobj(flat)
    A = torch.from_numpy(flat.view(np.float64) if cplx else flat).cuda()
    if cplx:
        A = A.view(torch.complex128)
    out = torch.empty(len(mats), dtype=torch.complex128 if cplx else torch.float64, device="cuda")
    (px.perm_c128 if cplx else px.perm_f64)(A, [n] * len(mats), [i * n * n for i in range(len(mats))], out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("cplx", [True, False])
def test_power_of_two_scaling_is_exact_through_the_final_rounding(cplx):
    """Scaling every entry by 2^k moves each row scale by -k and leaves the
    staged integers, the walk and the exact sums unchanged, so the single final
    rounding gives exactly perm(A) 2^(n k) while that stays a normal double;
    in the subnormal range the result is within one subnormal step of it, and
    past the top of the range it is +-inf."""
    import paper_2602_10141_b300 as px
    old = px.permx_set_fp_arith(1)
    try:
        g = np.random.default_rng(21)
        n = 8
        if cplx:
            A = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(2)
        else:
            A = g.standard_normal((n, n))
        ks = [0, -100, -60, 40, 100, -132, -134, 130]
        got = _perm_batch([A * 2.0 ** k for k in ks])
        base = got[0]
        assert abs(base) > 2.0 ** -10
        parts = (lambda z: (z.real, z.imag)) if cplx else (lambda z: (z,))
        for k, v in zip(ks, got):
            for b, x in zip(parts(base), parts(v)):
                try:
                    want = math.ldexp(float(b), n * k)
                except OverflowError:
                    want = math.copysign(math.inf, b)
                if math.isinf(want):
                    assert x == want, (k, x)
                elif abs(want) >= 2.0 ** -1022:
                    assert x == want, (k, x, want)
                else:
                    assert abs(x - want) <= 2.0 ** -1074, (k, x, want)
    finally:
        px.permx_set_fp_arith(old)
