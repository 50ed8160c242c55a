// Integer-mantissa arithmetic for the float64 / complex128 Gray walks
// (host + device; the kernels are in ryser_x64.cuh).  See ryser_x64.cuh for
// the representation.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "common.cuh"

#if !defined(__CUDACC__) && !defined(__host__)
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace permx {

// ---------------------------------------------------------------------------
// arithmetic helpers (host+device so that the library's self-test can check
// them against exact 128-bit arithmetic on the CPU)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int x64_clz(uint64_t v) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

__host__ __device__ __forceinline__ uint32_t x64_hiword(int64_t x) { return (uint32_t)((uint64_t)x >> 32); }

// Signed 32x32 -> 64-bit multiply-add, a b + c: one mad.wide.s32 on the GPU
// (the addition rides on the integer-multiply pipe); the host computes the
// same exact integer.
__host__ __device__ __forceinline__ int64_t x64_madw(int32_t a, int32_t b, int64_t c) {
#ifdef __CUDA_ARCH__
    long long r;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(b), "l"((long long)c));
    return r;
#else
    return (int64_t)a * (int64_t)b + c;
#endif
}

// Signed 32x32 -> 64-bit product (mul.wide.s32): the first term of a chain of
// multiply-adds, so that no zero addend has to be held in registers.
__host__ __device__ __forceinline__ int64_t x64_mulw(int32_t a, int32_t b) {
#ifdef __CUDA_ARCH__
    long long r;
    asm("mul.wide.s32 %0, %1, %2;" : "=l"(r) : "r"(a), "r"(b));
    return r;
#else
    return (int64_t)a * (int64_t)b;
#endif
}

// Balanced 32-bit limbs a = hi 2^32 + lo with lo in [-2^31, 2^31): every
// partial product is then a signed 32x32 -> 64 multiply.  hi is the high word
// plus the low word's top bit.
struct XLimbs {
    int32_t hi, lo;
};
__host__ __device__ __forceinline__ XLimbs x64_limbs(int64_t a) {
    const uint32_t al = (uint32_t)(uint64_t)a;
    return XLimbs{(int32_t)x64_hiword(a) + (int32_t)(al >> 31), (int32_t)al};
}

// (a * b) >> 62 for |a|, |b| <= 2^62 + 2^20 (the result fits; every partial
// product keeps a margin of 2^31), truncated: the result is within [-2, +1]
// of floor(a*b / 2^62).  The low product a0*b0 (< 2^62 in size) is dropped;
// the rest is 4 (a1 b1 + floor(mid / 2^32)) + bits 30..31 of mid, with
// mid = a1 b0 + a0 b1, all in multiply-adds.
__host__ __device__ __forceinline__ int64_t x64_mulhi62(int64_t a, int64_t b) {
    const XLimbs x = x64_limbs(a), y = x64_limbs(b);
    const int64_t mid = x64_madw(x.lo, y.hi, x64_mulw(x.hi, y.lo));
    const int64_t r = x64_madw(x.hi, y.hi, mid >> 32);
    return (int64_t)(((uint64_t)r << 2) | (((uint64_t)mid >> 30) & 3u));
}

// (a * b) >> 64 for |a| <= 2^62 + 2^20, |b| < 2^63 - 2^32, truncated (within
// [-2, +1] of the floor): a1 b1 + floor(mid / 2^32).  The walks use it for the
// chain factors, whose row sums are staged two bits larger for it
// (|R| < 2^62 + 2^17).
__host__ __device__ __forceinline__ int64_t x64_mulhi64(int64_t a, int64_t b) {
    const XLimbs x = x64_limbs(a), y = x64_limbs(b);
    const int64_t mid = x64_madw(x.lo, y.hi, x64_mulw(x.hi, y.lo));
    return x64_madw(x.hi, y.hi, mid >> 32);
}

// Complex product (ar + i ai)(br + i bi) >> SH by components (SH = 64: chain
// factor, b a staged row sum; SH = 62: combining factor, b a mantissa), for
// |ar| + |ai| <= 2^62 + 2^20 and |br| + |bi| <= 2^62 + 2^20: three products
// (Karatsuba), re = k1 - k3, im = k1 + k2, each k within [-2, +1] of its
// floor, so each component is within 4 of the exact (ar br - ai bi) 2^-SH
// (resp. (ar bi + ai br) 2^-SH).  A schoolbook form on twelve chained
// multiply-adds (the subtraction as a product with -ai) issues fewer
// instructions (64.8 against 67.4 per complex term at n = 20) but its longer
// dependency chains made it 2 % slower at n = 23 on B300.
template <int SH>
__host__ __device__ __forceinline__ void x64c_mulhi(int64_t ar, int64_t ai, int64_t br, int64_t bi, int64_t& re,
                                                    int64_t& im) {
    const int64_t k1 = SH == 64 ? x64_mulhi64(ar + ai, br) : x64_mulhi62(ar + ai, br);
    const int64_t k2 = SH == 64 ? x64_mulhi64(ar, bi - br) : x64_mulhi62(ar, bi - br);
    const int64_t k3 = SH == 64 ? x64_mulhi64(ai, br + bi) : x64_mulhi62(ai, br + bi);
    re = k1 - k3;
    im = k1 + k2;
}

// Normalisation works on the high 32-bit word only: |x| is at most 2^62, so
// the top bit of a non-tiny value is in the high word, a 32-bit clz finds it
// and the shift stays below 32 (two funnel-shift instructions).  A value whose
// high word is zero (|x| < 2^32, only when a row sum is tiny) is shifted by
// the largest such amount and stays partly normalised: its term is tiny and
// its absolute error is still bounded by the scale of typical terms.
__host__ __device__ __forceinline__ uint32_t x64_mag_hi(int64_t x) {
    const uint32_t h = x64_hiword(x);
    return h ^ (uint32_t)((int32_t)h >> 31);   // |x| >> 32 (one less for negative x)
}
__host__ __device__ __forceinline__ int x64_clz32(uint32_t v) {
#ifdef __CUDA_ARCH__
    return __clz((int)v);
#else
    return v ? __builtin_clz(v) : 32;
#endif
}
// x << s for 0 <= s <= 31, as two 32-bit word operations
__host__ __device__ __forceinline__ int64_t x64_shl(int64_t x, int s) {
    const uint32_t lo = (uint32_t)(uint64_t)x, hi = x64_hiword(x);
#ifdef __CUDA_ARCH__
    const uint32_t nhi = __funnelshift_l(lo, hi, s);
#else
    const uint32_t nhi = s ? (hi << s) | (lo >> (32 - s)) : hi;
#endif
    return (int64_t)(((uint64_t)nhi << 32) | (uint32_t)(lo << s));
}

// round(a 2^k) to the nearest integer, ties to even, for a finite double a
// with |a 2^k| < 2^62 (how staging turns an entry into the walk's integer):
// integer operations on a's sign, exponent and 53-bit significand, with one
// rounding (llrint(ldexp(a, k)) rounds twice when ldexp lands in the
// subnormal range).
__host__ __device__ __forceinline__ int64_t x64_scaled_round(double a, int k) {
#ifdef __CUDA_ARCH__
    const uint64_t bits = (uint64_t)__double_as_longlong(a);
#else
    uint64_t bits;
    __builtin_memcpy(&bits, &a, sizeof bits);
#endif
    const int be = (int)((bits >> 52) & 0x7ff);
    const uint64_t frac = bits & ((1ull << 52) - 1);
    const uint64_t m = be ? (frac | (1ull << 52)) : frac;      // |a| = m 2^(be - 1075), or m 2^-1074 if subnormal
    const int sh = (be ? be : 1) - 1075 + k;                     // |a| 2^k = m 2^sh
    uint64_t q;
    if (sh >= 0) {
        q = m << sh;                                            // < 2^62 by the caller's bound
    } else if (sh >= -53) {
        const int d = -sh;
        q = m >> d;
        const uint64_t rem = m & ((1ull << d) - 1), half = 1ull << (d - 1);
        q += (rem > half || (rem == half && (q & 1))) ? 1 : 0;
    } else {
        q = 0;                                                  // |a| 2^k < 1/2
    }
    return (bits >> 63) ? -(int64_t)q : (int64_t)q;
}

struct XReal { int64_t m; int e; };
struct XCplx { int64_t re, im; int e; };

// real: mantissa target |m| in [2^61, 2^62] (up to 2^62 + 2^20 where a staged
// row sum or a product of such enters un-normalised: the shift is never negative)
// Position of the most significant non-sign bit of the high word (-1 when the
// word is 0 or -1): bfind.s32 on the GPU, the same value from the folded
// magnitude on the host.
__host__ __device__ __forceinline__ int x64_top_hi(int64_t x) {
#ifdef __CUDA_ARCH__
    int r;
    asm("bfind.s32 %0, %1;" : "=r"(r) : "r"((int32_t)x64_hiword(x)));
    return r;
#else
    return 31 - x64_clz32(x64_mag_hi(x));
#endif
}
// Shift that puts the top non-sign bit (position `top` of the high word) at
// bit T-1 of the 64-bit value: T - 33 - top, at least 0 and at most T - 32
// (top >= -1), so 33 <= T <= 63 keeps it within a funnel shift.
template <int T>
__host__ __device__ __forceinline__ int x64_norm_shift_top(int top) {
    const int s = T - 33 - top;
    return s < 0 ? 0 : s;
}

__host__ __device__ __forceinline__ XReal x64_from_int(int64_t r) {
    const int s = x64_norm_shift_top<62>(x64_top_hi(r));
    return XReal{x64_shl(r, s), -s};
}
// The head of a product chain: a staged row sum (|R| < 2^62 + 2^17) is already a
// valid chain-factor operand, so it enters as it is (exponent 0) when a chain
// factor follows (norm = false): that factor then truncates on the row sum's
// own grid, as if the head were 2^62 in size, which the error bound counts.
// A chain that is only its head goes to the combining products normalised.
__host__ __device__ __forceinline__ XReal x64_head(int64_t R, bool norm) {
    return norm ? x64_from_int(R) : XReal{R, 0};
}
__host__ __device__ __forceinline__ XReal x64_mul(XReal a, int64_t m2, int e2) {
    const int64_t x = x64_mulhi62(a.m, m2);
    const int s = x64_norm_shift_top<62>(x64_top_hi(x));
    return XReal{x64_shl(x, s), a.e + e2 + 62 - s};
}
// a times a staged row sum R (|R| < 2^62 + 2^32): the chain factor
__host__ __device__ __forceinline__ XReal x64_mul_row(XReal a, int64_t R) {
    const int64_t x = x64_mulhi64(a.m, R);
    const int s = x64_norm_shift_top<62>(x64_top_hi(x));
    return XReal{x64_shl(x, s), a.e + 64 - s};
}

// complex: larger component target in [2^60, 2^61]; the invariant the products
// need is |re| + |im| <= 2^62 + 2^20, which every product keeps
__host__ __device__ __forceinline__ XCplx x64c_from_int(int64_t re, int64_t im) {
    const int t1 = x64_top_hi(re), t2 = x64_top_hi(im);
    const int s = x64_norm_shift_top<61>(t1 > t2 ? t1 : t2);
    return XCplx{x64_shl(re, s), x64_shl(im, s), -s};
}
__host__ __device__ __forceinline__ XCplx x64c_head(int64_t re, int64_t im, bool norm) {
    return norm ? x64c_from_int(re, im) : XCplx{re, im, 0};
}
// (a.re + i a.im) * (br + i bi) * 2^-62, |br| + |bi| <= 2^62 + 2^20: the combining factor
__host__ __device__ __forceinline__ XCplx x64c_mul(XCplx a, int64_t br, int64_t bi, int eb) {
    int64_t re, im;
    x64c_mulhi<62>(a.re, a.im, br, bi, re, im);
    const int t1 = x64_top_hi(re), t2 = x64_top_hi(im);
    const int s = x64_norm_shift_top<61>(t1 > t2 ? t1 : t2);
    return XCplx{x64_shl(re, s), x64_shl(im, s), a.e + eb + 62 - s};
}
// a times a staged complex row sum (|br| + |bi| < 2^62 + 2^17): the chain factor
__host__ __device__ __forceinline__ XCplx x64c_mul_row(XCplx a, int64_t br, int64_t bi) {
    int64_t re, im;
    x64c_mulhi<64>(a.re, a.im, br, bi, re, im);
    const int t1 = x64_top_hi(re), t2 = x64_top_hi(im);
    const int s = x64_norm_shift_top<61>(t1 > t2 ? t1 : t2);
    return XCplx{x64_shl(re, s), x64_shl(im, s), a.e + 64 - s};
}

// A term from its four product chains t[0..min(n, 4)) (chain q holds rows
// q, q + 4, ...): (t0 t1)(t2 t3), or the shorter forms for n < 4.  Leaving
// the last factor un-normalised (the accumulator takes any mantissa below
// 2^63) measured within +-2 % either way on B300 and is not done.
__host__ __device__ __forceinline__ XReal x64_term(const XReal (&t)[4], int n) {
    XReal p = t[0];
    if (n >= 2) p = x64_mul(p, t[1].m, t[1].e);
    if (n >= 4) {
        const XReal p23 = x64_mul(t[2], t[3].m, t[3].e);
        p = x64_mul(p, p23.m, p23.e);
    } else if (n == 3) {
        p = x64_mul(p, t[2].m, t[2].e);
    }
    return p;
}
__host__ __device__ __forceinline__ XCplx x64c_term(const XCplx (&t)[4], int n) {
    XCplx p = t[0];
    if (n >= 2) p = x64c_mul(p, t[1].re, t[1].im, t[1].e);
    if (n >= 4) {
        const XCplx p23 = x64c_mul(t[2], t[3].re, t[3].im, t[3].e);
        p = x64c_mul(p, p23.re, p23.im, p23.e);
    } else if (n == 3) {
        p = x64c_mul(p, t[2].re, t[2].im, t[2].e);
    }
    return p;
}

// Fixed-point sum of one chunk's terms: value = acc * 2^E.  The first
// term fixes E 24 bits below its mantissa's lowest bit range; a term more
// than 2^40 above the accumulator scale rescales it first, so at most 2^12
// terms never overflow 128 bits.  Terms far below (shift < -62) round to 0.
struct XAcc {
    __int128 acc;
    int E;
    bool set;
};
__host__ __device__ __forceinline__ void x64_acc_init(XAcc& a) {
    a.acc = 0;
    a.E = 0;
    a.set = false;
}
__host__ __device__ __forceinline__ void x64_acc_add(XAcc& a, int64_t m, int e, bool negate) {
    if (m == 0) return;
    if (!a.set) {
        a.E = e - 24;
        a.set = true;
    }
    int sh = e - a.E;
    if (sh > 40) {                     // rare: a much larger term, rescale the accumulator
        const int d = sh - 40;
        a.acc = d < 127 ? (a.acc >> d) : (a.acc < 0 ? -1 : 0);
        a.E += d;
        sh = 40;
    }
    if (sh <= -63) return;
    // v = m 2^sh (sh in [0, 40]) or floor(m 2^sh) (sh in (-63, 0)) as two 64-bit
    // words: a 64-bit shift and a sign or funnel word instead of a general
    // 128-bit variable shift (same value)
    const int64_t ms = sh >= 0 ? m : (m >> (-sh));
    const uint64_t vl = sh > 0 ? (uint64_t)m << sh : (uint64_t)ms;
    const int64_t vh = sh > 0 ? (m >> (64 - sh)) : (ms >> 63);
    const __int128 v = (__int128)(((unsigned __int128)(uint64_t)vh << 64) | vl);
    a.acc = negate ? a.acc - v : a.acc + v;
}
// a <- a + b, both aligned to the larger exponent (the smaller-exponent one
// is shifted right).  The operation is symmetric in a and b, so a fixed
// butterfly of merges gives the same bits on every lane and in every batch.
// A term is below 2^103 on its accumulator's grid (|mantissa| <= 2^62 + 2^20,
// shift <= 40), a chunk of at most 2^16 terms below 2^119, and 32 merges keep
// the sum below 2^124.
__host__ __device__ __forceinline__ __int128 x64_sar128(__int128 v, int d) {
    return d <= 0 ? v : (d < 127 ? (v >> d) : (v < 0 ? (__int128)-1 : (__int128)0));
}
__host__ __device__ __forceinline__ void x64_acc_merge(XAcc& a, const XAcc& b) {
    if (!b.set) return;
    if (!a.set) {
        a = b;
        return;
    }
    const int E = a.E > b.E ? a.E : b.E;
    a.acc = x64_sar128(a.acc, E - a.E) + x64_sar128(b.acc, E - b.E);
    a.E = E;
}

// The double nearest to acc * 2^(E + extra), ties to even, in integer
// operations only (B300's FP64 latency makes a handful of FP64 operations cost
// more than the whole conversion): the one rounding of an exact sum.
// Subnormal results are rounded once at their own precision; too large ones
// give +-inf.
__host__ __device__ __forceinline__ double x64_acc_to_double(const XAcc& a, int extra) {
    if (!a.set || a.acc == 0) return 0.0;
    const bool neg = a.acc < 0;
    const unsigned __int128 m = neg ? (unsigned __int128)0 - (unsigned __int128)a.acc : (unsigned __int128)a.acc;
    const uint64_t mh = (uint64_t)(m >> 64), ml = (uint64_t)m;
    const int b = mh ? 127 - x64_clz(mh) : 63 - x64_clz(ml);   // top bit of m
    const int F = a.E + extra;                                 // the value is m * 2^F
    int lsb = F + b - 52;                                      // lowest bit of a 53-bit significand
    if (lsb < -1074) lsb = -1074;
    const int sh = lsb - F;
    uint64_t q;
    if (sh <= 0) {
        q = (uint64_t)(m << (-sh));                            // exact, below 2^53
    } else if (sh > 128) {
        q = 0;                                                 // below half the smallest subnormal
    } else if (sh == 128) {
        q = m > ((unsigned __int128)1 << 127) ? 1 : 0;
    } else {
        q = (uint64_t)(m >> sh);
        const unsigned __int128 rem = m - ((unsigned __int128)q << sh), half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (q & 1))) ++q;
    }
    if (q >> 53) {                                             // rounded up to 2^53
        q >>= 1;
        ++lsb;
    }
    uint64_t bits;
    if (q >= (1ull << 52) && lsb + 1075 >= 2047) bits = 0x7ff0000000000000ull;   // overflow
    else bits = ((uint64_t)(lsb + 1074) << 52) + q;            // normal or subnormal (lsb = -1074)
    if (neg) bits |= 0x8000000000000000ull;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double d;
    memcpy(&d, &bits, sizeof d);
    return d;
#endif
}

// A lane group's sum as the partial it leaves for the finalisation
__host__ __device__ __forceinline__ XPart x64_part(const XAcc& a, int scale, bool nonfinite) {
    XPart p;
    p.lo = (uint64_t)a.acc;
    p.hi = (int64_t)(a.acc >> 64);
    p.e = a.E + scale;
    p.flag = nonfinite ? 2 : (a.set ? 1 : 0);
    p.pad = 0;
    return p;
}
__host__ __device__ __forceinline__ XAcc x64_acc_of_part(const XPart& p) {
    XAcc a;
    a.acc = (__int128)(((unsigned __int128)(uint64_t)p.hi << 64) | p.lo);
    a.E = p.e;
    a.set = p.flag == 1;
    return a;
}

// acc * 2^(E + scale) as a double-double (hi + lo): the host self-test's view
// of an accumulator (the kernels use x64_acc_to_double at the finalisation)
__host__ __device__ __forceinline__ void x64_acc_to_dd(const XAcc& a, int scale, double& hi, double& lo) {
    if (!a.set || a.acc == 0) {
        hi = 0.0;
        lo = 0.0;
        return;
    }
    const __int128 v = a.acc;
    const int64_t top = (int64_t)(v >> 64);
    const uint64_t bot = (uint64_t)v;
    // hi: v rounded (the two conversions round separately; the remainder fixes it)
    double h = (double)top * 18446744073709551616.0 + (double)bot;
    // exact remainder v - h in 128-bit integers (|h| < 2^127, h has 53 significant bits)
    int he = 0;
    const double hm = frexp(h, &he);                 // h = hm * 2^he, 0.5 <= |hm| < 1
    const int64_t hmi = (int64_t)ldexp(hm, 53);      // exact integer mantissa
    const int shift = he - 53;
    const __int128 hv = shift >= 0 ? ((__int128)hmi << shift) : ((__int128)hmi >> (-shift));
    const __int128 r = v - hv;                       // a few ulps of h
    const double l = (double)(int64_t)(r >> 32) * 4294967296.0 + (double)(uint32_t)(uint64_t)r;
    hi = ldexp(h, a.E + scale);
    lo = ldexp(l, a.E + scale);
}

}  // namespace permx
