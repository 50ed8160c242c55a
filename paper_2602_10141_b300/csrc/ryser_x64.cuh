// Gray-code Ryser for float64 / complex128 matrices on the integer pipes
// ("x64" arithmetic; paper §2.2 walk, Nijenhuis-Wilf form).
//
// B300 executes FP64 at about 1/74 of its FP32 rate, while 32-bit integer
// multiplies and adds issue at 1/2 to 1/1 of it.  This walk therefore keeps
// everything in integers:
//  - row i is scaled by 2^sigma_i (S 2^sigma_i in [2^62, 2^63) for the
//    float64 sum S of |a_ij|; complex: of |Re| + |Im|) and rounded to even
//    int64 entries A_ij (each entry moves by at most 2^-62 sum_j |a_ij|), so
//    every Gray-walk row sum R_i = X_i + sum_{j in S} A_ij of the rounded
//    matrix is exact (no drift) and |R_i| < 2^62 + 2^17 (complex: |Re R_i| +
//    |Im R_i|; S may undercount the exact sum by up to 64 ulps);
//  - a product of row sums is a float with a signed mantissa m (|m| in
//    [2^61, 2^62 + 2^20]; complex: |Re m| + |Im m| <= 2^62 + 2^20) and an int
//    exponent.  A chain factor is m R >> 64, a combining factor m m' >> 62,
//    each one truncated 64x64 -> 128-bit product from three signed
//    32x32 -> 64-bit multiplies, then a leading-zero normalisation (a chain's
//    head row sum enters its first chain factor as it is, exponent 0, and a
//    chain that is a single row sum enters the combining products as R
//    itself), so a term carries a truncation error of at most 16n times
//    sum_i prod_{k != i} |R_k| (complex: 64n; in a chain's first factor the
//    head counts as 2^62), i.e. about 2^-58 relative per factor;
//  - each chunk adds its terms into a 128-bit fixed-point accumulator whose
//    grid follows the chunk's first term (error at most 2^-80 of the sum of
//    the term magnitudes); lane groups merge their chunk sums in integers and
//    leave one 128-bit partial per group (XPart, with the staging scale
//    2^-sum(sigma) in its exponent), which the finalisation merges the same
//    way and rounds to double once.
// The result is therefore not exact; relative precision per factor is about
// 2^-58 (float64: 2^-53), and the tests check these bounds against exact
// rational arithmetic.
#pragma once
#include "common.cuh"
#include "ryser_fp.cuh"
#include "x64_arith.cuh"

namespace permx {

// Reduction of the lanes' chunk accumulators over aligned groups of
// `lanes` lanes (xor butterfly of symmetric merges), in integers, which keeps
// the slow FP64 pipe out of the walk altogether.
__device__ __forceinline__ void x64_group_merge(XAcc& a, int lanes, int first = 1) {
    for (int d = first; d < lanes; d <<= 1) {
        XAcc b;
        const uint64_t lo = (uint64_t)a.acc, hi = (uint64_t)(a.acc >> 64);
        const uint64_t blo = (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)lo, d);
        const uint64_t bhi = (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)hi, d);
        b.acc = (__int128)(((unsigned __int128)bhi << 64) | blo);
        b.E = __shfl_xor_sync(0xffffffffu, a.E, d);
        b.set = __shfl_xor_sync(0xffffffffu, (int)a.set, d) != 0;
        x64_acc_merge(a, b);
    }
}

// ---------------------------------------------------------------------------
// kernels.  Staged layout per matrix (int64 words): columns 0..n-1 of A,
// column n = X (Nijenhuis-Wilf offset), each `ld` entries (complex: re, im
// interleaved per entry), then one word holding -sum_i sigma_i.
// ---------------------------------------------------------------------------
// Resident blocks of 256 threads per SM that the register budget targets:
// two (128 registers per thread) while the row sums and product chains fit
// without spilling, one beyond.
// resident blocks of 256 threads per SM the register budget targets; 3 blocks (80 registers) fit the
// real walk up to n = 20 without spills but measured 6 % slower there
template <int N> constexpr int x64r_minb() { return N <= 24 ? 2 : 1; }
template <int N> constexpr int x64c_minb() { return N <= 16 ? 2 : 1; }   // 3 blocks (80 registers) spill even at n = 8

template <int N>
__global__ void __launch_bounds__(kRyserThreads, x64r_minb<N>()) ryser_x64r_kernel(const FpLaunch L) {
    grid_dep_wait();   // the set-up kernel before it has completed (pdl.cuh)
    constexpr int NP = pad2(N);
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t chunk_mask = (1ull << L.log2_chunks) - 1;
    const int lg = L.log2_chunks >= 5 ? 5 : L.log2_chunks;
    const int G = 1 << lg;
    for (uint64_t base = L.item_begin + (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         base < L.item_end; base += stride) {
        const uint64_t item = base + lane;
        bool valid = item < L.item_end;
        const double* cold = L.colT;
        uint64_t c = 0, slot = 0;
        XAcc acc;
        x64_acc_init(acc);
        int scale = 0;
        bool nonfinite = false;
        if (valid) decode_fp_item(L, item, chunk_mask, lg, valid, cold, c, slot);
        if (valid) {
            const int64_t* col = reinterpret_cast<const int64_t*>(cold);
            const uint64_t ks = c << L.ell;
            // the walk counts k modulo 2^(ell+1) in 32 bits: bit ell of k is
            // bit 0 of the chunk index, and the steps read bits 0..ell only
            const uint32_t kb = (uint32_t)(c & 1) << L.ell, kz = kb + (1u << L.ell);
            int64_t R[N];
#pragma unroll
            for (int i = 0; i < N; ++i) R[i] = col[N * NP + i];             // X_i
            const uint64_t S0 = ks ^ (ks >> 1);
#pragma unroll 1
            for (int j = 0; j < N; ++j) {
                if (!((S0 >> j) & 1)) continue;
                const longlong2* c2 = reinterpret_cast<const longlong2*>(col + j * NP);
#pragma unroll
                for (int q = 0; q < NP / 2; ++q) {
                    const longlong2 v = __ldg(c2 + q);
                    R[2 * q] += v.x;
                    if (2 * q + 1 < N) R[2 * q + 1] += v.y;
                }
            }
            scale = (int)col[(N + 1) * NP];
            nonfinite = col[(N + 1) * NP + 1] != 0;
            for (uint32_t k = kb; k < kz; ++k) {
                if (k > kb) {
                    const int j = __ffs((int)k) - 1;
                    const longlong2* c2 = reinterpret_cast<const longlong2*>(col + j * NP);
                    if ((k >> (j + 1)) & 1) {
#pragma unroll
                        for (int q = 0; q < NP / 2; ++q) {
                            const longlong2 v = __ldg(c2 + q);
                            R[2 * q] -= v.x;
                            if (2 * q + 1 < N) R[2 * q + 1] -= v.y;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < NP / 2; ++q) {
                            const longlong2 v = __ldg(c2 + q);
                            R[2 * q] += v.x;
                            if (2 * q + 1 < N) R[2 * q + 1] += v.y;
                        }
                    }
                }
                // four interleaved product chains, then combined
                XReal t[4];
#pragma unroll
                for (int q = 0; q < 4 && q < N; ++q) t[q] = x64_head(R[q], q + 4 >= N);
#pragma unroll
                for (int i = 4; i < N; ++i) t[i & 3] = x64_mul_row(t[i & 3], R[i]);
                const XReal p = x64_term(t, N);
                x64_acc_add(acc, p.m, p.e, k & 1);
            }
        }
        x64_group_merge(acc, G);
        if ((lane & (G - 1)) == 0 && valid) reinterpret_cast<XPart*>(L.partial)[slot] = x64_part(acc, scale, nonfinite);
    }
    if (L.fin) fused_finalize_x64(L);
}

template <int N>
__global__ void __launch_bounds__(kRyserThreads, x64c_minb<N>()) ryser_x64c_kernel(const FpLaunch L) {
    grid_dep_wait();   // the set-up kernel before it has completed (pdl.cuh)
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t chunk_mask = (1ull << L.log2_chunks) - 1;
    const int lg = L.log2_chunks >= 5 ? 5 : L.log2_chunks;
    const int G = 1 << lg;
    for (uint64_t base = L.item_begin + (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         base < L.item_end; base += stride) {
        const uint64_t item = base + lane;
        bool valid = item < L.item_end;
        const double* cold = L.colT;
        uint64_t c = 0, slot = 0;
        XAcc ar, ai;
        x64_acc_init(ar);
        x64_acc_init(ai);
        int scale = 0;
        bool nonfinite = false;
        if (valid) decode_fp_item(L, item, chunk_mask, lg, valid, cold, c, slot);
        if (valid) {
            const longlong2* col = reinterpret_cast<const longlong2*>(cold);
            const uint64_t ks = c << L.ell;
            // the walk counts k modulo 2^(ell+1) in 32 bits: bit ell of k is
            // bit 0 of the chunk index, and the steps read bits 0..ell only
            const uint32_t kb = (uint32_t)(c & 1) << L.ell, kz = kb + (1u << L.ell);
            int64_t Rr[N], Ri[N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const longlong2 x = __ldg(col + N * N + i);
                Rr[i] = x.x;
                Ri[i] = x.y;
            }
            const uint64_t S0 = ks ^ (ks >> 1);
#pragma unroll 1
            for (int j = 0; j < N; ++j) {
                if (!((S0 >> j) & 1)) continue;
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const longlong2 v = __ldg(col + j * N + i);
                    Rr[i] += v.x;
                    Ri[i] += v.y;
                }
            }
            scale = (int)reinterpret_cast<const int64_t*>(col + (N + 1) * N)[0];
            nonfinite = reinterpret_cast<const int64_t*>(col + (N + 1) * N)[1] != 0;
            for (uint32_t k = kb; k < kz; ++k) {
                if (k > kb) {
                    const int j = __ffs((int)k) - 1;
                    if ((k >> (j + 1)) & 1) {
#pragma unroll
                        for (int i = 0; i < N; ++i) {
                            const longlong2 v = __ldg(col + j * N + i);
                            Rr[i] -= v.x;
                            Ri[i] -= v.y;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < N; ++i) {
                            const longlong2 v = __ldg(col + j * N + i);
                            Rr[i] += v.x;
                            Ri[i] += v.y;
                        }
                    }
                }
                XCplx t[4];
#pragma unroll
                for (int q = 0; q < 4 && q < N; ++q) t[q] = x64c_head(Rr[q], Ri[q], q + 4 >= N);
#pragma unroll
                for (int i = 4; i < N; ++i) t[i & 3] = x64c_mul_row(t[i & 3], Rr[i], Ri[i]);
                const XCplx p = x64c_term(t, N);
                x64_acc_add(ar, p.re, p.e, k & 1);
                x64_acc_add(ai, p.im, p.e, k & 1);
            }
        }
        x64_group_merge(ar, G);
        x64_group_merge(ai, G);
        if ((lane & (G - 1)) == 0 && valid) {
            XPart* out = reinterpret_cast<XPart*>(L.partial) + 2 * slot;
            out[0] = x64_part(ar, scale, nonfinite);
            out[1] = x64_part(ai, scale, nonfinite);
        }
    }
    if (L.fin) fused_finalize_x64(L);
}

// Complex rows wider than 16: two lanes share a chunk.  Lane h of a pair
// owns rows [h*H, h*H + H) (H = ceil(N/2); the odd lane has N - H rows when
// N is odd), updates and multiplies only those, and the pair combines its two
// half products with one shuffle exchange and one more factor, formed in the
// same operand order on both lanes so both hold the identical term.  Halving
// the row registers lets two blocks reside per SM.  A warp covers 16 chunks,
// so lane groups are min(chunks, 16) chunks wide.
template <int N>
__global__ void __launch_bounds__(kRyserThreads, 2) ryser_x64c2_kernel(const FpLaunch L) {
    grid_dep_wait();   // the set-up kernel before it has completed (pdl.cuh)
    constexpr int H = (N + 1) / 2;
    const int lane = threadIdx.x & 31;
    const int h = lane & 1;
    const int rows = h ? N - H : H;
    const int r0 = h * H;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x / 2;
    const uint64_t chunk_mask = (1ull << L.log2_chunks) - 1;
    const int lg = L.log2_chunks >= 4 ? 4 : L.log2_chunks;
    const int G = 1 << lg;
    for (uint64_t base = L.item_begin + ((uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) / 2;
         base < L.item_end; base += stride) {
        const uint64_t item = base + (lane >> 1);
        bool valid = item < L.item_end;
        const double* cold = L.colT;
        uint64_t c = 0, slot = 0;
        XAcc acc;                // even lane of a pair: Re of the terms; odd lane: Im
        x64_acc_init(acc);
        int scale = 0;
        bool nonfinite = false;
        if (valid) decode_fp_item(L, item, chunk_mask, lg, valid, cold, c, slot);
        const unsigned pair_mask = __ballot_sync(0xffffffffu, valid);   // both lanes of a pair agree
        if (valid) {
            const longlong2* col = reinterpret_cast<const longlong2*>(cold);
            const uint64_t ks = c << L.ell;
            // the walk counts k modulo 2^(ell+1) in 32 bits: bit ell of k is
            // bit 0 of the chunk index, and the steps read bits 0..ell only
            const uint32_t kb = (uint32_t)(c & 1) << L.ell, kz = kb + (1u << L.ell);
            int64_t Rr[H], Ri[H];
#pragma unroll
            for (int i = 0; i < H; ++i) {
                Rr[i] = 0;
                Ri[i] = 0;
                if (i < rows) {
                    const longlong2 x = __ldg(col + N * N + r0 + i);
                    Rr[i] = x.x;
                    Ri[i] = x.y;
                }
            }
            const uint64_t S0 = ks ^ (ks >> 1);
#pragma unroll 1
            for (int j = 0; j < N; ++j) {
                if (!((S0 >> j) & 1)) continue;
#pragma unroll
                for (int i = 0; i < H; ++i) {
                    if (i < rows) {
                        const longlong2 v = __ldg(col + j * N + r0 + i);
                        Rr[i] += v.x;
                        Ri[i] += v.y;
                    }
                }
            }
            scale = (int)reinterpret_cast<const int64_t*>(col + (N + 1) * N)[0];
            nonfinite = reinterpret_cast<const int64_t*>(col + (N + 1) * N)[1] != 0;
            for (uint32_t k = kb; k < kz; ++k) {
                if (k > kb) {
                    const int j = __ffs((int)k) - 1;
                    const longlong2* cj = col + j * N + r0;
                    if ((k >> (j + 1)) & 1) {
#pragma unroll
                        for (int i = 0; i < H; ++i) {
                            if (i < rows) {
                                const longlong2 v = __ldg(cj + i);
                                Rr[i] -= v.x;
                                Ri[i] -= v.y;
                            }
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < H; ++i) {
                            if (i < rows) {
                                const longlong2 v = __ldg(cj + i);
                                Rr[i] += v.x;
                                Ri[i] += v.y;
                            }
                        }
                    }
                }
                // the lane's half product (rows >= 4 for n >= 8, so all four chains start)
                XCplx t[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) t[q] = x64c_head(Rr[q], Ri[q], q + 4 >= N - H);
#pragma unroll
                for (int i = 4; i < H; ++i)
                    if (i < rows) t[i & 3] = x64c_mul_row(t[i & 3], Rr[i], Ri[i]);
                XCplx p = x64c_mul(t[0], t[1].re, t[1].im, t[1].e);
                const XCplx p23 = x64c_mul(t[2], t[3].re, t[3].im, t[3].e);
                p = x64c_mul(p, p23.re, p23.im, p23.e);
                // exchange halves; both lanes multiply (lane 0's half) x (lane 1's half)
                XCplx o;
                o.re = (int64_t)__shfl_xor_sync(pair_mask, (long long)p.re, 1);
                o.im = (int64_t)__shfl_xor_sync(pair_mask, (long long)p.im, 1);
                o.e = __shfl_xor_sync(pair_mask, p.e, 1);
                const XCplx a = h ? o : p, b = h ? p : o;
                // each lane forms only the component it accumulates, un-normalised:
                // Re = k1 - k3, Im = k1 + k2 (the Karatsuba products of x64c_mulhi)
                const int64_t k1 = x64_mulhi62(a.re + a.im, b.re);
                const int64_t kx = x64_mulhi62(h ? a.re : a.im, h ? b.im - b.re : b.re + b.im);
                x64_acc_add(acc, h ? k1 + kx : k1 - kx, a.e + b.e + 62, k & 1);
            }
        }
        // merge even lanes with even lanes (Re) and odd with odd (Im), then the
        // group's leader takes the Im sum from its odd neighbour
        x64_group_merge(acc, 2 * G, 2);
        XAcc ai;
        {
            const uint64_t lo = (uint64_t)acc.acc, hi = (uint64_t)(acc.acc >> 64);
            const uint64_t blo = (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)lo, 1);
            const uint64_t bhi = (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)hi, 1);
            ai.acc = (__int128)(((unsigned __int128)bhi << 64) | blo);
            ai.E = __shfl_xor_sync(0xffffffffu, acc.E, 1);
            ai.set = __shfl_xor_sync(0xffffffffu, (int)acc.set, 1) != 0;
        }
        const XAcc ar = acc;
        if ((lane & (2 * G - 1)) == 0 && valid) {
            XPart* out = reinterpret_cast<XPart*>(L.partial) + 2 * slot;
            out[0] = x64_part(ar, scale, nonfinite);
            out[1] = x64_part(ai, scale, nonfinite);
        }
    }
    if (L.fin) fused_finalize_x64(L);
}

// Four lanes per chunk (complex, 8 <= n <= 16), for launches too small to
// give every SM sub-partition a warp of the one-lane kernel (a lone matrix, a
// small serving step).  Lane q of a quad owns rows i = q (mod 4) of its chunk,
// keeps their row sums and forms product chain q exactly as the one-lane
// kernel does (R_q, then times R_{q+4}, R_{q+8}, ...); the quad exchanges its
// four chains and every lane combines them in the one-lane kernel's order
// ((t0 t1)(t2 t3)) and adds the term to its (identical) chunk accumulators.
// A block of four warps holds 32 consecutive chunks, so the lane groups'
// merge tree is the one-lane kernel's: levels of chunk distance 1, 2, 4
// between lanes 4, 8, 16 apart, levels 8 and 16 between warps through shared
// memory.  Every result bit equals the one-lane kernel's.
constexpr int kQuadThreads = 128;
template <int N> constexpr bool x64c_quad_ok() { return N >= 8 && N <= 16 && !x64c_paired(N); }

__device__ __forceinline__ void xacc_store(long long* d, const XAcc& a) {
    d[0] = (long long)(unsigned long long)(uint64_t)a.acc;
    d[1] = (long long)(uint64_t)((unsigned __int128)a.acc >> 64);
    d[2] = a.E;
    d[3] = a.set;
}
__device__ __forceinline__ XAcc xacc_load(const long long* d) {
    XAcc a;
    a.acc = (__int128)(((unsigned __int128)(uint64_t)d[1] << 64) | (uint64_t)d[0]);
    a.E = (int)d[2];
    a.set = d[3] != 0;
    return a;
}
__device__ __forceinline__ XCplx shfl_cplx(unsigned mask, const XCplx& t, int src) {
    XCplx o;
    o.re = (int64_t)__shfl_sync(mask, (long long)t.re, src);
    o.im = (int64_t)__shfl_sync(mask, (long long)t.im, src);
    o.e = __shfl_sync(mask, t.e, src);
    return o;
}

template <int N>
__global__ void __launch_bounds__(kQuadThreads) ryser_x64c4_kernel(const FpLaunch L) {
    grid_dep_wait();   // the set-up kernel before it has completed (pdl.cuh)
    static_assert(N >= 8 && N <= 16, "the four-lane walk covers 8 <= n <= 16");
    constexpr int RQ = (N + 3) / 4;                 // rows of lane 0 (lanes with q >= N % 4 may own one fewer)
    __shared__ long long sh[4][2][4];               // per warp: (re, im) accumulators for the cross-warp levels
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, q = lane & 3;
    const int cl = 8 * w + (lane >> 2);             // chunk within the block's 32
    const unsigned quad = 0xFu << (lane & ~3);
    const uint64_t chunk_mask = (1ull << L.log2_chunks) - 1;
    const int lg = L.log2_chunks >= 5 ? 5 : L.log2_chunks;
    const int G = 1 << lg;
    for (uint64_t base = L.item_begin + (uint64_t)blockIdx.x * 32; base < L.item_end;
         base += (uint64_t)gridDim.x * 32) {
        const uint64_t item = base + cl;
        bool valid = item < L.item_end;
        const double* cold = L.colT;
        uint64_t c = 0, slot = 0;
        XAcc ar, ai;
        x64_acc_init(ar);
        x64_acc_init(ai);
        int scale = 0;
        bool nonfinite = false;
        if (valid) decode_fp_item(L, item, chunk_mask, lg, valid, cold, c, slot);
        if (valid) {
            const longlong2* col = reinterpret_cast<const longlong2*>(cold);
            const uint64_t ks = c << L.ell;
            // the walk counts k modulo 2^(ell+1) in 32 bits: bit ell of k is
            // bit 0 of the chunk index, and the steps read bits 0..ell only
            const uint32_t kb = (uint32_t)(c & 1) << L.ell, kz = kb + (1u << L.ell);
            int64_t Rr[RQ], Ri[RQ];
#pragma unroll
            for (int k = 0; k < RQ; ++k) {
                Rr[k] = 0;
                Ri[k] = 0;
                if (q + 4 * k < N) {
                    const longlong2 x = __ldg(col + N * N + q + 4 * k);
                    Rr[k] = x.x;
                    Ri[k] = x.y;
                }
            }
            // a lone matrix runs one warp per SM sub-partition, so latency is
            // the cost: every column's loads are issued at once (no branch on
            // the subset bits; a column outside S0 adds 0), and each step's
            // column is loaded one step ahead
            const uint64_t S0 = ks ^ (ks >> 1);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const int64_t in = -(int64_t)((S0 >> j) & 1);
#pragma unroll
                for (int k = 0; k < RQ; ++k) {
                    if (q + 4 * k < N) {
                        const longlong2 v = __ldg(col + j * N + q + 4 * k);
                        Rr[k] += v.x & in;
                        Ri[k] += v.y & in;
                    }
                }
            }
            scale = (int)reinterpret_cast<const int64_t*>(col + (N + 1) * N)[0];
            nonfinite = reinterpret_cast<const int64_t*>(col + (N + 1) * N)[1] != 0;
            longlong2 nxt[RQ];                       // column of the step into k + 1
#pragma unroll
            for (int r = 0; r < RQ; ++r) nxt[r] = make_longlong2(0, 0);
            if (kb + 1 < kz) {
                const int j = __ffs((int)(kb + 1)) - 1;
#pragma unroll
                for (int r = 0; r < RQ; ++r)
                    if (q + 4 * r < N) nxt[r] = __ldg(col + j * N + q + 4 * r);
            }
            for (uint32_t k = kb; k < kz; ++k) {
                if (k > kb) {
                    const int j = __ffs((int)k) - 1;
                    const int64_t neg = -(int64_t)((k >> (j + 1)) & 1);   // the column leaves S
#pragma unroll
                    for (int r = 0; r < RQ; ++r) {
                        // +v or -v: (v ^ neg) - neg
                        Rr[r] += (nxt[r].x ^ neg) - neg;
                        Ri[r] += (nxt[r].y ^ neg) - neg;
                    }
                    if (k + 1 < kz) {
                        const int jn = __ffs((int)(k + 1)) - 1;
#pragma unroll
                        for (int r = 0; r < RQ; ++r)
                            if (q + 4 * r < N) nxt[r] = __ldg(col + jn * N + q + 4 * r);
                    }
                }
                // chain q (rows q, q+4, q+8, ...), as the one-lane kernel forms t[q]
                XCplx t = x64c_head(Rr[0], Ri[0], q + 4 >= N);
#pragma unroll
                for (int r = 1; r < RQ; ++r)
                    if (q + 4 * r < N) t = x64c_mul_row(t, Rr[r], Ri[r]);
                const int q0 = lane & ~3;
                const XCplx t0 = shfl_cplx(quad, t, q0), t1 = shfl_cplx(quad, t, q0 + 1);
                const XCplx t2 = shfl_cplx(quad, t, q0 + 2), t3 = shfl_cplx(quad, t, q0 + 3);
                const XCplx tq[4] = {t0, t1, t2, t3};   // the one-lane walk's four chains
                const XCplx pr = x64c_term(tq, N);
                x64_acc_add(ar, pr.re, pr.e, k & 1);
                x64_acc_add(ai, pr.im, pr.e, k & 1);
            }
        }
        // the lane groups' merge tree over chunks: distances 1, 2, 4 inside the warp
        for (int d = 1; d < G && d < 8; d <<= 1) {
            XAcc b;
            const uint64_t lo = (uint64_t)ar.acc, hi = (uint64_t)(ar.acc >> 64);
            b.acc = (__int128)(((unsigned __int128)(uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)hi, 4 * d)
                                << 64) |
                               (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)lo, 4 * d));
            b.E = __shfl_xor_sync(0xffffffffu, ar.E, 4 * d);
            b.set = __shfl_xor_sync(0xffffffffu, (int)ar.set, 4 * d) != 0;
            x64_acc_merge(ar, b);
            const uint64_t lo2 = (uint64_t)ai.acc, hi2 = (uint64_t)(ai.acc >> 64);
            b.acc = (__int128)(((unsigned __int128)(uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)hi2, 4 * d)
                                << 64) |
                               (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)lo2, 4 * d));
            b.E = __shfl_xor_sync(0xffffffffu, ai.E, 4 * d);
            b.set = __shfl_xor_sync(0xffffffffu, (int)ai.set, 4 * d) != 0;
            x64_acc_merge(ai, b);
        }
        // distances 8 and 16 between warps (every lane of a warp holds its warp's subtree)
        for (int d = 8; d < G; d <<= 1) {
            if (lane == 0) {
                xacc_store(sh[w][0], ar);
                xacc_store(sh[w][1], ai);
            }
            __syncthreads();
            const int pw = w ^ (d >> 3);
            const XAcc br = xacc_load(sh[pw][0]), bi = xacc_load(sh[pw][1]);
            __syncthreads();
            x64_acc_merge(ar, br);
            x64_acc_merge(ai, bi);
        }
        if (q == 0 && (cl & (G - 1)) == 0 && valid) {
            XPart* out = reinterpret_cast<XPart*>(L.partial) + 2 * slot;
            out[0] = x64_part(ar, scale, nonfinite);
            out[1] = x64_part(ai, scale, nonfinite);
        }
    }
    if (L.fin) fused_finalize_x64(L);
}

template <int N>
cudaError_t launch_x64r(const FpLaunch& L, int grid, int threads, cudaStream_t s) {
    if (L.ell < 0 || L.ell > 30) return cudaErrorInvalidValue;   // 32-bit step counter
    return launch_dependent(ryser_x64r_kernel<N>, (unsigned)grid, (unsigned)threads, s, L);
}
template <int N>
cudaError_t launch_x64c(const FpLaunch& L, int grid, int threads, cudaStream_t s) {
    if (L.ell < 0 || L.ell > 30) return cudaErrorInvalidValue;   // 32-bit step counter
    if constexpr (x64c_quad_ok<N>()) {
        // fewer one-lane warps than SM sub-partitions: four lanes per chunk (same bits)
        const uint64_t items = L.item_end - L.item_begin;
        if (items < (uint64_t)sm_count() * 128) {
            return launch_dependent(ryser_x64c4_kernel<N>, (unsigned)((items + 31) / 32), (unsigned)kQuadThreads, s, L);
        }
    }
    if constexpr (x64c_paired(N)) return launch_dependent(ryser_x64c2_kernel<N>, (unsigned)grid, (unsigned)threads, s, L);
    else return launch_dependent(ryser_x64c_kernel<N>, (unsigned)grid, (unsigned)threads, s, L);
}
template <int N>
int blocks_per_sm_x64r() {
    static std::atomic<int> slot{0};
    return occupancy_blocks(slot, ryser_x64r_kernel<N>);
}
template <int N>
int blocks_per_sm_x64c() {
    static std::atomic<int> slot{0};
    if constexpr (x64c_paired(N)) return occupancy_blocks(slot, ryser_x64c2_kernel<N>);
    else return occupancy_blocks(slot, ryser_x64c_kernel<N>);
}

}  // namespace permx
