// Gray-code Ryser over F_p (paper §2.1 field, §2.2 Gray-code blocks).
//
// One thread owns one chunk of L = 2^ell consecutive Gray indices k of one
// matrix.  At the chunk start it forms the row sums r_i = sum_{j in S} a_ij of
// S = k ^ (k >> 1) from scratch; then every step k -> k+1 toggles column
// j = ctz(k+1): r_i += a_ij if that bit of S turns on, r_i -= a_ij if it turns
// off.  The term prod_i r_i enters with sign (-1)^{|S_k|} = (-1)^k, and the
// chunk contributes the signed sum D of its terms.
//
// Arithmetic: row sums are residues in [0, p), p < 2^31; modular add/sub use
// one add and an unsigned min.  Products use signed Montgomery reduction with
// R = 2^32 (the signed variant of Seiler, "Faster AVX2 optimized NTT
// multiplication for Ring-LWE lattice cryptography", 2018): for |a|, |b| < p,
// T = a*b (signed 64-bit), m = T * p^{-1} mod R taken as a signed 32-bit
// value, and t = (T - m p) / R = hi(T) - hi(m p) exactly, since T and m p
// agree in their low 32 bits.  |T - m p| < p 2^31 + 2^31 p, so |t| < p: the
// product stays in (-p, p) with no correction step, and the next product
// takes it as it is.  The product of n row sums by n-1 such steps carries
// R^{-(n-1)}; the finalize step multiplies it back.  Terms are summed in
// int64 without reduction (|D| < L 2^31 <= 2^61) and reduced once per chunk.
#pragma once
#include "common.cuh"
#include "finalize.cuh"
#include "pdl.cuh"

namespace permx {

// Pipe placement.  The products need one mul.wide, one mul.lo and one mul.hi
// each, all on the integer-multiply (fmaheavy) pipe, and that pipe bounds the
// walk.  ptxas is free to issue a two-operand integer add as a multiply-add
// on the same pipe, and does so for a share of the Montgomery subtractions
// and row-sum adds.  The walk therefore adds z, a launch parameter that is
// always 0 and unknown to the compiler, to each of them: a three-operand add
// has only the ALU form (IADD3), which leaves the multiply pipe to the
// multiplies (S_33 walk: 131 -> 100 multiply-pipe instructions per Gray step;
// the benchmark's five-prime step 259.4 -> 251.1 ms).
__device__ __forceinline__ uint32_t mod_add(uint32_t r, uint32_t a, uint32_t p, uint32_t z = 0) {
    uint32_t s = r + a + z;       // < 2p < 2^32
    return min(s, s - p);         // s - p wraps to > p when s < p
}
__device__ __forceinline__ uint32_t mod_sub(uint32_t r, uint32_t a, uint32_t p, uint32_t z = 0) {
    uint32_t d = r - a + z;       // wraps to > 2^31 > p when r < a
    return min(d, d + p);
}
#ifndef PERMX_MODP_SIGNED
#define PERMX_MODP_SIGNED 1   // 0: unsigned Montgomery with a correction to [0, p) per product
#endif

#if PERMX_MODP_SIGNED
typedef int32_t mont_t;       // product-tree values in (-p, p)
// a * b * 2^-32 mod p for |a|, |b| < p, result in (-p, p)
__device__ __forceinline__ int32_t mont_mul(int32_t a, int32_t b, uint32_t p, uint32_t pinv, int32_t z) {
    const long long T = (long long)a * b;
    const int32_t m = (int32_t)((uint32_t)(unsigned long long)T * pinv);
    const int32_t mh = __mulhi(m, (int32_t)p);
    return (int32_t)(T >> 32) - mh + z;
}
#else
typedef uint32_t mont_t;      // product-tree values in [0, p)
// (-p, p) -> [0, p): a negative value wraps above p, so the unsigned min picks r + p
__device__ __forceinline__ uint32_t mont_fix(uint32_t r, uint32_t p) { return min(r, r + p); }
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, uint32_t p, uint32_t pinv, int32_t z) {
    uint64_t T = (uint64_t)a * b + (uint32_t)z;
    uint32_t m = (uint32_t)T * pinv;
    uint32_t mh = __umulhi(m, p);
    uint32_t r = (uint32_t)(T >> 32) - mh;   // true value in (-p, p)
    return mont_fix(r, p);
}
#endif

// prod_i r_i * R^{-(N-1)} by a balanced tree (depth log2 N) for ILP (four
// interleaved chains measured 1 % slower at n = 33); each level multiplies its
// first half by its second half (1 % faster than pairing neighbours).  The
// level loop has a fixed trip count so that, fully unrolled, every index is a
// compile-time constant and v[] stays in registers.
template <int N>
__device__ __forceinline__ mont_t prod_tree(const uint32_t (&r)[N], uint32_t p, uint32_t pinv, int32_t z) {
    static_assert(N <= 64, "tree depth");
    mont_t v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = (mont_t)r[i];
#pragma unroll
    for (int lvl = 0; lvl < 6; ++lvl) {
        const int w = (N + (1 << lvl) - 1) >> lvl;   // live values at this level
        if (w > 1) {
            const int h = (w + 1) / 2;         // pair i with i + h; an odd middle one stays
#pragma unroll
            for (int i = 0; i < N / 2; ++i)
                if (i < w / 2) v[i] = mont_mul(v[i], v[i + h], p, pinv, z);
        }
    }
    return v[0];
}

// Two product trees formed level by level together (the paired steps' r and
// r2): each level's products of both trees are independent, so the compiler
// sees them side by side.  Same tree shape as prod_tree.
template <int N>
__device__ __forceinline__ void prod_tree2(const uint32_t (&r)[N], const uint32_t (&r2)[N], uint32_t p,
                                           uint32_t pinv, int32_t z, mont_t& out1, mont_t& out2) {
    mont_t v[N], w[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        v[i] = (mont_t)r[i];
        w[i] = (mont_t)r2[i];
    }
#pragma unroll
    for (int lvl = 0; lvl < 6; ++lvl) {
        const int n_live = (N + (1 << lvl) - 1) >> lvl;
        if (n_live > 1) {
            const int h = (n_live + 1) / 2;    // pair i with i + h; an odd middle one stays
#pragma unroll
            for (int i = 0; i < N / 2; ++i)
                if (i < n_live / 2) {
                    v[i] = mont_mul(v[i], v[i + h], p, pinv, z);
                    w[i] = mont_mul(w[i], w[i + h], p, pinv, z);
                }
        }
    }
    out1 = v[0];
    out2 = w[0];
}

// dst_i = src_i +- (column j)_i mod p
template <int N, bool SUB>
__device__ __forceinline__ void column_step(uint32_t (&dst)[N], const uint32_t (&src)[N],
                                            const uint32_t* __restrict__ cj, uint32_t p, uint32_t z) {
    constexpr int NP = pad4(N);
    const uint4* c4 = reinterpret_cast<const uint4*>(cj);
#pragma unroll
    for (int q = 0; q < NP / 4; ++q) {
        uint4 v = __ldg(c4 + q);
        uint32_t a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (4 * q + e < N)
                dst[4 * q + e] = SUB ? mod_sub(src[4 * q + e], a[e], p, z) : mod_add(src[4 * q + e], a[e], p, z);
        }
    }
}

template <int N, bool SUB>
__device__ __forceinline__ void apply_column(uint32_t (&r)[N], const uint32_t* __restrict__ cj, uint32_t p) {
    constexpr int NP = pad4(N);
    const uint4* c4 = reinterpret_cast<const uint4*>(cj);
#pragma unroll
    for (int q = 0; q < NP / 4; ++q) {
        uint4 v = __ldg(c4 + q);
        uint32_t a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (4 * q + e < N) r[4 * q + e] = SUB ? mod_sub(r[4 * q + e], a[e], p) : mod_add(r[4 * q + e], a[e], p);
        }
    }
}

#ifndef PERMX_MODP_PAIR_MAX_N
// Paired steps up to n = 46.  From n = 42 ptxas spills some of the second
// row-sum copy at 128 registers, and the pairs still win: S_n Gray windows of
// 2^36 steps gain 2-9 % at n = 41-46.  At n = 47, 48 the spills cost more than
// the pairs gain; one block per SM with no spills was slower at every n > 40.
#define PERMX_MODP_PAIR_MAX_N 46
#endif
#ifndef PERMX_MODP_MINB
#define PERMX_MODP_MINB 2   // resident blocks of 256 threads per SM the register budget targets
#endif

// Step into Gray index k (k >= 1): column j = ctz(k) enters the subset if bit
// j+1 of k is clear, leaves it otherwise.
template <int N>
__device__ __forceinline__ void toggle_column(uint32_t (&r)[N], const uint32_t* __restrict__ col, uint32_t k,
                                              uint32_t p) {
    constexpr int NP = pad4(N);
    const int j = __ffs((int)k) - 1;
    if ((k >> (j + 1)) & 1) apply_column<N, true>(r, col + j * NP, p);
    else apply_column<N, false>(r, col + j * NP, p);
}

template <int N>
__global__ void __launch_bounds__(kRyserThreads, PERMX_MODP_MINB) ryser_modp_kernel(const ModpLaunch L) {
    grid_dep_wait();   // the set-up kernel before it has completed (pdl.cuh)
    constexpr int NP = pad4(N);
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t chunk_mask = (1ull << L.log2_chunks) - 1;
    const uint32_t z0 = L.zero;   // 0, opaque to the compiler (pipe placement, above)
    // lanes holding chunks of the same matrix form aligned groups of G lanes
    const int G = L.log2_chunks >= 5 ? 32 : (1 << L.log2_chunks);
    // warp-aligned loop: every lane of a warp runs the same number of iterations
    for (uint64_t base = L.item_begin + (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         base < L.item_end; base += stride) {
        const uint64_t item = base + lane;
        // decode the item: matrix columns, prime, accumulator and chunk index
        bool valid = item < L.item_end;
        const uint32_t* col = L.colT;
        unsigned long long* acc = L.acc;
        uint32_t p = 1, pinv = 1;
        uint64_t c = 0;
        if (valid) {
            if (L.segs) {
                const SegDesc& sg = L.segs[find_segment(L.segs, L.nsegs, item)];
                c = sg.chunk0 + (item - (uint64_t)sg.item_start);
                valid = c < sg.chunk_end;
                col += sg.col_off;
                acc += sg.out_off;
                p = sg.p;
                pinv = sg.pinv;
            } else {
                const int64_t m = (int64_t)(item >> L.log2_chunks);
                c = item & chunk_mask;
                col += m * L.mat_stride;
                acc += m;
                p = __ldg(L.p + m);
                pinv = __ldg(L.pinv + m);
            }
        }
        uint32_t part = 0;
        const uint64_t k0 = c << L.ell;
        uint64_t ks = k0, ke = k0 + (1ull << L.ell);
        ks = ks > L.k_lo ? ks : L.k_lo;
        ke = ke < L.k_hi ? ke : L.k_hi;
        if (valid && ks < ke) {
            // chunk start: row sums of S = gray(ks) from scratch
            uint32_t r[N];
#pragma unroll
            for (int i = 0; i < N; ++i) r[i] = 0;
            if (L.nw) apply_column<N, false>(r, col + N * NP, p);   // r_i = x_i
            const uint64_t S0 = ks ^ (ks >> 1);
#pragma unroll 1
            for (int j = 0; j < N; ++j)
                if ((S0 >> j) & 1) apply_column<N, false>(r, col + j * NP, p);

            long long D = 0;                   // sum of (-1)^k prod_i r_i over the chunk
            // the walk counts k modulo 2^(ell+1) in 32 bits (ell <= 30): bit ell
            // of k is bit 0 of the chunk index, and every step of the chunk
            // reads bits 0..ell only (toggled column, its sign, the parity)
            const uint32_t cb = (uint32_t)(c & 1) << L.ell;
            uint32_t k = (uint32_t)(ks - k0) + cb;
            const uint32_t ke32 = (uint32_t)(ke - k0) + cb;
            if (k & 1) {                       // a window may start on an odd index
                D -= prod_tree<N>(r, p, pinv, (int32_t)z0);
                ++k;
                if (k < ke32) toggle_column<N>(r, col, k, p);
            }
            // pairs (k even, k+1): the step k -> k+1 toggles column 0; both
            // products are formed from independent arrays, which doubles the
            // instruction-level parallelism of the product trees.  r2 is
            // computed from r and the next r from r2, so no array is copied.
            // A pair's two products are summed one pair later, so no instruction
            // of the pair waits for the trees' last levels and the next pair's
            // column steps and trees issue behind them.  The loop tests once
            // per pair: the step after the last pair is taken too and unused.
            // The pairs' even and odd products are summed apart, each offset
            // by p into [0, 2p) (unsigned: no sign extension); every pair adds
            // one of each, so the offsets cancel in Eu - Ou (< 2^(ell+31)).
            mont_t pe = 0, po = 0;
            unsigned long long Eu = 0, Ou = 0;
            const uint32_t kp = ke32 - ((ke32 - k) & 1);   // pairs cover [k, kp)
            if (N <= PERMX_MODP_PAIR_MAX_N && k < kp) {
                do {
                    uint32_t r2[N];
                    if ((k >> 1) & 1) column_step<N, true>(r2, r, col, p, z0);
                    else column_step<N, false>(r2, r, col, p, z0);
                    mont_t te, to;
                    prod_tree2<N>(r, r2, p, pinv, (int32_t)z0, te, to);
                    Eu += ((uint32_t)pe + p);
                    Ou += ((uint32_t)po + p);
                    pe = te;
                    po = to;
                    k += 2;
                    // the next step, also after the last pair (then unused; the
                    // column index is clamped so the loads stay in the table)
                    const int j = min(__ffs((int)k) - 1, min(N - 1, 30));
                    if ((k >> (j + 1)) & 1) column_step<N, true>(r, r2, col + j * NP, p, z0);
                    else column_step<N, false>(r, r2, col + j * NP, p, z0);
                } while (k < kp);
            }
            Eu += ((uint32_t)pe + p);
            Ou += ((uint32_t)po + p);
            D += (long long)(Eu - Ou);
            for (; k < ke32; ++k) {            // remaining steps one at a time
                const long long t = prod_tree<N>(r, p, pinv, (int32_t)z0);
                D += (k & 1) ? -t : t;
                if (k + 1 < ke32) toggle_column<N>(r, col, k + 1, p);
            }
            const long long d = D % (long long)p;       // |D| < 2^(ell+31) <= 2^61
            part = (uint32_t)(d < 0 ? d + (long long)p : d);
        }
        // sum the group's partials mod p (all lanes of a group share m and p)
        for (int d = 1; d < G; d <<= 1) part = mod_add(part, __shfl_xor_sync(0xffffffffu, part, d), p);
        if ((lane & (G - 1)) == 0 && valid && part) atomicAdd(acc, (unsigned long long)part);
    }
    if (L.fin) fused_finalize_modp(L);
}

template <int N>
cudaError_t launch_modp(const ModpLaunch& L, int grid, int threads, cudaStream_t s) {
    if (L.ell < 0 || L.ell > kModpMaxEll) return cudaErrorInvalidValue;   // 32-bit step counter
    return launch_dependent(ryser_modp_kernel<N>, (unsigned)grid, (unsigned)threads, s, L);
}

template <int N>
int blocks_per_sm_modp() {
    static std::atomic<int> slot{0};
    return occupancy_blocks(slot, ryser_modp_kernel<N>);
}

}  // namespace permx
