// Gray-code Ryser in IEEE float64 / complex128 (paper §2.2 Gray-code blocks;
// §1 Note: compensated summation of the alternating outer sum).
//
// Same walk as the F_p kernel: one thread per chunk of L = 2^ell Gray indices,
// row sums formed from scratch at the chunk start, then one column toggled per
// step (r_i = fma(sgn, a_ij, r_i), sgn = +-1, which rounds exactly like
// r_i +- a_ij).  Products use four interleaved chains.  The signed terms
// (-1)^k prod_i r_i are added plainly in blocks of 16 steps and every block
// is folded into a (sum, compensation) pair with Knuth's TwoSum, so the
// accumulation error stays at the level of one product's rounding.  Each
// chunk writes its pair to its own slot; a fixed-order reduction combines
// the slots of a matrix, which makes the result independent of scheduling.
#pragma once
#include "common.cuh"
#include "finalize.cuh"
#include "pdl.cuh"

namespace permx {

__device__ __forceinline__ void two_sum_acc(double& s, double& comp, double x) {
    double t = s + x;
    double bp = t - s;
    double err = (s - (t - bp)) + (x - bp);
    s = t;
    comp += err;
}

template <int N>
__device__ __forceinline__ double prod_real(const double (&r)[N]) {
    double t[4] = {1.0, 1.0, 1.0, 1.0};
#pragma unroll
    for (int i = 0; i < N; ++i) t[i & 3] = (i < 4) ? r[i] : t[i & 3] * r[i];
    if (N == 1) return t[0];
    if (N == 2) return t[0] * t[1];
    if (N == 3) return (t[0] * t[1]) * t[2];
    return (t[0] * t[1]) * (t[2] * t[3]);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

template <int N>
__device__ __forceinline__ double2 prod_cplx(const double2 (&r)[N]) {
    double2 t[4];
#pragma unroll
    for (int i = 0; i < N; ++i) t[i & 3] = (i < 4) ? r[i] : cmul(t[i & 3], r[i]);
    if (N == 1) return t[0];
    if (N == 2) return cmul(t[0], t[1]);
    if (N == 3) return cmul(cmul(t[0], t[1]), t[2]);
    return cmul(cmul(t[0], t[1]), cmul(t[2], t[3]));
}

// Merge of two (sum, compensation) pairs; the TwoSum error term is exact, so
// the result does not depend on the order of the two operands.
__device__ __forceinline__ void pair_add(double& s, double& c, double s2, double c2) {
    double t = s + s2;
    double bp = t - s;
    double err = (s - (t - bp)) + (s2 - bp);
    s = t;
    c = (c + c2) + err;
}

// Lanes of one group (G consecutive chunks of one matrix) combine their pairs
// by an xor butterfly; every lane ends with the same pair.
__device__ __forceinline__ void group_reduce(double& s, double& c, int G) {
    for (int d = 1; d < G; d <<= 1) {
        double s2 = __shfl_xor_sync(0xffffffffu, s, d);
        double c2 = __shfl_xor_sync(0xffffffffu, c, d);
        pair_add(s, c, s2, c2);
    }
}

// Item -> (columns, chunk index, partial slot) for batch and segment mode.
__device__ __forceinline__ void decode_fp_item(const FpLaunch& L, uint64_t item, uint64_t chunk_mask, int lg,
                                               bool& valid, const double*& col, uint64_t& c, uint64_t& slot) {
    if (L.segs) {
        const SegDesc& sg = L.segs[find_segment(L.segs, L.nsegs, item)];
        c = sg.chunk0 + (item - (uint64_t)sg.item_start);
        valid = c < sg.chunk_end;
        col += sg.col_off;
        slot = (uint64_t)sg.out_off + (c >> lg);
    } else {
        const int64_t m = (int64_t)(item >> L.log2_chunks);
        c = item & chunk_mask;
        col += m * L.mat_stride;
        slot = (item - L.item_begin) >> lg;
    }
}

template <int N>
__global__ void __launch_bounds__(kRyserThreads, 1) ryser_f64_kernel(const FpLaunch L) {
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
        double s = 0.0, comp = 0.0;
        bool valid = item < L.item_end;
        const double* col = L.colT;
        uint64_t c = 0, slot = 0;
        if (valid) decode_fp_item(L, item, chunk_mask, lg, valid, col, c, slot);
        if (valid) {
            const uint64_t ks = c << L.ell, ke = ks + (1ull << L.ell);
            double r[N];
#pragma unroll
            for (int i = 0; i < N; ++i) r[i] = L.nw ? col[N * NP + i] : 0.0;   // x_i or 0
            const uint64_t S0 = ks ^ (ks >> 1);
#pragma unroll 1
            for (int j = 0; j < N; ++j) {
                if (!((S0 >> j) & 1)) continue;
                const double2* c2 = reinterpret_cast<const double2*>(col + j * NP);
#pragma unroll
                for (int q = 0; q < NP / 2; ++q) {
                    double2 v = __ldg(c2 + q);
                    r[2 * q] += v.x;
                    if (2 * q + 1 < N) r[2 * q + 1] += v.y;
                }
            }
            double blk = (ks & 1) ? -prod_real<N>(r) : prod_real<N>(r);
            for (uint64_t k = ks + 1; k < ke; ++k) {
                const int j = __ffsll((long long)k) - 1;
                const double sgn = ((k >> (j + 1)) & 1) ? -1.0 : 1.0;
                const double2* c2 = reinterpret_cast<const double2*>(col + j * NP);
#pragma unroll
                for (int q = 0; q < NP / 2; ++q) {
                    double2 v = __ldg(c2 + q);
                    r[2 * q] = fma(sgn, v.x, r[2 * q]);
                    if (2 * q + 1 < N) r[2 * q + 1] = fma(sgn, v.y, r[2 * q + 1]);
                }
                const double t = prod_real<N>(r);
                blk = (k & 1) ? blk - t : blk + t;
                if ((k & 15) == 15) {
                    two_sum_acc(s, comp, blk);
                    blk = 0.0;
                }
            }
            two_sum_acc(s, comp, blk);
        }
        group_reduce(s, comp, G);
        if ((lane & (G - 1)) == 0 && valid) reinterpret_cast<double2*>(L.partial)[slot] = make_double2(s, comp);
    }
    if (L.fin) fused_finalize_fp(L);
}

template <int N>
__global__ void __launch_bounds__(kRyserThreads, 1) ryser_c128_kernel(const FpLaunch L) {
    grid_dep_wait();   // the set-up kernel before it has completed (pdl.cuh)
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t chunk_mask = (1ull << L.log2_chunks) - 1;
    const int lg = L.log2_chunks >= 5 ? 5 : L.log2_chunks;
    const int G = 1 << lg;
    for (uint64_t base = L.item_begin + (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         base < L.item_end; base += stride) {
        const uint64_t item = base + lane;
        double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;
        bool valid = item < L.item_end;
        const double* cold = L.colT;
        uint64_t c = 0, slot = 0;
        if (valid) decode_fp_item(L, item, chunk_mask, lg, valid, cold, c, slot);
        if (valid) {
            const uint64_t ks = c << L.ell, ke = ks + (1ull << L.ell);
            const double2* col = reinterpret_cast<const double2*>(cold);
            double2 r[N];
#pragma unroll
            for (int i = 0; i < N; ++i) r[i] = L.nw ? __ldg(col + N * N + i) : make_double2(0.0, 0.0);
            const uint64_t S0 = ks ^ (ks >> 1);
#pragma unroll 1
            for (int j = 0; j < N; ++j) {
                if (!((S0 >> j) & 1)) continue;
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    double2 v = __ldg(col + j * N + i);
                    r[i].x += v.x;
                    r[i].y += v.y;
                }
            }
            double2 t0 = prod_cplx<N>(r);
            double br = (ks & 1) ? -t0.x : t0.x, bi = (ks & 1) ? -t0.y : t0.y;
            for (uint64_t k = ks + 1; k < ke; ++k) {
                const int j = __ffsll((long long)k) - 1;
                const double sgn = ((k >> (j + 1)) & 1) ? -1.0 : 1.0;
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    double2 v = __ldg(col + j * N + i);
                    r[i].x = fma(sgn, v.x, r[i].x);
                    r[i].y = fma(sgn, v.y, r[i].y);
                }
                const double2 t = prod_cplx<N>(r);
                if (k & 1) { br -= t.x; bi -= t.y; } else { br += t.x; bi += t.y; }
                if ((k & 15) == 15) {
                    two_sum_acc(sr, cr, br);
                    two_sum_acc(si, ci, bi);
                    br = 0.0;
                    bi = 0.0;
                }
            }
            two_sum_acc(sr, cr, br);
            two_sum_acc(si, ci, bi);
        }
        group_reduce(sr, cr, G);
        group_reduce(si, ci, G);
        if ((lane & (G - 1)) == 0 && valid) {
            double2* out = reinterpret_cast<double2*>(L.partial) + 2 * slot;
            out[0] = make_double2(sr, cr);
            out[1] = make_double2(si, ci);
        }
    }
    if (L.fin) fused_finalize_fp(L);
}

template <int N>
cudaError_t launch_f64(const FpLaunch& L, int grid, int threads, cudaStream_t s) {
    return launch_dependent(ryser_f64_kernel<N>, (unsigned)grid, (unsigned)threads, s, L);
}
template <int N>
cudaError_t launch_c128(const FpLaunch& L, int grid, int threads, cudaStream_t s) {
    return launch_dependent(ryser_c128_kernel<N>, (unsigned)grid, (unsigned)threads, s, L);
}
template <int N>
int blocks_per_sm_f64() {
    static std::atomic<int> slot{0};
    return occupancy_blocks(slot, ryser_f64_kernel<N>);
}
template <int N>
int blocks_per_sm_c128() {
    static std::atomic<int> slot{0};
    return occupancy_blocks(slot, ryser_c128_kernel<N>);
}

}  // namespace permx
