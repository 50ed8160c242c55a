// Finalisation of batched permanents (paper §2.2: the chunk partials of one
// matrix summed into its permanent), as block-level device functions that
// both the finalize kernels and the walk kernels' last block use, so a
// matrix gets the same bits whichever of them finishes it.
#pragma once
#include "common.cuh"
#include "x64_arith.cuh"

namespace permx {

constexpr int kFinalThreads = 128;

__device__ __forceinline__ void dd_pair_add(double& s, double& c, double s2, double c2) {
    double t = s + s2;
    double bp = t - s;
    double err = (s - (t - bp)) + (s2 - bp);
    s = t;
    c = (c + c2) + err;
}

__device__ __forceinline__ uint32_t mulmod_u64(uint64_t a, uint64_t b, uint32_t p) {
    return (uint32_t)((a % p) * (b % p) % p);
}

// perm mod p from a matrix's accumulated chunk residues: undo the Montgomery
// factors (and the Nijenhuis-Wilf factor 2) and apply the sign.
__device__ __forceinline__ uint32_t finalize_modp_value(unsigned long long acc, const ModpFinal& x) {
    uint32_t v = mulmod_u64(acc % x.p, x.rfix, x.p);
    if (x.negate && v) v = x.p - v;
    return v;
}

// One matrix's (sum, compensation) partial slots summed in a fixed order by
// kFinalThreads virtual threads, which the block's threads (any multiple of 32)
// take in turn; every thread of the block must call it (it synchronises the
// block).  Virtual thread v folds partials v, v + kFinalThreads, ... in order,
// then a fixed binary tree (level h adds v + h into v).  Virtual threads at
// or past the partial count hold the pair (0, 0), and adding it leaves a pair
// unchanged, so the tree starts at the first level whose upper half holds
// partials; its last five levels run in warp 0 with shuffles.  The result
// depends on neither the block size nor the thread that runs a virtual
// thread.  Partials are read through L2 (another block may have written them
// during this kernel).
__device__ __forceinline__ void finalize_fp_block(const double* __restrict__ partial, const FpFinal& x, int cplx,
                                                  void* __restrict__ out, double (&sh)[4][kFinalThreads]) {
    const int t = threadIdx.x, bd = blockDim.x;
    const int w = cplx ? 4 : 2;
    for (int v = t; v < kFinalThreads; v += bd) {
        double s0 = 0.0, c0 = 0.0, s1 = 0.0, c1 = 0.0;
        for (int64_t q = v; q < x.count; q += kFinalThreads) {
            const double* pq = partial + (x.first + q) * w;
            dd_pair_add(s0, c0, __ldcg(pq), __ldcg(pq + 1));
            if (cplx) dd_pair_add(s1, c1, __ldcg(pq + 2), __ldcg(pq + 3));
        }
        sh[0][v] = s0; sh[1][v] = c0; sh[2][v] = s1; sh[3][v] = c1;
    }
    __syncthreads();
    const int live = x.count < kFinalThreads ? (int)x.count : kFinalThreads;
    int h = kFinalThreads / 2;
    while (h > 0 && h >= live) h >>= 1;       // levels that would add only (0, 0) pairs
    for (; h >= 32; h >>= 1) {
        for (int v = t; v < h; v += bd) {
            double a = sh[0][v], ac = sh[1][v];
            dd_pair_add(a, ac, sh[0][v + h], sh[1][v + h]);
            sh[0][v] = a; sh[1][v] = ac;
            if (cplx) {
                double b = sh[2][v], bc = sh[3][v];
                dd_pair_add(b, bc, sh[2][v + h], sh[3][v + h]);
                sh[2][v] = b; sh[3][v] = bc;
            }
        }
        __syncthreads();
    }
    if (t < 32) {
        double a = sh[0][t], ac = sh[1][t], b = sh[2][t], bc = sh[3][t];
        for (; h > 0; h >>= 1) {
            const double a2 = __shfl_down_sync(0xffffffffu, a, h), ac2 = __shfl_down_sync(0xffffffffu, ac, h);
            const double b2 = __shfl_down_sync(0xffffffffu, b, h), bc2 = __shfl_down_sync(0xffffffffu, bc, h);
            if (t < h) {
                dd_pair_add(a, ac, a2, ac2);
                if (cplx) dd_pair_add(b, bc, b2, bc2);
            }
        }
        if (t == 0) {
            const double sg = (x.negate ? -1.0 : 1.0) * (x.twice ? 2.0 : 1.0);
            const double re = sg * (a + ac);
            if (cplx) {
                const double im = sg * (b + bc);
                reinterpret_cast<double2*>(out)[x.out_index] = make_double2(re, im);
            } else {
                reinterpret_cast<double*>(out)[x.out_index] = re;
            }
        }
    }
    __syncthreads();   // sh is reused by the next matrix
}

// Integer mode: one matrix's XPart slots (one per lane group and component)
// merged in the same fixed order as finalize_fp_block (virtual thread v folds
// partials v, v + kFinalThreads, ..., then a fixed binary tree), with the
// symmetric integer merge of the chunk accumulators, and rounded to double
// once.  The merges align to the larger exponent (bits below the larger
// sum's grid, 2^-80 of its terms, are dropped); no floating-point operation
// precedes the final rounding.  Every thread of the block must call it.
struct XFinSh {
    unsigned long long lo[2][kFinalThreads];
    long long hi[2][kFinalThreads];
    int e[2][kFinalThreads];
    int f[2][kFinalThreads];   // bit 0: a sum is set, bit 1: non-finite entry seen
};
__device__ __forceinline__ void xfin_store(XFinSh& sh, int c, int v, const XAcc& a, int nf) {
    sh.lo[c][v] = (unsigned long long)(uint64_t)a.acc;
    sh.hi[c][v] = (long long)(a.acc >> 64);
    sh.e[c][v] = a.E;
    sh.f[c][v] = (a.set ? 1 : 0) | (nf ? 2 : 0);
}
__device__ __forceinline__ XAcc xfin_load(const XFinSh& sh, int c, int v, int& nf) {
    XAcc a;
    a.acc = (__int128)(((unsigned __int128)(uint64_t)sh.hi[c][v] << 64) | (uint64_t)sh.lo[c][v]);
    a.E = sh.e[c][v];
    a.set = (sh.f[c][v] & 1) != 0;
    nf = (sh.f[c][v] >> 1) & 1;
    return a;
}
__device__ __forceinline__ XAcc xfin_shfl_down(const XAcc& a, int h) {
    XAcc b;
    const uint64_t lo = (uint64_t)a.acc, hi = (uint64_t)(a.acc >> 64);
    const uint64_t blo = (uint64_t)__shfl_down_sync(0xffffffffu, (unsigned long long)lo, h);
    const uint64_t bhi = (uint64_t)__shfl_down_sync(0xffffffffu, (unsigned long long)hi, h);
    b.acc = (__int128)(((unsigned __int128)bhi << 64) | blo);
    b.E = __shfl_down_sync(0xffffffffu, a.E, h);
    b.set = __shfl_down_sync(0xffffffffu, (int)a.set, h) != 0;
    return b;
}
__device__ __forceinline__ void finalize_x64_block(const XPart* __restrict__ partial, const FpFinal& x, int cplx,
                                                   void* __restrict__ out, XFinSh& sh) {
    const int t = threadIdx.x, bd = blockDim.x;
    const int nc = cplx ? 2 : 1;
    for (int v = t; v < kFinalThreads; v += bd) {
        XAcc a[2];
        int nf = 0;
        x64_acc_init(a[0]);
        x64_acc_init(a[1]);
        for (int64_t q = v; q < x.count; q += kFinalThreads) {
            for (int c = 0; c < nc; ++c) {
                const longlong2* pq = reinterpret_cast<const longlong2*>(partial + (x.first + q) * nc + c);
                const longlong2 w0 = __ldcg(pq), w1 = __ldcg(pq + 1);
                XPart p;
                p.lo = (uint64_t)w0.x;
                p.hi = w0.y;
                p.e = (int32_t)(uint32_t)(uint64_t)w1.x;
                p.flag = (int32_t)(uint32_t)((uint64_t)w1.x >> 32);
                nf |= p.flag == 2;
                x64_acc_merge(a[c], x64_acc_of_part(p));
            }
        }
        for (int c = 0; c < 2; ++c) xfin_store(sh, c, v, a[c], nf);
    }
    __syncthreads();
    const int live = x.count < kFinalThreads ? (int)x.count : kFinalThreads;
    int h = kFinalThreads / 2;
    while (h > 0 && h >= live) h >>= 1;       // levels that would merge only empty sums
    for (; h >= 32; h >>= 1) {
        for (int v = t; v < h; v += bd) {
            for (int c = 0; c < nc; ++c) {
                int nf0, nf1;
                XAcc a = xfin_load(sh, c, v, nf0);
                x64_acc_merge(a, xfin_load(sh, c, v + h, nf1));
                xfin_store(sh, c, v, a, nf0 | nf1);
            }
        }
        __syncthreads();
    }
    if (t < 32) {
        int nf0, nf1;
        XAcc a = xfin_load(sh, 0, t, nf0), b = xfin_load(sh, 1, t, nf1);
        int nf = nf0 | nf1;
        for (; h > 0; h >>= 1) {
            const XAcc a2 = xfin_shfl_down(a, h);
            const XAcc b2 = cplx ? xfin_shfl_down(b, h) : b;
            const int nf2 = __shfl_down_sync(0xffffffffu, nf, h);
            if (t < h) {
                x64_acc_merge(a, a2);
                if (cplx) x64_acc_merge(b, b2);
                nf |= nf2;
            }
        }
        if (t == 0) {
            const int ex = x.twice ? 1 : 0;
            double re = x64_acc_to_double(a, ex), im = cplx ? x64_acc_to_double(b, ex) : 0.0;
            if (x.negate) {
                re = -re;
                im = -im;
            }
            if (nf) re = im = __longlong_as_double(0x7ff8000000000000ll);
            if (cplx) reinterpret_cast<double2*>(out)[x.out_index] = make_double2(re, im);
            else reinterpret_cast<double*>(out)[x.out_index] = re;
        }
    }
    __syncthreads();   // sh is reused by the next matrix
}

// True in exactly one block of the launch, the last to get here: every
// thread's earlier global writes are fenced before the block takes its
// ticket, so that block sees all of them.  It resets the counter to 0 for
// the next launch.  Every thread of every block must call it.
__device__ __forceinline__ bool last_block(unsigned* done) {
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        is_last = atomicAdd(done, 1u) == gridDim.x - 1;
        if (is_last) *done = 0;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// Walk-kernel epilogues (batch mode, small groups).
__device__ __forceinline__ void fused_finalize_fp(const FpLaunch& L) {
    __shared__ double sh[4][kFinalThreads];
    if (!last_block(L.done)) return;
    for (int m = 0; m < L.nfin; ++m) finalize_fp_block(L.part_all, L.fin[m], L.cplx, L.out, sh);
}
__device__ __forceinline__ void fused_finalize_x64(const FpLaunch& L) {
    __shared__ XFinSh sh;
    if (!last_block(L.done)) return;
    for (int m = 0; m < L.nfin; ++m)
        finalize_x64_block(reinterpret_cast<const XPart*>(L.part_all), L.fin[m], L.cplx, L.out, sh);
}
__device__ __forceinline__ void fused_finalize_modp(const ModpLaunch& L) {
    if (!last_block(L.done)) return;
    for (int m = threadIdx.x; m < L.nfin; m += blockDim.x)
        L.out[L.fin[m].out_index] = finalize_modp_value(__ldcg(L.acc + m), L.fin[m]);
}

}  // namespace permx
