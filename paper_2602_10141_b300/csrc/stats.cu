// Sample statistics of a batch of permanents (perm_sample_stats, and
// perm_sample_histogram over caller-supplied edges): the
// distributional measurements of paper §3-§7 taken over the batched output
// without copying it to the host.
//
// Two passes over the values, each a fixed grid of blocks with a fixed-order
// block tree, then one block that combines the block partials in index order.
// Pass 1 sums Re z, Im z, |z|^2, |z|^4, z^2 and takes min / max |z|^2 and the
// three counts; pass 2 sums the central powers of Re z and Im z about the
// pass-1 means (two passes, so variances and kurtoses do not lose digits when
// the mean is large), and the powers of d = log|z| - c, c = log(E|z|^2) / 2,
// which the last kernel turns into central moments of log|z|.  The shift c
// is within a few units of the mean of log|z| for any sample, so the
// conversion loses at most a few digits, and each value needs one logarithm
// (the float64 log dominates the kernels' cost on B300's FP64 pipe).  The grid
// depends on the count only, so a given input gives the same bits every time.
//
// Decisions that produce counts use |z|^2 = rn(rn(re*re) + rn(im*im)) (no
// fused multiply-add) and |z| = sqrt(|z|^2), correctly rounded, so any IEEE
// double implementation of the same formulas takes the same decisions.
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"
#include "permx.h"

namespace permx {
namespace {

constexpr int kT = 256;          // threads per block
constexpr int kMaxBlocks = 1184; // 148 SMs x 8
constexpr int kS1 = 9;           // pass-1 doubles: re, im, abs2, abs4, z2re, z2im, (unused), min, max
constexpr int kC1 = 3;           // pass-1 counts: nonzero, above, real
constexpr int kS2 = 9;           // pass-2 doubles: c2re, c2im, c11, c3re, c4re, d, d2, d3, d4

int grid_for(int64_t count) {
    const int64_t b = (count + 8 * kT - 1) / (8 * kT);
    return (int)(b < 1 ? 1 : (b > kMaxBlocks ? kMaxBlocks : b));
}

__device__ __forceinline__ void load_value(const double* v, int cplx, int64_t i, double& re, double& im) {
    if (cplx) {
        const double2 z = reinterpret_cast<const double2*>(v)[i];
        re = z.x;
        im = z.y;
    } else {
        re = v[i];
        im = 0.0;
    }
}

__device__ __forceinline__ double abs2_rn(double re, double im) {
    return __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
}

// fixed-order tree over the block; op 0 = sum, 1 = min, 2 = max
template <typename T>
__device__ T block_tree(T x, T* sh, int op) {
    const int t = threadIdx.x;
    sh[t] = x;
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
        if (t < s) {
            const T a = sh[t], b = sh[t + s];
            sh[t] = op == 0 ? a + b : (op == 1 ? (b < a ? b : a) : (b > a ? b : a));
        }
        __syncthreads();
    }
    const T r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kT) stats_pass1_kernel(const double* __restrict__ v, int cplx, int64_t count,
                                                         double thr, double tol, double* __restrict__ part,
                                                         long long* __restrict__ cpart) {
    __shared__ double shd[kT];
    __shared__ long long shc[kT];
    double s[kS1] = {0, 0, 0, 0, 0, 0, 0, __longlong_as_double(0x7ff0000000000000ll),
                     __longlong_as_double(0xfff0000000000000ll)};
    long long c[kC1] = {0, 0, 0};
    const int64_t stride = (int64_t)gridDim.x * kT;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < count; i += stride) {
        double re, im;
        load_value(v, cplx, i, re, im);
        const double a2 = abs2_rn(re, im);
        s[0] += re;
        s[1] += im;
        s[2] += a2;
        s[3] += a2 * a2;
        s[4] += re * re - im * im;
        s[5] += 2.0 * re * im;
        if (a2 > 0.0) ++c[0];
        s[7] = a2 < s[7] ? a2 : s[7];
        s[8] = a2 > s[8] ? a2 : s[8];
        if (a2 >= thr) ++c[1];
        // tol = 0 (the common case) reduces to im == 0 for finite values; no square root
        if (tol == 0.0 ? im == 0.0 : fabs(im) <= __dmul_rn(tol, __dsqrt_rn(a2))) ++c[2];
    }
    for (int q = 0; q < kS1; ++q) {
        const double r = block_tree(s[q], shd, q == 7 ? 1 : (q == 8 ? 2 : 0));
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kS1 + q] = r;
    }
    for (int q = 0; q < kC1; ++q) {
        const long long r = block_tree(c[q], shc, 0);
        if (threadIdx.x == 0) cpart[(int64_t)blockIdx.x * kC1 + q] = r;
    }
}

// one block: pass-1 partials -> totals (tot[0..kS1), ctot[0..kC1))
__global__ void __launch_bounds__(kT) stats_reduce1_kernel(const double* __restrict__ part,
                                                           const long long* __restrict__ cpart, int nb,
                                                           double* __restrict__ tot, long long* __restrict__ ctot) {
    __shared__ double shd[kT];
    __shared__ long long shc[kT];
    for (int q = 0; q < kS1; ++q) {
        const int op = q == 7 ? 1 : (q == 8 ? 2 : 0);
        double x = op == 0 ? 0.0 : part[q];
        for (int b = threadIdx.x; b < nb; b += kT) {
            const double y = part[(int64_t)b * kS1 + q];
            x = op == 0 ? x + y : (op == 1 ? (y < x ? y : x) : (y > x ? y : x));
        }
        const double r = block_tree(x, shd, op);
        if (threadIdx.x == 0) tot[q] = r;
    }
    for (int q = 0; q < kC1; ++q) {
        long long x = 0;
        for (int b = threadIdx.x; b < nb; b += kT) x += cpart[(int64_t)b * kC1 + q];
        const long long r = block_tree(x, shc, 0);
        if (threadIdx.x == 0) ctot[q] = r;
    }
}

__global__ void __launch_bounds__(kT) stats_pass2_kernel(const double* __restrict__ v, int cplx, int64_t count,
                                                         const double* __restrict__ tot,
                                                         const long long* __restrict__ ctot,
                                                         double* __restrict__ part) {
    __shared__ double shd[kT];
    const double mre = tot[0] / (double)count, mim = tot[1] / (double)count;
    const double shift = tot[2] > 0.0 ? 0.5 * log(tot[2] / (double)count) : 0.0;
    double s[kS2] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t stride = (int64_t)gridDim.x * kT;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < count; i += stride) {
        double re, im;
        load_value(v, cplx, i, re, im);
        const double dr = re - mre, di = im - mim;
        const double dr2 = dr * dr;
        s[0] += dr2;
        s[1] += di * di;
        s[2] += dr * di;
        s[3] += dr2 * dr;
        s[4] += dr2 * dr2;
        const double a2 = abs2_rn(re, im);
        if (a2 > 0.0) {
            const double d = 0.5 * log(a2) - shift;
            const double d2 = d * d;
            s[5] += d;
            s[6] += d2;
            s[7] += d2 * d;
            s[8] += d2 * d2;
        }
    }
    for (int q = 0; q < kS2; ++q) {
        const double r = block_tree(s[q], shd, 0);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kS2 + q] = r;
    }
}

__global__ void __launch_bounds__(kT) stats_final_kernel(const double* __restrict__ part, int nb, int64_t count,
                                                         const double* __restrict__ tot,
                                                         const long long* __restrict__ ctot,
                                                         perm_stats_t* __restrict__ out) {
    __shared__ double shd[kT];
    double c[kS2];
    for (int q = 0; q < kS2; ++q) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nb; b += kT) x += part[(int64_t)b * kS2 + q];
        c[q] = block_tree(x, shd, 0);
    }
    if (threadIdx.x != 0) return;
    const double N = (double)count;
    const long long nz = ctot[0];
    perm_stats_t r;
    r.count = count;
    r.count_nonzero = nz;
    r.count_above = ctot[1];
    r.count_real = ctot[2];
    r.mean_re = tot[0] / N;
    r.mean_im = tot[1] / N;
    r.var_re = c[0] / N;
    r.var_im = c[1] / N;
    r.cov_re_im = c[2] / N;
    r.skew_re = (c[3] / N) / (r.var_re * sqrt(r.var_re));
    r.exkurt_re = (c[4] / N) / (r.var_re * r.var_re) - 3.0;
    r.mean_abs2 = tot[2] / N;
    r.mean_abs4 = tot[3] / N;
    r.mean_z2_re = tot[4] / N;
    r.mean_z2_im = tot[5] / N;
    r.min_abs2 = tot[7];
    r.max_abs2 = tot[8];
    // central moments of log|z| from the raw moments of d = log|z| - shift
    const double M = (double)nz;   // nz = 0 gives NaN log moments
    const double shift = tot[2] > 0.0 ? 0.5 * log(tot[2] / N) : 0.0;
    const double m1 = c[5] / M, r2 = c[6] / M, r3 = c[7] / M, r4 = c[8] / M;
    const double v = r2 - m1 * m1;
    const double k3 = r3 - 3.0 * m1 * r2 + 2.0 * m1 * m1 * m1;
    const double k4 = r4 - 4.0 * m1 * r3 + 6.0 * m1 * m1 * r2 - 3.0 * m1 * m1 * m1 * m1;
    r.log_mean = shift + m1;
    r.log_var = v;
    r.log_skew = k3 / (v * sqrt(v));
    r.log_exkurt = k4 / (v * v) - 3.0;
    *out = r;
}

// Histogram over caller-supplied edges (sorted, in shared memory): bin b holds
// edges[b] <= x < edges[b+1]; counts[0] is below edges[0], counts[nedges] at or
// above the last edge; NaN is not counted.  Integer counts: any order gives the
// same result.
constexpr int kMaxEdges = 4097;
__global__ void __launch_bounds__(kT) hist_kernel(const double* __restrict__ v, int cplx, int64_t count, int kind,
                                                  const double* __restrict__ edges, int nedges,
                                                  unsigned long long* __restrict__ counts) {
    extern __shared__ unsigned char smem[];
    double* se = reinterpret_cast<double*>(smem);
    unsigned int* sc = reinterpret_cast<unsigned int*>(se + nedges);
    for (int i = threadIdx.x; i < nedges; i += kT) se[i] = edges[i];
    for (int i = threadIdx.x; i <= nedges; i += kT) sc[i] = 0u;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * kT;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < count; i += stride) {
        double re, im;
        load_value(v, cplx, i, re, im);
        const double x = kind == PERMX_HIST_ABS2 ? abs2_rn(re, im) : (kind == PERMX_HIST_RE ? re : im);
        if (x != x) continue;
        int lo = 0, hi = nedges;               // first edge > x, by bisection: bin = that index
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (se[mid] <= x) lo = mid + 1;
            else hi = mid;
        }
        atomicAdd(&sc[lo], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= nedges; i += kT)
        if (sc[i]) atomicAdd(&counts[i], (unsigned long long)sc[i]);
}

}  // namespace
}  // namespace permx

using namespace permx;

extern "C" int perm_sample_histogram(int field, const void* values, int64_t count, int kind, const double* edges,
                                     int32_t nedges, int64_t* counts, void* stream) {
    clear_error();
    if (field != PERMX_FIELD_C128 && field != PERMX_FIELD_F64)
        return fail(PERMX_EINVAL, "histograms take complex128 or float64 values");
    if (!edges || !counts || (!values && count > 0)) return fail(PERMX_EINVAL, "NULL argument");
    if (count < 0) return fail(PERMX_EINVAL, "negative count");
    if (kind != PERMX_HIST_ABS2 && kind != PERMX_HIST_RE && kind != PERMX_HIST_IM)
        return fail(PERMX_EINVAL, "unknown histogram quantity");
    if (nedges < 1 || nedges > kMaxEdges) return fail(PERMX_EINVAL, "need 1..4097 edges");
    for (int i = 0; i < nedges; ++i) {
        if (!(edges[i] == edges[i]) || (i > 0 && !(edges[i - 1] < edges[i])))
            return fail(PERMX_EINVAL, "edges must be strictly increasing and not NaN");
    }
    if (reinterpret_cast<uintptr_t>(values) % (field == PERMX_FIELD_C128 ? 16 : 8) ||
        reinterpret_cast<uintptr_t>(counts) % 8)
        return fail(PERMX_EINVAL, "misaligned values or counts");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PERMX_CUDA(cudaMemsetAsync(counts, 0, sizeof(int64_t) * (size_t)(nedges + 1), s));
    if (count == 0) return PERMX_OK;
    // copy from a pageable host buffer of our own: the runtime stages such a
    // copy before returning, so the caller may reuse `edges` at once even when
    // it lives in pinned memory
    const std::vector<double> host_edges(edges, edges + nedges);
    void* d_edges = nullptr;
    PERMX_CUDA(ws_alloc(&d_edges, sizeof(double) * (size_t)nedges, s));
    cudaError_t e = cudaMemcpyAsync(d_edges, host_edges.data(), sizeof(double) * (size_t)nedges,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const size_t shmem = sizeof(double) * (size_t)nedges + sizeof(unsigned int) * (size_t)(nedges + 1);
        if (shmem > 48 * 1024) e = cudaFuncSetAttribute(hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)shmem);
        if (e == cudaSuccess) {
            hist_kernel<<<grid_for(count), kT, shmem, s>>>(static_cast<const double*>(values),
                                                            field == PERMX_FIELD_C128, count, kind,
                                                            static_cast<const double*>(d_edges), nedges,
                                                            reinterpret_cast<unsigned long long*>(counts));
            e = cudaGetLastError();
        }
    }
    ws_free(d_edges, s);
    if (e != cudaSuccess) return cuda_fail(e, "perm_sample_histogram");
    return PERMX_OK;
}

extern "C" int perm_sample_stats(int field, const void* values, int64_t count, double threshold, double real_tol,
                                 perm_stats_t* out, void* stream) {
    clear_error();
    if (field != PERMX_FIELD_C128 && field != PERMX_FIELD_F64)
        return fail(PERMX_EINVAL, "sample statistics take complex128 or float64 values");
    if (!values || !out) return fail(PERMX_EINVAL, "NULL argument");
    if (count < 1) return fail(PERMX_EINVAL, "count must be at least 1");
    if (!(real_tol >= 0.0)) return fail(PERMX_EINVAL, "real_tol must be >= 0");
    if (reinterpret_cast<uintptr_t>(values) % (field == PERMX_FIELD_C128 ? 16 : 8) ||
        reinterpret_cast<uintptr_t>(out) % 8)
        return fail(PERMX_EINVAL, "misaligned values or output");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = grid_for(count);
    const size_t words = (size_t)nb * (kS1 + kC1 + kS2) + kS1 + kC1;
    void* ws = nullptr;
    PERMX_CUDA(ws_alloc(&ws, 8 * words, s));
    double* part1 = static_cast<double*>(ws);
    long long* cpart1 = reinterpret_cast<long long*>(part1 + (size_t)nb * kS1);
    double* part2 = reinterpret_cast<double*>(cpart1 + (size_t)nb * kC1);
    double* tot = part2 + (size_t)nb * kS2;
    long long* ctot = reinterpret_cast<long long*>(tot + kS1);
    const double* v = static_cast<const double*>(values);
    const int cplx = field == PERMX_FIELD_C128;
    stats_pass1_kernel<<<nb, kT, 0, s>>>(v, cplx, count, threshold, real_tol, part1, cpart1);
    stats_reduce1_kernel<<<1, kT, 0, s>>>(part1, cpart1, nb, tot, ctot);
    stats_pass2_kernel<<<nb, kT, 0, s>>>(v, cplx, count, tot, ctot, part2);
    stats_final_kernel<<<1, kT, 0, s>>>(part2, nb, count, tot, ctot, out);
    const cudaError_t e = cudaGetLastError();
    ws_free(ws, s);
    if (e != cudaSuccess) return cuda_fail(e, "perm_sample_stats launch");
    return PERMX_OK;
}
