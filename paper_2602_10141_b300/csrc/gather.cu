// Permanents of submatrices (perm_c128_gather / perm_f64_gather): the
// boson-sampling amplitudes perm(U_T) of paper §8 ("Connections to boson
// sampling"), where U_T takes rows r_1..r_n and columns c_1..c_n of an m x m
// interferometer matrix U (indices may repeat: several photons in one mode).
//
// The index lists are checked on the host, uploaded once, and one gather
// kernel writes every n x n submatrix contiguously into a workspace from the
// library pool; the batched Gray-code path then runs on that workspace
// exactly as perm_c128 / perm_f64 would on caller-supplied matrices, so each
// result has the same bits as perm_c128 on the explicitly extracted matrix.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "batch.h"
#include "common.cuh"
#include "permx.h"

namespace permx {
namespace {

template <typename T>
__global__ void gather_kernel(const T* __restrict__ U, int64_t ldu, const int32_t* __restrict__ rows,
                              const int32_t* __restrict__ cols, int32_t n, int64_t total, T* __restrict__ dst) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / nn;
        const int64_t rc = e - b * nn;
        const int32_t r = (int32_t)(rc / n), c = (int32_t)(rc - (int64_t)r * n);
        dst[e] = U[(int64_t)__ldg(rows + b * n + r) * ldu + __ldg(cols + b * n + c)];
    }
}

template <typename T>
int gather_run(const T* U, int32_t m, int64_t ldu, const int32_t* rows, const int32_t* cols, int32_t n,
               int64_t batch, T* out, bool cplx, cudaStream_t s) {
    if (!U || !rows || !cols || !out) return fail(PERMX_EINVAL, "NULL argument");
    if (m < 1 || ldu < m) return fail(PERMX_EINVAL, "need m >= 1 and ldu >= m");
    if (n < 1 || n > PERMX_MAX_N_FP) return fail(PERMX_EINVAL, "n out of range [1, 32]");
    if (batch < 0) return fail(PERMX_EINVAL, "negative batch");
    if (batch == 0) return PERMX_OK;
    if (cplx && (reinterpret_cast<uintptr_t>(U) % 16 || reinterpret_cast<uintptr_t>(out) % 16))
        return fail(PERMX_EINVAL, "complex128 arrays must be 16-byte aligned");
    const int64_t idx = batch * n;
    for (int64_t k = 0; k < idx; ++k)
        if (rows[k] < 0 || rows[k] >= m || cols[k] < 0 || cols[k] >= m)
            return fail(PERMX_EINVAL, "index " + std::to_string(k) + " outside [0, m)");
    const int64_t total = idx * n;
    const size_t idx_bytes = ((sizeof(int32_t) * (size_t)idx + 255) / 256) * 256;
    void* ws = nullptr;
    PERMX_CUDA(ws_alloc(&ws, 2 * idx_bytes + sizeof(T) * (size_t)total, s));
    int32_t* d_rows = static_cast<int32_t*>(ws);
    int32_t* d_cols = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(ws) + idx_bytes);
    T* d_sub = reinterpret_cast<T*>(static_cast<unsigned char*>(ws) + 2 * idx_bytes);
    // the indices go through a private pageable copy: a copy from pageable memory
    // has left the source by the time cudaMemcpyAsync returns (it waits for the
    // stream's earlier work first), so the caller may reuse rows and cols, pinned
    // or not, as soon as this call returns
    const std::vector<int32_t> hrows(rows, rows + idx), hcols(cols, cols + idx);
    cudaError_t e = cudaMemcpyAsync(d_rows, hrows.data(), sizeof(int32_t) * (size_t)idx, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_cols, hcols.data(), sizeof(int32_t) * (size_t)idx, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const int64_t want = (total + 255) / 256, cap = (int64_t)sm_count() * 16;
        const int blocks = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
        gather_kernel<T><<<blocks, 256, 0, s>>>(U, ldu, d_rows, d_cols, n, total, d_sub);
        e = cudaGetLastError();
    }
    int rc = PERMX_OK;
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "gather");
    } else {
        std::vector<int32_t> nv((size_t)batch, n);
        std::vector<int64_t> off((size_t)batch);
        for (int64_t b = 0; b < batch; ++b) off[(size_t)b] = b * (int64_t)n * n;
        rc = run_fp_batch(reinterpret_cast<const double*>(d_sub), nv.data(), off.data(), batch, out, cplx, s);
    }
    ws_free(ws, s);
    return rc;
}

}  // namespace
}  // namespace permx

using namespace permx;

extern "C" {

int perm_c128_gather(const perm_c128_t* U, int32_t m, int64_t ldu, const int32_t* rows, const int32_t* cols,
                     int32_t n, int64_t batch, perm_c128_t* out, void* stream) {
    clear_error();
    return gather_run(U, m, ldu, rows, cols, n, batch, out, true, static_cast<cudaStream_t>(stream));
}

int perm_f64_gather(const double* U, int32_t m, int64_t ldu, const int32_t* rows, const int32_t* cols, int32_t n,
                    int64_t batch, double* out, void* stream) {
    clear_error();
    return gather_run(U, m, ldu, rows, cols, n, batch, out, false, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
