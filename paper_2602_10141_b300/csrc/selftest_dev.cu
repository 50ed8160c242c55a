// Device side of the self-test hooks: the integer-mantissa products as the
// GPU computes them (inline-PTX multiply-adds), for comparison with the host
// forms of the same functions and with exact integer arithmetic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "x64_arith.cuh"

namespace permx {

__global__ void x64_mulhi_kernel(const int64_t* __restrict__ a, const int64_t* __restrict__ b, int64_t count,
                                 int64_t* __restrict__ hi62, int64_t* __restrict__ hi64) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        hi62[i] = x64_mulhi62(a[i], b[i]);
        hi64[i] = x64_mulhi64(a[i], b[i]);
    }
}

__global__ void x64c_mulhi_kernel(const int64_t* __restrict__ in4, int64_t count, int64_t* __restrict__ out4) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        const int64_t* q = in4 + 4 * i;
        int64_t* o = out4 + 4 * i;
        x64c_mulhi<64>(q[0], q[1], q[2], q[3], o[0], o[1]);
        x64c_mulhi<62>(q[0], q[1], q[2], q[3], o[2], o[3]);
    }
}

}  // namespace permx

using namespace permx;

extern "C" int permx_x64_mulhi_device(const int64_t* a, const int64_t* b, int64_t count, int64_t* hi62,
                                      int64_t* hi64) {
    if (!a || !b || !hi62 || !hi64 || count < 1 || count > (1 << 20)) return fail(PERMX_EINVAL, "bad arguments");
    const size_t bytes = (size_t)count * sizeof(int64_t);
    int64_t* d = nullptr;
    PERMX_CUDA(cudaMalloc(&d, 4 * bytes));
    cudaError_t e = cudaMemcpy(d, a, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + count, b, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        x64_mulhi_kernel<<<(unsigned)((count + 255) / 256), 256>>>(d, d + count, count, d + 2 * count, d + 3 * count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(hi62, d + 2 * count, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hi64, d + 3 * count, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? PERMX_OK : cuda_fail(e, "x64 mulhi self-test");
}

extern "C" int permx_x64c_mulhi_device(const int64_t* in4, int64_t count, int64_t* out4) {
    if (!in4 || !out4 || count < 1 || count > (1 << 20)) return fail(PERMX_EINVAL, "bad arguments");
    const size_t bytes = (size_t)count * 4 * sizeof(int64_t);
    int64_t* d = nullptr;
    PERMX_CUDA(cudaMalloc(&d, 2 * bytes));
    cudaError_t e = cudaMemcpy(d, in4, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        x64c_mulhi_kernel<<<(unsigned)((count + 255) / 256), 256>>>(d, count, d + 4 * count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out4, d + 4 * count, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? PERMX_OK : cuda_fail(e, "x64c mulhi self-test");
}
