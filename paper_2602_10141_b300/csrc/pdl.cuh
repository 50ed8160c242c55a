// Programmatic dependent launch (sm_90 and later): a walk kernel is launched
// so that the GPU may schedule its blocks while the set-up kernel before it in
// the stream still runs; every walk block first waits (griddepcontrol.wait)
// until that kernel has completed and its writes are visible, so nothing the
// walk reads is touched early.  The set-up kernels allow the early launch as
// they start (griddepcontrol.launch_dependents).  Launched without the
// attribute, or after a non-kernel stream operation, the wait returns at once.
#pragma once
#include <cuda_runtime.h>

namespace permx {

__device__ __forceinline__ void grid_dep_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
__device__ __forceinline__ void grid_dep_allow() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// kernel<<<grid, threads, 0, s>>>(L) with the programmatic stream
// serialization attribute
template <typename L>
cudaError_t launch_dependent(void (*kernel)(L), unsigned grid, unsigned threads, cudaStream_t s, const L& arg) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, arg);
}

}  // namespace permx
