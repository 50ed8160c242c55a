// Explicit instantiations of the complex128 Ryser kernel for n in [PERMX_NLO, PERMX_NHI].
#include "ryser_fp.cuh"

namespace permx {
#define PERMX_INST(N)                                                                  \
    template cudaError_t launch_c128<N>(const FpLaunch&, int, int, cudaStream_t);           \
    template int blocks_per_sm_c128<N>();
#include "inst_range.inc"
}  // namespace permx
