// Explicit instantiations of the integer-mantissa complex128 Ryser kernel for n in [PERMX_NLO, PERMX_NHI].
#include "ryser_x64.cuh"

namespace permx {
#define PERMX_INST(N)                                                                  \
    template cudaError_t launch_x64c<N>(const FpLaunch&, int, int, cudaStream_t);           \
    template int blocks_per_sm_x64c<N>();
#include "inst_range.inc"
}  // namespace permx
