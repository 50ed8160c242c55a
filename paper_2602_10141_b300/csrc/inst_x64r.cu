// Explicit instantiations of the integer-mantissa float64 Ryser kernel for n in [PERMX_NLO, PERMX_NHI].
#include "ryser_x64.cuh"

namespace permx {
#define PERMX_INST(N)                                                                  \
    template cudaError_t launch_x64r<N>(const FpLaunch&, int, int, cudaStream_t);           \
    template int blocks_per_sm_x64r<N>();
#include "inst_range.inc"
}  // namespace permx
