// Explicit instantiations of the F_p Ryser kernel for n in [PERMX_NLO, PERMX_NHI].
// The build compiles this file several times with different ranges, in parallel.
#include "ryser_modp.cuh"

namespace permx {
#define PERMX_INST(N)                                                                  \
    template cudaError_t launch_modp<N>(const ModpLaunch&, int, int, cudaStream_t);         \
    template int blocks_per_sm_modp<N>();
#include "inst_range.inc"
}  // namespace permx
