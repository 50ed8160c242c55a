// Explicit instantiations of the float64 Ryser kernel for n in [PERMX_NLO, PERMX_NHI].
#include "ryser_fp.cuh"

namespace permx {
#define PERMX_INST(N)                                                                  \
    template cudaError_t launch_f64<N>(const FpLaunch&, int, int, cudaStream_t);            \
    template int blocks_per_sm_f64<N>();
#include "inst_range.inc"
}  // namespace permx
