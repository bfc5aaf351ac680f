// k_lmm_halton.cu -- LMM caplet kernels for the halton generator.
#include "k_lmm.cuh"

namespace rqmc {
template cudaError_t launch_caplets_seq<kRasrap>(const Plan &pl, cudaStream_t st);
}  // namespace rqmc
