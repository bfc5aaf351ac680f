// k_lmm_sobol.cu -- LMM caplet kernels for the sobol generator.
#include "k_lmm.cuh"

namespace rqmc {
template cudaError_t launch_caplets_seq<kSobolDS>(const Plan &pl, cudaStream_t st);
}  // namespace rqmc
