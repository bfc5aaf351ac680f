// k_lmm_philox.cu -- LMM caplet kernels for the philox generator.
#include "k_lmm.cuh"

namespace rqmc {
template cudaError_t launch_caplets_seq<kPhilox>(const Plan &pl, cudaStream_t st);
}  // namespace rqmc
