// k_batch_sobol.cu -- batched persistent kernel for the sobol generator.
#include "k_batch.cuh"

namespace rqmc {
template cudaError_t launch_batch_seq<kSobolDS>(const BatchLaunch &bl, int kind, cudaStream_t st);
}  // namespace rqmc
