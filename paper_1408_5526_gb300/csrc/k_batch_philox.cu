// k_batch_philox.cu -- batched persistent kernel for the philox generator.
#include "k_batch.cuh"

namespace rqmc {
template cudaError_t launch_batch_seq<kPhilox>(const BatchLaunch &bl, int kind, cudaStream_t st);
}  // namespace rqmc
