// k_batch_halton.cu -- batched persistent kernel for the halton generator.
#include "k_batch.cuh"

namespace rqmc {
template cudaError_t launch_batch_seq<kRasrap>(const BatchLaunch &bl, int kind, cudaStream_t st);
}  // namespace rqmc
