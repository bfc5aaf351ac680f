// k_adjoint_philox.cu -- pathwise adjoint kernels for the philox generator.
#include "k_adjoint.cuh"

namespace rqmc {
template int adjoint_seq<kPhilox, false>(const Plan &pl, cudaStream_t st, int mode);
}  // namespace rqmc
