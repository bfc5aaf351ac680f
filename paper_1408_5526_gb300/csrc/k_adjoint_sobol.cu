// k_adjoint_sobol.cu -- pathwise adjoint kernels for the sobol generator.
#include "k_adjoint.cuh"

namespace rqmc {
template int adjoint_seq<kSobolDS, false>(const Plan &pl, cudaStream_t st, int mode);
}  // namespace rqmc
