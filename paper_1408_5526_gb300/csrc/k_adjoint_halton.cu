// k_adjoint_halton.cu -- pathwise adjoint kernels for the halton generator.
#include "k_adjoint.cuh"

namespace rqmc {
template int adjoint_seq<kRasrap, false>(const Plan &pl, cudaStream_t st, int mode);
}  // namespace rqmc
