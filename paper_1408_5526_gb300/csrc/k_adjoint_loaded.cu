// k_adjoint_loaded.cu -- pathwise adjoint kernels that read their normals (written beforehand
// by the point-stream run kernel) instead of generating them: one set serves every sequence
// (the generator is not used; the nominal SEQ only types the unused path state).
#include "k_adjoint.cuh"

namespace rqmc {
template int adjoint_seq<kPhilox, true>(const Plan &pl, cudaStream_t st, int mode);
}  // namespace rqmc
