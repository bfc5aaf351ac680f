// k_adjoint.cu -- dispatch of the pathwise adjoint kernels by sequence (or, for plans whose
// normals are written beforehand, to the one set of kernels that reads them).
#include "rqmc_internal.h"

namespace rqmc {

template <int SEQ, bool ZG>
int adjoint_seq(const Plan &pl, cudaStream_t st, int mode);

cudaError_t launch_adjoint(const Plan &pl, cudaStream_t st) {
    if (pl.znorm) return (cudaError_t)adjoint_seq<kPhilox, true>(pl, st, 0);
#define RQMC_L(S) adjoint_seq<S, false>(pl, st, 0)
    return (cudaError_t)RQMC_SEQ_DISPATCH(pl.seq, RQMC_L);
#undef RQMC_L
}

int adjoint_grid(const Plan &pl) {
    if (pl.znorm) return adjoint_seq<kPhilox, true>(pl, 0, 1);
#define RQMC_L(S) adjoint_seq<S, false>(pl, 0, 1)
    return RQMC_SEQ_DISPATCH(pl.seq, RQMC_L);
#undef RQMC_L
}

}  // namespace rqmc
