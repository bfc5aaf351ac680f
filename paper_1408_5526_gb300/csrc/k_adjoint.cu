// k_adjoint.cu -- dispatch of the pathwise adjoint kernels by sequence.
#include "rqmc_internal.h"

namespace rqmc {

template <int SEQ>
int adjoint_seq(const Plan &pl, cudaStream_t st, int mode);

cudaError_t launch_adjoint(const Plan &pl, cudaStream_t st) {
#define RQMC_L(S) adjoint_seq<S>(pl, st, 0)
    return (cudaError_t)RQMC_SEQ_DISPATCH(pl.seq, RQMC_L);
#undef RQMC_L
}

int adjoint_grid(const Plan &pl) {
#define RQMC_L(S) adjoint_seq<S>(pl, 0, 1)
    return RQMC_SEQ_DISPATCH(pl.seq, RQMC_L);
#undef RQMC_L
}

}  // namespace rqmc
