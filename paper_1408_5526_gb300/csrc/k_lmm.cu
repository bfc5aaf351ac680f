// k_lmm.cu -- dispatch of the LMM caplet kernels by sequence.
#include "rqmc_internal.h"

namespace rqmc {

template <int SEQ>
cudaError_t launch_caplets_seq(const Plan &pl, cudaStream_t st);

cudaError_t launch_caplets_loaded(const Plan &pl, cudaStream_t st);

cudaError_t launch_caplets(const Plan &pl, cudaStream_t st) {
    if (pl.znorm && pl.prec == RQMC_FP32) return launch_caplets_loaded(pl, st);
#define RQMC_L(S) launch_caplets_seq<S>(pl, st)
    return RQMC_SEQ_DISPATCH(pl.seq, RQMC_L);
#undef RQMC_L
}

}  // namespace rqmc
