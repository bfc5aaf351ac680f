// k_lmm_loaded.cu -- FP32 LMM caplet kernels that read their normals (written beforehand by
// the point-stream run kernel) instead of generating them: one kernel per bucket serves every
// sequence (the generator is not used; the nominal SEQ only types the unused path state).
#include "k_lmm.cuh"

namespace rqmc {
cudaError_t launch_caplets_loaded(const Plan &pl, cudaStream_t st) {
    switch (pl.nf_bucket) {
        case 16: return launch_lmm_t<16, kPhilox, float, true>(pl, pl.lmm32, st);
        case 40: return launch_lmm_t<40, kPhilox, float, true>(pl, pl.lmm32, st);
        case 80: return launch_lmm_t<80, kPhilox, float, true>(pl, pl.lmm32, st);
        case 160: return launch_lmm_t<160, kPhilox, float, true>(pl, pl.lmm32, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace rqmc
