// k_lmm.cu -- fused LIBOR-market-model caplet kernel (Sec. 5).
//
// One thread = one path of one replication.  Per time step t (grid t_i = T_i, h = delta):
// coordinate t of the point (Halton/Rasrap digits, Sobol', or Philox) -> Phi^-1 -> one
// log-Euler step of every alive forward under the spot measure,
//     log L_n += sigma_n mu_n h - sigma_n^2 h / 2 + sigma_n sqrt(h) Z,
//     mu_n = sum_{j=eta}^{n} delta L_j sigma_j / (1 + delta L_j)   (a running prefix),
// then L_{t+1}(T_{t+1}) is fixed, the spot numeraire is advanced by (1 + delta L_{t+1}) and
// the caplet payoffs delta (L_{t+1} - K)^+ / prod_{j<=t+1}(1 + delta L_j(T_j)) are summed
// over the warp and accumulated per warp (Kahan in FP32).
//
// The forwards live in registers (NF-slot buckets 16/40/80/160; an instrument with nf
// forwards uses slots NF-nf..NF-1).  Each step jumps into the unrolled slot sequence at
// the first alive slot (a switch that falls through), so exactly the alive forwards are
// updated and no per-slot guard is executed.
#include "paths_common.cuh"

namespace rqmc {

template <typename T>
__device__ __forceinline__ T model_exp(T x);
template <>
__device__ __forceinline__ float model_exp<float>(float x) { return ex2_approx(x); }   // constants carry log2 e
template <>
__device__ __forceinline__ double model_exp<double>(double x) { return exp(x); }

template <int K, int NF, typename T>
__device__ __forceinline__ void lmm_upd(T (&L)[NF], const LmmModel<T> &md, T z, T &S) {
    if constexpr (K < NF) {
        const T x = md.dl * L[K];
        const T a = x * fast_rcp<T>(T(1) + x);        // delta L_j / (1 + delta L_j), old L_j
        S = fmaT(md.sg[K], a, S);                      // prefix sum including j = n
        const T e = fmaT(md.cdr[K], S, fmaT(md.cz[K], z, md.cc[K]));
        L[K] *= model_exp<T>(e);
    }
}

template <int NF, typename T>
__global__ void __launch_bounds__(256) lmm_caplet_kernel(const GenParams g, const LmmModel<T> md, const RedParams r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *acc = reinterpret_cast<T *>(smem_raw);
    T *cmp = acc + nw * r.nout;
    T *wacc = acc + warp * r.nout, *wcmp = cmp + warp * r.nout;
    zero_acc(acc, cmp, nw * r.nout);
    __syncthreads();
    uint32_t u0, u1;
    unit_range(r, u0, u1);
    const int slot0 = NF - md.nf;
    for (uint32_t u = u0; u < u1; ++u) {
        const int m = (int)(u / r.tiles_per_m);
        const uint32_t tile = u % r.tiles_per_m;
        for (int pp = 0; pp < r.ppt; ++pp) {
            const uint32_t i = tile * r.tile + (uint32_t)(pp * blockDim.x + threadIdx.x);
            const bool active = i < r.N;
            if (!__any_sync(0xffffffffu, active)) break;
            PathGen pg;
            pg.init(g, m, active ? i : 0u);
            T L[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) L[k] = md.L0[k];
            T disc = md.disc0;
            for (int t = 0; t < md.nf; ++t) {
                const T z = NormalOf<T>::get(pg, t);
                T S = T(0);
                const int first = slot0 + t;
                switch (first) {
#define RQMC_UPD(k) \
    case (k):       \
        lmm_upd<(k)>(L, md, z, S);
                    RQMC_C160(RQMC_UPD)
#undef RQMC_UPD
                    default:
                        break;
                }
                T Lf = L[0];
                switch (first) {
#define RQMC_PICK(k)                           \
    case (k):                                  \
        if constexpr ((k) < NF) Lf = L[(k)];   \
        break;
                    RQMC_C160(RQMC_PICK)
#undef RQMC_PICK
                    default:
                        break;
                }
                disc *= fast_rcp<T>(T(1) + md.dl * Lf);
                const int ob = t * md.nK;
                for (int kk = 0; kk < md.nK; ++kk) {
                    const T x = Lf - md.K[kk];
                    const T pay = (active && x > T(0)) ? md.dl * x * disc : T(0);
                    warp_accumulate<T>(pay, wacc, wcmp, ob + kk, lane);
                }
            }
        }
        flush_unit(r, u, acc, cmp);
    }
}

template <int NF, typename T>
static cudaError_t launch_lmm_t(const Plan &pl, const LmmModel<T> &md, cudaStream_t st) {
    auto kern = lmm_caplet_kernel<NF, T>;
    const int threads = pl.threads;
    const size_t smem = 2ull * (threads / 32) * pl.red.nout * sizeof(T);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (occ < 1) occ = 1;
    unsigned grid = (unsigned)std::min<unsigned long long>(pl.red.units, (unsigned long long)occ * sms);
    if (pl.grid > 0) grid = (unsigned)std::min<unsigned long long>(pl.red.units, (unsigned long long)pl.grid);
    kern<<<grid, threads, smem, st>>>(pl.gen, md, pl.red);
    return cudaGetLastError();
}

cudaError_t launch_caplets(const Plan &pl, cudaStream_t st) {
    const bool f32 = pl.prec == RQMC_FP32;
    switch (pl.nf_bucket) {
        case 16: return f32 ? launch_lmm_t<16>(pl, pl.lmm32, st) : launch_lmm_t<16>(pl, pl.lmm64, st);
        case 40: return f32 ? launch_lmm_t<40>(pl, pl.lmm32, st) : launch_lmm_t<40>(pl, pl.lmm64, st);
        case 80: return f32 ? launch_lmm_t<80>(pl, pl.lmm32, st) : launch_lmm_t<80>(pl, pl.lmm64, st);
        case 160: return f32 ? launch_lmm_t<160>(pl, pl.lmm32, st) : launch_lmm_t<160>(pl, pl.lmm64, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rqmc
