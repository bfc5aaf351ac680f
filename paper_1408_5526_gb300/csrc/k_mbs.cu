// k_mbs.cu -- fused mortgage-backed-security kernel (Sec. 6, Caflisch's model).
//
// One thread = one path: for month k = 1..M, coordinate k-1 -> Phi^-1 -> xi_k = sigma z_k,
//   i_k = K0 e^{xi_k} i_{k-1},  w_k = K1 + K2 atan(K3 i_k + K4),
//   m_k = c r_k ((1 - w_k) + w_k c_k),  v += u_k m_k  (Kahan in FP32),
//   u_{k+1} = u_k / (1 + i_k),  r_{k+1} = r_k (1 - w_k).
// The path value v is summed over the warp and accumulated per warp and unit.
#include "k_mbs.cuh"

namespace rqmc {

// Paths per thread in lockstep: in FP32 mbs_paths32(SEQ) (their coordinates share the
// dimension's constants, and a Sobol' point blockDim away costs a few XORs), one in FP64.
template <typename T, int SEQ>
constexpr int mbs_ilp() {
    return sizeof(T) == 4 ? mbs_paths32(SEQ) : 1;
}

template <typename T, int SEQ, bool STAGED>
__global__ void __launch_bounds__(256) mbs_kernel(const GenParams g, const MbsModel<T> md, const RedParams r) {
    constexpr int P = mbs_ilp<T, SEQ>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *acc = reinterpret_cast<T *>(smem_raw + stage_bytes(g));
    T *cmp = acc + nw;
    T *ck = cmp + nw;
    for (int k = threadIdx.x; k <= md.months; k += blockDim.x) ck[k] = md.ck[k];
    zero_acc(acc, cmp, nw);
    uint32_t u0, u1;
    unit_range(r, u0, u1);
    GenView gv;
    int staged_m = -1;
    for (uint32_t u = u0; u < u1; ++u) {
        const int m = (int)(u / r.tiles_per_m);
        const uint32_t tile = u % r.tiles_per_m;
        if (m != staged_m) {
            __syncthreads();
            load_tables<STAGED>(g, m, smem_raw, gv);
            staged_m = m;
        }
        __syncthreads();
        for (int pp = 0; pp < r.ppt; pp += P) {
            PathGen<SEQ> pg[P];
            bool act[P];
            bool any = false;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const uint32_t i = tile * r.tile + (uint32_t)((pp + p) * blockDim.x + threadIdx.x);
                act[p] = pp + p < r.ppt && i < r.N;
                any = any || act[p];
                pg[p].init(gv, act[p] ? i : 0u);
            }
            if (!__any_sync(0xffffffffu, any)) break;
            T v[P];
            mbs_paths<T, SEQ, P>(pg, md, ck, v);
#pragma unroll
            for (int p = 0; p < P; ++p) warp_accumulate<T>(act[p] ? v[p] : T(0), acc + warp, cmp + warp, 0, lane);
        }
        flush_unit(r, u, acc, cmp);
    }
}

template <typename T, int SEQ>
static cudaError_t launch_mbs_t(const Plan &pl, const MbsModel<T> &md, cudaStream_t st) {
    auto kern = pl.gen.stage ? mbs_kernel<T, SEQ, true> : mbs_kernel<T, SEQ, false>;
    const int threads = pl.threads;
    const size_t smem = stage_bytes(pl.gen) + (2ull * (threads / 32) + md.months + 1) * sizeof(T);
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

template <int SEQ>
static cudaError_t launch_mbs_seq(const Plan &pl, cudaStream_t st) {
    return pl.prec == RQMC_FP32 ? launch_mbs_t<float, SEQ>(pl, pl.mbs32, st) : launch_mbs_t<double, SEQ>(pl, pl.mbs64, st);
}

cudaError_t launch_mbs(const Plan &pl, cudaStream_t st) {
#define RQMC_L(S) launch_mbs_seq<S>(pl, st)
    return RQMC_SEQ_DISPATCH(pl.seq, RQMC_L);
#undef RQMC_L
}

}  // namespace rqmc
