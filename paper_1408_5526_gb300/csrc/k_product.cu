// k_product.cu -- product test integrand f(x) = prod_j (|4 x_j - 2| + a_j)/(1 + a_j) and the
// final replication reduction theta_N^m = (1/N) sum_i f(q_i^m) (Sec. 1).
#include "paths_common.cuh"

namespace rqmc {

template <typename T, int SEQ, bool STAGED>
__global__ void __launch_bounds__(256) product_kernel(const GenParams g, const ProductModel<T> md,
                                                      const RedParams r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *acc = reinterpret_cast<T *>(smem_raw + stage_bytes(g));
    T *cmp = acc + nw;
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
        for (int pp = 0; pp < r.ppt; ++pp) {
            const uint32_t i = tile * r.tile + (uint32_t)(pp * blockDim.x + threadIdx.x);
            const bool active = i < r.N;
            if (!__any_sync(0xffffffffu, active)) break;
            PathGen<SEQ> pg;
            pg.init(gv, active ? i : 0u);
            T f = T(1);
            for (int j = 0; j < md.s; ++j) {
                const T x = Draw<T>::uniform(pg, j);
                f *= (fabs(T(4) * x - T(2)) + md.a[j]) * md.inv1pa[j];
            }
            warp_accumulate<T>(active ? f : T(0), acc + warp, cmp + warp, 0, lane);
        }
        flush_unit(r, u, acc, cmp);
    }
}

template <typename T, int SEQ>
static cudaError_t launch_product_t(const Plan &pl, const ProductModel<T> &md, cudaStream_t st) {
    auto kern = pl.gen.stage ? product_kernel<T, SEQ, true> : product_kernel<T, SEQ, false>;
    const int threads = pl.threads;
    const size_t smem = stage_bytes(pl.gen) + 2ull * (threads / 32) * sizeof(T);
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
static cudaError_t launch_product_seq(const Plan &pl, cudaStream_t st) {
    return pl.prec == RQMC_FP32 ? launch_product_t<float, SEQ>(pl, pl.prod32, st)
                                : launch_product_t<double, SEQ>(pl, pl.prod64, st);
}

cudaError_t launch_product(const Plan &pl, cudaStream_t st) {
#define RQMC_L(S) launch_product_seq<S>(pl, st)
    return RQMC_SEQ_DISPATCH(pl.seq, RQMC_L);
#undef RQMC_L
}

// theta[m][o] = (sum over the tiles of replication m, in tile order) / N
// theta[m][o] = (sum over the replication's tiles of partials[m][tile][o]) / N.  A CTA of 32 x 8
// threads serves 32 outputs of one replication: thread (x, y) sums the y-th contiguous eighth
// of the tiles for output x (the 32 reads of a tile are one 256-byte row), and the eight part
// sums are added in y order, so the result does not depend on scheduling.
constexpr int kThetaSlices = 8;
__global__ void __launch_bounds__(32 * kThetaSlices) theta_kernel(const double *__restrict__ partials, int nout,
                                                                  uint32_t tiles_per_m, double N,
                                                                  double *__restrict__ theta) {
    __shared__ double part[kThetaSlices][32];
    const int o = blockIdx.x * 32 + threadIdx.x, m = blockIdx.y;
    const uint32_t t0 = (uint32_t)(((unsigned long long)threadIdx.y * tiles_per_m) / kThetaSlices);
    const uint32_t t1 = (uint32_t)(((unsigned long long)(threadIdx.y + 1) * tiles_per_m) / kThetaSlices);
    double s = 0.0;
    if (o < nout) {
        const double *p = partials + (size_t)m * tiles_per_m * nout + o;
        for (uint32_t t = t0; t < t1; ++t) s += p[(size_t)t * nout];
    }
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && o < nout) {
        double tot = 0.0;
#pragma unroll
        for (int k = 0; k < kThetaSlices; ++k) tot += part[k][threadIdx.x];
        theta[(size_t)m * nout + o] = tot / N;
    }
}

cudaError_t launch_theta(const Plan &pl, double *theta_dev, cudaStream_t st) {
    const dim3 grid((unsigned)((pl.red.nout + 31) / 32), (unsigned)pl.M), block(32, kThetaSlices);
    theta_kernel<<<grid, block, 0, st>>>(pl.red.partials, pl.red.nout, pl.red.tiles_per_m, (double)pl.N, theta_dev);
    return cudaGetLastError();
}

}  // namespace rqmc
