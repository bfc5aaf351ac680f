// k_points.cu -- point-stream kernel: coordinates of M randomizations of N points,
// layout out[(m*s + j)*N + i] (the generator-throughput setting of Sec. 4, Table 2).
// Rows (m, j) are cut into chunks of ITEMS*blockDim consecutive points; a thread writes
// ITEMS coordinates blockDim apart so every warp store is one contiguous 128-byte (FP32)
// segment, and computes them in lockstep (shared digit / bit loop and inverse-CDF
// polynomial).  Philox rows come four dimensions at a time from one counter.
#include "paths_common.cuh"

namespace rqmc {

constexpr int kPtItems = 8;

template <int TR, typename T>
__device__ __forceinline__ T value_from_u32(uint32_t x) {
    if constexpr (TR == RQMC_RAW) return (T)x;
    else if constexpr (sizeof(T) == 4) {
        const Unif32 v = unif32_from_u32(x);
        if constexpr (TR == RQMC_NORMAL) return ndtri32(v);
        else return v.lower ? v.q : 1.0f - v.q;
    } else {
        const Unif64 v = unif64_from_u32(x);
        if constexpr (TR == RQMC_NORMAL) return ndtri64(v);
        else return v.lower ? v.q : 1.0 - v.q;
    }
}

template <int TR, typename T>
__global__ void __launch_bounds__(256) points_kernel(const GenParams g, uint32_t N, uint32_t chunks,
                                                     unsigned long long nrows, T *__restrict__ out) {
    const uint32_t span = blockDim.x * kPtItems;
    const unsigned long long total = nrows * chunks;
    for (unsigned long long b = blockIdx.x; b < total; b += gridDim.x) {
        const unsigned long long row = b / chunks;
        const uint32_t base = (uint32_t)(b % chunks) * span + threadIdx.x;
        if (g.seq == kPhilox) {
            const int nb = (g.s + 3) >> 2;
            const int m = (int)(row / nb), jb = (int)(row % nb);
#pragma unroll 2
            for (int it = 0; it < kPtItems; ++it) {
                const uint32_t i = base + it * blockDim.x;
                if (i >= N) break;
                const unsigned long long n = g.offset + i;
                const U32x4 w = philox4x32_10((uint32_t)n, (uint32_t)((n >> 32) & 0xFFFFu) | ((uint32_t)jb << 16),
                                              (uint32_t)m, kTagPath | (g.inst << 8), g.key0, g.key1);
                const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = 4 * jb + q;
                    if (j < g.s) out[((size_t)m * g.s + j) * N + i] = value_from_u32<TR, T>(ws[q]);
                }
            }
        } else {
            // Halton / Sobol' rows: the ITEMS points of the thread advance in lockstep
            const int m = (int)(row / g.s), j = (int)(row % g.s);
            T *dst = out + row * N;
            if (base >= N) continue;
            uint32_t ii[kPtItems];
            bool ok[kPtItems];
#pragma unroll
            for (int it = 0; it < kPtItems; ++it) {
                const uint32_t i = base + it * blockDim.x;
                ok[it] = i < N;
                ii[it] = ok[it] ? i : base;   // past the end: recompute a valid point, store nothing
            }
            if (g.seq == kSobolDS) {
                uint32_t n[kPtItems], x[kPtItems];
#pragma unroll
                for (int it = 0; it < kPtItems; ++it) n[it] = (uint32_t)(g.offset + ii[it]);
                sobol_lockstep<kPtItems>(g.sobV + (size_t)m * g.sobV_mstride + 32 * j, __ldg(g.sobShift + row), n,
                                         g.sob_bits, x);
                if constexpr (TR == RQMC_NORMAL && sizeof(T) == 4) {
                    Unif32 u[kPtItems];
                    float z[kPtItems];
#pragma unroll
                    for (int it = 0; it < kPtItems; ++it) u[it] = unif32_from_u32(x[it]);
                    ndtri32_lockstep<kPtItems>(u, z);
#pragma unroll
                    for (int it = 0; it < kPtItems; ++it)
                        if (ok[it]) dst[ii[it]] = z[it];
                } else {
#pragma unroll
                    for (int it = 0; it < kPtItems; ++it)
                        if (ok[it]) dst[ii[it]] = value_from_u32<TR, T>(x[it]);
                }
            } else {
                const HaltonDim h = g.hdim[row];   // one copy in registers, shared by the items
                const uint16_t *sig = g.sigma + (size_t)m * g.sig_len;
                uint32_t R[kPtItems], c[kPtItems];
                halton_R_lockstep<kPtItems>(h, sig + h.sig_off, ii, R, c);
                if constexpr (TR == RQMC_RAW) {
#pragma unroll
                    for (int it = 0; it < kPtItems; ++it)
                        if (ok[it]) dst[ii[it]] = (T)halton_num(h, R[it], c[it]);
                } else if constexpr (sizeof(T) == 4) {
                    Unif32 u[kPtItems];
#pragma unroll
                    for (int it = 0; it < kPtItems; ++it) u[it] = unif32_halton(h, R[it], c[it]);
                    if constexpr (TR == RQMC_NORMAL) {
                        float z[kPtItems];
                        ndtri32_lockstep<kPtItems>(u, z);
#pragma unroll
                        for (int it = 0; it < kPtItems; ++it)
                            if (ok[it]) dst[ii[it]] = z[it];
                    } else {
#pragma unroll
                        for (int it = 0; it < kPtItems; ++it)
                            if (ok[it]) dst[ii[it]] = u[it].lower ? u[it].q : 1.0f - u[it].q;
                    }
                } else {
#pragma unroll
                    for (int it = 0; it < kPtItems; ++it) {
                        const Unif64 v = unif64_halton(h, R[it], c[it]);
                        T val;
                        if constexpr (TR == RQMC_NORMAL) val = ndtri64(v);
                        else val = v.lower ? v.q : 1.0 - v.q;
                        if (ok[it]) dst[ii[it]] = val;
                    }
                }
            }
        }
    }
}

template <int TR, typename T>
static cudaError_t launch_points_t(const Plan &pl, void *out, cudaStream_t st) {
    auto kern = points_kernel<TR, T>;
    const int threads = 256;
    const uint32_t span = threads * kPtItems;
    const uint32_t chunks = (uint32_t)((pl.N + span - 1) / span);
    const unsigned long long nrows =
        pl.seq == kPhilox ? (unsigned long long)pl.M * ((pl.s + 3) / 4) : (unsigned long long)pl.M * pl.s;
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0);
    if (occ < 1) occ = 1;
    const unsigned long long total = nrows * chunks;
    const unsigned grid = (unsigned)std::min<unsigned long long>(total, (unsigned long long)occ * sms * 4);
    kern<<<grid, threads, 0, st>>>(pl.gen, (uint32_t)pl.N, chunks, nrows, reinterpret_cast<T *>(out));
    return cudaGetLastError();
}

cudaError_t launch_points(const Plan &pl, int tr, void *out, cudaStream_t st) {
    if (tr == RQMC_RAW) return launch_points_t<RQMC_RAW, unsigned long long>(pl, out, st);
    const bool f32 = pl.prec == RQMC_FP32;
    if (tr == RQMC_UNIFORM)
        return f32 ? launch_points_t<RQMC_UNIFORM, float>(pl, out, st) : launch_points_t<RQMC_UNIFORM, double>(pl, out, st);
    return f32 ? launch_points_t<RQMC_NORMAL, float>(pl, out, st) : launch_points_t<RQMC_NORMAL, double>(pl, out, st);
}

}  // namespace rqmc
