// paths_common.cuh -- unit scheduling and the per-unit replication reduction shared by the
// fused path kernels.
//
// Work unit u = (replication m = u / tiles_per_m, tile = u % tiles_per_m): `tile`
// consecutive points i of replication m.  CTA c processes the contiguous unit range
// [c U / G, (c+1) U / G), so a grid of G = (SMs x resident CTAs) CTAs is balanced to
// within one unit.  Within a unit each warp accumulates its per-step payload in shared
// memory; at the end of the unit the warps' accumulators are added in double in warp
// order and written to partials[u][o].  No float atomics: the result is bit-identical
// from run to run and independent of G.
#pragma once
#include "rqmc_internal.h"

namespace rqmc {

__device__ __forceinline__ void unit_range(const RedParams &r, uint32_t &u0, uint32_t &u1) {
    u0 = (uint32_t)(((unsigned long long)blockIdx.x * r.units) / gridDim.x);
    u1 = (uint32_t)(((unsigned long long)(blockIdx.x + 1) * r.units) / gridDim.x);
}

// acc / cmp: [nwarps][nout] Kahan pairs (cmp unused in FP64 mode, kept zero).
template <typename T>
__device__ __forceinline__ void zero_acc(T *acc, T *cmp, int n) {
    for (int o = threadIdx.x; o < n; o += blockDim.x) {
        acc[o] = T(0);
        cmp[o] = T(0);
    }
}

template <typename T>
__device__ __forceinline__ void flush_unit(const RedParams &r, uint32_t u, T *acc, T *cmp) {
    __syncthreads();
    const int nw = blockDim.x >> 5, nout = r.nout;
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) {
            s += (double)acc[w * nout + o] - (double)cmp[w * nout + o];
            acc[w * nout + o] = T(0);
            cmp[w * nout + o] = T(0);
        }
        r.partials[(size_t)u * nout + o] = s;
    }
    __syncthreads();
}

// Lane 0 adds a warp total into the warp's accumulator slot o (Kahan in FP32).
template <typename T>
__device__ __forceinline__ void warp_accumulate(T v, T *acc, T *cmp, int o, int lane) {
    v = warp_sum(v);
    if (lane == 0) {
        T s = acc[o], c = cmp[o];
        kahan_add(s, c, v);
        acc[o] = s;
        cmp[o] = c;
    }
}

template <>
__device__ __forceinline__ void warp_accumulate<double>(double v, double *acc, double *, int o, int lane) {
    v = warp_sum(v);
    if (lane == 0) acc[o] += v;
}

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// Uniform u = (num + 1/2)/D and normal z of dimension j for the current path.
template <typename T>
struct Draw;
template <>
struct Draw<float> {
    template <int SEQ>
    static __device__ __forceinline__ float uniform(PathGen<SEQ> &pg, int j) {
        const Unif32 v = pg.unif32(j);
        return v.lower ? v.q : 1.0f - v.q;
    }
    template <int SEQ>
    static __device__ __forceinline__ float normal(PathGen<SEQ> &pg, int j) { return ndtri32(pg.unif32(j)); }
};
template <>
struct Draw<double> {
    template <int SEQ>
    static __device__ __forceinline__ double uniform(PathGen<SEQ> &pg, int j) {
        const Unif64 v = pg.unif64(j);
        return v.lower ? v.q : 1.0 - v.q;
    }
    template <int SEQ>
    static __device__ __forceinline__ double normal(PathGen<SEQ> &pg, int j) { return ndtri64(pg.unif64(j)); }
};

template <typename T>
__device__ __forceinline__ T fast_exp2(T x);
template <>
__device__ __forceinline__ float fast_exp2<float>(float x) { return ex2_approx(x); }
template <>
__device__ __forceinline__ double fast_exp2<double>(double x) { return exp2(x); }

template <typename T>
__device__ __forceinline__ T fast_rcp(T x);
template <>
__device__ __forceinline__ float fast_rcp<float>(float x) { return rcp_approx(x); }
template <>
__device__ __forceinline__ double fast_rcp<double>(double x) { return 1.0 / x; }

// 0..NF-1 case labels for jump tables (k is a constant expression).
#define RQMC_C1(X, k) X(k)
#define RQMC_C2(X, k) RQMC_C1(X, k) RQMC_C1(X, (k) + 1)
#define RQMC_C4(X, k) RQMC_C2(X, k) RQMC_C2(X, (k) + 2)
#define RQMC_C8(X, k) RQMC_C4(X, k) RQMC_C4(X, (k) + 4)
#define RQMC_C16(X, k) RQMC_C8(X, k) RQMC_C8(X, (k) + 8)
#define RQMC_C32(X, k) RQMC_C16(X, k) RQMC_C16(X, (k) + 16)
#define RQMC_C160(X) RQMC_C32(X, 0) RQMC_C32(X, 32) RQMC_C32(X, 64) RQMC_C32(X, 96) RQMC_C32(X, 128)

}  // namespace rqmc
