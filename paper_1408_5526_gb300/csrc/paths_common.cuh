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

// Asynchronous 4-byte global -> shared copies (waited for by the issuing thread only).
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
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

// ------------------------------------------------------------------ lockstep generation
// P coordinates of one dimension at once (P paths of a thread, or P points of a stream):
// they share the dimension's constants and advance together through the digit or bit loop
// and the inverse-CDF polynomial, so each loop iteration carries P independent dependency
// chains.  Every value is bit-identical to the one-at-a-time routines.

// Halton/Rasrap: R and carry of the points lo0 + i[p] (see halton_R); sg = sigma of the dim.
template <int P>
__device__ __forceinline__ void halton_R_lockstep(const HaltonDim &h, const uint16_t *__restrict__ sg,
                                                  const uint32_t (&i)[P], uint32_t (&R)[P], uint32_t (&c)[P]) {
    uint32_t low[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        low[p] = h.lo0 + i[p];
        c[p] = low[p] >= h.pL ? 1u : 0u;
        low[p] -= c[p] ? h.pL : 0u;
        R[p] = 0u;
    }
    if (h.p == 2) {   // base 2: bit reversal, sigma the identity or the swap
        const uint32_t flip = sg[0] != 0 ? (1u << h.L) - 1u : 0u;
#pragma unroll
        for (int p = 0; p < P; ++p) R[p] = (__brev(low[p]) >> (32u - h.L)) ^ flip;
        return;
    }
    const uint32_t pb = h.p, mg = h.magic;
    for (uint32_t k = 0; k < h.L; ++k) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            uint32_t q = __umulhi(low[p], mg);
            uint32_t d = low[p] - q * pb;
            if ((int32_t)d < 0) {   // the rounded-up reciprocal overshot by one
                d += pb;
                q -= 1;
            }
            R[p] = R[p] * pb + (uint32_t)sg[d];
            low[p] = q;
        }
    }
}

// Sobol': x = shift ^ XOR of V_k over the set bits of n[p].  The construction is linear,
// x(n') = x(n) ^ (XOR of V_k over the set bits of n ^ n'): the first point runs the bit
// loop, the others (a fixed stride apart) differ from it in a few bits and cost a few XORs.
template <int P>
__device__ __forceinline__ void sobol_lockstep(const uint32_t *__restrict__ Vj, uint32_t shift,
                                               const uint32_t (&n)[P], int bits, uint32_t (&x)[P]) {
    uint32_t x0 = shift;
#pragma unroll 4
    for (int k = 0; k < bits; ++k) x0 ^= ((n[0] >> k) & 1u) ? Vj[k] : 0u;
    x[0] = x0;
#pragma unroll
    for (int p = 1; p < P; ++p) {
        uint32_t xp = x0;
        for (uint32_t d = n[p] ^ n[0]; d != 0u; d &= d - 1u) xp ^= Vj[__ffs(d) - 1];
        x[p] = xp;
    }
}

// Phi^-1 of P uniforms: the central polynomial for all of them in straight-line code, the
// tail branches only where some value needs them (about 0.3 % of the values).
template <int P>
__device__ __forceinline__ void ndtri32_lockstep(const Unif32 (&u)[P], float (&z)[P]) {
    float v[P], y[P], r[P];
    bool central = true;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float q = u[p].q;
        v[p] = ndtri32_v(q);
        y[p] = fmaf(-2.0f, q, 1.0f);
        central = central && v[p] > (float)RQMC_NDTRI_V_SPLIT;
        r[p] = erfinv_central32(v[p]);
    }
    if (!central) {
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (!(v[p] > (float)RQMC_NDTRI_V_SPLIT)) r[p] = erfinv_tail32(v[p]);
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float x = y[p] * r[p];
        z[p] = u[p].lower ? -x : x;
    }
}

// FP32 normals of dimension j for the P lockstep paths of a thread (the values of P calls
// of Draw<float>::normal).
template <int SEQ, int P>
__device__ __forceinline__ void normals32(PathGen<SEQ> (&pg)[P], int j, float (&z)[P]) {
    Unif32 u[P];
    const GenView &v = pg[0].v;   // every path of the thread shares the replication's view
    if constexpr (SEQ == kPhilox) {
#pragma unroll
        for (int p = 0; p < P; ++p) u[p] = unif32_from_u32(pg[p].philox_word(j));
    } else if constexpr (SEQ == kSobolDS) {
        uint32_t n[P], x[P];
#pragma unroll
        for (int p = 0; p < P; ++p) n[p] = (uint32_t)pg[p].n;
        sobol_lockstep<P>(v.V + 32 * j, v.shift[j], n, v.sob_bits, x);
#pragma unroll
        for (int p = 0; p < P; ++p) u[p] = unif32_from_u32(x[p]);
    } else {
        const HaltonDim &h = v.hd[j];
        uint32_t i[P], R[P], c[P];
#pragma unroll
        for (int p = 0; p < P; ++p) i[p] = pg[p].i;
        halton_R_lockstep<P>(h, v.sig + h.sig_off, i, R, c);
#pragma unroll
        for (int p = 0; p < P; ++p) u[p] = unif32_halton(h, R[p], c[p]);
    }
    ndtri32_lockstep<P>(u, z);
}

// FP32 normals of two dimensions j0, j1 of one path (the values of two Draw<float>::normal
// calls): the Sobol' bit loop and the Halton digit loops of the two dimensions run together.
template <int SEQ>
__device__ __forceinline__ void normals32_two_dims(PathGen<SEQ> &pg, int j0, int j1, float &z0, float &z1) {
    Unif32 u[2];
    const GenView &v = pg.v;
    if constexpr (SEQ == kPhilox) {
        u[0] = unif32_from_u32(pg.philox_word(j0));
        u[1] = unif32_from_u32(pg.philox_word(j1));
    } else if constexpr (SEQ == kSobolDS) {
        const uint32_t *V0 = v.V + 32 * j0, *V1 = v.V + 32 * j1;
        const uint32_t n = (uint32_t)pg.n;
        uint32_t x0 = v.shift[j0], x1 = v.shift[j1];
#pragma unroll 4
        for (int k = 0; k < v.sob_bits; ++k) {
            const bool b = (n >> k) & 1u;
            x0 ^= b ? V0[k] : 0u;
            x1 ^= b ? V1[k] : 0u;
        }
        u[0] = unif32_from_u32(x0);
        u[1] = unif32_from_u32(x1);
    } else {
        const HaltonDim &h0 = v.hd[j0], &h1 = v.hd[j1];
        uint32_t c0, c1;
        const uint32_t R0 = halton_R(h0, v.sig, pg.i, c0);
        const uint32_t R1 = halton_R(h1, v.sig, pg.i, c1);
        u[0] = unif32_halton(h0, R0, c0);
        u[1] = unif32_halton(h1, R1, c1);
    }
    float z[2];
    ndtri32_lockstep<2>(u, z);
    z0 = z[0];
    z1 = z[1];
}

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
