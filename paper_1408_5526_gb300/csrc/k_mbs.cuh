// k_mbs.cuh -- paths of the mortgage-backed-security model (Sec. 6), shared by the MBS
// kernel and the batched kernel.
#pragma once
#include "atan_coeffs.h"
#include "paths_common.cuh"

namespace rqmc {

template <typename T>
__device__ __forceinline__ T mbs_exp(T x);
template <>
__device__ __forceinline__ float mbs_exp<float>(float x) { return ex2_approx(x); }
template <>
__device__ __forceinline__ double mbs_exp<double>(double x) { return exp(x); }

// FP32 arctangent without branches: t = min(|x|, 1/|x|) in [0, 1], atan(t) = t P(t^2) with
// our own fit (fit_atan.py), reflected by atan(a) = pi/2 - atan(1/a) for a > 1.
__device__ __forceinline__ float mbs_atan(float x) {
    constexpr float C[] = RQMC_ATAN_C;
    const float a = fabsf(x);
    const float t = fminf(a, rcp_approx(a));
    const float r = t * horner(C, t * t);
    return copysignf(a > 1.0f ? 1.5707963267948966f - r : r, x);
}
__device__ __forceinline__ double mbs_atan(double x) { return atan(x); }

// P paths in lockstep (same arithmetic per path as P = 1): they share the c_k loads and
// the control flow and give the thread P independent dependency chains.
template <typename T, int SEQ, int P>
__device__ __forceinline__ void mbs_paths(PathGen<SEQ> (&pg)[P], const MbsModel<T> &md, const T *__restrict__ ck,
                                          T (&out)[P]) {
    T ip[P], u[P], rr[P], v[P], vc[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        ip[p] = md.i0;
        u[p] = md.u1;
        rr[p] = T(1);
        v[p] = T(0);
        vc[p] = T(0);
    }
    for (int k = 1; k <= md.months; ++k) {
        const T c = ck[k];
        T zs[P];
        if constexpr (sizeof(T) == 4) {
            normals32<SEQ, P>(pg, k - 1, zs);   // the P paths' normals of month k together
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p) zs[p] = Draw<T>::normal(pg[p], k - 1);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const T z = zs[p];
            const T ik = ip[p] * mbs_exp<T>(fmaT(md.sz, z, md.lk0));
            const T w = fmaT(md.K2, mbs_atan(fmaT(md.K3, ik, md.K4)), md.K1);
            const T mk = md.c * rr[p] * ((T(1) - w) + w * c);
            if constexpr (sizeof(T) == 4) kahan_add(v[p], vc[p], u[p] * mk);
            else v[p] += u[p] * mk;
            u[p] *= fast_rcp<T>(T(1) + ik);
            rr[p] *= T(1) - w;
            ip[p] = ik;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) out[p] = v[p] - vc[p];
}

}  // namespace rqmc
