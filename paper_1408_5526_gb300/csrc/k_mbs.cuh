// k_mbs.cuh -- one path of the mortgage-backed-security model (Sec. 6), shared by the MBS
// kernel and the batched kernel.
#pragma once
#include "paths_common.cuh"

namespace rqmc {

template <typename T>
__device__ __forceinline__ T mbs_exp(T x);
template <>
__device__ __forceinline__ float mbs_exp<float>(float x) { return ex2_approx(x); }
template <>
__device__ __forceinline__ double mbs_exp<double>(double x) { return exp(x); }

__device__ __forceinline__ float mbs_atan(float x) { return atanf(x); }
__device__ __forceinline__ double mbs_atan(double x) { return atan(x); }

template <typename T, int SEQ>
__device__ __forceinline__ T mbs_path(PathGen<SEQ> &pg, const MbsModel<T> &md, const T *__restrict__ ck) {
    T ip = md.i0, u = md.u1, rr = T(1), v = T(0), vc = T(0);
    for (int k = 1; k <= md.months; ++k) {
        const T z = Draw<T>::normal(pg, k - 1);
        const T ik = ip * mbs_exp<T>(fmaT(md.sz, z, md.lk0));
        const T w = fmaT(md.K2, mbs_atan(fmaT(md.K3, ik, md.K4)), md.K1);
        const T mk = md.c * rr * ((T(1) - w) + w * ck[k]);
        if constexpr (sizeof(T) == 4) kahan_add(v, vc, u * mk);
        else v += u * mk;
        u *= fast_rcp<T>(T(1) + ik);
        rr *= T(1) - w;
        ip = ik;
    }
    return v - vc;
}

}  // namespace rqmc
