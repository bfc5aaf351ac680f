// k_adjoint.cuh -- pathwise adjoint of an LMM caplet strip (not in the paper; the model
// and the estimator are Sec. 5's), instantiated per sequence by k_adjoint_{halton,sobol,philox}.cu.
//
// Objective per path: V = sum_n sum_k w_{n,k} delta (L_n(T_n) - K_k)^+ D_n with the spot
// numeraire D_n = prod_{j<=n} (1 + delta L_j(T_j))^-1.  Forwards live in registers as
// X_n = log2(delta L_n); one log-Euler step of slot n (d factors) is
//     a_n = 1 / (1 + 2^-X_n)               (= delta L_n / (1 + delta L_n))
//     A_n = sum_{j<=n, alive} sigma_j a_j   (d-vector prefix)
//     X_n += log2 e (h sigma_n.A_n + sqrt(h) sigma_n.Z - h |sigma_n|^2 / 2).
// Forward sweep (as in the caplet kernel, 8-step blocks with a register shift) stores,
// per step, the pre-step X of the forward fixed at that step and every updated a_n in a
// per-thread column of global scratch (coalesced across the warp).  Reverse sweep: with
// Xb_n = dV/dX_n in registers and B_n = sum_{m>=n} Xb_m sigma_m,
//     sigma_bar_n = log2 e [Xb_n (h A_n + sqrt(h) Z - h sigma_n) + h a_n B_n]
//     Xb_n       += h (sigma_n.B_n) a_n (1 - a_n)
// and at the fixing of forward n (Y = its post-step X, L = 2^Y / delta, G_n = sum_{m>=n} P_m)
//     Xb_n       += ln 2 [sum_k w_{n,k} delta 1{L > K_k} D_n L - a(Y) G_n].
// The normals of a step are regenerated from the counter, never stored.  At the end
// dV/dL_n(0) = Xb_n / (L_n(0) ln 2) and dV/dvol_n = sum over steps of sigma_bar_n . b_n.
// Per-thread value / delta / vega accumulators sit in global columns; each (replication,
// tile) unit sums its CTA's columns in double into its own partial row.
#pragma once
#include "paths_common.cuh"

namespace rqmc {

template <int D>
__device__ __forceinline__ float dotv(const float (&x)[D], const float (&y)[D]) {
    float s = x[0] * y[0];
    if constexpr (D == 2) s = fmaf(x[1], y[1], s);
    return s;
}

__device__ __forceinline__ float4 lds4(const float4 *p) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}

// Shared memory: [generator stage][(sigma_1, sigma_2, b_1, b_2) x NF][cc x NF]
template <int NF>
__host__ __device__ __forceinline__ size_t adj_smem_layout(const GenParams &g, size_t *o_cst, size_t *o_cc) {
    size_t off = align16(stage_bytes(g));
    *o_cst = off;
    off = align16(off + sizeof(float4) * NF);
    *o_cc = off;
    off = align16(off + sizeof(float) * NF);
    return off;
}

// one forward step of slot k (forward sweep): store a_k, advance the prefix and X_k
template <int D>
__device__ __forceinline__ void adj_fwd_update(float &X, const float4 c, float cc, float (&A)[D], const float (&Az)[D],
                                               float hl, float *&st, uint32_t T) {
    const float a = rcp_approx(1.0f + ex2_approx(-X));
    *st = a;
    st += T;
    A[0] = fmaf(c.x, a, A[0]);
    float inc = fmaf(c.x, fmaf(A[0], hl, Az[0]), cc);
    if constexpr (D == 2) {
        A[1] = fmaf(c.y, a, A[1]);
        inc = fmaf(c.y, fmaf(A[1], hl, Az[1]), inc);
    }
    X += inc;
}

template <int NF, int D, int SEQ>
__global__ void __launch_bounds__(128, NF <= 40 ? 4 : 2) lmm_adjoint_kernel(const GenParams g, const AdjModel md,
                                                                            const AdjScratch sc, const RedParams r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    size_t o_cst, o_cc;
    adj_smem_layout<NF>(g, &o_cst, &o_cc);
    float4 *cst = reinterpret_cast<float4 *>(smem_raw + o_cst);
    float *ccs = reinterpret_cast<float *>(smem_raw + o_cc);
    for (int k = threadIdx.x; k < NF; k += blockDim.x) {
        cst[k] = make_float4(md.sg[k][0], md.sg[k][1], md.b[k][0], md.b[k][1]);
        ccs[k] = md.cc[k];
    }
    const uint32_t T = sc.T;                              // threads in the grid: column stride
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    float *acc = sc.acc + gt;                             // [1 + 2 NF] rows: value, delta, vega
    const int nf = md.nf, nK = md.nK;
    const float l2e = 1.4426950408889634f, ln2 = 0.6931471805599453f;
    const float hl = md.h * l2e, sqhl = md.sqh * l2e, dl = md.dl, inv_dl = md.inv_dl;
    uint32_t u0, u1;
    unit_range(r, u0, u1);
    GenView gv;
    int staged_m = -1;
    for (uint32_t u = u0; u < u1; ++u) {
        const int m = (int)(u / r.tiles_per_m);
        const uint32_t tile = u % r.tiles_per_m;
        if (m != staged_m) {
            __syncthreads();
            stage_tables(g, m, smem_raw, gv);
            staged_m = m;
        }
        __syncthreads();
        for (int pp = 0; pp < r.ppt; ++pp) {
            const uint32_t i = tile * r.tile + (uint32_t)(pp * blockDim.x + threadIdx.x);
            const bool active = i < r.N;
            if (!__any_sync(0xffffffffu, active)) break;
            PathGen<SEQ> pg;
            pg.init(gv, active ? i : 0u);
            float X[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) X[k] = md.X0[k];
            float *st = sc.store + gt;
            // ---------------- forward sweep
            float disc = md.disc0, value = 0.0f;
            const int nblk = (nf + 7) >> 3;
            for (int b = 0; b < nblk; ++b) {
                const int ngrp = (nf - 8 * b + 7) >> 3;
                const float4 *cb = cst + 8 * b;
                const float *ccb = ccs + 8 * b;
                const int nst = min(8, nf - 8 * b);
                for (int tp = 0; tp < nst; ++tp) {
                    const int t = 8 * b + tp;
                    float Az[D], A[D];
#pragma unroll
                    for (int f = 0; f < D; ++f) {
                        Az[f] = sqhl * Draw<float>::normal(pg, t * D + f);
                        A[f] = 0.0f;
                    }
                    float Xpre = X[0];
                    switch (tp) {
#define RQMC_XP(k) \
    case (k):      \
        Xpre = X[(k)]; \
        break;
                        RQMC_XP(1) RQMC_XP(2) RQMC_XP(3) RQMC_XP(4) RQMC_XP(5) RQMC_XP(6) RQMC_XP(7)
#undef RQMC_XP
                        default:
                            break;
                    }
                    *st = Xpre;
                    st += T;
                    switch (tp) {
#define RQMC_G0(k)                                                                          \
    case (k):                                                                               \
        adj_fwd_update<D>(X[(k)], lds4(cb + (k)), ccb[(k)], A, Az, hl, st, T);
                        RQMC_G0(0) RQMC_G0(1) RQMC_G0(2) RQMC_G0(3) RQMC_G0(4) RQMC_G0(5) RQMC_G0(6) RQMC_G0(7)
#undef RQMC_G0
                        default:
                            break;
                    }
#pragma unroll
                    for (int gi = 1; gi < NF / 8; ++gi) {
                        if (gi < ngrp) {
#pragma unroll
                            for (int k = 0; k < 8; ++k)
                                adj_fwd_update<D>(X[8 * gi + k], lds4(cb + 8 * gi + k), ccb[8 * gi + k], A, Az, hl, st, T);
                        }
                    }
                    float Y = X[0];
                    switch (tp) {
#define RQMC_PK(k) \
    case (k):      \
        Y = X[(k)]; \
        break;
                        RQMC_PK(1) RQMC_PK(2) RQMC_PK(3) RQMC_PK(4) RQMC_PK(5) RQMC_PK(6) RQMC_PK(7)
#undef RQMC_PK
                        default:
                            break;
                    }
                    const float e = ex2_approx(Y);
                    disc *= rcp_approx(1.0f + e);
                    const float L = e * inv_dl;
                    float pn = 0.0f;
                    float *pr = acc + (size_t)(1 + 2 * NF + t * nK) * T;   // unweighted caplet prices
                    for (int kk = 0; kk < nK; ++kk) {
                        const float x = L - md.K[kk];
                        const float c = x > 0.0f ? dl * x * disc : 0.0f;
                        pn = fmaf(md.w[t][kk], c, pn);
                        if (active) pr[(size_t)kk * T] += c;
                    }
                    value += pn;
                }
#pragma unroll
                for (int k = 0; k + 8 < NF; ++k) X[k] = X[k + 8];
            }
            // ---------------- reverse sweep (X now holds the adjoints Xb); skipped for zero weights
            float Dcur = disc, G = 0.0f;
            const int nblk_rev = md.reverse ? nblk : 0;
#pragma unroll
            for (int k = 0; k < NF; ++k) X[k] = 0.0f;
            for (int b = nblk_rev - 1; b >= 0; --b) {
                if (b != nblk - 1) {
#pragma unroll
                    for (int k = NF - 1; k >= 8; --k) X[k] = X[k - 8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) X[k] = 0.0f;
                }
                const int ngrp = (nf - 8 * b + 7) >> 3;
                const float4 *cb = cst + 8 * b;
                const float *ccb = ccs + 8 * b;
                float *vg = acc + (size_t)(1 + NF + 8 * b) * T;   // vega column of original slot 8b
                const int nst = min(8, nf - 8 * b);
                for (int tp = nst - 1; tp >= 0; --tp) {
                    const int t = 8 * b + tp;
                    const int cnt = 8 * ngrp - tp;                // a-values stored at this step
                    st -= (size_t)(cnt + 1) * T;
                    const float Xpre = *st;
                    const float *sa = st + T;                     // a of shifted slot tp + q at sa[q T]
                    float Zs[D];
#pragma unroll
                    for (int f = 0; f < D; ++f) Zs[f] = Draw<float>::normal(pg, t * D + f);
                    // prefix total A over the updated slots
                    float Atot[D];
#pragma unroll
                    for (int f = 0; f < D; ++f) Atot[f] = 0.0f;
                    for (int q = 0; q < cnt; ++q) {
                        const float a = sa[(size_t)q * T];
                        const float4 c = lds4(cb + tp + q);
                        Atot[0] = fmaf(c.x, a, Atot[0]);
                        if constexpr (D == 2) Atot[1] = fmaf(c.y, a, Atot[1]);
                    }
                    // post-step value of the fixed forward (slot tp, first in the prefix),
                    // with the forward sweep's exact operations
                    const float4 c0 = lds4(cb + tp);
                    const float a0 = sa[0];
                    float inc = fmaf(c0.x, fmaf(fmaf(c0.x, a0, 0.0f), hl, sqhl * Zs[0]), ccb[tp]);
                    if constexpr (D == 2) inc = fmaf(c0.y, fmaf(fmaf(c0.y, a0, 0.0f), hl, sqhl * Zs[1]), inc);
                    const float Y = Xpre + inc;
                    const float e = ex2_approx(Y);
                    const float aY = e * rcp_approx(1.0f + e);
                    const float L = e * inv_dl;
                    float pn = 0.0f, dpn = 0.0f;   // sum w (L-K)^+ and sum w 1{L > K}, times delta below
                    for (int kk = 0; kk < nK; ++kk) {
                        const float x = L - md.K[kk];
                        if (x > 0.0f) {
                            pn = fmaf(md.w[t][kk], x, pn);
                            dpn += md.w[t][kk];
                        }
                    }
                    dpn *= dl;
                    G = fmaf(pn * dl, Dcur, G);
                    // an inactive lane (past N) follows a dummy path with zero adjoint source
                    const float ybar = active ? ln2 * (dpn * Dcur * L - aY * G) : 0.0f;
                    Dcur *= 1.0f + e;                             // D_{n-1} = D_n (1 + delta L_n)
                    // back through the step, slots from the last updated down to tp
                    float B[D], Ar[D];
#pragma unroll
                    for (int f = 0; f < D; ++f) {
                        B[f] = 0.0f;
                        Ar[f] = Atot[f];
                    }
                    auto back = [&](float &Xb, int q) {
                        const float a = sa[(size_t)q * T];
                        const float4 c = lds4(cb + tp + q);
                        B[0] = fmaf(Xb, c.x, B[0]);
                        float sB = c.x * B[0];
                        float sbar0 = l2e * fmaf(Xb, fmaf(md.h, Ar[0] - c.x, md.sqh * Zs[0]), md.h * a * B[0]);
                        float v = sbar0 * c.z;
                        Ar[0] = fmaf(-c.x, a, Ar[0]);
                        if constexpr (D == 2) {
                            B[1] = fmaf(Xb, c.y, B[1]);
                            sB = fmaf(c.y, B[1], sB);
                            const float sbar1 =
                                l2e * fmaf(Xb, fmaf(md.h, Ar[1] - c.y, md.sqh * Zs[1]), md.h * a * B[1]);
                            v = fmaf(sbar1, c.w, v);
                            Ar[1] = fmaf(-c.y, a, Ar[1]);
                        }
                        float *vq = vg + (size_t)(tp + q) * T;
                        *vq += v;
                        Xb = fmaf(md.h * sB, a * (1.0f - a), Xb);
                    };
#pragma unroll
                    for (int gi = NF / 8 - 1; gi >= 1; --gi) {
                        if (gi < ngrp) {
#pragma unroll
                            for (int k = 7; k >= 0; --k) back(X[8 * gi + k], 8 * gi + k - tp);
                        }
                    }
#pragma unroll
                    for (int k = 7; k >= 0; --k) {
                        if (k < tp) break;
                        if (k == tp) X[k] += ybar;                 // payoff adjoint of the fixed forward
                        back(X[k], k - tp);
                    }
                }
            }
            if (active) {
                acc[0] += value;
#pragma unroll
                for (int k = 0; k < NF; ++k)
                    if (k < nf) acc[(size_t)(1 + k) * T] += X[k] * md.invL0ln2[k];
            }
        }
        // ---------------- unit flush: sum the CTA's columns in double
        __syncthreads();
        const int nrow = 1 + 2 * nf + nf * nK;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        const uint32_t col0 = blockIdx.x * blockDim.x;
        for (int rw = warp; rw < nrow; rw += nw) {
            const int row = rw == 0 ? 0 : rw <= nf ? rw : rw <= 2 * nf ? 1 + NF + (rw - 1 - nf) : 1 + 2 * NF + (rw - 1 - 2 * nf);
            float *p = sc.acc + (size_t)row * T + col0;
            double s = 0.0;
            for (int c = lane; c < (int)blockDim.x; c += 32) {
                s += (double)p[c];
                p[c] = 0.0f;
            }
            s = warp_sum(s);
            if (lane == 0) r.partials[(size_t)u * nrow + rw] = s;
        }
        __syncthreads();
    }
}

}  // namespace rqmc

namespace rqmc {

template <int NF, int D, int SEQ>
static cudaError_t launch_adj_t(const Plan &pl, cudaStream_t st) {
    auto kern = lmm_adjoint_kernel<NF, D, SEQ>;
    size_t a, b;
    const size_t smem = adj_smem_layout<NF>(pl.gen, &a, &b);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<pl.grid, pl.threads, smem, st>>>(pl.gen, *pl.adjm, pl.adjs, pl.red);
    return cudaGetLastError();
}

template <int NF, int D, int SEQ>
static int grid_adj_t(const Plan &pl) {
    auto kern = lmm_adjoint_kernel<NF, D, SEQ>;
    size_t a, b;
    const size_t smem = adj_smem_layout<NF>(pl.gen, &a, &b);
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, pl.threads, smem);
    if (occ < 1) occ = 1;
    return (int)std::min<unsigned long long>(pl.red.units, (unsigned long long)occ * sms);
}

// mode 0: launch, mode 1: return the persistent grid size
template <int SEQ>
int adjoint_seq(const Plan &pl, cudaStream_t st, int mode) {
    const bool two = pl.adjm->d == 2;
    if (pl.nf_bucket == 40) {
        if (mode) return two ? grid_adj_t<40, 2, SEQ>(pl) : grid_adj_t<40, 1, SEQ>(pl);
        return (int)(two ? launch_adj_t<40, 2, SEQ>(pl, st) : launch_adj_t<40, 1, SEQ>(pl, st));
    }
    if (mode) return two ? grid_adj_t<80, 2, SEQ>(pl) : grid_adj_t<80, 1, SEQ>(pl);
    return (int)(two ? launch_adj_t<80, 2, SEQ>(pl, st) : launch_adj_t<80, 1, SEQ>(pl, st));
}

}  // namespace rqmc
