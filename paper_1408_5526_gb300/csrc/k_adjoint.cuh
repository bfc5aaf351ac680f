// k_adjoint.cuh -- pathwise adjoint of an LMM caplet strip (not in the paper; the model
// and the estimator are Sec. 5's), instantiated per sequence by k_adjoint_{halton,sobol,philox}.cu.
//
// Objective per path: V = sum_n sum_k w_{n,k} delta (L_n(T_n) - K_k)^+ D_n with the spot
// numeraire D_n = prod_{j<=n} (1 + delta L_j(T_j))^-1.  Forwards live in registers as
// X_n = log2(delta L_n); one log-Euler step of slot n (d factors) is
//     a_n = 1 / (1 + 2^-X_n)               (= delta L_n / (1 + delta L_n))
//     A_n = sum_{j<=n, alive} sigma_j a_j   (d-vector prefix)
//     X_n += log2 e (h sigma_n.A_n + sqrt(h) sigma_n.Z - h |sigma_n|^2 / 2).
// Each thread keeps its path's X_n (then the adjoints) in a shared-memory column and loops
// over the alive forwards with rolled loops, so the code stays small and about 60
// registers give ~20 warps per SM.  The forward sweep stores, per step, a header (the
// pre-step X of the forward fixed at that step, the step's prefix total A) and the a_n in
// 16-byte chunks aligned to absolute forward slots, interleaved by thread in global scratch:
// one coalesced 128-bit store (and, in the reverse sweep, one 128-bit load) per four
// forwards.  The vega accumulators use the same chunking.  Reverse sweep: with
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

// Shared memory: [generator stage][(sigma_1, sigma_2, b_1, b_2) x NF][cc x NF]
//                [per-thread state x NF x blockDim]  (forward X, then the adjoints Xb)
template <int NF>
__host__ __device__ __forceinline__ size_t adj_smem_layout(const GenParams &g, int threads, size_t *o_cst,
                                                           size_t *o_cc, size_t *o_st) {
    size_t off = align16(stage_bytes(g));
    *o_cst = off;
    off = align16(off + sizeof(float4) * NF);
    *o_cc = off;
    off = align16(off + sizeof(float) * NF);
    *o_st = off;
    off = align16(off + sizeof(float) * NF * (size_t)threads);
    return off;
}

// Resident CTAs per SM that the register budget must allow: the shared-memory state columns
// limit residency to 2 CTAs of 256 threads (4 of 128) for the staged sequences anyway, so up
// to 128 registers cost no occupancy and let the unrolled chunk code keep its loads in flight.
#ifndef RQMC_ADJ_MIN_BLOCKS
#define RQMC_ADJ_MIN_BLOCKS 2
#endif

template <int NF, int D, int SEQ>
__global__ void __launch_bounds__(256, RQMC_ADJ_MIN_BLOCKS) lmm_adjoint_kernel(const GenParams g, const AdjModel md, const AdjScratch sc,
                                                         const RedParams r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    size_t o_cst, o_cc, o_st;
    adj_smem_layout<NF>(g, blockDim.x, &o_cst, &o_cc, &o_st);
    float4 *cst = reinterpret_cast<float4 *>(smem_raw + o_cst);
    float *ccs = reinterpret_cast<float *>(smem_raw + o_cc);
    float *xs = reinterpret_cast<float *>(smem_raw + o_st) + threadIdx.x;   // slot n at xs[n * blockDim]
    const int bd = blockDim.x;
    for (int k = threadIdx.x; k < NF; k += blockDim.x) {
        cst[k] = make_float4(md.sg[k][0], md.sg[k][1], md.b[k][0], md.b[k][1]);
        ccs[k] = md.cc[k];
    }
    const uint32_t T = sc.T;                              // threads in the grid: column stride
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    // accumulators: vega as float4 chunks [NF/4][T], then value [T], delta [NF][T], prices [nf nK][T]
    float4 *__restrict__ vega4 = reinterpret_cast<float4 *>(sc.acc) + gt;
    float *accs = sc.acc + (size_t)NF * T + gt;
    const int nf = md.nf, nK = md.nK, nch = (nf + 3) >> 2;
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
            // slots nf .. 4 nch - 1 are padding with zero volatility: they stay constant and feed
            // nothing into the drifts, the adjoints or the vegas, so full chunks need no checks
            for (int n = 0; n < 4 * nch; ++n) xs[n * bd] = md.X0[n];
            // records, in float4 units: per step a header (X of the fixed forward, the step's
            // prefix total A) and the a_n of chunks t/4 .. nch-1 (absolute slots, dead slots 0)
            float4 *__restrict__ rec = reinterpret_cast<float4 *>(sc.store) + gt;
            // ---------------- forward sweep
            float disc = md.disc0, value = 0.0f;
            for (int t = 0; t < nf; ++t) {
                float Az[D], A[D];
#pragma unroll
                for (int f = 0; f < D; ++f) {
                    Az[f] = sqhl * Draw<float>::normal(pg, t * D + f);
                    A[f] = 0.0f;
                }
                const float Xpre = xs[t * bd];
                float4 *hdr = rec;
                rec += T;
                // one chunk of four slots, slots below jlo are fixed forwards (a = 0)
                auto fwd_chunk = [&](int c, int jlo) {
                    float av[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int n = 4 * c + j;
                        av[j] = 0.0f;
                        if (j >= jlo) {
                            const float4 cn = cst[n];
                            const float X = xs[n * bd];
                            const float a = rcp_approx(1.0f + ex2_approx(-X));
                            av[j] = a;
                            A[0] = fmaf(cn.x, a, A[0]);
                            float inc = fmaf(cn.x, fmaf(A[0], hl, Az[0]), ccs[n]);
                            if constexpr (D == 2) {
                                A[1] = fmaf(cn.y, a, A[1]);
                                inc = fmaf(cn.y, fmaf(A[1], hl, Az[1]), inc);
                            }
                            xs[n * bd] = X + inc;
                        }
                    }
                    *rec = make_float4(av[0], av[1], av[2], av[3]);
                    rec += T;
                };
                fwd_chunk(t >> 2, t & 3);
                for (int c = (t >> 2) + 1; c < nch; ++c) fwd_chunk(c, 0);
                *hdr = make_float4(Xpre, A[0], D == 2 ? A[1] : 0.0f, 0.0f);
                const float e = ex2_approx(xs[t * bd]);
                disc *= rcp_approx(1.0f + e);
                const float L = e * inv_dl;
                float pn = 0.0f;
                float *pr = accs + (size_t)(1 + NF + t * nK) * T;   // unweighted caplet prices
                for (int kk = 0; kk < nK; ++kk) {
                    const float x = L - md.K[kk];
                    const float cpl = x > 0.0f ? dl * x * disc : 0.0f;
                    pn = fmaf(md.w[t][kk], cpl, pn);
                    if (active) atomicAdd(pr + (size_t)kk * T, cpl);   // own column: a plain reduction
                }
                value += pn;
            }
            // ---------------- reverse sweep (xs now holds the adjoints Xb); skipped for zero weights
            for (int n = 0; n < 4 * nch; ++n) xs[n * bd] = 0.0f;
            float Dcur = disc, G = 0.0f;
            for (int t = md.reverse ? nf - 1 : -1; t >= 0; --t) {
                const int c0 = t >> 2;
                rec -= (size_t)(1 + nch - c0) * T;
                const float4 h4 = rec[0];
                const float4 *__restrict__ ch = rec + T;      // chunk c at ch[(c - c0) T]
                // software pipeline: the next chunk's a_n and vega are loaded one chunk ahead
                float4 a4n = ch[(size_t)(nch - 1 - c0) * T];
                float4 v4n = vega4[(size_t)(nch - 1) * T];
                float Ar[D], Zs[D];
                Ar[0] = h4.y;
                if constexpr (D == 2) Ar[1] = h4.z;
#pragma unroll
                for (int f = 0; f < D; ++f) Zs[f] = Draw<float>::normal(pg, t * D + f);
                // post-step value of the fixed forward, with the forward sweep's operations
                const float4 ct = cst[t];
                const float4 ac = ch[0];
                const float a0 = (t & 3) == 0 ? ac.x : (t & 3) == 1 ? ac.y : (t & 3) == 2 ? ac.z : ac.w;
                float inc = fmaf(ct.x, fmaf(fmaf(ct.x, a0, 0.0f), hl, sqhl * Zs[0]), ccs[t]);
                if constexpr (D == 2) inc = fmaf(ct.y, fmaf(fmaf(ct.y, a0, 0.0f), hl, sqhl * Zs[1]), inc);
                const float Y = h4.x + inc;
                const float e = ex2_approx(Y);
                const float aY = e * rcp_approx(1.0f + e);
                const float L = e * inv_dl;
                float pn = 0.0f, dpn = 0.0f;   // sum w (L-K)^+ and sum w 1{L > K}
                for (int kk = 0; kk < nK; ++kk) {
                    const float x = L - md.K[kk];
                    if (x > 0.0f) {
                        pn = fmaf(md.w[t][kk], x, pn);
                        dpn += md.w[t][kk];
                    }
                }
                G = fmaf(pn * dl, Dcur, G);
                // an inactive lane (past N) follows a dummy path with zero adjoint source
                xs[t * bd] += active ? ln2 * (dpn * dl * Dcur * L - aY * G) : 0.0f;
                Dcur *= 1.0f + e;                             // D_{n-1} = D_n (1 + delta L_n)
                float B[D];
#pragma unroll
                for (int f = 0; f < D; ++f) B[f] = 0.0f;
                auto rev_chunk = [&](int c, int jlo, const float4 a4, const float4 v4) {
                    const float aa[4] = {a4.x, a4.y, a4.z, a4.w};
                    float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                    for (int j = 3; j >= 0; --j) {
                        const int n = 4 * c + j;
                        if (j >= jlo) {
                            const float a = aa[j];
                            const float4 cn = cst[n];
                            const float Xb = xs[n * bd];
                            B[0] = fmaf(Xb, cn.x, B[0]);
                            float sB = cn.x * B[0];
                            float v = cn.z * l2e * fmaf(Xb, fmaf(md.h, Ar[0] - cn.x, md.sqh * Zs[0]), md.h * a * B[0]);
                            Ar[0] = fmaf(-cn.x, a, Ar[0]);
                            if constexpr (D == 2) {
                                B[1] = fmaf(Xb, cn.y, B[1]);
                                sB = fmaf(cn.y, B[1], sB);
                                v = fmaf(cn.w * l2e, fmaf(Xb, fmaf(md.h, Ar[1] - cn.y, md.sqh * Zs[1]), md.h * a * B[1]), v);
                                Ar[1] = fmaf(-cn.y, a, Ar[1]);
                            }
                            vv[j] += v;
                            xs[n * bd] = fmaf(md.h * sB, a * (1.0f - a), Xb);
                        }
                    }
                    vega4[(size_t)c * T] = make_float4(vv[0], vv[1], vv[2], vv[3]);
                };
                for (int c = nch - 1; c > c0; --c) {
                    const float4 a4 = a4n, v4 = v4n;
                    a4n = ch[(size_t)(c - 1 - c0) * T];
                    v4n = vega4[(size_t)(c - 1) * T];
                    rev_chunk(c, 0, a4, v4);
                }
                rev_chunk(c0, t & 3, a4n, v4n);
            }
            if (active) {
                atomicAdd(accs, value);
                for (int n = 0; n < nf; ++n) atomicAdd(accs + (size_t)(1 + n) * T, xs[n * bd] * md.invL0ln2[n]);
            }
        }
        // ---------------- unit flush: sum the CTA's columns in double
        __syncthreads();
        const int nrow = 1 + 2 * nf + nf * nK;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        const uint32_t col0 = blockIdx.x * blockDim.x;
        for (int rw = warp; rw < nrow; rw += nw) {
            // output row rw: value, delta_n, vega_n, prices; columns of this CTA's threads
            float *p;
            int cs;   // float stride between consecutive threads
            if (rw == 0) { p = sc.acc + (size_t)NF * T + col0; cs = 1; }
            else if (rw <= nf) { p = sc.acc + (size_t)(NF + rw) * T + col0; cs = 1; }
            else if (rw <= 2 * nf) {
                const int n = rw - 1 - nf;
                p = sc.acc + ((size_t)(n >> 2) * T + col0) * 4 + (n & 3);
                cs = 4;
            } else { p = sc.acc + (size_t)(NF + 1 + NF + (rw - 1 - 2 * nf)) * T + col0; cs = 1; }
            double s = 0.0;
            for (int c = lane; c < (int)blockDim.x; c += 32) {
                s += (double)__ldcg(p + (size_t)c * cs);   // from L2: the columns were reduced there
                p[(size_t)c * cs] = 0.0f;
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
    size_t a, b, c;
    const size_t smem = adj_smem_layout<NF>(pl.gen, pl.threads, &a, &b, &c);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<pl.grid, pl.threads, smem, st>>>(pl.gen, *pl.adjm, pl.adjs, pl.red);
    return cudaGetLastError();
}

template <int NF, int D, int SEQ>
static int grid_adj_t(const Plan &pl, int mode) {
    auto kern = lmm_adjoint_kernel<NF, D, SEQ>;
    size_t a, b, c;
    const size_t smem = adj_smem_layout<NF>(pl.gen, pl.threads, &a, &b, &c);
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, pl.threads, smem);
    if (mode == 2) return occ;
    if (occ < 1) occ = 1;
    return (int)std::min<unsigned long long>(pl.red.units, (unsigned long long)occ * sms);
}

// mode 0: launch, mode 1: return the persistent grid size, mode 2: resident CTAs per SM
template <int SEQ>
int adjoint_seq(const Plan &pl, cudaStream_t st, int mode) {
    const bool two = pl.adjm->d == 2;
    if (pl.nf_bucket == 40) {
        if (mode) return two ? grid_adj_t<40, 2, SEQ>(pl, mode) : grid_adj_t<40, 1, SEQ>(pl, mode);
        return (int)(two ? launch_adj_t<40, 2, SEQ>(pl, st) : launch_adj_t<40, 1, SEQ>(pl, st));
    }
    if (mode) return two ? grid_adj_t<80, 2, SEQ>(pl, mode) : grid_adj_t<80, 1, SEQ>(pl, mode);
    return (int)(two ? launch_adj_t<80, 2, SEQ>(pl, st) : launch_adj_t<80, 1, SEQ>(pl, st));
}

}  // namespace rqmc
