// k_adjoint.cuh -- pathwise adjoint of an LMM caplet strip (not in the paper; the model
// and the estimator are Sec. 5's), instantiated per sequence by k_adjoint_{halton,sobol,philox}.cu.
//
// Objective per path: V = sum_n sum_k w_{n,k} delta (L_n(T_n) - K_k)^+ D_n with the spot
// numeraire D_n = prod_{j<=n} (1 + delta L_j(T_j))^-1.  Forwards are carried as
// X_n = log2(delta L_n); one log-Euler step of slot n (d factors) is
//     a_n = 1 / (1 + 2^-X_n)               (= delta L_n / (1 + delta L_n))
//     A_n = sum_{j<=n, alive} sigma_j a_j   (d-vector prefix)
//     X_n += log2 e (h sigma_n.A_n + sqrt(h) sigma_n.Z - h |sigma_n|^2 / 2).
// Each thread keeps its path's X_n in a shared-memory column with a compile-time stride and
// loops over the alive forwards four slots (one chunk) at a time.  The forward sweep stores
// one record per step: the step's prefix total A (d floats).  The reverse sweep walks the
// alive slots of a step top-down and RECONSTRUCTS the pre-step state from the post-step one:
// with E = h A_n + sqrt(h) Z running down from the stored total (E -= h sigma_n a_n past
// slot n), the step's increment of slot n is log2 e sigma_n.E - h |sigma_n|^2 log2 e / 2, so
//     X_n(t) = X_n(t+1) - (log2 e sigma_n.E + cc_n),   a_n = 1 / (1 + 2^-X_n(t)),
// and the shared-memory column walks back from X(T) to X(0) (rounding moves it by about one
// ulp per step).  With Xb_n = dV/dX_n and B_n = sum_{m>=n} Xb_m sigma_m, the reverse step
// applies, top-down,
//     sigma_bar_n = log2 e [Xb_n (h A_n + sqrt(h) Z - h sigma_n) + h a_n B_n]
//     Xb_n       += h (sigma_n.B_n) a_n (1 - a_n)
// and at the fixing of forward n (Y = its post-step X, L = 2^Y / delta, G_n = sum_{m>=n} P_m)
//     Xb_n       += ln 2 [sum_k w_{n,k} delta 1{L > K_k} D_n L - a(Y) G_n].
// The adjoints Xb live in per-thread global columns (16-byte chunks, loaded two chunks ahead;
// the columns stay in L2; the two top chunks, first in every step, stay in registers across
// steps), the vega accumulators likewise, updated by vector reductions that
// the thread does not wait for.  The normals of a step are regenerated from the counter, never
// stored.  At the end dV/dL_n(0) = Xb_n / (L_n(0) ln 2) and dV/dvol_n = sum over steps of
// sigma_bar_n . b_n.  Per-thread value / delta / vega / price accumulators sit in global
// columns; each (replication, tile) unit sums its CTA's columns in double into its own row.
#pragma once
#include "paths_common.cuh"

namespace rqmc {

// Fire-and-forget vector reduction into global memory (no value returned, so the issuing
// thread never waits on it).  Each address is one thread's own column, and reductions from
// one thread to one address take effect in program order, so the sums are deterministic.
__device__ __forceinline__ void red_add_v4(float4 *p, const float (&v)[4]) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3])
                 : "memory");
}

// Threads per CTA.  Fixed, so that a thread's state column has a compile-time stride and
// every shared-memory access of the sweeps is an immediate offset from one pointer.
constexpr int kAdjThreads = kAdjointThreads;

// Shared memory: [generator stage][forward constants (sigma_1, sigma_2, cc, 0) x NF]
//                [reverse constants (h sigma_1, h sigma_2, b_1 log2 e, b_2 log2 e) x NF]
//                [reconstruction constants (sigma_1 log2 e, sigma_2 log2 e, cc, 0) x NF]
//                [per-thread state x NF x kAdjThreads]  (X)
template <int NF>
__host__ __device__ __forceinline__ size_t adj_smem_layout(const GenParams &g, size_t *o_fw, size_t *o_rv,
                                                           size_t *o_st) {
    size_t off = align16(stage_bytes(g));
    *o_fw = off;
    off += sizeof(float4) * NF;
    *o_rv = off;
    off += sizeof(float4) * 2 * NF;
    *o_st = off;
    off = align16(off + sizeof(float) * NF * (size_t)kAdjThreads);
    return off;
}

// The shared-memory state columns (NF floats per thread, 40 KB per 128-thread CTA at 80
// forwards) allow five CTAs per SM; the register budget that five CTAs leave (102 per thread)
// holds the kernel without spills.  Measured on the Greeks workload: 20 warps per SM at 128
// threads per CTA ran 5 % faster than 16 warps at 256.
#ifndef RQMC_ADJ_MIN_BLOCKS
#define RQMC_ADJ_MIN_BLOCKS 5
#endif

// ZG: the normals are read from zg ([M][D nf][N], written beforehand by the point-stream run
// kernel from the plan's generator, one step ahead of their use) instead of generated; g.stage
// is then 0 and no generator table is staged.
template <int NF, int D, int SEQ, bool ZG = false>
__global__ void __launch_bounds__(kAdjThreads, RQMC_ADJ_MIN_BLOCKS)
    lmm_adjoint_kernel(const GenParams g, const AdjModel md, const AdjScratch sc, const RedParams r,
                       const float *__restrict__ zg) {
    constexpr int BD = kAdjThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    size_t o_fw, o_rv, o_st;
    adj_smem_layout<NF>(g, &o_fw, &o_rv, &o_st);
    float4 *cfw = reinterpret_cast<float4 *>(smem_raw + o_fw);
    float4 *crv = reinterpret_cast<float4 *>(smem_raw + o_rv);
    float4 *crc = crv + NF;
    float *xcol = reinterpret_cast<float *>(smem_raw + o_st) + threadIdx.x;   // slot n at xcol[n BD]
    const float l2e = 1.4426950408889634f, ln2 = 0.6931471805599453f;
    for (int k = threadIdx.x; k < NF; k += BD) {
        cfw[k] = make_float4(md.sg[k][0], md.sg[k][1], md.cc[k], 0.0f);
        crv[k] = make_float4(md.h * md.sg[k][0], md.h * md.sg[k][1], md.b[k][0] * l2e, md.b[k][1] * l2e);
        crc[k] = make_float4(md.sg[k][0] * l2e, md.sg[k][1] * l2e, md.cc[k], 0.0f);
    }
    const uint32_t T = sc.T;                              // threads in the grid: column stride
    const uint32_t gt = blockIdx.x * BD + threadIdx.x;
    // accumulators: vega as float4 chunks [NF/4][T], then value [T], delta [NF][T], prices [nf nK][T]
    float4 *const vega4 = reinterpret_cast<float4 *>(sc.acc) + gt;
    float *accs = sc.acc + (size_t)NF * T + gt;
    float4 *const xb4 = reinterpret_cast<float4 *>(sc.xb) + gt;   // adjoints Xb as float4 chunks [NF/4][T]
    float2 *const rec = reinterpret_cast<float2 *>(sc.store) + gt; // per step t: prefix total A at rec[t T]
    const int nf = md.nf, nK = md.nK, nch = (nf + 3) >> 2;
    const float h = md.h, inv_h = 1.0f / md.h, hl = md.h * l2e, sqhl = md.sqh * l2e, dl = md.dl, inv_dl = md.inv_dl;
    uint32_t u0, u1;
    unit_range(r, u0, u1);
    GenView gv;
    int staged_m = -1;
    for (uint32_t u = u0; u < u1; ++u) {
        const int m = (int)(u / r.tiles_per_m);
        const uint32_t tile = u % r.tiles_per_m;
        if (m != staged_m) {
            __syncthreads();
            if constexpr (ZG) view_tables(g, m, gv);
            else stage_tables(g, m, smem_raw, gv);
            staged_m = m;
        }
        __syncthreads();
        for (int pp = 0; pp < r.ppt; ++pp) {
            const uint32_t i = tile * r.tile + (uint32_t)(pp * BD + threadIdx.x);
            const bool active = i < r.N;
            if (!__any_sync(0xffffffffu, active)) break;
            PathGen<SEQ> pg;
            pg.init(gv, active ? i : 0u);
            // loaded normals of step t: dims D t, D t + 1 of this path's column
            const float *zrow = ZG ? zg + (size_t)m * (size_t)(D * nf) * r.N + pg.i : nullptr;
            auto zload = [&](int t, float &a, float &b) {
                a = zrow[(size_t)(D * t) * r.N];
                b = D == 2 ? zrow[(size_t)(D * t + 1) * r.N] : 0.0f;
            };
            float zn0 = 0.0f, zn1 = 0.0f;
            if constexpr (ZG) zload(0, zn0, zn1);
            // slots nf .. 4 nch - 1 are padding with zero volatility: they stay constant and feed
            // nothing into the drifts, the adjoints or the vegas, so full chunks need no checks
            for (int n = 0; n < 4 * nch; ++n) xcol[n * BD] = md.X0[n];
            // ---------------- forward sweep
            float disc = md.disc0, value = 0.0f;
            for (int t = 0; t < nf; ++t) {
                float Az0, Az1 = 0.0f, A0 = 0.0f, A1 = 0.0f;
                if constexpr (ZG) {
                    Az0 = sqhl * zn0;
                    Az1 = sqhl * zn1;
                    if (t + 1 < nf) zload(t + 1, zn0, zn1);
                } else if constexpr (D == 2) {
                    float z0, z1;
                    normals32_two_dims<SEQ>(pg, 2 * t, 2 * t + 1, z0, z1);
                    Az0 = sqhl * z0;
                    Az1 = sqhl * z1;
                } else {
                    Az0 = sqhl * Draw<float>::normal(pg, t);
                }
                // one chunk of four slots; slots below jlo are fixed forwards.  All loads come
                // before the stores, so the four exponentials overlap.
                auto fwd_chunk = [&](int c, int jlo) {
                    float *px = xcol + c * (4 * BD);
                    const float4 *pc = cfw + 4 * c;
                    float X[4], a[4];
                    float4 cn[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        X[j] = px[j * BD];
                        cn[j] = pc[j];
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) a[j] = j >= jlo ? rcp_approx(1.0f + ex2_approx(-X[j])) : 0.0f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (j >= jlo) {
                            A0 = fmaf(cn[j].x, a[j], A0);
                            float inc = fmaf(cn[j].x, fmaf(A0, hl, Az0), cn[j].z);
                            if constexpr (D == 2) {
                                A1 = fmaf(cn[j].y, a[j], A1);
                                inc = fmaf(cn[j].y, fmaf(A1, hl, Az1), inc);
                            }
                            px[j * BD] = X[j] + inc;
                        }
                    }
                };
                fwd_chunk(t >> 2, t & 3);
                for (int c = (t >> 2) + 1; c < nch; ++c) fwd_chunk(c, 0);
                rec[(size_t)t * T] = make_float2(A0, A1);
                const float e = ex2_approx(xcol[t * BD]);
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
            // ---------------- reverse sweep (skipped for zero weights): xcol walks back to X(0),
            // the adjoints accumulate in the thread's global columns
            for (int c = 0; c < nch; ++c) xb4[(size_t)c * T] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float Dcur = disc, G = 0.0f;
            // the two top chunks (nch-1, nch-2) are processed first in every step: their values
            // carry over in registers; the others are loaded two chunks ahead from the columns
            float4 top0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), top1 = top0;
            float2 At_next = md.reverse ? rec[(size_t)(nf - 1) * T] : make_float2(0.0f, 0.0f);
            if constexpr (ZG) {
                if (md.reverse) zload(nf - 1, zn0, zn1);
            }
            for (int t = md.reverse ? nf - 1 : -1; t >= 0; --t) {
                const int c0 = t >> 2, jt = t & 3;
                const float2 At = At_next;
                if (t > 0) At_next = rec[(size_t)(t - 1) * T];   // one step ahead
                const float4 *q = xb4 + (ptrdiff_t)(nch - 3) * (ptrdiff_t)T;   // chunk nch-3 (read only when it exists)
                float4 p0 = top0;
                float4 p1 = nch - 2 >= c0 ? top1 : top0;
                float Z0, Z1 = 0.0f;
                if constexpr (ZG) {
                    Z0 = zn0;
                    Z1 = zn1;
                    if (t > 0) zload(t - 1, zn0, zn1);
                } else if constexpr (D == 2) {
                    normals32_two_dims<SEQ>(pg, 2 * t, 2 * t + 1, Z0, Z1);
                } else {
                    Z0 = Draw<float>::normal(pg, t);
                }
                // the fixed forward's post-step value is the column's current value
                const float Y = xcol[t * BD];
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
                const float src = active ? ln2 * (dpn * dl * Dcur * L - aY * G) : 0.0f;
                Dcur *= 1.0f + e;                             // D_{n-1} = D_n (1 + delta L_n)
                // top-down over the alive slots n: E = h A_n + sqrt(h) Z (A_n the step's prefix
                // sum through n) and hB = h B_n = h sum_{m>=n} Xb_m sigma_m, per factor; the
                // update of Xb_n is h (sigma.B) a (1 - a) = (h sigma . hB) a (1 - a) / h
                float E0 = fmaf(h, At.x, md.sqh * Z0), E1 = fmaf(h, At.y, md.sqh * Z1);
                float hB0 = 0.0f, hB1 = 0.0f;
                float4 *vg = vega4 + (size_t)(nch - 1) * T;
                auto rev_chunk = [&](int c, int jlo, float4 xb) {
                    float *px = xcol + c * (4 * BD);
                    const float4 *pc = crv + 4 * c;
                    const float4 *pq = crc + 4 * c;
                    float Xb[4] = {xb.x, xb.y, xb.z, xb.w}, vv[4], Xp[4];
                    float4 cn[4], cr[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        Xp[j] = px[j * BD];
                        cn[j] = pc[j];
                        cr[j] = pq[j];
                    }
#pragma unroll
                    for (int j = 3; j >= 0; --j) {
                        vv[j] = 0.0f;
                        if (j >= jlo) {
                            // pre-step state of slot n and its drift factor a_n
                            float inc = fmaf(cr[j].x, E0, cr[j].z);
                            if constexpr (D == 2) inc = fmaf(cr[j].y, E1, inc);
                            const float Xn = Xp[j] - inc;
                            const float a = rcp_approx(1.0f + ex2_approx(-Xn));
                            px[j * BD] = Xn;
                            // sigma_bar = Xb (h (A_n - sigma_n) + sqrt(h) Z) + h a_n B_n, per factor
                            hB0 = fmaf(Xb[j], cn[j].x, hB0);
                            float S = cn[j].x * hB0;              // h^2 sigma.B
                            float v = cn[j].z * fmaf(Xb[j], E0 - cn[j].x, a * hB0);
                            E0 = fmaf(-cn[j].x, a, E0);
                            if constexpr (D == 2) {
                                hB1 = fmaf(Xb[j], cn[j].y, hB1);
                                S = fmaf(cn[j].y, hB1, S);
                                v = fmaf(cn[j].w, fmaf(Xb[j], E1 - cn[j].y, a * hB1), v);
                                E1 = fmaf(-cn[j].y, a, E1);
                            }
                            vv[j] = v;
                            Xb[j] = fmaf(S, inv_h * fmaf(-a, a, a), Xb[j]);   // + h (sigma.B) a (1 - a)
                        }
                    }
                    const float4 nv = make_float4(Xb[0], Xb[1], Xb[2], Xb[3]);
                    xb4[(size_t)c * T] = nv;
                    if (c == nch - 1) top0 = nv;
                    if (c == nch - 2) top1 = nv;
                    red_add_v4(vg, vv);
                    vg -= T;
                };
                for (int c = nch - 1; c > c0; --c) {
                    const float4 xb = p0;
                    p0 = p1;
                    if (c - 2 >= c0) {
                        p1 = *q;
                        q -= T;
                    }
                    rev_chunk(c, 0, xb);
                }
                // the fixing's source enters the fixed forward's adjoint before its chunk
                p0.x += jt == 0 ? src : 0.0f;
                p0.y += jt == 1 ? src : 0.0f;
                p0.z += jt == 2 ? src : 0.0f;
                p0.w += jt == 3 ? src : 0.0f;
                rev_chunk(c0, jt, p0);
            }
            if (active) {
                atomicAdd(accs, value);
                for (int c = 0; c < nch; ++c) {
                    const float4 xb = xb4[(size_t)c * T];
                    const float xs[4] = {xb.x, xb.y, xb.z, xb.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int n = 4 * c + j;
                        if (n < nf) atomicAdd(accs + (size_t)(1 + n) * T, xs[j] * md.invL0ln2[n]);
                    }
                }
            }
        }
        // ---------------- unit flush: sum the CTA's columns in double
        __syncthreads();
        const int nrow = 1 + 2 * nf + nf * nK;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = BD >> 5;
        const uint32_t col0 = blockIdx.x * BD;
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
            for (int c = lane; c < BD; c += 32) {
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

template <int NF, int D, int SEQ, bool ZG = false>
static cudaError_t launch_adj_t(const Plan &pl, cudaStream_t st) {
    auto kern = lmm_adjoint_kernel<NF, D, SEQ, ZG>;
    GenParams g = pl.gen;
    if (ZG) g.stage = 0;   // no generator table is read
    size_t a, b, c;
    const size_t smem = adj_smem_layout<NF>(g, &a, &b, &c);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<pl.grid, kAdjThreads, smem, st>>>(g, *pl.adjm, pl.adjs, pl.red,
                                             ZG ? static_cast<const float *>(pl.znorm) : nullptr);
    return cudaGetLastError();
}

template <int NF, int D, int SEQ, bool ZG = false>
static int grid_adj_t(const Plan &pl, int mode) {
    auto kern = lmm_adjoint_kernel<NF, D, SEQ, ZG>;
    GenParams g = pl.gen;
    if (ZG) g.stage = 0;
    size_t a, b, c;
    const size_t smem = adj_smem_layout<NF>(g, &a, &b, &c);
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kAdjThreads, smem);
    if (occ < 1) occ = 1;
    return (int)std::min<unsigned long long>(pl.red.units, (unsigned long long)occ * sms);
}

// mode 0: launch, mode 1: return the persistent grid size
// ZG: the kernels that read pl.znorm (one set for every sequence, instantiated only by
// k_adjoint_loaded.cu)
template <int SEQ, bool ZG = false>
int adjoint_seq(const Plan &pl, cudaStream_t st, int mode) {
    const bool two = pl.adjm->d == 2;
    if (pl.nf_bucket == 40) {
        if (mode) return two ? grid_adj_t<40, 2, SEQ, ZG>(pl, mode) : grid_adj_t<40, 1, SEQ, ZG>(pl, mode);
        return (int)(two ? launch_adj_t<40, 2, SEQ, ZG>(pl, st) : launch_adj_t<40, 1, SEQ, ZG>(pl, st));
    }
    if (mode) return two ? grid_adj_t<80, 2, SEQ, ZG>(pl, mode) : grid_adj_t<80, 1, SEQ, ZG>(pl, mode);
    return (int)(two ? launch_adj_t<80, 2, SEQ, ZG>(pl, st) : launch_adj_t<80, 1, SEQ, ZG>(pl, st));
}

}  // namespace rqmc
