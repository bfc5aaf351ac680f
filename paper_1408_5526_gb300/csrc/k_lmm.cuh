// k_lmm.cuh -- fused LIBOR-market-model caplet kernel (Sec. 5), instantiated per sequence
// by k_lmm_halton.cu, k_lmm_sobol.cu and k_lmm_philox.cu.
//
// One thread = one path of one replication.  Per time step t (grid t_i = T_i, h = delta):
// coordinate t of the point (Halton/Rasrap digits, Sobol', or Philox) -> Phi^-1 -> one
// log-Euler step of every alive forward under the spot measure,
//     log L_n += sigma_n (h mu'_n + sqrt(h) Z) - sigma_n^2 h / 2,
//     mu'_n = sum_{j=eta}^{n} sigma_j delta L_j / (1 + delta L_j)   (a running prefix),
// then L_{t+1}(T_{t+1}) is fixed, the spot numeraire is advanced by (1 + delta L_{t+1}) and
// the caplet payoffs delta (L_{t+1} - K)^+ / prod_{j<=t+1}(1 + delta L_j(T_j)) are staged
// for the warp reduction.
//
// Layout: the forwards live in registers as X_n = log(delta L_n) (base 2 in FP32).  Within
// a step the drift is carried as W_n = h mu'_n + sqrt(h) Z (in log2 units), so one forward
// costs ex2 + rcp + 4 FP32 ops: a = 1 / (1 + 2^-X), W += (h sigma_n) a, X += sigma_n W + cc_n.
// FP32 strips of up to 40 forwards drop the + cc_n: they carry X~_n = X_n - t cc_n and read,
// per step t and forward n, the constant g = 2^(-t cc_n) from a table, so that 1 + 2^-X =
// 1 + g 2^-X~ is one FMA.  In FP32 the factor h sigma_n is folded into the denominator,
// d' = (1 + g 2^-X~) / (h sigma_n) = G 2^-X~ + H with the constants G = g / (h sigma_n) and
// H = 1 / (h sigma_n), so that the drift term h sigma_n a_n is 1/d'.  Two lockstep paths share
// one reciprocal, 1/d0' = d1' / (d0' d1') and 1/d1' = d0' / (d0' d1'): per forward and pair of
// paths two ex2, one rcp and seven FP32 operations.  Single-path strips (80 and 160 forwards)
// pair adjacent forwards the same way outside the first group of a block.  Forward n sits in slot n-1 of an
// NF-slot array (NF = 16/40/80/160).  Steps run in blocks of 8; after each block the
// array shifts down by 8 slots, so at step tp of a block the alive slots are tp..7 of
// group 0 (entered through an 8-way fall-through switch) plus whole groups of 8 that a
// uniform test skips once they are dead.  The code holds NF update bodies, not NF^2/2.
// Per-forward constants (sigma_n, h sigma_n, -sigma_n^2 h/2 or g, in log2 units) come from
// shared memory as one 16-byte (FP32) load shared by the thread's paths.  Payoffs are written to a padded per-warp transpose buffer and summed
// once per block (lane r sums row r), then added to the warp's Kahan accumulator.
#pragma once
#include "paths_common.cuh"

namespace rqmc {

template <typename T>
struct LmmMath;
// ld.shared of one forward's constants at the point of use (volatile: the compiler
// must not hoist the 2 x NF constants of a block into registers).
// Per-forward constants: x = sigma_n, y = h sigma_n (h in the state's log units), z = cc_n.
struct LmmC64 {
    double x, y, z, w;
};
template <>
struct LmmMath<float> {
    using C = float4;
    static constexpr int PAD = 36;   // row stride of the transpose buffer (conflict-free 16-byte reads)
    static __device__ __forceinline__ float expb(float x) { return ex2_approx(x); }
    static __device__ __forceinline__ float rcp(float x) { return rcp_approx(x); }
    static __device__ __forceinline__ float4 lds(const float4 *p) {
        float4 v;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "r"((unsigned)__cvta_generic_to_shared(p)));
        return v;
    }
    static __device__ __forceinline__ float2 lds2(const float2 *p) {
        float2 v;
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y)
                     : "r"((unsigned)__cvta_generic_to_shared(p)));
        return v;
    }
};
template <>
struct LmmMath<double> {
    using C = LmmC64;
    static constexpr int PAD = 34;
    static __device__ __forceinline__ double expb(double x) { return exp(x); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ LmmC64 lds(const LmmC64 *p) {
        LmmC64 v;
        const unsigned a = (unsigned)__cvta_generic_to_shared(p);
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
        asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v.z) : "r"(a + 16));
        v.w = 0.0;
        return v;
    }
};

// FP32 strips of up to 40 forwards use the per-(step, forward) constant table (g-table).
template <int NF, typename T>
__host__ __device__ constexpr bool lmm_gtab() {
    return sizeof(T) == 4 && NF <= 40;
}
// FP32 strips of 80 and 160 forwards (one path per thread) use the pair table: per pair q of
// adjacent slots (2q, 2q + 1) the static (sigma, H, sigma, H) as one float4, per step t and pair
// the (G, G) of the two slots as one float2, and per step the fixing factor 2^((t+1) cc_t).
template <int NF, typename T>
__host__ __device__ constexpr bool lmm_ptab() {
    return sizeof(T) == 4 && NF > 40;
}

// The folded drift constant H = 1 / (h sigma_n); a zero (or vanishing) h sigma_n is replaced by
// 2^-40 of the same sign, whose drift term h sigma_n a_n <= 2^-40 is far below the FP32
// rounding of W, so that d' and the product of a pair of them stay finite.
__host__ __device__ __forceinline__ float lmm_fold_inv(float hs) {
    const float m = 9.094947e-13f;   // 2^-40
    return 1.0f / (fabsf(hs) < m ? copysignf(m, hs) : hs);
}

// One forward of one path.  FP64: c = (sigma, h sigma, cc, 0), X the log-forward.  FP32 (g-table):
// c = (sigma, G, H, 2^(t cc)) and X = X~ (see the header: the drift term is 1/d').
template <bool GT, typename T>
__device__ __forceinline__ void lmm_update(T &X, const typename LmmMath<T>::C c, T &W) {
    const T e = LmmMath<T>::expb(-X);
    if constexpr (sizeof(T) == 4) {
        static_assert(GT, "FP32 log-Euler strips read the g-table or the pair table");
        W += LmmMath<T>::rcp(fmaT(e, c.y, c.z));   // h sigma delta L / (1 + delta L)
        X = fmaT(c.x, W, X);
    } else {
        const T a = LmmMath<T>::rcp(T(1) + e);   // delta L / (1 + delta L), old L
        W = fmaT(c.y, a, W);                     // drift through j = n
        X = fmaT(c.x, W, X) + c.z;
    }
}

// One forward of one path under the Euler scheme (eq. L_n_discrete), X = delta L:
// a = X / (1 + X), W += h sigma a, X *= 1 + sigma W.
template <typename T>
__device__ __forceinline__ void lmm_update_euler(T &X, const typename LmmMath<T>::C c, T &W) {
    const T a = X * LmmMath<T>::rcp(T(1) + X);
    W = fmaT(c.y, a, W);
    X = fmaT(X * c.x, W, X);
}

// The same forward for two lockstep FP32 paths with one reciprocal: r = 1 / (d0' d1'), so the
// drift terms are r d1' and r d0'.
template <bool GT, typename T>
__device__ __forceinline__ void lmm_update2(T &X0, T &X1, const typename LmmMath<T>::C c, T &W0, T &W1) {
    static_assert(sizeof(T) == 4 && GT, "lockstep pairs share reciprocals in FP32 g-table strips");
    const T e0 = LmmMath<T>::expb(-X0), e1 = LmmMath<T>::expb(-X1);
    const T d0 = fmaT(e0, c.y, c.z), d1 = fmaT(e1, c.y, c.z);
    const T r = LmmMath<T>::rcp(d0 * d1);
    W0 = fmaT(r, d1, W0);
    W1 = fmaT(r, d0, W1);
    X0 = fmaT(c.x, W0, X0);
    X1 = fmaT(c.x, W1, X1);
}

template <typename T>
__device__ __forceinline__ T row_sum32(const T *row) {
    T s[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int c = 0; c < 32; c += 4) {
        s[0] += row[c];
        s[1] += row[c + 1];
        s[2] += row[c + 2];
        s[3] += row[c + 3];
    }
    return (s[0] + s[1]) + (s[2] + s[3]);
}

// Scalars of one LMM caplet strip as the path code uses them.
template <typename T>
struct LmmScal {
    int nf, nK;
    T dl, inv_dl, disc0, hc, sqhc;
};

// Constants in shared memory: with the g-table [NF + 1 steps][NF forwards], row t holding
// (sigma_n, G = 2^(-t cc_n) H, H, 2^(t cc_n)), H = 1 / (h sigma_n); with the pair table
// [NF/2] float4 (sigma_2q, H_2q, sigma_2q+1, H_2q+1), [NF + 1][NF/2] float2 (G_2q, G_2q+1) and
// [NF] float 2^((t+1) cc_t); otherwise [NF] of (sigma_n, h sigma_n, cc_n, 0) (FP64, Euler scheme).
// The Euler scheme reads the first NF entries of the region in that last layout.
template <int NF, typename T>
__host__ __device__ constexpr size_t lmm_cst_count() {   // in units of LmmMath<T>::C
    return lmm_gtab<NF, T>()   ? (size_t)NF * (NF + 1)   // the Euler scheme uses the first NF
           : lmm_ptab<NF, T>() ? (size_t)NF / 2 + (size_t)(NF + 1) * NF / 4 + (size_t)NF / 4
                               : (size_t)NF;
}

// Fill the constants and the initial state X0 (all threads of the CTA; the caller synchronises).
template <int NF, typename T, bool EU = false>
__device__ __forceinline__ void lmm_fill_constants(const LmmModel<T> &md, typename LmmMath<T>::C *cst, T *X0) {
    using CC = typename LmmMath<T>::C;
    if constexpr (lmm_gtab<NF, T>() && !EU) {
        for (int k = threadIdx.x; k < NF * (NF + 1); k += blockDim.x) {
            const int t = k / NF, n = k % NF;
            const float x = (float)t * md.cc[n];   // t cc_n in log2 units
            const float H = lmm_fold_inv(md.hc * md.sig[n]);
            cst[k] = CC{md.sig[n], exp2f(-x) * H, H, exp2f(x)};
        }
    } else if constexpr (lmm_ptab<NF, T>() && !EU) {
        constexpr int NP = NF / 2;
        float2 *gt = reinterpret_cast<float2 *>(cst + NP);
        float *wf = reinterpret_cast<float *>(gt + (NF + 1) * NP);
        for (int q = threadIdx.x; q < NP; q += blockDim.x)
            cst[q] = CC{md.sig[2 * q], lmm_fold_inv(md.hc * md.sig[2 * q]), md.sig[2 * q + 1],
                        lmm_fold_inv(md.hc * md.sig[2 * q + 1])};
        for (int k = threadIdx.x; k < (NF + 1) * NP; k += blockDim.x) {
            const int t = k / NP, q = k % NP;
            gt[k] = make_float2(exp2f(-(float)t * md.cc[2 * q]) * lmm_fold_inv(md.hc * md.sig[2 * q]),
                                exp2f(-(float)t * md.cc[2 * q + 1]) * lmm_fold_inv(md.hc * md.sig[2 * q + 1]));
        }
        for (int t = threadIdx.x; t < NF; t += blockDim.x) wf[t] = exp2f((float)(t + 1) * md.cc[t]);
    } else {
        for (int k = threadIdx.x; k < NF; k += blockDim.x) cst[k] = CC{md.sig[k], md.hc * md.sig[k], md.cc[k], T(0)};
    }
    for (int k = threadIdx.x; k < NF; k += blockDim.x) X0[k] = md.X0[k];
}

// Shared memory: [generator stage][constants][X0 x NF, K x 8][normals zsets x 8 x P x threads]
//                [transpose buffers][acc][cmp]
// zsets = 2 when the normals are loaded: the next block's are copied in while a block runs.
template <int NF, typename T, int P = 1>
__host__ __device__ __forceinline__ size_t lmm_smem_layout(const GenParams &g, int nw, int nK, int nout,
                                                           size_t *o_cst, size_t *o_x0, size_t *o_z, size_t *o_buf,
                                                           size_t *o_acc, int zsets = 1) {
    size_t off = stage_bytes(g);
    *o_cst = off;
    off = align16(off + sizeof(typename LmmMath<T>::C) * lmm_cst_count<NF, T>());
    *o_x0 = off;
    off = align16(off + sizeof(T) * (NF + kMaxStrikes));
    *o_z = off;
    off = align16(off + sizeof(T) * 8 * P * 32 * (size_t)nw * (size_t)zsets);
    *o_buf = off;
    off = align16(off + sizeof(T) * (size_t)nw * 8 * nK * LmmMath<T>::PAD);
    *o_acc = off;
    off += 2 * sizeof(T) * (size_t)nw * nout;
    return off;
}

// Strips of at least this many forward slots keep the step loop of a block rolled.
#ifndef RQMC_LMM_ROLL_MIN_NF
#define RQMC_LMM_ROLL_MIN_NF 80
#endif

// CTAs per SM to plan registers for: forwards take NF (FP32) or 2 NF (FP64) registers.
#ifndef RQMC_LMM_EXTRA_REGS
#define RQMC_LMM_EXTRA_REGS 44
#endif
template <int NF, typename T>
constexpr int lmm_ilp();
template <int NF, typename T>
constexpr int lmm_min_blocks() {
    constexpr int regs = (int)(NF * sizeof(T) / 4) * lmm_ilp<NF, T>() + RQMC_LMM_EXTRA_REGS;
    return regs <= 64 ? 4 : regs <= 85 ? 3 : regs <= 128 ? 2 : 1;
}

// P paths in lockstep (1 or 2 in the caplet kernel, up to 4 in the batch): forwards in registers, per-step payoffs (summed over
// the P paths) into the warp's transpose buffer, block sums into the warp's Kahan
// accumulators (wacc/wcmp, indexed by output t nK + k).  The P paths share every constant
// load and all control flow, and give each warp P independent dependency chains.
// ZG: the normals are not generated here but read from zg, normals [step][zN] written
// beforehand from the same generator (by the point-stream kernel for a plan's replication,
// zi0 = 0; by the batch kernel for an item's points from zi0 on): path i takes
// zg[t zN + i - zi0], copied into the thread's shared columns a block ahead.
// DK: Ks holds delta K and the payoff is (delta L - delta K)^+ D; otherwise Ks holds K and the
// payoff is delta (L - K)^+ D with L = delta L / delta (the same value up to rounding).
template <int NF, int SEQ, typename T, int P, bool EU = false, bool ZG = false, bool DK = true>
__device__ __forceinline__ void lmm_path(PathGen<SEQ> (&pg)[P], const bool (&active)[P], const LmmScal<T> &sc,
                                         const typename LmmMath<T>::C *cst, const T *X0, const T *Ks, T *zb,
                                         T *wbuf, T *wacc, T *wcmp, const int lane, const T *zg = nullptr,
                                         size_t zN = 0, uint32_t zi0 = 0) {
    using M = LmmMath<T>;
    using CC = typename M::C;
    constexpr int PAD = M::PAD;
    constexpr bool GT = lmm_gtab<NF, T>() && !EU;
    constexpr bool PG = lmm_ptab<NF, T>() && !EU;
    static_assert(!PG || P == 1, "the pair table serves one path per thread");
    constexpr int NP = NF / 2;
    // pair table (PG): static pair constants, per-step G pairs, fixing factors
    const float4 *pc = reinterpret_cast<const float4 *>(cst);
    const float2 *pgt = reinterpret_cast<const float2 *>(pc + NP);
    const float *pwf = reinterpret_cast<const float *>(pgt + (size_t)(NF + 1) * NP);
    const int nf = sc.nf, nK = sc.nK;
    const T sqhc = sc.sqhc;
    const int zs = P * blockDim.x;   // stride of one step in the normals buffer
    T X[P][NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const T x0 = X0[k];
#pragma unroll
        for (int p = 0; p < P; ++p) X[p][k] = x0;
    }
    T disc[P];
#pragma unroll
    for (int p = 0; p < P; ++p) disc[p] = sc.disc0;
    const int nblk = (nf + 7) >> 3;
    // loaded normals: block bb's go to set bb & 1 of the thread's columns by asynchronous copies
    auto zload = [&](const int bb) {
        if (bb < nblk) {
            const int nb = min(8, nf - 8 * bb);
            T *dst = zb + (bb & 1) * 8 * zs;
#pragma unroll
            for (int tp = 0; tp < 8; ++tp)
#pragma unroll
                for (int p = 0; p < P; ++p)
                    if (tp < nb)
                        cp_async4(dst + tp * zs + p * blockDim.x, zg + (size_t)(8 * bb + tp) * zN + (pg[p].i - zi0));
        }
        cp_async_commit();   // an empty group past the last block keeps the wait count uniform
    };
    if constexpr (ZG) zload(0);
    for (int b = 0; b < nblk; ++b) {
        const int ngrp = (nf - 8 * b + 7) >> 3;   // groups of 8 shifted slots still alive
        const CC *cb0 = cst + 8 * b;              // constants of original slot 8b + k (row 0)
        const int nst = min(8, nf - 8 * b);
        // phase A: the block's normals (copied in during the previous block, or one short
        // generator loop)
        T *zbb = zb;
        if constexpr (ZG) {
            zload(b + 1);          // the set it overwrites was last read in block b - 1
            cp_async_wait<1>();    // block b's copies have landed
            zbb = zb + (b & 1) * 8 * zs;
        } else {
            for (int tp = 0; tp < nst; ++tp) {
                if constexpr (sizeof(T) == 4) {
                    float z[P];
                    normals32<SEQ, P>(pg, 8 * b + tp, z);
#pragma unroll
                    for (int p = 0; p < P; ++p) zb[tp * zs + p * blockDim.x] = z[p];
                } else {
#pragma unroll
                    for (int p = 0; p < P; ++p) zb[tp * zs + p * blockDim.x] = Draw<T>::normal(pg[p], 8 * b + tp);
                }
            }
        }
        // phase B: forward updates and payoffs (each thread reads back its own columns).  The
        // step loop of the wider strips stays rolled: eight copies of an 80- or 160-slot update
        // body would overflow the instruction cache.
        auto step = [&](const int tp) {
            T W[P];
#pragma unroll
            for (int p = 0; p < P; ++p) W[p] = sqhc * zbb[tp * zs + p * blockDim.x];
            const CC *cb = GT ? cb0 + (size_t)(8 * b + tp) * NF : cb0;   // this step's row
            const float4 *pcb = pc + 4 * b;                                // PG: pairs of the block's slots
            const float2 *pgr = pgt + (size_t)(8 * b + tp) * NP + 4 * b;   // PG: this step's G pairs
            // PG, one slot k of the block: (sigma, H) and G from its pair's entries
            auto update_slot_pg = [&](const int k) {
                if constexpr (PG) {
                    const float4 c4 = M::lds(pcb + (k >> 1));
                    const float2 g2 = M::lds2(pgr + (k >> 1));
                    const float sg = (k & 1) ? c4.z : c4.x, H = (k & 1) ? c4.w : c4.y, G = (k & 1) ? g2.y : g2.x;
                    T &x = X[0][k];
                    W[0] += M::rcp(fmaT(M::expb(-x), G, H));
                    x = fmaT(sg, W[0], x);
                }
            };
            // slot k of the P paths: FP32 pairs share a reciprocal, an odd path goes alone
            auto update_slot = [&](const int k, const CC c) {
                if constexpr (EU) {
#pragma unroll
                    for (int p = 0; p < P; ++p) lmm_update_euler<T>(X[p][k], c, W[p]);
                } else if constexpr (sizeof(T) == 4) {
                    if constexpr (GT) {
#pragma unroll
                        for (int p = 0; p + 1 < P; p += 2) lmm_update2<GT, T>(X[p][k], X[p + 1][k], c, W[p], W[p + 1]);
                        if constexpr (P % 2 == 1) lmm_update<GT, T>(X[P - 1][k], c, W[P - 1]);
                    }
                } else {
#pragma unroll
                    for (int p = 0; p < P; ++p) lmm_update<GT, T>(X[p][k], c, W[p]);
                }
            };
            // group 0: alive slots tp..7, entered through a fall-through switch
            switch (tp) {
#define RQMC_G0(k)                           \
    case (k): {                              \
        if constexpr (PG) {                  \
            update_slot_pg(k);               \
        } else {                             \
            const CC c = M::lds(cb + (k));   \
            update_slot(k, c);               \
        }                                    \
    }
                RQMC_G0(0) RQMC_G0(1) RQMC_G0(2) RQMC_G0(3) RQMC_G0(4) RQMC_G0(5) RQMC_G0(6) RQMC_G0(7)
#undef RQMC_G0
                default:
                    break;
            }
#pragma unroll
            for (int gi = 1; gi < NF / 8; ++gi) {
                if (gi < ngrp) {
                    if constexpr (PG) {
                        // one path: adjacent forwards share a reciprocal, 1/d'_k = d'_(k+1) r and
                        // 1/d'_(k+1) = d'_k r with r = 1/(d'_k d'_(k+1))
#pragma unroll
                        for (int k = 0; k < 8; k += 2) {
                            static_assert(sizeof(T) == 4, "pair table in FP32 only");
                            const float4 c4 = M::lds(pcb + 4 * gi + (k >> 1));
                            const float2 g2 = M::lds2(pgr + 4 * gi + (k >> 1));
                            T &x0 = X[0][8 * gi + k], &x1 = X[0][8 * gi + k + 1];
                            const T d0 = fmaT(M::expb(-x0), g2.x, c4.y);
                            const T d1 = fmaT(M::expb(-x1), g2.y, c4.w);
                            const T r = M::rcp(d0 * d1);
                            W[0] = fmaT(r, d1, W[0]);
                            x0 = fmaT(c4.x, W[0], x0);
                            W[0] = fmaT(r, d0, W[0]);
                            x1 = fmaT(c4.z, W[0], x1);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const CC c = M::lds(cb + 8 * gi + k);
                            update_slot(8 * gi + k, c);
                        }
                    }
                }
            }
            // L_{t+1}(T_{t+1}) = b^X / delta sits in shifted slot tp
            T Xf[P];
#pragma unroll
            for (int p = 0; p < P; ++p) Xf[p] = X[p][0];
            switch (tp) {
#define RQMC_PK(k)                                                       \
    case (k):                                                            \
        _Pragma("unroll") for (int p = 0; p < P; ++p) Xf[p] = X[p][(k)]; \
        break;
                RQMC_PK(1) RQMC_PK(2) RQMC_PK(3) RQMC_PK(4) RQMC_PK(5) RQMC_PK(6) RQMC_PK(7)
#undef RQMC_PK
                default:
                    break;
            }
            // DK: the payoff delta (L - K)^+ D as (delta L - delta K)^+ D, strikes staged as delta K
            T Lf[P], dd[P];
            // with the g-table the fixed forward's X_n = X~_n + (t+1) cc_n: one more factor 2^((t+1) cc_n)
            T gfix = T(1);
            if constexpr (GT) gfix = cst[(size_t)(8 * b + tp + 1) * NF + 8 * b + tp].w;
            if constexpr (PG) gfix = pwf[8 * b + tp];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const T e = EU ? Xf[p] : ((GT || PG) ? M::expb(Xf[p]) * gfix : M::expb(Xf[p]));   // delta L
                disc[p] *= M::rcp(T(1) + e);
                if constexpr (DK) {
                    Lf[p] = e;
                    dd[p] = active[p] ? disc[p] : T(0);
                } else {
                    Lf[p] = e * sc.inv_dl;
                    dd[p] = active[p] ? sc.dl * disc[p] : T(0);
                }
            }
            T *row = wbuf + (size_t)tp * nK * PAD + lane;
            for (int kk = 0; kk < nK; ++kk) {
                const T K = Ks[kk];
                T pay = T(0);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    pay = fmaT(fmax(Lf[p] - K, T(0)), dd[p], pay);
                }
                row[kk * PAD] = pay;
            }
        };
        if constexpr (NF >= RQMC_LMM_ROLL_MIN_NF) {
#pragma unroll 1
            for (int tp = 0; tp < nst; ++tp) step(tp);
        } else {
            for (int tp = 0; tp < nst; ++tp) step(tp);
        }
        __syncwarp();
        const int nrows = nst * nK;
        for (int rw = lane; rw < nrows; rw += 32) {
            const T v = row_sum32<T>(wbuf + (size_t)rw * PAD);
            const int o = 8 * b * nK + rw;
            T s = wacc[o], c = wcmp[o];
            if constexpr (sizeof(T) == 4) kahan_add(s, c, v);
            else s += v;
            wacc[o] = s;
            wcmp[o] = c;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k + 8 < NF; ++k) {
#pragma unroll
            for (int p = 0; p < P; ++p) X[p][k] = X[p][k + 8];
        }
    }
}

// Paths per thread in lockstep for a bucket: two where the registers allow it.
template <int NF, typename T>
constexpr int lmm_ilp() {
#ifdef RQMC_LMM_ILP
    return (NF * (int)sizeof(T) / 4) <= 40 ? RQMC_LMM_ILP : 1;
#else
    return (NF * (int)sizeof(T) / 4) <= 40 ? 2 : 1;
#endif
}

// ZG: normals read from zg ([M][nf][N], see lmm_path); g.stage is then 0 and no generator
// table is staged.
template <int NF, int SEQ, typename T, bool EU, bool ZG>
__global__ void __launch_bounds__(256, lmm_min_blocks<NF, T>()) lmm_caplet_kernel(const GenParams g, const LmmModel<T> md, const RedParams r,
                                                                            const T *__restrict__ zg) {
    using M = LmmMath<T>;
    using CC = typename M::C;
    constexpr int PAD = M::PAD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nK = md.nK, nout = r.nout;
    constexpr int P = lmm_ilp<NF, T>();
    size_t o_cst, o_x0, o_z, o_buf, o_acc;
    lmm_smem_layout<NF, T, P>(g, nw, nK, nout, &o_cst, &o_x0, &o_z, &o_buf, &o_acc, ZG ? 2 : 1);
    T *zb = reinterpret_cast<T *>(smem_raw + o_z) + threadIdx.x;   // [zsets][8][P][blockDim], own columns
    CC *cst = reinterpret_cast<CC *>(smem_raw + o_cst);
    T *X0 = reinterpret_cast<T *>(smem_raw + o_x0);
    T *Ks = X0 + NF;
    T *wbuf = reinterpret_cast<T *>(smem_raw + o_buf) + (size_t)warp * 8 * nK * PAD;
    T *acc = reinterpret_cast<T *>(smem_raw + o_acc);
    T *cmp = acc + nw * nout;
    T *wacc = acc + warp * nout, *wcmp = cmp + warp * nout;
    lmm_fill_constants<NF, T, EU>(md, cst, X0);
    if (threadIdx.x < kMaxStrikes) Ks[threadIdx.x] = md.dl * md.K[threadIdx.x];   // delta K (DK payoff form)
    zero_acc(acc, cmp, nw * nout);
    const LmmScal<T> sc{md.nf, md.nK, md.dl, md.inv_dl, md.disc0, md.hc, md.sqhc};
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
        for (int pp = 0; pp < r.ppt; pp += P) {
            PathGen<SEQ> pg[P];
            bool active[P];
            bool any = false;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const uint32_t i = tile * r.tile + (uint32_t)((pp + p) * blockDim.x + threadIdx.x);
                active[p] = pp + p < r.ppt && i < r.N;
                any = any || active[p];
                pg[p].init(gv, active[p] ? i : 0u);
            }
            if (!__any_sync(0xffffffffu, any)) break;
            lmm_path<NF, SEQ, T, P, EU, ZG>(pg, active, sc, cst, X0, Ks, zb, wbuf, wacc, wcmp, lane,
                                            ZG ? zg + (size_t)m * md.nf * r.N : nullptr, r.N);
        }
        flush_unit(r, u, acc, cmp);
    }
}

template <int NF, int SEQ, typename T, bool ZG = false>
static cudaError_t launch_lmm_t(const Plan &pl, const LmmModel<T> &md, cudaStream_t st) {
    auto kern = pl.scheme == RQMC_EULER ? lmm_caplet_kernel<NF, SEQ, T, true, ZG> : lmm_caplet_kernel<NF, SEQ, T, false, ZG>;
    GenParams g = pl.gen;
    if (ZG) g.stage = 0;   // no generator table is read
    const int threads = pl.threads;
    size_t a, b, c, d, e2;
    const size_t smem = lmm_smem_layout<NF, T, lmm_ilp<NF, T>()>(g, threads / 32, md.nK, pl.red.nout, &a, &b, &c, &d,
                                                                 &e2, ZG ? 2 : 1);
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
    kern<<<grid, threads, smem, st>>>(g, md, pl.red, ZG ? reinterpret_cast<const T *>(pl.znorm) : nullptr);
    return cudaGetLastError();
}

template <int SEQ>
cudaError_t launch_caplets_seq(const Plan &pl, cudaStream_t st) {
    const bool f32 = pl.prec == RQMC_FP32;
    switch (pl.nf_bucket) {
        case 16: return f32 ? launch_lmm_t<16, SEQ>(pl, pl.lmm32, st) : launch_lmm_t<16, SEQ>(pl, pl.lmm64, st);
        case 40: return f32 ? launch_lmm_t<40, SEQ>(pl, pl.lmm32, st) : launch_lmm_t<40, SEQ>(pl, pl.lmm64, st);
        case 80: return f32 ? launch_lmm_t<80, SEQ>(pl, pl.lmm32, st) : launch_lmm_t<80, SEQ>(pl, pl.lmm64, st);
        case 160: return f32 ? launch_lmm_t<160, SEQ>(pl, pl.lmm32, st) : launch_lmm_t<160, SEQ>(pl, pl.lmm64, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rqmc
