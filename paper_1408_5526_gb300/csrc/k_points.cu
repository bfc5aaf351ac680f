// k_points.cu -- point-stream kernel: coordinates of M randomizations of N points,
// layout out[(m*s + j)*N + i] (the generator-throughput setting of Sec. 4, Table 2).
// Rows (m, j) are cut into chunks of ITEMS*blockDim consecutive points; a thread writes
// ITEMS coordinates blockDim apart so every warp store is one contiguous 128-byte (FP32)
// segment, and computes them in lockstep (shared digit / bit loop and inverse-CDF
// polynomial).  Philox rows come four dimensions at a time from one counter.
#include <cstring>

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

// ------------------------------------------------------------------ runs of consecutive points
// Halton/Rasrap and Sobol' rows with N a multiple of 8 (and a 16-byte aligned buffer): a lane
// owns runs of kRun = 8 consecutive points, a warp 32 runs = one chunk of 256 consecutive
// points of a row, and a warp task kSegChunks chunks.  The lane writes its run with 16-byte
// vector stores, so every store instruction of the warp covers consecutive bytes.
//   Sobol': x(n) for the lane's first point once per task (bit loop), then per chunk the
//   direction numbers of the index bits that change from n to n + 256 (the same bits in
//   every lane when the offset is a multiple of 256), and inside a run (n a multiple of 8)
//   x(n + k) = x(n) ^ (XOR of V_b over the bits b of k).
//   Halton/Rasrap: Algorithm 2's odometer restated for SIMD lanes.  Write the low part of the
//   run's first point as q p + d0; the run's points are d = d0 + k (k < 8) with q, or, past a
//   wrap of the lowest digit, d - p with q + 1.  With the permuted digit sums of the higher
//   digits R'(q) and R'(q + 1) computed once per run, a point costs one sigma lookup:
//   R = sigma(d) p^(L-1) + R'(.).  FP32 uniforms and normals never form R: the exact side
//   test and the value follow from sigma(d) and per-run constants (HaltonRow::split).  For
//   p >= 7 a run wraps at most once; bases 2, 3 and 5 take the direct digit expansion.
constexpr int kRun = 8;
constexpr int kSegChunks = 8;

// sum_{k=1}^{L-1} sigma(d_k) p^(L-1-k) over the digits d_1, d_2, ... of q (least significant
// first), in Horner order.
__device__ __forceinline__ uint32_t halton_high(const HaltonDim &h, const uint16_t *__restrict__ sg, uint32_t q) {
    uint32_t r = 0;
    for (uint32_t k = 1; k < h.L; ++k) {
        uint32_t qq = __umulhi(q, h.magic);
        uint32_t d = q - qq * h.p;
        if ((int32_t)d < 0) {
            d += h.p;
            qq -= 1;
        }
        r = r * h.p + (uint32_t)sg[d];
        q = qq;
    }
    return r;
}

// halton_high of q (into *r0) and of q + 1 modulo p^(L-1) (into *r1) from one pass over the
// digits of q: the digits of q + 1 are those of q with a carry that runs through the low digits
// equal to p - 1.
__device__ __forceinline__ void halton_high2(const HaltonDim &h, const uint16_t *__restrict__ sg, uint32_t q,
                                             uint32_t *r0, uint32_t *r1) {
    uint32_t a = 0, b = 0, cy = 1;
    for (uint32_t k = 1; k < h.L; ++k) {
        uint32_t qq = __umulhi(q, h.magic);
        uint32_t d = q - qq * h.p;
        if ((int32_t)d < 0) {
            d += h.p;
            qq -= 1;
        }
        uint32_t e = d + cy;
        cy = e == h.p ? 1u : 0u;
        e = cy ? 0u : e;
        a = a * h.p + (uint32_t)sg[d];
        b = b * h.p + (uint32_t)sg[e];
        q = qq;
    }
    *r0 = a;
    *r1 = b;
}

template <typename T, int RUN = kRun>
__device__ __forceinline__ void store_run(T *dst, const T (&v)[RUN]) {
    static_assert(RUN % 4 == 0, "runs of whole 16-byte stores");
    if constexpr (sizeof(T) == 4) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
        for (int q = 0; q < RUN / 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
        ulonglong2 *d2 = reinterpret_cast<ulonglong2 *>(dst);
#pragma unroll
        for (int q = 0; q < RUN / 2; ++q) {
            ulonglong2 w;
            memcpy(&w.x, &v[2 * q], 8);
            memcpy(&w.y, &v[2 * q + 1], 8);
            d2[q] = w;
        }
    }
}

// Values of the run from raw Sobol' words.
template <int TR, typename T, int RUN = kRun>
__device__ __forceinline__ void run_from_u32(const uint32_t (&x)[RUN], T (&v)[RUN]) {
    if constexpr (TR == RQMC_NORMAL && sizeof(T) == 4) {
        Unif32 u[RUN];
        float z[RUN];
#pragma unroll
        for (int k = 0; k < RUN; ++k) u[k] = unif32_from_u32(x[k]);
        ndtri32_lockstep<RUN>(u, z);
#pragma unroll
        for (int k = 0; k < RUN; ++k) v[k] = z[k];
    } else {
#pragma unroll
        for (int k = 0; k < RUN; ++k) v[k] = value_from_u32<TR, T>(x[k]);
    }
}

// One Halton row's constants as scalars: the carry-dependent fields are picked with selects,
// so the row stays in registers (a HaltonDim indexed by the carry would live in local memory).
struct HaltonRow {
    unsigned long long P, S0, S1;
    double invD;
    uint32_t pL, thr0, thr1;   // halton_lower(h, R, c) is R < thr_c
    float inv_pL, a0, a1, b0, b1;
    // the split R = sigma(d) p^(L-1) + R' of the FP32 runs (run_halton32): thr_c = thi_c p^(L-1) + tlo_c
    uint32_t pLm1, thi0, tlo0, thi1, tlo1;
    float inv_p, pm1f;
    __device__ __forceinline__ explicit HaltonRow(const HaltonDim &h)
        : P(h.P), S0(h.S[0]), S1(h.S[1]), invD(h.invD), pL(h.pL), thr0((h.pL >> 1) + (h.tie & 1u)),
          thr1((h.pL >> 1) + ((h.tie >> 1) & 1u)), inv_pL(h.inv_pL), a0(h.a[0]), a1(h.a[1]), b0(h.b[0]), b1(h.b[1]),
          pLm1(h.pL / h.p), thi0(thr0 / pLm1), tlo0(thr0 % pLm1), thi1(thr1 / pLm1), tlo1(thr1 % pLm1),
          inv_p(1.0f / (float)h.p), pm1f((float)(h.p - 1u)) {}
    // Run constants of the points with higher-digit sum R' and carry c: the point with lowest
    // digit sigma = sigma(d) has R = sigma p^(L-1) + R' and lies in the lower half exactly when
    // sigma < T (R < thr_c, R' < p^(L-1)); then u = sigma / p + A, else 1 - u with
    // 1 - u = (p - 1 - sigma) / p + B:  A = R' / p^L + a_c,  B = (p^(L-1) - 1 - R') / p^L + b_c.
    __device__ __forceinline__ void split(uint32_t Rp, uint32_t c, uint32_t &T, float &A, float &B) const {
        T = (c ? thi1 : thi0) + (Rp < (c ? tlo1 : tlo0) ? 1u : 0u);
        A = fmaf((float)Rp, inv_pL, c ? a1 : a0);
        B = fmaf((float)(pLm1 - 1u - Rp), inv_pL, c ? b1 : b0);
    }
    __device__ __forceinline__ unsigned long long num(uint32_t R, uint32_t c) const {
        return (unsigned long long)R * P + (c ? S1 : S0);
    }
    // the values of unif32_halton / unif64_halton
    __device__ __forceinline__ Unif32 unif32(uint32_t R, uint32_t c) const {
        const bool lo = R < (c ? thr1 : thr0);
        const uint32_t Rs = lo ? R : pL - 1u - R;
        const float off = c ? (lo ? a1 : b1) : (lo ? a0 : b0);
        return Unif32{fmaf((float)Rs, inv_pL, off), lo};
    }
    __device__ __forceinline__ Unif64 unif64(uint32_t R, uint32_t c) const {
        const unsigned long long n = num(R, c);
        const unsigned long long D1 = (unsigned long long)pL * P - 1ull;
        const bool lo = n <= D1 - n;
        return Unif64{((double)(lo ? n : D1 - n) + 0.5) * invD, lo};
    }
};

// One lane's run of kRun points (p >= 7): lowest digit d0 of its first point, the higher-digit
// sums R'(q0) and R'(q0 + 1) and the carries before and after the wrap of the lowest digit
// (R1 = R0 where no lane of the warp wraps).
struct HaltonRun {
    uint32_t d0, R0, R1, c0, c1;
    bool any_wrap;   // warp-uniform: some lane's run wraps its lowest digit
};
__device__ __forceinline__ HaltonRun halton_run(const HaltonDim &h, const uint16_t *__restrict__ sg, uint32_t i0,
                                                uint32_t pLm1) {
    HaltonRun r;
    uint32_t low = h.lo0 + i0;
    r.c0 = low >= h.pL ? 1u : 0u;
    low -= r.c0 ? h.pL : 0u;
    uint32_t q0 = __umulhi(low, h.magic);
    r.d0 = low - q0 * h.p;
    if ((int32_t)r.d0 < 0) {
        r.d0 += h.p;
        q0 -= 1;
    }
    // the run reaches p^L: the low part wraps into the carry (and q0 + 1 to 0)
    r.c1 = q0 + 1 == pLm1 ? 1u : r.c0;
    // R'(q0 + 1) only where some lane's run wraps its lowest digit: always for small p, in
    // about 256/p of the warps for p > 256
    r.any_wrap = __any_sync(0xffffffffu, r.d0 + (kRun - 1) >= h.p);
    if (r.any_wrap) {
        halton_high2(h, sg, q0, &r.R0, &r.R1);
    } else {
        r.R0 = halton_high(h, sg, q0);
        r.R1 = r.R0;
    }
    return r;
}

// FP32 uniforms or normals of a run (p >= 7) from the split of HaltonRow::split: a point costs
// one permutation lookup (the padded table, see kSigPad), one integer compare and two FMAs.
template <int TR>
__device__ __forceinline__ void run_halton32(const HaltonRow &hr, const HaltonRun &r, const uint16_t *__restrict__ sg,
                                             uint32_t p, float (&v)[kRun]) {
    uint32_t T0;
    float A0, B0;
    hr.split(r.R0, r.c0, T0, A0, B0);
    const uint16_t *sb = sg + r.d0;   // sb[k] = sigma((d0 + k) mod p)
    Unif32 u[kRun];
    if (!r.any_wrap) {
#pragma unroll
        for (int k = 0; k < kRun; ++k) {
            const uint32_t sk = sb[k];
            const float fs = (float)sk;
            const bool lo = sk < T0;
            u[k] = Unif32{lo ? fmaf(fs, hr.inv_p, A0) : fmaf(hr.pm1f - fs, hr.inv_p, B0), lo};
        }
    } else {
        uint32_t T1;
        float A1, B1;
        hr.split(r.R1, r.c1, T1, A1, B1);
        const uint32_t kw = p - r.d0;   // points k >= kw are past the wrap: R'(q0 + 1), carry c1
#pragma unroll
        for (int k = 0; k < kRun; ++k) {
            const bool w = (uint32_t)k >= kw;
            const uint32_t sk = sb[k];
            const float fs = (float)sk;
            const bool lo = sk < (w ? T1 : T0);
            u[k] = Unif32{lo ? fmaf(fs, hr.inv_p, w ? A1 : A0) : fmaf(hr.pm1f - fs, hr.inv_p, w ? B1 : B0), lo};
        }
    }
    if constexpr (TR == RQMC_NORMAL) {
        ndtri32_lockstep<kRun>(u, v);
    } else {
#pragma unroll
        for (int k = 0; k < kRun; ++k) v[k] = u[k].lower ? u[k].q : 1.0f - u[k].q;
    }
}

template <int TR, typename T>
__device__ __forceinline__ void run_from_halton(const HaltonRow &h, const uint32_t (&R)[kRun],
                                                const uint32_t (&c)[kRun], T (&v)[kRun]) {
    if constexpr (TR == RQMC_RAW) {
#pragma unroll
        for (int k = 0; k < kRun; ++k) v[k] = (T)h.num(R[k], c[k]);
    } else if constexpr (sizeof(T) == 4) {
        Unif32 u[kRun];
#pragma unroll
        for (int k = 0; k < kRun; ++k) u[k] = h.unif32(R[k], c[k]);
        if constexpr (TR == RQMC_NORMAL) {
            float z[kRun];
            ndtri32_lockstep<kRun>(u, z);
#pragma unroll
            for (int k = 0; k < kRun; ++k) v[k] = z[k];
        } else {
#pragma unroll
            for (int k = 0; k < kRun; ++k) v[k] = u[k].lower ? u[k].q : 1.0f - u[k].q;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kRun; ++k) {
            const Unif64 w = h.unif64(R[k], c[k]);
            v[k] = TR == RQMC_NORMAL ? ndtri64(w) : (w.lower ? w.q : 1.0 - w.q);
        }
    }
}

// Any transform and precision: the run's integer digit sums R (the odometer for p >= 7, the
// digit expansion for bases 2, 3 and 5), then the values of unif32/unif64_halton.
template <int TR, typename T>
__device__ __forceinline__ void run_halton_digits(const HaltonRow &hr, const HaltonDim &h,
                                                  const uint16_t *__restrict__ sg, uint32_t i0, uint32_t pLm1,
                                                  T (&v)[kRun]) {
    uint32_t R[kRun], cc[kRun];
    if (h.p >= 7) {
        const HaltonRun r = halton_run(h, sg, i0, pLm1);
        const uint32_t kw = h.p - r.d0;
#pragma unroll
        for (int k = 0; k < kRun; ++k) {
            const bool w = (uint32_t)k >= kw;
            R[k] = (uint32_t)sg[r.d0 + k] * pLm1 + (w ? r.R1 : r.R0);
            cc[k] = w ? r.c1 : r.c0;
        }
    } else {
        uint32_t ii[kRun];
#pragma unroll
        for (int k = 0; k < kRun; ++k) ii[k] = i0 + k;
        halton_R_lockstep<kRun>(h, sg, ii, R, cc);
    }
    run_from_halton<TR, T>(hr, R, cc, v);
}

template <int TR, typename T, int SEQ>
__global__ void __launch_bounds__(256) points_run_kernel(const GenParams g, uint32_t N, uint32_t tasks_per_row,
                                                         unsigned long long ntasks, T *__restrict__ out) {
    const uint32_t lane = threadIdx.x & 31;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const uint32_t seg_pts = 32u * kRun * kSegChunks;
    for (unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < ntasks;
         w += warps) {
        const unsigned long long row = w / tasks_per_row;
        const uint32_t seg0 = (uint32_t)(w % tasks_per_row) * seg_pts;
        const int m = (int)(row / g.s), j = (int)(row % g.s);
        T *dst = out + row * N;
        if constexpr (SEQ == kSobolDS) {
            const uint32_t *V = g.sobV + (size_t)m * g.sobV_mstride + 32 * j;
            const uint32_t v0 = __ldg(V), v1 = __ldg(V + 1), v2 = __ldg(V + 2);
            const uint32_t comb[kRun] = {0u, v0, v1, v0 ^ v1, v2, v2 ^ v0, v2 ^ v1, v2 ^ v1 ^ v0};
            uint32_t n = (uint32_t)(g.offset + seg0 + kRun * lane);   // first point of the lane's run
            uint32_t x = __ldg(g.sobShift + row);
            for (int k = 0; k < g.sob_bits; ++k) x ^= ((n >> k) & 1u) ? __ldg(V + k) : 0u;
            for (int c = 0; c < kSegChunks; ++c) {
                const uint32_t i0 = seg0 + 256u * c + kRun * lane;
                if (c > 0) {
                    const uint32_t n2 = n + 256u;
                    for (uint32_t d = n ^ n2; d != 0u; d &= d - 1u) x ^= __ldg(V + (__ffs(d) - 1));
                    n = n2;
                }
                if (seg0 + 256u * c >= N) break;   // warp-uniform
                uint32_t xs[kRun];
#pragma unroll
                for (int k = 0; k < kRun; ++k) xs[k] = x ^ comb[k];
                T v[kRun];
                run_from_u32<TR, T>(xs, v);
                if (i0 < N) store_run<T>(dst + i0, v);
            }
        } else {
            const HaltonDim &hg = g.hdim[row];
            const HaltonRow hr(hg);
            HaltonDim h;   // the digit fields only (no carry-indexed field is read from it)
            h.p = hg.p;
            h.L = hg.L;
            h.pL = hg.pL;
            h.lo0 = hg.lo0;
            h.magic = hg.magic;
            const uint16_t *sg = g.sigma + (size_t)m * g.sig_len + hg.sig_off;
            const uint32_t pLm1 = h.pL / h.p;   // p^(L-1)
            for (int c = 0; c < kSegChunks; ++c) {
                if (seg0 + 256u * c >= N) break;   // warp-uniform
                const uint32_t i0 = min(seg0 + 256u * c + kRun * lane, N - kRun);   // past the end: a valid run, not stored
                T v[kRun];
                if constexpr (sizeof(T) == 4 && TR != RQMC_RAW) {
                    if (h.p >= 7) run_halton32<TR>(hr, halton_run(h, sg, i0, pLm1), sg, h.p, v);
                    else run_halton_digits<TR, T>(hr, h, sg, i0, pLm1, v);
                } else {
                    run_halton_digits<TR, T>(hr, h, sg, i0, pLm1, v);
                }
                if (seg0 + 256u * c + kRun * lane < N) store_run<T>(dst + i0, v);
            }
        }
    }
}

// Philox rows in runs: a warp task is (replication, block of 4 dimensions, 2048 consecutive
// points); a lane takes runs of PR consecutive points, one Philox call each gives the point's 4
// coordinates of the block, and the lane writes each of the 4 rows' PR values with vector stores.
template <int TR, typename T>
__global__ void __launch_bounds__(256) points_run_philox_kernel(const GenParams g, uint32_t N, uint32_t tasks_per_row,
                                                                unsigned long long ntasks, T *__restrict__ out) {
    // FP32 normals take runs of 4 points: the 4 x 4 Philox words and the inverse-CDF state
    // fit in 71 registers (3 CTAs per SM) instead of 109
    constexpr int PR = TR == RQMC_NORMAL && sizeof(T) == 4 ? 4 : kRun;
    constexpr uint32_t chunk = 32u * PR;
    const uint32_t lane = threadIdx.x & 31;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const uint32_t seg_pts = 32u * kRun * kSegChunks;
    const int nb = (g.s + 3) >> 2;
    for (unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < ntasks;
         w += warps) {
        const unsigned long long rb = w / tasks_per_row;   // (m, block of 4 dimensions)
        const uint32_t seg0 = (uint32_t)(w % tasks_per_row) * seg_pts;
        const int m = (int)(rb / nb), jb = (int)(rb % nb);
        for (uint32_t c = 0; c < seg_pts / chunk; ++c) {
            if (seg0 + chunk * c >= N) break;   // warp-uniform
            const uint32_t i0 = seg0 + chunk * c + PR * lane;
            if (i0 >= N) continue;
            uint32_t x[4][PR];
#pragma unroll
            for (int k = 0; k < PR; ++k) {
                const unsigned long long n = g.offset + i0 + k;
                const U32x4 r = philox4x32_10((uint32_t)n, (uint32_t)((n >> 32) & 0xFFFFu) | ((uint32_t)jb << 16),
                                              (uint32_t)m, kTagPath | (g.inst << 8), g.key0, g.key1);
                x[0][k] = r.x;
                x[1][k] = r.y;
                x[2][k] = r.z;
                x[3][k] = r.w;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 4 * jb + q;
                if (j < g.s) {
                    T v[PR];
                    run_from_u32<TR, T, PR>(x[q], v);
                    store_run<T, PR>(out + ((size_t)m * g.s + j) * N + i0, v);
                }
            }
        }
    }
}

template <int TR, typename T, int SEQ>
static cudaError_t launch_points_run(const Plan &pl, void *out, cudaStream_t st) {
    void (*kern)(const GenParams, uint32_t, uint32_t, unsigned long long, T *);
    if constexpr (SEQ == kPhilox) kern = points_run_philox_kernel<TR, T>;
    else kern = points_run_kernel<TR, T, SEQ>;
    const int threads = 256;
    const uint32_t seg_pts = 32u * kRun * kSegChunks;
    const uint32_t tasks_per_row = (uint32_t)((pl.N + seg_pts - 1) / seg_pts);
    const unsigned long long rows = SEQ == kPhilox ? (unsigned long long)pl.M * ((pl.s + 3) / 4)
                                                   : (unsigned long long)pl.M * pl.s;
    const unsigned long long ntasks = rows * tasks_per_row;
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0);
    if (occ < 1) occ = 1;
    const unsigned long long blocks = (ntasks + threads / 32 - 1) / (threads / 32);
    const unsigned grid = (unsigned)std::min<unsigned long long>(blocks, (unsigned long long)occ * sms * 4);
    kern<<<grid, threads, 0, st>>>(pl.gen, (uint32_t)pl.N, tasks_per_row, ntasks, reinterpret_cast<T *>(out));
    return cudaGetLastError();
}

// The run kernels apply when every run of 8 points starts on a 16-byte boundary (N a multiple
// of 8, the buffer 16-byte aligned) and, for Sobol', the offset is a multiple of 8 (the runs'
// index bits 0..2 are then the point's position in the run).
bool points_runs_eligible(const Plan &pl) {
    return pl.N % kRun == 0 && (pl.seq == kPhilox || pl.offset % kRun == 0);
}
static bool points_runs_apply(const Plan &pl, const void *out) {
    return points_runs_eligible(pl) && ((uintptr_t)out & 15u) == 0;
}

template <int TR, typename T>
static cudaError_t launch_points_runs_t(const Plan &pl, void *out, cudaStream_t st) {
    if (pl.gen.seq == kPhilox) return launch_points_run<TR, T, kPhilox>(pl, out, st);
    return pl.gen.seq == kSobolDS ? launch_points_run<TR, T, kSobolDS>(pl, out, st)
                                  : launch_points_run<TR, T, kRasrap>(pl, out, st);
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
    const bool f32 = pl.prec == RQMC_FP32;
    if (points_runs_apply(pl, out)) {
        if (tr == RQMC_RAW) return launch_points_runs_t<RQMC_RAW, unsigned long long>(pl, out, st);
        if (tr == RQMC_UNIFORM)
            return f32 ? launch_points_runs_t<RQMC_UNIFORM, float>(pl, out, st)
                       : launch_points_runs_t<RQMC_UNIFORM, double>(pl, out, st);
        return f32 ? launch_points_runs_t<RQMC_NORMAL, float>(pl, out, st)
                   : launch_points_runs_t<RQMC_NORMAL, double>(pl, out, st);
    }
    if (tr == RQMC_RAW) return launch_points_t<RQMC_RAW, unsigned long long>(pl, out, st);
    if (tr == RQMC_UNIFORM)
        return f32 ? launch_points_t<RQMC_UNIFORM, float>(pl, out, st) : launch_points_t<RQMC_UNIFORM, double>(pl, out, st);
    return f32 ? launch_points_t<RQMC_NORMAL, float>(pl, out, st) : launch_points_t<RQMC_NORMAL, double>(pl, out, st);
}

}  // namespace rqmc
