// rqmc_common.cuh -- device building blocks of the RQMC hot path (sm_103a).
//
//   * Philox4x32-10 (Salmon et al., SC'11), the Sec. 2 counter-based stream and
//     the source of every randomization
//   * counter-based random-start permuted van der Corput (Sec. 3.1, Algorithm 3,
//     eq. perm) in exact integer digit arithmetic
//   * Sobol' in binary counter order with a digital shift (Sec. 3.2)
//   * the inverse normal CDF (our own fit, Giles' polynomial form) in FP32, and
//     in FP64 with one Halley correction on erfc
//   * warp-shuffle reductions
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ndtri_coeffs.h"

namespace rqmc {

constexpr int kMaxStrikes = 8;

// ------------------------------------------------------------------ SFU wrappers (PTX ISA)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------------------ Philox4x32-10
struct U32x4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// Ten rounds; each round multiplies words 0 and 2 by 0xD2511F53 / 0xCD9E8D57,
// mixes the high halves into words 1 and 3 with the key, and bumps the key by
// the Weyl constants 0x9E3779B9 / 0xBB67AE85.
__host__ __device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                        uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = mulhi32(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = mulhi32(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U32x4{c0, c1, c2, c3};
}

// Counter tags (low byte of counter word 3; the instrument index sits above it).
enum : uint32_t { kTagPath = 0, kTagStart = 1, kTagPerm = 2, kTagShift = 3, kTagScramble = 4 };

// ------------------------------------------------------------------ sequence descriptors
// kSobolLMS is a plan-level sequence only: its kernels run the kSobolDS code on
// per-replication (scrambled) direction numbers.
enum Seq : int { kHaltonRS = 0, kRasrap = 1, kSobolDS = 2, kPhilox = 3, kSobolLMS = 4 };

// Per (replication m, dimension j) description of the random-start permuted van der
// Corput points phi_p^sigma(n0 + offset + i), i < N, split at digit L:
//   low  = lo0 + i                      (lo0 = (n0+offset) mod p^L, carry c = low >= p^L)
//   R    = sum_{k<L} sigma(d_k) p^(L-1-k) over the digits d_k of low mod p^L
//   num  = R * P + S[c]                 (P = p^(K+1-L); S[c] = the permuted high digits
//                                        of (n0+offset) div p^L + c at positions L..K)
// num / p^(K+1) is exactly the point of eq. (perm) with all K start positions permuted.
// Each dimension's permutation sigma(0..p-1) is followed by sigma(0..kSigPad-1) once more (indices
// taken mod p), so that sigma of d = d0 + k, k < kSigPad, with d0 < p, is entry d0 + k whether
// or not the lowest digit wraps.
constexpr uint32_t kSigPad = 8;

struct __align__(16) HaltonDim {
    unsigned long long P;
    unsigned long long S[2];
    double invD;             // 1 / p^(K+1) (FP64 conversion)
    uint32_t p, L, pL, lo0;
    uint32_t magic;          // floor(2^32 / p) + 1: q = umulhi(x, magic) is floor(x/p) or one more
    uint32_t sig_off;        // offset of sigma_{m,j} inside replication m's permutation table
                             // (p entries, then sigma(0..kSigPad-1) again, see kSigPad)
    float inv_pL;            // FP32 conversion: u = R / p^L + (S[c] + 1/2) / D
    float a[2];              // (S[c] + 1/2) / D
    float b[2];              // (P - 1 - S[c] + 1/2) / D, the complement's tail
    uint32_t tie;            // bit c: p^L odd and 2 S[c] <= P - 1, i.e. the middle R = (p^L - 1)/2
                             // puts num = R P + S[c] in the lower half (see halton_lower)
};

struct GenParams {
    int seq;
    int s;
    int M;
    uint32_t key0, key1;
    uint32_t inst;           // instrument index (batched launches)
    unsigned long long offset;
    const HaltonDim *hdim;   // [M][s]
    const uint16_t *sigma;   // [M][sig_len]
    unsigned long long sig_len;
    const uint32_t *sobV;    // [s][32], or [M][s][32] when scrambled per replication
    unsigned long long sobV_mstride;   // 0, or 32 s for per-replication tables
    const uint32_t *sobShift;// [M][s]
    int sob_bits;            // bits of offset + N - 1
    int stage_sig;           // 1: a replication's permutations are staged in shared memory
    int stage;               // 1: a replication's per-dimension tables are staged in shared
                             //    memory; 0 (very large s): the kernels read them from global
};

// Per-replication view of the generator tables used by the path kernels; the tables
// of replication m are staged in shared memory when the CTA starts working on m
// (the permutations only when they fit, see stage_bytes()).
struct GenView {
    int seq, s, sob_bits;
    uint32_t key0, key1, inst;
    int m;
    unsigned long long offset;
    const HaltonDim *hd;     // [s]
    const uint16_t *sig;     // permutations of replication m
    const uint32_t *V;       // [s][32]
    const uint32_t *shift;   // [s]
};

__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared-memory bytes the staging of one replication's tables takes.
__host__ __device__ __forceinline__ size_t stage_bytes(const GenParams &g) {
    if (!g.stage) return 0;
    if (g.seq == kHaltonRS || g.seq == kRasrap)
        return align16(sizeof(HaltonDim) * g.s) + (g.stage_sig ? align16(2 * g.sig_len) : 0);
    if (g.seq == kSobolDS) return align16(4ull * 32 * g.s) + align16(4ull * g.s);
    return 0;
}

// All threads of the CTA call this (no barrier inside; the caller synchronises).  Every
// pointer of the view points into shared memory, which the compiler can see, so the
// generators' table reads compile to shared-memory loads.
__device__ __forceinline__ void stage_tables(const GenParams &g, int m, unsigned char *sm, GenView &v) {
    v.seq = g.seq;
    v.s = g.s;
    v.sob_bits = g.sob_bits;
    v.key0 = g.key0;
    v.key1 = g.key1;
    v.inst = g.inst;
    v.m = m;
    v.offset = g.offset;
    v.hd = nullptr;
    v.sig = nullptr;
    v.V = nullptr;
    v.shift = nullptr;
    if (g.seq == kHaltonRS || g.seq == kRasrap) {
        HaltonDim *hd = reinterpret_cast<HaltonDim *>(sm);
        const uint4 *src = reinterpret_cast<const uint4 *>(g.hdim + (size_t)m * g.s);
        uint4 *dst = reinterpret_cast<uint4 *>(hd);
        const int n16 = (int)(sizeof(HaltonDim) / 16) * g.s;
        for (int k = threadIdx.x; k < n16; k += blockDim.x) dst[k] = src[k];
        v.hd = hd;
        const uint16_t *gs = g.sigma + (size_t)m * g.sig_len;
        if (g.stage_sig) {
            uint16_t *ss = reinterpret_cast<uint16_t *>(sm + align16(sizeof(HaltonDim) * g.s));
            for (unsigned long long k = threadIdx.x; k < g.sig_len; k += blockDim.x) ss[k] = gs[k];
            v.sig = ss;
        } else {
            v.sig = gs;
        }
    } else if (g.seq == kSobolDS) {
        uint32_t *V = reinterpret_cast<uint32_t *>(sm);
        uint32_t *sh = reinterpret_cast<uint32_t *>(sm + align16(4ull * 32 * g.s));
        const uint32_t *Vm = g.sobV + (size_t)m * g.sobV_mstride;
        for (int k = threadIdx.x; k < 32 * g.s; k += blockDim.x) V[k] = Vm[k];
        for (int k = threadIdx.x; k < g.s; k += blockDim.x) sh[k] = g.sobShift[(size_t)m * g.s + k];
        v.V = V;
        v.shift = sh;
    }
}

// View of replication m's tables where they are, in global memory (for s too large to stage;
// g.stage == 0).  A separate function, so that kernels which stage keep pointers the
// compiler knows to be shared.
__device__ __forceinline__ void view_tables(const GenParams &g, int m, GenView &v) {
    v.seq = g.seq;
    v.s = g.s;
    v.sob_bits = g.sob_bits;
    v.key0 = g.key0;
    v.key1 = g.key1;
    v.inst = g.inst;
    v.m = m;
    v.offset = g.offset;
    v.hd = nullptr;
    v.sig = nullptr;
    v.V = nullptr;
    v.shift = nullptr;
    if (g.seq == kHaltonRS || g.seq == kRasrap) {
        v.hd = g.hdim + (size_t)m * g.s;
        v.sig = g.sigma + (size_t)m * g.sig_len;
    } else if (g.seq == kSobolDS) {
        v.V = g.sobV + (size_t)m * g.sobV_mstride;
        v.shift = g.sobShift + (size_t)m * g.s;
    }
}

template <bool STAGED>
__device__ __forceinline__ void load_tables(const GenParams &g, int m, unsigned char *sm, GenView &v) {
    if constexpr (STAGED) stage_tables(g, m, sm, v);
    else view_tables(g, m, v);
}

// ------------------------------------------------------------------ Halton digits
// Digits of low = lo0 + i in base p, each mapped through sigma and accumulated in
// Horner order (sigma(d_0) most significant).  Exact; no divergence (L is uniform).
__device__ __forceinline__ uint32_t halton_R(const HaltonDim &h, const uint16_t *__restrict__ sig, uint32_t i,
                                             uint32_t &carry) {
    uint32_t low = h.lo0 + i;
    carry = low >= h.pL ? 1u : 0u;
    low -= carry ? h.pL : 0u;
    const uint16_t *sg = sig + h.sig_off;
    if (h.p == 2) {   // base 2: the digits are bits and sigma is the identity or the swap
        const uint32_t rev = __brev(low) >> (32u - h.L);
        return sg[0] != 0 ? rev ^ ((1u << h.L) - 1u) : rev;
    }
    uint32_t r = 0;
    for (uint32_t k = 0; k < h.L; ++k) {
        uint32_t q = __umulhi(low, h.magic);
        uint32_t d = low - q * h.p;
        if ((int32_t)d < 0) {   // the rounded-up reciprocal overshot by one
            d += h.p;
            q -= 1;
        }
        r = r * h.p + (uint32_t)sg[d];
        low = q;
    }
    return r;
}

__device__ __forceinline__ unsigned long long halton_num(const HaltonDim &h, uint32_t R, uint32_t c) {
    return (unsigned long long)R * h.P + h.S[c];
}

// u <= 1/2 side test, exact: num <= D-1-num, i.e. 2 (R P + S[c]) <= p^L P - 1.  That holds
// for every 2R <= p^L - 2 (as S[c] <= P - 1), for no 2R >= p^L, and for 2R = p^L - 1 exactly
// when 2 S[c] <= P - 1; so it is R < floor(p^L / 2) + (bit c of tie).
__device__ __forceinline__ bool halton_lower(const HaltonDim &h, uint32_t R, uint32_t c) {
    return R < (h.pL >> 1) + ((h.tie >> c) & 1u);
}

// ------------------------------------------------------------------ Sobol'
__device__ __forceinline__ uint32_t sobol_x(const uint32_t *__restrict__ V, uint32_t shift, uint32_t n, int nbits) {
    uint32_t x = shift;
#pragma unroll 4
    for (int k = 0; k < nbits; ++k)
        if ((n >> k) & 1u) x ^= V[k];
    return x;
}

// ------------------------------------------------------------------ uniforms
// Every coordinate is delivered as (q, lower): q = (min(num, D-1-num) + 1/2)/D and
// lower = (num <= D-1-num).  u = lower ? q : 1 - q.
struct Unif32 {
    float q;
    bool lower;
};
struct Unif64 {
    double q;
    bool lower;
};

__device__ __forceinline__ Unif32 unif32_from_u32(uint32_t x) {
    const bool lower = x < 0x80000000u;
    const uint32_t qx = lower ? x : ~x;
    return Unif32{fmaf((float)qx, 2.3283064365386963e-10f, 1.1641532182693481e-10f), lower};
}
__device__ __forceinline__ Unif64 unif64_from_u32(uint32_t x) {
    const bool lower = x < 0x80000000u;
    const uint32_t qx = lower ? x : ~x;
    return Unif64{((double)qx + 0.5) * 2.3283064365386963e-10, lower};
}
__device__ __forceinline__ Unif32 unif32_halton(const HaltonDim &h, uint32_t R, uint32_t c) {
    const bool lower = halton_lower(h, R, c);
    const uint32_t Rs = lower ? R : h.pL - 1u - R;
    return Unif32{fmaf((float)Rs, h.inv_pL, lower ? h.a[c] : h.b[c]), lower};
}
__device__ __forceinline__ Unif64 unif64_halton(const HaltonDim &h, uint32_t R, uint32_t c) {
    const unsigned long long num = halton_num(h, R, c);
    const unsigned long long D1 = (unsigned long long)h.pL * h.P - 1ull;   // D - 1
    const bool lower = num <= D1 - num;
    const unsigned long long qn = lower ? num : D1 - num;
    return Unif64{((double)qn + 0.5) * h.invD, lower};
}

// Stateful per-thread coordinate source for one path (fixed m and point i) of sequence
// SEQ (compile time).  Philox words come four dimensions at a time and are cached.
template <int SEQ>
struct PathGen {
    GenView v;              // by value: the fields stay in (uniform) registers
    uint32_t i;
    unsigned long long n;   // offset + i
    int blk;
    U32x4 words;

    __device__ __forceinline__ void init(const GenView &gv, uint32_t i_) {
        v = gv;
        i = i_;
        n = gv.offset + i_;
        blk = -1;
    }
    __device__ __forceinline__ uint32_t philox_word(int j) {
        if ((j >> 2) != blk) {
            blk = j >> 2;
            words = philox4x32_10((uint32_t)n, (uint32_t)((n >> 32) & 0xFFFFu) | ((uint32_t)blk << 16),
                                  (uint32_t)v.m, kTagPath | (v.inst << 8), v.key0, v.key1);
        }
        const int w = j & 3;
        return w == 0 ? words.x : w == 1 ? words.y : w == 2 ? words.z : words.w;
    }
    __device__ __forceinline__ Unif32 unif32(int j) {
        if constexpr (SEQ == kPhilox) {
            return unif32_from_u32(philox_word(j));
        } else if constexpr (SEQ == kSobolDS) {
            return unif32_from_u32(sobol_x(v.V + 32 * j, v.shift[j], (uint32_t)n, v.sob_bits));
        } else {
            const HaltonDim &h = v.hd[j];
            uint32_t c;
            const uint32_t R = halton_R(h, v.sig, i, c);
            return unif32_halton(h, R, c);
        }
    }
    __device__ __forceinline__ Unif64 unif64(int j) {
        if constexpr (SEQ == kPhilox) {
            return unif64_from_u32(philox_word(j));
        } else if constexpr (SEQ == kSobolDS) {
            return unif64_from_u32(sobol_x(v.V + 32 * j, v.shift[j], (uint32_t)n, v.sob_bits));
        } else {
            const HaltonDim &h = v.hd[j];
            uint32_t c;
            const uint32_t R = halton_R(h, v.sig, i, c);
            return unif64_halton(h, R, c);
        }
    }
};

// Runtime sequence -> compile-time generator (HALTON_RS and RASRAP share one code path).
#define RQMC_SEQ_DISPATCH(seq, F)                                \
    ((seq) == kPhilox                            ? F(kPhilox)    \
     : ((seq) == kSobolDS || (seq) == kSobolLMS) ? F(kSobolDS)   \
                                                 : F(kRasrap))

// ------------------------------------------------------------------ inverse normal CDF
// erfinv(y)/y as a polynomial in w = -ln(4q(1-q)) (three branches, coefficients
// fitted by fit_ndtri.py); Phi^-1(u) = -/+ sqrt(2) y P(w), y = 1 - 2q.  The FP32 routines
// take the central branch as one polynomial in v = log2(q(1-q)) = -w/ln 2 - 2 that includes
// the factor sqrt(2) (RQMC_NDTRI_V), so no scaling or shift is spent before or after it.
template <typename T, int N>
__device__ __forceinline__ T horner(const T (&c)[N], T x) {
    T p = c[N - 1];
#pragma unroll
    for (int k = N - 2; k >= 0; --k) p = p * x + c[k];
    return p;
}

// sqrt(2) erfinv(y)/y from v = log2(q(1-q)): central polynomial for v > V_SPLIT (w < W_SPLIT),
// else the tail polynomials in sqrt(w).
__device__ __forceinline__ float erfinv_central32(float v) {
    constexpr float V[] = RQMC_NDTRI_V;
    return horner(V, v);
}
__device__ __forceinline__ float erfinv_tail32(float v) {
    constexpr float T[] = RQMC_NDTRI_T;
    constexpr float U[] = RQMC_NDTRI_U;
    const float w = -0.6931471805599453f * (v + 2.0f);
    const float sw = sqrt_approx(w);
    const float r = w < (float)RQMC_NDTRI_W_SPLIT2 ? horner(T, sw - (float)RQMC_NDTRI_T_MID)
                                                   : horner(U, sw - (float)RQMC_NDTRI_U_MID);
    return 1.4142135623730951f * r;
}
__device__ __forceinline__ float ndtri32_v(float q) { return lg2_approx(q * (1.0f - q)); }

__device__ __forceinline__ float ndtri32(Unif32 v) {
    const float q = v.q;
    const float lv = ndtri32_v(q);
    const float y = fmaf(-2.0f, q, 1.0f);
    const float x = y * (lv > (float)RQMC_NDTRI_V_SPLIT ? erfinv_central32(lv) : erfinv_tail32(lv));
    return v.lower ? -x : x;
}

__device__ __forceinline__ double erfinv_ratio64(double w) {
    constexpr double C[] = RQMC_NDTRI_C;
    constexpr double T[] = RQMC_NDTRI_T;
    constexpr double U[] = RQMC_NDTRI_U;
    if (w < RQMC_NDTRI_W_SPLIT) return horner(C, w - RQMC_NDTRI_W_MID);
    const double sw = sqrt(w);
    if (w < RQMC_NDTRI_W_SPLIT2) return horner(T, sw - RQMC_NDTRI_T_MID);
    return horner(U, sw - RQMC_NDTRI_U_MID);
}

// FP64: polynomial start (~1e-7 relative), then one Halley step on
// F(x) = erfc(-x/sqrt 2)/2 - q, which brings x to full double precision.
__device__ __forceinline__ double ndtri64(Unif64 v) {
    const double q = v.q;
    const double w = -log(4.0 * q * (1.0 - q));
    const double y = 1.0 - 2.0 * q;
    double x = -1.4142135623730951 * y * erfinv_ratio64(w);   // Phi^-1(q) <= 0
    if (q < 0.5) {
        const double F = 0.5 * erfc(-x * 0.7071067811865476) - q;
        const double dens = 0.3989422804014327 * exp(-0.5 * x * x);
        const double t = F / dens;
        x = x - t / (1.0 + 0.5 * x * t);
    }
    return v.lower ? x : -x;
}

// ------------------------------------------------------------------ reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ void kahan_add(T &sum, T &comp, T x) {
    const T y = x - comp;
    const T t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

}  // namespace rqmc
