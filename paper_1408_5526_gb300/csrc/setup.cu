// setup.cu -- randomization of every (replication m, dimension j) on the device.
//
// Halton / Rasrap (Sec. 3.1, Algorithm 3 step (1); readings c1, c2, c4): a 64-bit
// Philox word U gives omega = U / 2^64; its first K base-p digits, reversed, give
// the start n0 with |phi_p(n0) - omega| < p^-K.  The digit permutation sigma is a
// Fisher-Yates shuffle driven by Philox words (identity for random-start Halton).
// Sobol' (Sec. 3.2): direction numbers from the Joe-Kuo table by the primitive
// polynomial recurrence (host, once per process); digital shift per (m, j).
#include <cstring>
#include <mutex>

#include "rqmc_internal.h"

namespace rqmc {

// ------------------------------------------------------------------ primes
std::vector<uint32_t> first_primes(int s) {
    std::vector<uint32_t> out;
    out.reserve(s);
    for (uint32_t c = 2; (int)out.size() < s; ++c) {
        bool prime = true;
        for (uint32_t q : out) {
            if (q * q > c) break;
            if (c % q == 0) { prime = false; break; }
        }
        if (prime) out.push_back(c);
    }
    return out;
}

// ------------------------------------------------------------------ Sobol' directions
static std::mutex g_sobol_mu;
static std::vector<uint32_t> g_sobV;   // [n][32], V[k-1] = m_k 2^(32-k)
static int g_sob_dims = 0;

bool sobol_table_ready(int s) {
    std::lock_guard<std::mutex> lk(g_sobol_mu);
    return s <= g_sob_dims;
}
const std::vector<uint32_t> &sobol_directions() { return g_sobV; }

}  // namespace rqmc

using namespace rqmc;

extern "C" rqmc_status rqmc_set_sobol_table(const int64_t *poly, const int64_t *vinit, int n_dims, int max_deg) {
    if (!poly || !vinit || n_dims < 1 || n_dims > kMaxDims || max_deg < 1 || max_deg > 32) {
        set_error("rqmc_set_sobol_table: bad arguments");
        return RQMC_EINVAL;
    }
    std::vector<uint32_t> V((size_t)n_dims * 32);
    for (int j = 0; j < n_dims; ++j) {
        uint64_t m[33];
        if (j == 0) {
            for (int k = 1; k <= 32; ++k) m[k] = 1;   // van der Corput in base 2
        } else {
            const uint64_t P = (uint64_t)poly[j];
            int deg = 63 - __builtin_clzll(P | 1ull);
            if (deg < 1 || deg > max_deg) {
                set_error("rqmc_set_sobol_table: polynomial degree out of range");
                return RQMC_EINVAL;
            }
            for (int k = 1; k <= deg && k <= 32; ++k) m[k] = (uint64_t)vinit[(size_t)j * max_deg + k - 1];
            // m_k = 2 a_1 m_{k-1} xor ... xor 2^(deg-1) a_{deg-1} m_{k-deg+1} xor 2^deg m_{k-deg} xor m_{k-deg}
            for (int k = deg + 1; k <= 32; ++k) {
                uint64_t v = m[k - deg] ^ (m[k - deg] << deg);
                for (int i = 1; i < deg; ++i)
                    if ((P >> (deg - i)) & 1ull) v ^= m[k - i] << i;
                m[k] = v;
            }
        }
        for (int k = 1; k <= 32; ++k) {
            if (!(m[k] & 1ull) || m[k] >= (1ull << k)) {
                set_error("rqmc_set_sobol_table: direction numbers must be odd and below 2^k");
                return RQMC_EINVAL;
            }
            V[(size_t)j * 32 + k - 1] = (uint32_t)(m[k] << (32 - k));
        }
    }
    std::lock_guard<std::mutex> lk(g_sobol_mu);
    g_sobV.swap(V);
    g_sob_dims = n_dims;
    return RQMC_OK;
}

namespace rqmc {

// ------------------------------------------------------------------ device setup kernels
__device__ __forceinline__ unsigned long long high_numerator(unsigned long long H, const BaseConst &b,
                                                             const uint16_t *sg, bool &ok) {
    // digits of H occupy positions L, L+1, ...; positions < K are all permuted
    // (zeros included), position K only when nonzero, nothing may lie beyond K.
    unsigned long long num = 0, w = b.P / b.p;   // weight p^(K - L) of position L
    for (uint32_t k = b.L; k <= b.K; ++k) {
        const unsigned long long a = H % b.p;
        H /= b.p;
        if (k < b.K) num += (unsigned long long)sg[a] * w;
        else if (a != 0) num += sg[a];
        w /= b.p;
    }
    ok = (H == 0);
    return num;
}

// One thread per (m, j).  Bases up to kSetupSmemP shuffle their permutation in a private
// shared-memory row (the Fisher-Yates swaps are dependent random accesses, far slower in
// global memory) and copy it out at the end; larger bases shuffle in place in global memory.
constexpr uint32_t kSetupSmemP = 256;
constexpr int kSetupThreads = 64;
__global__ void __launch_bounds__(kSetupThreads)
    setup_halton_kernel(const BaseConst *__restrict__ bases, int s, int M, uint32_t key0, uint32_t key1,
                        uint32_t inst, unsigned long long offset, unsigned long long N, int identity,
                        HaltonDim *__restrict__ hdim, uint16_t *__restrict__ sigma, unsigned long long sig_len,
                        uint32_t *status) {
    __shared__ uint16_t work[kSetupThreads][kSetupSmemP + kSigPad];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * s) return;
    const int m = idx / s, j = idx % s;
    const BaseConst b = bases[j];
    // start: leading K base-p digits of omega = U / 2^64, reversed
    const U32x4 w = philox4x32_10((uint32_t)j, 0u, (uint32_t)m, kTagStart | (inst << 8), key0, key1);
    const unsigned long long U = (unsigned long long)w.x | ((unsigned long long)w.y << 32);
    unsigned long long lead = __umul64hi(U, b.pK);
    unsigned long long n0 = 0, pw = b.pK / b.p;   // p^(K-1) receives the least significant digit of lead
    for (uint32_t t = 0; t < b.K; ++t) {
        n0 += (lead % b.p) * pw;
        lead /= b.p;
        pw /= b.p;
    }
    // permutation
    uint16_t *const gsg = sigma + (size_t)m * sig_len + b.sig_off;
    const bool local = b.p <= kSetupSmemP;
    uint16_t *sg = local ? work[threadIdx.x] : gsg;
    for (uint32_t a = 0; a < b.p; ++a) sg[a] = (uint16_t)a;
    if (!identity) {
        U32x4 r4{};
        for (uint32_t k = b.p - 1, t = 0; k >= 1; --k, ++t) {
            if ((t & 3u) == 0)
                r4 = philox4x32_10((uint32_t)j, t >> 2, (uint32_t)m, kTagPerm | (inst << 8), key0, key1);
            const uint32_t word = (t & 3u) == 0 ? r4.x : (t & 3u) == 1 ? r4.y : (t & 3u) == 2 ? r4.z : r4.w;
            const uint32_t r = (uint32_t)(((unsigned long long)word * (k + 1)) >> 32);
            const uint16_t tmp = sg[k];
            sg[k] = sg[r];
            sg[r] = tmp;
        }
    }
    for (uint32_t a = 0; a < kSigPad; ++a) sg[b.p + a] = sg[a % b.p];
    if (local)
        for (uint32_t a = 0; a < b.p + kSigPad; ++a) gsg[a] = sg[a];
    // split of n0 + offset at digit L
    const unsigned long long n0o = n0 + offset;
    bool ok = n0o >= n0 && n0o <= b.D - N;   // n0 + offset + N - 1 < p^(K+1)
    const unsigned long long lo0 = n0o % b.pL, H = n0o / b.pL;
    HaltonDim h;
    h.P = b.P;
    bool ok0 = true, ok1 = true;
    h.S[0] = high_numerator(H, b, sg, ok0);
    h.S[1] = high_numerator(H + 1, b, sg, ok1);
    h.invD = b.invD;
    h.p = b.p;
    h.L = b.L;
    h.pL = b.pL;
    h.lo0 = (uint32_t)lo0;
    h.magic = b.magic;
    h.sig_off = b.sig_off;
    h.inv_pL = b.inv_pL;
    for (int c = 0; c < 2; ++c) {
        h.a[c] = (float)(((double)h.S[c] + 0.5) * b.invD);
        h.b[c] = (float)(((double)(b.P - 1ull - h.S[c]) + 0.5) * b.invD);
    }
    h.tie = 0;
    for (int c = 0; c < 2; ++c)
        if ((b.pL & 1u) && h.S[c] <= b.P - 1ull - h.S[c]) h.tie |= 1u << c;
    hdim[idx] = h;
    if (!(ok && ok0)) atomicOr(status, 1u);
    (void)ok1;   // the carry case is reached only by points the range check admits
}

__global__ void setup_shift_kernel(int s, int M, uint32_t key0, uint32_t key1, uint32_t inst,
                                   uint32_t *__restrict__ shift) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * s) return;
    const int m = idx / s, j = idx % s;
    shift[idx] = philox4x32_10((uint32_t)j, 0u, (uint32_t)m, kTagShift | (inst << 8), key0, key1).x;
}

// Matousek's random linear scrambling (Sec. 3.2): per (m, j) a unit lower-triangular binary
// matrix L over the coordinate's binary digits (most significant first).  Row r (output
// digit r) is a 32-bit mask over the input digits (digit l = bit 31 - l) with the diagonal
// set and, left of it, the top r bits of Philox word r - 1 of counters (j, (r-1)/4, m,
// tag 4).  The map is linear, L(XOR_k n_k v_k) = XOR_k n_k (L v_k), so the replication's
// direction numbers are scrambled once here and the kernels run the plain Sobol' code.
__global__ void setup_scramble_kernel(int s, int M, uint32_t key0, uint32_t key1, uint32_t inst,
                                      const uint32_t *__restrict__ V, uint32_t *__restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * s) return;
    const int m = idx / s, j = idx % s;
    uint32_t rows[32];
    rows[0] = 0x80000000u;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const U32x4 w = philox4x32_10((uint32_t)j, (uint32_t)b, (uint32_t)m, kTagScramble | (inst << 8), key0, key1);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = 4 * b + q + 1;   // row r uses word r - 1
            if (r < 32) rows[r] = ((ws[q] >> (32 - r)) << (32 - r)) | (0x80000000u >> r);
        }
    }
    const uint32_t *Vj = V + 32 * j;
    uint32_t *o = out + (size_t)idx * 32;
    for (int k = 0; k < 32; ++k) {
        const uint32_t v = Vj[k];
        uint32_t y = 0;
#pragma unroll
        for (int r = 0; r < 32; ++r) y |= (uint32_t)(__popc(rows[r] & v) & 1) << (31 - r);
        o[k] = y;
    }
}

// ------------------------------------------------------------------ host side
static int halton_K(uint32_t p) {
    unsigned long long pw = p;
    int k = 0;
    while (pw <= ~0ull / p) { pw *= p; ++k; }
    return k;
}

static unsigned long long upow(uint32_t p, int e) {
    unsigned long long r = 1;
    for (int i = 0; i < e; ++i) r *= p;
    return r;
}

// Sizes and per-base constants; validates the point range.
rqmc_status generator_layout(Plan &pl, Carve &cv, GenLayout &gl) {
    const int s = pl.s, M = pl.M;
    gl = GenLayout{};
    if (pl.seq == kHaltonRS || pl.seq == kRasrap) {
        std::vector<uint32_t> P = first_primes(s);
        gl.bases.resize(s);
        unsigned long long off = 0;
        for (int j = 0; j < s; ++j) {
            BaseConst &b = gl.bases[j];
            b.p = P[j];
            b.K = (uint32_t)halton_K(b.p);
            uint32_t L = 1;
            unsigned long long pl_ = b.p;
            while (pl_ < pl.N) { pl_ *= b.p; ++L; }
            if (pl_ > (1ull << 31) || L > b.K) {
                set_error("Halton: N too large for base " + std::to_string(b.p) + " (p^L must stay <= 2^31)");
                return RQMC_EUNSUPPORTED;
            }
            b.L = L;
            b.pL = (uint32_t)pl_;
            b.pK = upow(b.p, (int)b.K);
            b.D = b.pK * b.p;
            b.P = upow(b.p, (int)(b.K + 1 - L));
            b.magic = (uint32_t)((1ull << 32) / b.p + 1ull);
            b.sig_off = (uint32_t)off;
            b.inv_pL = (float)(1.0 / (double)b.pL);
            b.invD = 1.0 / (double)b.D;
            off += b.p + kSigPad;
        }
        gl.sig_len = off;
        gl.hdim_off = cv.take(sizeof(HaltonDim) * (size_t)M * s);
        gl.sigma_off = cv.take(sizeof(uint16_t) * (size_t)M * off);
        gl.base_off = cv.take(sizeof(BaseConst) * (size_t)s);
    } else if (pl.seq == kSobolDS || pl.seq == kSobolLMS) {
        if (!sobol_table_ready(s)) {
            set_error("Sobol': direction table covers fewer than s dimensions (call rqmc_set_sobol_table)");
            return RQMC_ENOTABLE;
        }
        if (pl.offset + pl.N > (1ull << 32)) {
            set_error("Sobol': offset + N must not exceed 2^32");
            return RQMC_EUNSUPPORTED;
        }
        gl.sobV_off = cv.take(sizeof(uint32_t) * 32 * (size_t)s);
        gl.shift_off = cv.take(sizeof(uint32_t) * (size_t)M * s);
        if (pl.seq == kSobolLMS) gl.scr_off = cv.take(sizeof(uint32_t) * 32 * (size_t)M * s);
    } else {
        if (pl.offset + pl.N > (1ull << 48)) {
            set_error("Philox: offset + N must not exceed 2^48");
            return RQMC_EUNSUPPORTED;
        }
    }
    return RQMC_OK;
}

rqmc_status generator_init(Plan &pl, const GenLayout &gl, unsigned char *d, uint32_t *d_status, cudaStream_t st) {
    const int s = pl.s, M = pl.M;
    GenParams &g = pl.gen;
    g.seq = pl.seq == kSobolLMS ? kSobolDS : pl.seq;   // kernels run scrambled tables as plain ones
    g.s = s;
    g.M = M;
    g.key0 = (uint32_t)pl.seed;
    g.key1 = (uint32_t)(pl.seed >> 32);
    g.inst = pl.inst;
    g.offset = pl.offset;
    g.stage = 1;
    const int nthr = 128, nblk = (M * s + nthr - 1) / nthr;
    if (pl.seq == kHaltonRS || pl.seq == kRasrap) {
        g.hdim = reinterpret_cast<const HaltonDim *>(d + gl.hdim_off);
        g.sigma = reinterpret_cast<const uint16_t *>(d + gl.sigma_off);
        g.sig_len = gl.sig_len;
        g.stage_sig = 2ull * gl.sig_len <= 48ull * 1024 ? 1 : 0;
        BaseConst *db = reinterpret_cast<BaseConst *>(d + gl.base_off);
        if (cudaMemcpyAsync(db, gl.bases.data(), sizeof(BaseConst) * s, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return RQMC_ECUDA;
        setup_halton_kernel<<<(M * s + kSetupThreads - 1) / kSetupThreads, kSetupThreads, 0, st>>>(
            db, s, M, g.key0, g.key1, g.inst, pl.offset, pl.N, pl.seq == kHaltonRS ? 1 : 0,
            const_cast<HaltonDim *>(g.hdim), const_cast<uint16_t *>(g.sigma), gl.sig_len, d_status);
    } else if (pl.seq == kSobolDS || pl.seq == kSobolLMS) {
        uint32_t *V = reinterpret_cast<uint32_t *>(d + gl.sobV_off);
        uint32_t *sh = reinterpret_cast<uint32_t *>(d + gl.shift_off);
        {
            std::lock_guard<std::mutex> lk(g_sobol_mu);
            if (cudaMemcpyAsync(V, g_sobV.data(), sizeof(uint32_t) * 32 * (size_t)s, cudaMemcpyHostToDevice, st) !=
                cudaSuccess)
                return RQMC_ECUDA;
            // pageable source: the copy has been staged before cudaMemcpyAsync returns
        }
        setup_shift_kernel<<<nblk, nthr, 0, st>>>(s, M, g.key0, g.key1, g.inst, sh);
        g.sobV = V;
        g.sobV_mstride = 0;
        g.sobShift = sh;
        if (pl.seq == kSobolLMS) {
            uint32_t *scr = reinterpret_cast<uint32_t *>(d + gl.scr_off);
            setup_scramble_kernel<<<nblk, nthr, 0, st>>>(s, M, g.key0, g.key1, g.inst, V, scr);
            g.sobV = scr;
            g.sobV_mstride = 32ull * s;
        }
        unsigned long long last = pl.offset + pl.N - 1;
        int bits = 1;
        while (bits < 32 && (last >> bits) != 0) ++bits;
        g.sob_bits = bits;
    }
    // Per-dimension tables of one replication go to shared memory when they fit comfortably
    // (up to 64 KB: s <= ~800 for Halton, ~490 for Sobol'); beyond, the kernels read them
    // from global memory (L1/L2-cached), so every s up to the API's limit runs.
    g.stage = stage_bytes(g) <= 64ull * 1024 ? 1 : 0;
    return cudaGetLastError() == cudaSuccess ? RQMC_OK : RQMC_ECUDA;
}

}  // namespace rqmc
