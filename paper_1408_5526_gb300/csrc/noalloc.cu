// noalloc.cu -- caplet pricing that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they price: code that runs
// while a CUDA graph is being captured (cudaMalloc is not a capturable operation),
// callbacks that run inside another framework's memory allocator (re-entering it can
// deadlock), processes whose device memory is entirely reserved up front by a pool, and
// latency-critical services whose policy forbids allocation after start-up.  For them
// rqmc_price_caplets_noalloc runs the same caplet kernel as price_caplets, but its scratch
// space -- the randomization tables, the per-tile partial sums and a status word -- lives
// in one file-scope __device__ array that the driver creates when it loads this library's
// module.  That array is kNoAllocScratchBytes (16 MiB) on every GPU that loads the library
// and stays allocated until the process exits.
//
// The host needs the array's device address; a __device__ symbol named in host code is
// only a host-side stand-in.  The first call on each device therefore looks the address
// up with cudaGetSymbolAddress (with that device current) and caches it; make that first
// call before any stream capture begins.  All calls share the one array, so calls whose
// work overlaps on the GPU (different streams, or different host threads) race on it and
// must be serialised by the caller.  Every call rewrites the tables and every partial-sum
// row it reads, and clears the status word it uses, so nothing carries over between calls.
#include <cmath>
#include <mutex>
#include <string>

#include "rqmc_internal.h"

namespace rqmc {

constexpr size_t kNoAllocScratchBytes = 16u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_addr[64];   // device address of the array, per device ordinal

static rqmc_status noalloc_scratch(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        set_error("rqmc_price_caplets_noalloc: no usable current CUDA device");
        return RQMC_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("rqmc_price_caplets_noalloc: cudaGetSymbolAddress failed: ") +
                      cudaGetErrorString(e));
            return RQMC_ECUDA;
        }
        g_noalloc_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_addr[dev];
    return RQMC_OK;
}

template <typename T>
static void noalloc_fill_model(LmmModel<T> &md, const rqmc_lmm_params *p, const double *K, int nK, int bucket) {
    const double h = p->delta, sh = std::sqrt(p->delta);
    const double sc = sizeof(T) == 4 ? 1.4426950408889634 : 1.0;   // FP32 works in base 2
    md = LmmModel<T>{};
    md.nf = p->n_fwd;
    md.nK = nK;
    md.dl = (T)p->delta;
    md.inv_dl = (T)(1.0 / p->delta);
    md.disc0 = (T)(1.0 / (1.0 + p->delta * p->L0[0]));
    md.hc = (T)(h * sc);
    md.sqhc = (T)(sh * sc);
    for (int k = 0; k < nK; ++k) md.K[k] = (T)K[k];
    for (int slot = 0; slot < bucket; ++slot) {
        const int n = slot + 1;
        const bool real = n <= p->n_fwd;
        const double L0 = real ? p->L0[n] : p->L0[p->n_fwd];
        const double sg = real ? p->vol[n - 1] : 0.0;
        md.sig[slot] = (T)sg;
        md.cc[slot] = (T)(-0.5 * sg * sg * h * sc);
        md.X0[slot] = (T)(std::log(p->delta * L0) * sc);
    }
}

}  // namespace rqmc

using namespace rqmc;

extern "C" rqmc_status rqmc_price_caplets_noalloc(const rqmc_lmm_params *p, const double *strikes_host,
                                                  int n_strikes, int64_t N, int M, rqmc_sequence seq,
                                                  uint64_t seed, rqmc_precision prec, double *theta_dev,
                                                  void *stream) {
    // ---- arguments (the same limits as price_caplets)
    if (!p || !p->L0 || !p->vol || !strikes_host || !theta_dev) {
        set_error("rqmc_price_caplets_noalloc: parameters, strikes and theta_dev are required");
        return RQMC_EINVAL;
    }
    if (p->n_fwd < 1 || p->n_fwd > kMaxFwd || p->n_factors != 1 || p->scheme != RQMC_LOG_EULER ||
        !(p->delta > 0.0) || !std::isfinite(p->delta) || n_strikes < 1 || n_strikes > kMaxStrikes ||
        N < 1 || N > (int64_t(1) << 31) || M < 1 || M > 65535 || seq < 0 || seq > 4 ||
        (prec != RQMC_FP32 && prec != RQMC_FP64)) {
        set_error("rqmc_price_caplets_noalloc: argument out of range (one-factor log-Euler, 1..160 forwards, "
                  "1..8 strikes, N in 1..2^31, M in 1..65535)");
        return RQMC_EINVAL;
    }
    if (!(p->L0[0] > -1.0 / p->delta) || !std::isfinite(p->L0[0])) {
        set_error("rqmc_price_caplets_noalloc: 1 + delta L_0(0) must be positive");
        return RQMC_EINVAL;
    }
    for (int n = 1; n <= p->n_fwd; ++n)
        if (!(p->L0[n] > 0.0) || !std::isfinite(p->L0[n]) || !std::isfinite(p->vol[n - 1])) {
            set_error("rqmc_price_caplets_noalloc: initial forwards must be positive and finite");
            return RQMC_EINVAL;
        }
    for (int k = 0; k < n_strikes; ++k)
        if (!std::isfinite(strikes_host[k])) {
            set_error("rqmc_price_caplets_noalloc: strikes must be finite");
            return RQMC_EINVAL;
        }

    // ---- plan on the host stack; same launch shape as price_caplets
    Plan pl{};
    pl.kind = kCaplets;
    pl.prec = prec;
    pl.seq = seq;
    pl.s = p->n_fwd;
    pl.M = M;
    pl.N = (uint64_t)N;
    pl.offset = 0;
    pl.seed = seed;
    pl.inst = 0;
    pl.nf_bucket = p->n_fwd <= 16 ? 16 : p->n_fwd <= 40 ? 40 : p->n_fwd <= 80 ? 80 : 160;
    const int nout = p->n_fwd * n_strikes;
    pl.threads = 256;
    pl.ppt = prec == RQMC_FP32 ? 2 : 1;
    pl.nout = nout;
    pl.red.nout = nout;
    pl.red.ppt = pl.ppt;
    pl.red.tile = (uint32_t)(pl.threads * pl.ppt);
    pl.red.tiles_per_m = (uint32_t)((pl.N + pl.red.tile - 1) / pl.red.tile);
    pl.red.units = pl.red.tiles_per_m * (uint32_t)M;
    pl.red.N = (uint32_t)N;
    if (prec == RQMC_FP32) noalloc_fill_model(pl.lmm32, p, strikes_host, n_strikes, pl.nf_bucket);
    else noalloc_fill_model(pl.lmm64, p, strikes_host, n_strikes, pl.nf_bucket);

    // ---- carve the static scratch array
    Carve cv;
    GenLayout gl;
    rqmc_status rs = generator_layout(pl, cv, gl);
    if (rs != RQMC_OK) return rs;
    const size_t status_off = cv.take(sizeof(uint32_t) * 4);
    const size_t part_off = cv.take(sizeof(double) * (size_t)pl.red.units * nout);
    if (cv.off > kNoAllocScratchBytes) {
        set_error("rqmc_price_caplets_noalloc: this request needs " + std::to_string(cv.off) +
                  " bytes of scratch but the built-in array holds " + std::to_string(kNoAllocScratchBytes) +
                  " bytes; use price_caplets or a plan for larger N, M or n_fwd");
        return RQMC_EINVAL;
    }
    unsigned char *d = nullptr;
    if ((rs = noalloc_scratch(&d)) != RQMC_OK) return rs;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint32_t *status = reinterpret_cast<uint32_t *>(d + status_off);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(uint32_t) * 4, st);
    if (e != cudaSuccess) {
        set_error(std::string("rqmc_price_caplets_noalloc: ") + cudaGetErrorString(e));
        return RQMC_ECUDA;
    }
    if ((rs = generator_init(pl, gl, d, status, st)) != RQMC_OK) {
        set_error("rqmc_price_caplets_noalloc: generator setup launch failed");
        return rs;
    }
    pl.red.partials = reinterpret_cast<double *>(d + part_off);
    pl.red.status = status + 1;
    if ((e = launch_caplets(pl, st)) != cudaSuccess || (e = launch_theta(pl, theta_dev, st)) != cudaSuccess) {
        set_error(std::string("rqmc_price_caplets_noalloc: launch failed: ") + cudaGetErrorString(e));
        return RQMC_ECUDA;
    }
    return RQMC_OK;
}
