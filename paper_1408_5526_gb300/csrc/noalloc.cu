// noalloc.cu -- caplet pricing that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they price: callbacks that run
// inside another framework's memory allocator (re-entering it can deadlock), processes
// whose device memory is entirely reserved up front by a pool, and latency-critical
// services whose policy forbids allocation after start-up.  For them
// rqmc_price_caplets_noalloc runs the same caplet kernel as price_caplets, but its scratch
// space -- the randomization tables, the per-tile partial sums and a status word -- lives
// in one file-scope __device__ array that the driver creates when it loads this library's
// module.  That array is kNoAllocScratchBytes (16 MiB) on every GPU that loads the library
// and stays allocated until the process exits.
//
// The host needs the array's device address; a __device__ symbol named in host code is
// only a host-side stand-in.  The first call on each device therefore looks the address
// up with cudaGetSymbolAddress (with that device current) and caches it.  All calls share
// the one array, so calls whose work overlaps on the GPU (different streams, or different
// host threads) race on it and must be serialised by the caller.  Every call rewrites the
// tables and every partial-sum row it reads, and clears the status word it uses, so
// nothing carries over between calls.  The call is asynchronous: a status word set on the
// device (a randomized point range beyond a Halton start's digits) turns every theta value
// of the call into NaN, which the caller sees when it reads theta.
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

// theta[0..n) = NaN when the call's status word is set (runs after the theta reduction).
__global__ void noalloc_poison_kernel(const uint32_t *__restrict__ status, double *__restrict__ theta, int n) {
    if (status[0] == 0u) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) theta[k] = nan("");
}

}  // namespace rqmc

using namespace rqmc;

extern "C" rqmc_status rqmc_price_caplets_noalloc(const rqmc_lmm_params *p, const double *strikes_host,
                                                  int n_strikes, int64_t N, int M, rqmc_sequence seq,
                                                  uint64_t seed, rqmc_precision prec, double *theta_dev,
                                                  void *stream) {
    // ---- arguments: the checks price_caplets runs, plus the output pointer
    if (!theta_dev) {
        set_error("rqmc_price_caplets_noalloc: theta_dev is required");
        return RQMC_EINVAL;
    }
    LmmCurve curve;
    rqmc_status rs = lmm_curve(p, curve);
    if (rs != RQMC_OK) return rs;
    p = &curve.p;
    rs = check_lmm(p, strikes_host, n_strikes, false);
    if (rs != RQMC_OK) return rs;
    if ((rs = common_checks(p->n_fwd * p->n_factors, N, 0, M, seq, prec)) != RQMC_OK) return rs;

    // ---- plan on the host stack; same launch shape and model constants as price_caplets
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
    pl.nf_bucket = lmm_bucket(p->n_fwd);
    pl.scheme = p->scheme;
    const int nout = p->n_fwd * n_strikes;
    set_reduction(pl, nout, 256, prec == RQMC_FP32 ? 2 : 1);
    if (prec == RQMC_FP32) fill_lmm(pl.lmm32, p, strikes_host, n_strikes, pl.nf_bucket);
    else fill_lmm(pl.lmm64, p, strikes_host, n_strikes, pl.nf_bucket);

    // ---- carve the static scratch array
    Carve cv;
    GenLayout gl;
    if ((rs = generator_layout(pl, cv, gl)) != RQMC_OK) return rs;
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
    const int n = M * nout;
    noalloc_poison_kernel<<<(n + 255) / 256, 256, 0, st>>>(status, theta_dev, n);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        set_error(std::string("rqmc_price_caplets_noalloc: launch failed: ") + cudaGetErrorString(e));
        return RQMC_ECUDA;
    }
    return RQMC_OK;
}
