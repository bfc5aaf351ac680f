// api.cu -- the C ABI of librqmc.so (declared in include/rqmc.h): argument validation,
// plan construction (device tables, model constants, workspace), launches, and the
// synchronous one-shot estimators.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "rqmc_internal.h"

namespace rqmc {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

static std::mutex g_oneshot_mu;

static rqmc_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return RQMC_ECUDA;
}

static bool finite_all(const double *p, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

static void keep_pool_cached(int dev) {
    static std::once_flag flags[64];
    if (dev < 0 || dev >= 64) return;
    std::call_once(flags[dev], [dev]() {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

// ------------------------------------------------------------------ plan construction
struct ModelHost {
    std::vector<unsigned char> bytes;   // model tables to copy after the generator tables
    size_t off = 0;
};

rqmc_status common_checks(int s, int64_t N, int64_t offset, int M, int seq, int prec) {
    if (s < 1 || s > kMaxDims) { set_error("s must be in 1..4096"); return RQMC_EINVAL; }
    if (N < 1 || N > (int64_t(1) << 31)) { set_error("N must be in 1..2^31"); return RQMC_EINVAL; }
    if (offset < 0) { set_error("offset must be >= 0"); return RQMC_EINVAL; }
    if (M < 1 || M > 65535) { set_error("M must be in 1..65535"); return RQMC_EINVAL; }
    if (seq < 0 || seq > 4) { set_error("unknown sequence"); return RQMC_EINVAL; }
    if (prec != RQMC_FP64 && prec != RQMC_FP32) { set_error("unknown precision"); return RQMC_EINVAL; }
    return RQMC_OK;
}

void set_reduction(Plan &pl, int nout, int threads, int ppt) {
    pl.threads = threads;
    pl.ppt = ppt;
    pl.nout = nout;
    RedParams &r = pl.red;
    r.nout = nout;
    r.ppt = ppt;
    r.tile = (uint32_t)(threads * ppt);
    r.tiles_per_m = (uint32_t)((pl.N + r.tile - 1) / r.tile);
    r.units = r.tiles_per_m * (uint32_t)pl.M;
    r.N = (uint32_t)pl.N;
}

// Largest normals buffer of an FP32 caplet plan; above it the caplet kernel generates its
// normals itself.
static constexpr size_t kMaxNormalsBytes = 8ull << 30;

// Allocates one device block: generator tables, model tables, status words, partials
// (sized for the smallest tile, 32 paths, so launch knobs can change later).
static rqmc_status finish_plan(Plan *pl, const std::vector<unsigned char> &model, size_t model_align,
                               size_t partial_doubles, cudaStream_t st, size_t *model_off_out) {
    Carve cv;
    GenLayout gl;
    rqmc_status rs = generator_layout(*pl, cv, gl);
    if (rs != RQMC_OK) return rs;
    const size_t model_off = model.empty() ? 0 : cv.take(model.size(), model_align);
    const size_t status_off = cv.take(sizeof(uint32_t) * 4);
    const size_t part_off = cv.take(sizeof(double) * std::max<size_t>(partial_doubles, 1));
    cudaGetDevice(&pl->device);
    keep_pool_cached(pl->device);
    pl->d_bytes = cv.off;
    cudaError_t e = cudaMallocAsync(&pl->d_buf, pl->d_bytes, st);
    if (e != cudaSuccess) {
        pl->d_buf = nullptr;
        set_error(std::string("device allocation failed: ") + cudaGetErrorString(e));
        return RQMC_ENOMEM;
    }
    unsigned char *d = static_cast<unsigned char *>(pl->d_buf);
    uint32_t *status = reinterpret_cast<uint32_t *>(d + status_off);
    if ((e = cudaMemsetAsync(status, 0, sizeof(uint32_t) * 4, st)) != cudaSuccess) return cuda_fail(e, "memset");
    if (!model.empty()) {
        if ((e = cudaMemcpyAsync(d + model_off, model.data(), model.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "model upload");
    }
    rs = generator_init(*pl, gl, d, status, st);
    if (rs != RQMC_OK) {
        set_error("generator setup launch failed");
        return rs;
    }
    pl->red.partials = reinterpret_cast<double *>(d + part_off);
    pl->red.status = status + 1;
    if (model_off_out) *model_off_out = model_off;
    if (st == 0) {   // plans outlive this call and may run on any stream: finish the setup now
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "plan setup");
    }
    return RQMC_OK;
}

static size_t partial_capacity(const Plan &pl, int nout) {
    // smallest tile is 32 paths
    return (size_t)pl.M * (size_t)((pl.N + 31) / 32) * (size_t)nout;
}

static void destroy(Plan *pl, cudaStream_t st) {
    if (!pl) return;
    if (pl->kind == kBatch) batch_destroy(*pl);
    if (pl->d_buf) cudaFreeAsync(pl->d_buf, st);
    if (pl->znorm) cudaFreeAsync(pl->znorm, st);
    if (pl->adj_buf) {
        cudaStreamSynchronize(st);
        cudaFree(pl->adj_buf);
    }
    delete pl->adjm;
    delete pl;
}

int lmm_bucket(int nf) {
    if (nf <= 16) return 16;
    if (nf <= 40) return 40;
    if (nf <= 80) return 80;
    return 160;
}

template <typename T>
void fill_lmm(LmmModel<T> &md, const rqmc_lmm_params *p, const double *K, int nK, int bucket) {
    const bool euler = p->scheme == RQMC_EULER;
    const double h = p->delta, sh = std::sqrt(p->delta);
    // FP32 log-Euler works in base 2; Euler carries delta L itself, in natural units
    const double sc = (sizeof(T) == 4 && !euler) ? 1.4426950408889634 : 1.0;
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
        const int n = slot + 1;   // forward index; slots beyond nf hold inert padding
        const bool real = n <= p->n_fwd;
        const double L0 = real ? p->L0[n] : p->L0[p->n_fwd];
        const double sg = real ? p->vol[n - 1] : 0.0;
        md.sig[slot] = (T)sg;
        md.cc[slot] = euler ? T(0) : (T)(-0.5 * sg * sg * h * sc);
        md.X0[slot] = euler ? (T)(p->delta * L0) : (T)(std::log(p->delta * L0) * sc);
    }
}

template void fill_lmm<float>(LmmModel<float> &, const rqmc_lmm_params *, const double *, int, int);
template void fill_lmm<double>(LmmModel<double> &, const rqmc_lmm_params *, const double *, int, int);

rqmc_status lmm_curve(const rqmc_lmm_params *in, LmmCurve &c) {
    if (!in) { set_error("LMM parameters missing"); return RQMC_EINVAL; }
    c.p = *in;
    c.L0.clear();
    if (in->init == 0) return RQMC_OK;
    if (in->init != 1) { set_error("init must be 0 (forwards) or 1 (bond prices)"); return RQMC_EINVAL; }
    if (!in->L0 || in->n_fwd < 1 || in->n_fwd > kMaxFwd || !(in->delta > 0.0) || !std::isfinite(in->delta)) {
        set_error("bond prices need n_fwd in 1..160, delta > 0 and nf + 2 prices");
        return RQMC_EINVAL;
    }
    const int nf = in->n_fwd;
    for (int n = 0; n < nf + 2; ++n)
        if (!(in->L0[n] > 0.0) || !std::isfinite(in->L0[n])) {
            set_error("bond prices must be positive and finite");
            return RQMC_EINVAL;
        }
    c.L0.resize(nf + 1);
    for (int n = 0; n <= nf; ++n) c.L0[n] = (in->L0[n] - in->L0[n + 1]) / (in->delta * in->L0[n + 1]);   // eq. BL
    c.p.L0 = c.L0.data();
    c.p.init = 0;
    return RQMC_OK;
}

rqmc_status check_lmm(const rqmc_lmm_params *p, const double *K, int nK, bool adjoint) {
    if (!p || !p->L0 || !p->vol) { set_error("LMM parameters missing"); return RQMC_EINVAL; }
    if (p->n_fwd < 1 || p->n_fwd > kMaxFwd) { set_error("n_fwd must be in 1..160"); return RQMC_EINVAL; }
    if (p->n_factors < 1 || p->n_factors > 2 || (!adjoint && p->n_factors != 1)) {
        set_error(adjoint ? "n_factors must be 1 or 2" : "price_caplets runs one-factor models (n_factors = 1)");
        return adjoint ? RQMC_EINVAL : RQMC_EUNSUPPORTED;
    }
    if (p->n_factors > 1 && !p->loadings) { set_error("loadings required for n_factors > 1"); return RQMC_EINVAL; }
    if (p->scheme != RQMC_LOG_EULER && p->scheme != RQMC_EULER) { set_error("unknown scheme"); return RQMC_EINVAL; }
    if (adjoint && p->scheme != RQMC_LOG_EULER) { set_error("the adjoint runs the log-Euler scheme"); return RQMC_EUNSUPPORTED; }
    if (!(p->delta > 0.0) || !std::isfinite(p->delta)) { set_error("delta must be > 0"); return RQMC_EINVAL; }
    if (!finite_all(p->L0, p->n_fwd + 1) || !finite_all(p->vol, p->n_fwd)) {
        set_error("L0/vol must be finite");
        return RQMC_EINVAL;
    }
    if (!(p->L0[0] > -1.0 / p->delta)) { set_error("1 + delta L_0(0) must be positive"); return RQMC_EINVAL; }
    for (int n = 1; n <= p->n_fwd; ++n)
        if (!(p->L0[n] > 0.0)) { set_error("initial forwards L_n(0), n >= 1, must be positive"); return RQMC_EINVAL; }
    if (!K || nK < 1 || nK > kMaxStrikes || !finite_all(K, nK)) {
        set_error("strikes: 1..8 finite values");
        return RQMC_EINVAL;
    }
    if (p->n_fwd * nK > kMaxOutputs) { set_error("n_fwd * n_strikes must be <= 1280"); return RQMC_EINVAL; }
    return RQMC_OK;
}

static rqmc_status check_mbs(const rqmc_mbs_params *p) {
    if (!p) { set_error("MBS parameters missing"); return RQMC_EINVAL; }
    if (p->months < 1 || p->months > kMaxDims) { set_error("months must be in 1..4096"); return RQMC_EINVAL; }
    const double v[] = {p->i0, p->K1, p->K2, p->K3, p->K4, p->sigma, p->c};
    if (!finite_all(v, 7) || p->i0 <= -1.0 || p->sigma < 0.0) { set_error("MBS constants invalid"); return RQMC_EINVAL; }
    return RQMC_OK;
}

}  // namespace rqmc

using namespace rqmc;

struct rqmc_plan_s : public Plan {};

// ------------------------------------------------------------------ diagnostics
extern "C" const char *rqmc_status_string(rqmc_status st) {
    switch (st) {
        case RQMC_OK: return "ok";
        case RQMC_EINVAL: return "invalid argument";
        case RQMC_ENOMEM: return "out of memory";
        case RQMC_ECUDA: return "CUDA error";
        case RQMC_ETIMEOUT: return "device wait timed out";
        case RQMC_EUNSUPPORTED: return "unsupported request";
        case RQMC_ENOTABLE: return "Sobol' direction table missing";
    }
    return "unknown status";
}
extern "C" const char *rqmc_last_error(void) { return g_err.c_str(); }
extern "C" int rqmc_abi_version(void) { return 1; }

// ------------------------------------------------------------------ plans
static rqmc_status new_plan(PlanKind kind, int s, int64_t N, int64_t offset, int M, rqmc_sequence seq, uint64_t seed,
                            rqmc_precision prec, rqmc_plan **out) {
    rqmc_status rs = common_checks(s, N, offset, M, seq, prec);
    if (rs != RQMC_OK) return rs;
    if (!out) { set_error("plan pointer is NULL"); return RQMC_EINVAL; }
    auto *pl = new rqmc_plan_s();
    pl->kind = kind;
    pl->prec = prec;
    pl->seq = seq;
    pl->s = s;
    pl->M = M;
    pl->N = (uint64_t)N;
    pl->offset = (uint64_t)offset;
    pl->seed = seed;
    pl->inst = 0;
    *out = pl;
    return RQMC_OK;
}

extern "C" rqmc_status rqmc_plan_product(int s, int64_t N, int64_t offset, int M, rqmc_sequence seq, uint64_t seed,
                                         const double *a_host, rqmc_precision prec, rqmc_plan **plan) {
    if (!a_host || !finite_all(a_host, std::max(0, std::min(s, kMaxDims)))) {
        set_error("a: s finite weights required");
        return RQMC_EINVAL;
    }
    rqmc_plan *pl = nullptr;
    rqmc_status rs = new_plan(kProduct, s, N, offset, M, seq, seed, prec, &pl);
    if (rs != RQMC_OK) return rs;
    set_reduction(*pl, 1, 256, 2);
    const size_t es = prec == RQMC_FP32 ? 4 : 8;
    std::vector<unsigned char> model(2 * es * s);
    for (int j = 0; j < s; ++j) {
        const double a = a_host[j], ia = 1.0 / (1.0 + a_host[j]);
        if (es == 4) {
            float af = (float)a, iaf = (float)ia;
            std::memcpy(&model[j * 4], &af, 4);
            std::memcpy(&model[(s + j) * 4], &iaf, 4);
        } else {
            std::memcpy(&model[j * 8], &a, 8);
            std::memcpy(&model[(s + j) * 8], &ia, 8);
        }
    }
    size_t moff = 0;
    rs = finish_plan(pl, model, 16, partial_capacity(*pl, 1), 0, &moff);
    if (rs != RQMC_OK) { destroy(pl, 0); return rs; }
    unsigned char *d = static_cast<unsigned char *>(pl->d_buf) + moff;
    if (es == 4) pl->prod32 = ProductModel<float>{s, (const float *)d, (const float *)(d + 4 * s)};
    else pl->prod64 = ProductModel<double>{s, (const double *)d, (const double *)(d + 8 * s)};
    pl->launches = 2;
    *plan = pl;
    return RQMC_OK;
}

extern "C" rqmc_status rqmc_plan_caplets(const rqmc_lmm_params *p, const double *strikes_host, int n_strikes,
                                         int64_t N, int64_t offset, int M, rqmc_sequence seq, uint64_t seed,
                                         rqmc_precision prec, rqmc_plan **plan) {
    LmmCurve curve;
    rqmc_status rs = lmm_curve(p, curve);
    if (rs != RQMC_OK) return rs;
    p = &curve.p;
    rs = check_lmm(p, strikes_host, n_strikes, false);
    if (rs != RQMC_OK) return rs;
    rqmc_plan *pl = nullptr;
    rs = new_plan(kCaplets, p->n_fwd * p->n_factors, N, offset, M, seq, seed, prec, &pl);
    if (rs != RQMC_OK) return rs;
    const int nout = p->n_fwd * n_strikes;
    pl->nf_bucket = lmm_bucket(p->n_fwd);
    pl->scheme = p->scheme;
    set_reduction(*pl, nout, 256, prec == RQMC_FP32 ? 2 : 1);
    if (prec == RQMC_FP32) fill_lmm(pl->lmm32, p, strikes_host, n_strikes, pl->nf_bucket);
    else fill_lmm(pl->lmm64, p, strikes_host, n_strikes, pl->nf_bucket);
    rs = finish_plan(pl, {}, 16, partial_capacity(*pl, nout), 0, nullptr);
    if (rs != RQMC_OK) { destroy(pl, 0); return rs; }
    pl->launches = 2;
    // FP32: the normals come from the point-stream run kernel, which shares the digit and bit
    // work of consecutive points, and the caplet kernel reads one per path and step
    const size_t zbytes = sizeof(float) * (size_t)M * (size_t)pl->s * (size_t)N;
    if (prec == RQMC_FP32 && points_runs_eligible(*pl) && zbytes <= kMaxNormalsBytes) {
        cudaError_t e = cudaMallocAsync(&pl->znorm, zbytes, 0);
        if (e != cudaSuccess) {
            pl->znorm = nullptr;
            destroy(pl, 0);
            set_error(std::string("device allocation failed (normals): ") + cudaGetErrorString(e));
            return RQMC_ENOMEM;
        }
        pl->launches = 3;
    }
    *plan = pl;
    return RQMC_OK;
}

extern "C" rqmc_status rqmc_plan_mbs(const rqmc_mbs_params *p, int64_t N, int64_t offset, int M, rqmc_sequence seq,
                                     uint64_t seed, rqmc_precision prec, rqmc_plan **plan) {
    rqmc_status rs = check_mbs(p);
    if (rs != RQMC_OK) return rs;
    rqmc_plan *pl = nullptr;
    rs = new_plan(kMbs, p->months, N, offset, M, seq, seed, prec, &pl);
    if (rs != RQMC_OK) return rs;
    set_reduction(*pl, 1, 256, prec == RQMC_FP32 ? mbs_paths32(seq) : 1);   // FP32: lockstep paths per thread
    const int Mm = p->months;
    const double v = 1.0 / (1.0 + p->i0);
    std::vector<double> ck(Mm + 1, 0.0);
    for (int k = 1; k <= Mm; ++k) {   // c_k = sum_{j=0}^{M-k} (1+i0)^-j
        double acc = 0.0, pw = 1.0;
        for (int j = 0; j <= Mm - k; ++j) { acc += pw; pw *= v; }
        ck[k] = acc;
    }
    const size_t es = prec == RQMC_FP32 ? 4 : 8;
    std::vector<unsigned char> model(es * (Mm + 1));
    for (int k = 0; k <= Mm; ++k) {
        if (es == 4) { float f = (float)ck[k]; std::memcpy(&model[k * 4], &f, 4); }
        else std::memcpy(&model[k * 8], &ck[k], 8);
    }
    size_t moff = 0;
    rs = finish_plan(pl, model, 16, partial_capacity(*pl, 1), 0, &moff);
    if (rs != RQMC_OK) { destroy(pl, 0); return rs; }
    const unsigned char *d = static_cast<unsigned char *>(pl->d_buf) + moff;
    const double s2 = p->sigma * p->sigma;
    if (es == 4) {
        const double l2e = 1.4426950408889634;
        pl->mbs32 = MbsModel<float>{Mm, (float)p->i0, (float)p->K1, (float)p->K2, (float)p->K3, (float)p->K4,
                                    (float)p->c, (float)v, (float)(-0.5 * s2 * l2e), (float)(p->sigma * l2e),
                                    (const float *)d};
    } else {
        pl->mbs64 = MbsModel<double>{Mm, p->i0, p->K1, p->K2, p->K3, p->K4, p->c, v, -0.5 * s2, p->sigma,
                                     (const double *)d};
    }
    pl->launches = 2;
    *plan = pl;
    return RQMC_OK;
}

extern "C" int64_t rqmc_plan_output_size(const rqmc_plan *plan) {
    if (!plan) return -1;
    if (plan->kind == kBatch) return batch_output_size(*plan);
    if (plan->kind == kPoints) return (int64_t)plan->M * plan->s * (int64_t)plan->N;
    return (int64_t)plan->M * plan->nout;
}

extern "C" int rqmc_plan_launches(const rqmc_plan *plan) { return plan ? plan->launches : 0; }

extern "C" rqmc_status rqmc_plan_get_launch(const rqmc_plan *plan, int *threads, int *paths_per_thread) {
    if (!plan || !threads || !paths_per_thread) { set_error("plan and both outputs are required"); return RQMC_EINVAL; }
    *threads = plan->threads;
    *paths_per_thread = plan->ppt;
    return RQMC_OK;
}

extern "C" rqmc_status rqmc_plan_set_launch(rqmc_plan *plan, int threads, int paths_per_thread) {
    if (!plan) { set_error("plan is NULL"); return RQMC_EINVAL; }
    if (plan->kind == kAdjoint || plan->kind == kBatch || plan->kind == kPoints) {
        set_error("adjoint, batch and point-stream plans fix their launch shape when they are built");
        return RQMC_EUNSUPPORTED;
    }
    int t = threads > 0 ? threads : plan->threads;
    int p = paths_per_thread > 0 ? paths_per_thread : plan->ppt;
    if (t % 32 != 0 || t < 32 || t > 256 || p < 1 || p > 64) {
        set_error("threads must be a multiple of 32 in 32..256, paths_per_thread in 1..64");
        return RQMC_EINVAL;
    }
    if (plan->kind == kCaplets) {
        const size_t es = plan->prec == RQMC_FP32 ? 4 : 8;
        if (2ull * (t / 32) * plan->nout * es > 200 * 1024) { set_error("accumulators exceed shared memory"); return RQMC_EINVAL; }
    }
    set_reduction(*plan, plan->nout, t, p);
    return RQMC_OK;
}

extern "C" rqmc_status rqmc_plan_execute(rqmc_plan *plan, double *theta_dev, void *stream) {
    if (!plan || !theta_dev) { set_error("plan and theta_dev are required"); return RQMC_EINVAL; }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != plan->device) {   // its tables live there
        set_error("the plan was built on device " + std::to_string(plan->device) + ", the current device is " +
                  std::to_string(cur));
        return RQMC_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (plan->kind == kBatch) return batch_execute(*plan, theta_dev, st);
    cudaError_t e;
    if (plan->kind == kPoints) {   // the buffer holds the coordinates, not theta
        if ((e = launch_points(*plan, plan->transform, theta_dev, st)) != cudaSuccess)
            return cuda_fail(e, "points launch");
        return RQMC_OK;
    }
    switch (plan->kind) {
        case kProduct: e = launch_product(*plan, st); break;
        case kCaplets:
            e = plan->znorm ? launch_points(*plan, RQMC_NORMAL, plan->znorm, st) : cudaSuccess;
            if (e == cudaSuccess) e = launch_caplets(*plan, st);
            break;
        case kMbs: e = launch_mbs(*plan, st); break;
        case kAdjoint:
            e = plan->znorm ? launch_points(*plan, RQMC_NORMAL, plan->znorm, st) : cudaSuccess;
            if (e == cudaSuccess) e = launch_adjoint(*plan, st);
            break;
        default: set_error("plan kind cannot be executed"); return RQMC_EUNSUPPORTED;
    }
    if (e != cudaSuccess) return cuda_fail(e, "path kernel launch");
    if ((e = launch_theta(*plan, theta_dev, st)) != cudaSuccess) return cuda_fail(e, "reduction launch");
    return RQMC_OK;
}

extern "C" rqmc_status rqmc_plan_check(rqmc_plan *plan, void *stream) {
    if (!plan) { set_error("plan is NULL"); return RQMC_EINVAL; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (plan->kind == kBatch) {
        const cudaError_t e = cudaStreamSynchronize(st);
        return e == cudaSuccess ? RQMC_OK : cuda_fail(e, "batch");
    }
    uint32_t h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, reinterpret_cast<unsigned char *>(plan->red.status) - sizeof(uint32_t),
                                    sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (h[0]) { set_error("randomized point range exceeds the start digits (offset + N too large)"); return RQMC_EUNSUPPORTED; }
    if (h[1] == 2) { set_error("device wait timed out"); return RQMC_ETIMEOUT; }
    if (h[1]) { set_error("device-side check failed"); return RQMC_ECUDA; }
    return RQMC_OK;
}

extern "C" rqmc_status rqmc_plan_destroy(rqmc_plan *plan) {
    if (!plan) return RQMC_OK;
    destroy(plan, 0);
    return RQMC_OK;
}

// ------------------------------------------------------------------ point stream
static rqmc_status make_points_plan(int s, int64_t N, int64_t offset, int M, rqmc_sequence seq, uint64_t seed,
                                    rqmc_precision prec, rqmc_transform tr, cudaStream_t st, rqmc_plan **plan) {
    if (tr < RQMC_UNIFORM || tr > RQMC_RAW) { set_error("unknown transform"); return RQMC_EINVAL; }
    if ((int64_t)M * s * N > (int64_t(1) << 40)) { set_error("output too large"); return RQMC_EINVAL; }
    rqmc_plan *pl = nullptr;
    rqmc_status rs = new_plan(kPoints, s, N, offset, M, seq, seed, prec, &pl);
    if (rs != RQMC_OK) return rs;
    pl->transform = tr;
    rs = finish_plan(pl, {}, 16, 1, st, nullptr);
    if (rs != RQMC_OK) { destroy(pl, st); return rs; }
    pl->launches = 1;
    *plan = pl;
    return RQMC_OK;
}

extern "C" rqmc_status rqmc_plan_points(int s, int64_t N, int64_t offset, int M, rqmc_sequence seq, uint64_t seed,
                                        rqmc_precision prec, rqmc_transform tr, rqmc_plan **plan) {
    return make_points_plan(s, N, offset, M, seq, seed, prec, tr, 0, plan);
}

extern "C" rqmc_status rqmc_points(int s, int64_t N, int M, rqmc_sequence seq, uint64_t seed, int64_t offset,
                                   rqmc_precision prec, rqmc_transform tr, void *out, void *stream) {
    if (!out) { set_error("out is NULL"); return RQMC_EINVAL; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    rqmc_plan *pl = nullptr;
    rqmc_status rs = make_points_plan(s, N, offset, M, seq, seed, prec, tr, st, &pl);
    if (rs != RQMC_OK) return rs;
    cudaError_t e = launch_points(*pl, pl->transform, out, st);
    destroy(pl, st);   // stream-ordered free after the kernel
    if (e != cudaSuccess) return cuda_fail(e, "points launch");
    return RQMC_OK;
}

// ------------------------------------------------------------------ one-shot estimators
static rqmc_status run_oneshot(rqmc_plan *pl, double *theta_host, double *rq_host, double *sd_host, void *stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = rqmc_plan_output_size(pl);
    double *theta_dev = nullptr;
    cudaError_t e = cudaMallocAsync(&theta_dev, sizeof(double) * n, st);
    if (e != cudaSuccess) { destroy(pl, st); set_error("device allocation failed"); return RQMC_ENOMEM; }
    rqmc_status rs = rqmc_plan_execute(pl, theta_dev, stream);
    if (rs == RQMC_OK) {
        e = cudaMemcpyAsync(theta_host, theta_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rs = cuda_fail(e, "result copy");
    }
    if (rs == RQMC_OK) rs = rqmc_plan_check(pl, stream);   // synchronises
    cudaFreeAsync(theta_dev, st);
    const int M = pl->M, nout = pl->nout;
    destroy(pl, st);
    if (rs != RQMC_OK) return rs;
    for (int o = 0; o < nout; ++o) {
        double mean = 0.0;
        for (int m = 0; m < M; ++m) mean += theta_host[(size_t)m * nout + o];
        mean /= M;
        double ss = 0.0;
        for (int m = 0; m < M; ++m) {
            const double d = theta_host[(size_t)m * nout + o] - mean;
            ss += d * d;
        }
        if (rq_host) rq_host[o] = mean;
        if (sd_host) sd_host[o] = M > 1 ? std::sqrt(ss / (M - 1)) : 0.0;
    }
    return RQMC_OK;
}

extern "C" rqmc_status rqmc_integrate_product(int s, int64_t N, int M, rqmc_sequence seq, uint64_t seed,
                                              const double *a_host, rqmc_precision prec, double *theta_host,
                                              double *rq_host, double *sd_host, void *stream) {
    if (!theta_host) { set_error("theta_host is NULL"); return RQMC_EINVAL; }
    std::lock_guard<std::mutex> lk(g_oneshot_mu);
    rqmc_plan *pl = nullptr;
    rqmc_status rs = rqmc_plan_product(s, N, 0, M, seq, seed, a_host, prec, &pl);
    if (rs != RQMC_OK) return rs;
    return run_oneshot(pl, theta_host, rq_host, sd_host, stream);
}

extern "C" rqmc_status price_caplets(const rqmc_lmm_params *p, const double *strikes_host, int n_strikes, int64_t N,
                                     int M, rqmc_sequence seq, uint64_t seed, rqmc_precision prec, double *theta_host,
                                     double *rq_host, double *sd_host, void *stream) {
    if (!theta_host) { set_error("theta_host is NULL"); return RQMC_EINVAL; }
    std::lock_guard<std::mutex> lk(g_oneshot_mu);
    rqmc_plan *pl = nullptr;
    rqmc_status rs = rqmc_plan_caplets(p, strikes_host, n_strikes, N, 0, M, seq, seed, prec, &pl);
    if (rs != RQMC_OK) return rs;
    return run_oneshot(pl, theta_host, rq_host, sd_host, stream);
}

extern "C" rqmc_status price_mbs(const rqmc_mbs_params *p, int64_t N, int M, rqmc_sequence seq, uint64_t seed,
                                 rqmc_precision prec, double *theta_host, double *rq_host, double *sd_host,
                                 void *stream) {
    if (!theta_host) { set_error("theta_host is NULL"); return RQMC_EINVAL; }
    std::lock_guard<std::mutex> lk(g_oneshot_mu);
    rqmc_plan *pl = nullptr;
    rqmc_status rs = rqmc_plan_mbs(p, N, 0, M, seq, seed, prec, &pl);
    if (rs != RQMC_OK) return rs;
    return run_oneshot(pl, theta_host, rq_host, sd_host, stream);
}

// ------------------------------------------------------------------ pathwise adjoint
extern "C" rqmc_status rqmc_plan_adjoint(const rqmc_lmm_params *p, const double *strikes_host, int n_strikes,
                                         const double *weights_host, int64_t N, int64_t offset, int M,
                                         rqmc_sequence seq, uint64_t seed, rqmc_precision prec, int checkpoint,
                                         rqmc_plan **plan) {
    LmmCurve curve;
    rqmc_status rs = lmm_curve(p, curve);
    if (rs != RQMC_OK) return rs;
    p = &curve.p;
    rs = check_lmm(p, strikes_host, n_strikes, true);
    if (rs != RQMC_OK) return rs;
    if (p->n_fwd > kMaxAdjFwd) { set_error("adjoint: n_fwd must be <= 80"); return RQMC_EUNSUPPORTED; }
    if (prec != RQMC_FP32) { set_error("adjoint: FP32 paths only"); return RQMC_EUNSUPPORTED; }
    if (checkpoint < 0 || checkpoint > 1) {
        set_error("adjoint: checkpoint must be 0 or 1 (the forward sweep records every step)");
        return RQMC_EINVAL;
    }
    const int nf = p->n_fwd, d = p->n_factors;
    if (!weights_host || !finite_all(weights_host, nf * n_strikes)) {
        set_error("adjoint: n_fwd * n_strikes finite weights required");
        return RQMC_EINVAL;
    }
    if (d == 2 && !finite_all(p->loadings, 2 * nf)) { set_error("adjoint: loadings must be finite"); return RQMC_EINVAL; }
    rqmc_plan *pl = nullptr;
    rs = new_plan(kAdjoint, nf * d, N, offset, M, seq, seed, prec, &pl);
    if (rs != RQMC_OK) return rs;
    const int nout = 1 + 2 * nf + nf * n_strikes;
    pl->nf_bucket = nf <= 40 ? 40 : 80;
    pl->checkpoint = 1;
    set_reduction(*pl, nout, kAdjointThreads, 4);
    AdjModel *md = new AdjModel();
    std::memset(md, 0, sizeof(AdjModel));
    pl->adjm = md;
    const double l2e = 1.4426950408889634, h = p->delta;
    md->nf = nf;
    md->nK = n_strikes;
    md->d = d;
    md->dl = (float)p->delta;
    md->inv_dl = (float)(1.0 / p->delta);
    md->disc0 = (float)(1.0 / (1.0 + p->delta * p->L0[0]));
    md->h = (float)h;
    md->sqh = (float)std::sqrt(h);
    bool any_w = false;
    for (int k = 0; k < n_strikes; ++k) md->K[k] = (float)strikes_host[k];
    for (int n = 0; n < pl->nf_bucket; ++n) {
        const bool real = n < nf;
        double b0 = 1.0, b1 = 0.0;
        if (real && d == 2) { b0 = p->loadings[2 * n]; b1 = p->loadings[2 * n + 1]; }
        const double vol = real ? p->vol[n] : 0.0;
        const double L0 = real ? p->L0[n + 1] : p->L0[nf];
        md->sg[n][0] = (float)(vol * b0);
        md->sg[n][1] = (float)(vol * b1);
        md->b[n][0] = (float)b0;
        md->b[n][1] = (float)b1;
        md->cc[n] = (float)(-0.5 * h * vol * vol * (b0 * b0 + b1 * b1) * l2e);
        md->X0[n] = (float)(std::log2(p->delta * L0));
        md->invL0ln2[n] = (float)(1.0 / (L0 * 0.6931471805599453));
        if (real)
            for (int k = 0; k < n_strikes; ++k) {
                md->w[n][k] = (float)weights_host[n * n_strikes + k];
                any_w = any_w || weights_host[n * n_strikes + k] != 0.0;
            }
    }
    md->reverse = any_w ? 1 : 0;
    rs = finish_plan(pl, {}, 16, (size_t)pl->red.units * nout, 0, nullptr);
    if (rs != RQMC_OK) { destroy(pl, 0); return rs; }
    // the normals from the point-stream run kernel, as for caplet plans (before the grid query:
    // the kernels that read them are the ones launched).  Not for Philox: one counter call
    // gives a path four coordinates, so generating them in the sweeps is cheaper than the
    // buffer's round trip through HBM (66.6 against 68.8 ms at 80 forwards, two factors,
    // N = 2^18, M = 32).
    const size_t zbytes = sizeof(float) * (size_t)M * (size_t)pl->s * (size_t)N;
    if (pl->seq != kPhilox && points_runs_eligible(*pl) && zbytes <= kMaxNormalsBytes) {
        cudaError_t ez = cudaMallocAsync(&pl->znorm, zbytes, 0);
        if (ez != cudaSuccess) {
            pl->znorm = nullptr;
            destroy(pl, 0);
            set_error(std::string("device allocation failed (normals): ") + cudaGetErrorString(ez));
            return RQMC_ENOMEM;
        }
    }
    pl->grid = adjoint_grid(*pl);
    if (pl->grid < 1) { destroy(pl, 0); set_error("adjoint: occupancy query failed"); return RQMC_ECUDA; }
    // per-thread columns (stride T): records, one float2 per step (the step's prefix total A);
    // adjoints Xb, NF/4 float4 chunks; then the accumulators
    const uint32_t T = (uint32_t)pl->grid * (uint32_t)pl->threads + 96;   // + 96: rows not 64 KiB-periodic
    const size_t rec_floats = 2 * (size_t)nf, xb_floats = (size_t)pl->nf_bucket;
    const size_t rows = 1 + 2 * (size_t)pl->nf_bucket + (size_t)nf * n_strikes;   // vega chunks, value, delta, prices
    pl->adjs.T = T;
    const size_t bytes = sizeof(float) * (rec_floats + xb_floats + rows) * T;
    void *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (e != cudaSuccess) { destroy(pl, 0); set_error("adjoint: scratch allocation failed"); return RQMC_ENOMEM; }
    pl->adj_buf = buf;
    pl->adjs.store = static_cast<float *>(buf);
    pl->adjs.xb = static_cast<float *>(buf) + rec_floats * T;
    pl->adjs.acc = pl->adjs.xb + xb_floats * T;
    if ((e = cudaMemset(pl->adjs.acc, 0, sizeof(float) * rows * T)) != cudaSuccess) {
        destroy(pl, 0);
        return cuda_fail(e, "adjoint scratch clear");
    }
    pl->launches = pl->znorm ? 3 : 2;
    *plan = pl;
    return RQMC_OK;
}

extern "C" rqmc_status price_adjoint(const rqmc_lmm_params *p, const double *strikes_host, int n_strikes,
                                     const double *weights_host, int64_t N, int M, rqmc_sequence seq, uint64_t seed,
                                     rqmc_precision prec, int checkpoint, double *value_host, double *delta_host,
                                     double *vega_host, void *stream) {
    if (!value_host || !delta_host || !vega_host) { set_error("adjoint outputs are required"); return RQMC_EINVAL; }
    std::lock_guard<std::mutex> lk(g_oneshot_mu);
    rqmc_plan *pl = nullptr;
    rqmc_status rs =
        rqmc_plan_adjoint(p, strikes_host, n_strikes, weights_host, N, 0, M, seq, seed, prec, checkpoint, &pl);
    if (rs != RQMC_OK) return rs;
    const int nf = p->n_fwd, nout = pl->nout;
    std::vector<double> th((size_t)M * nout);
    rs = run_oneshot(pl, th.data(), nullptr, nullptr, stream);
    if (rs != RQMC_OK) return rs;
    for (int m = 0; m < M; ++m) {
        const double *row = th.data() + (size_t)m * nout;
        value_host[m] = row[0];
        for (int n = 0; n < nf; ++n) {
            delta_host[(size_t)m * nf + n] = row[1 + n];
            vega_host[(size_t)m * nf + n] = row[1 + nf + n];
        }
    }
    return RQMC_OK;
}

extern "C" rqmc_status price_batch(const rqmc_instrument *inst, int n, int M, rqmc_sequence seq, uint64_t seed,
                                   rqmc_precision prec, double *theta_host, void *stream) {
    if (!theta_host) { set_error("theta_host is NULL"); return RQMC_EINVAL; }
    std::lock_guard<std::mutex> lk(g_oneshot_mu);
    rqmc_plan *pl = nullptr;
    rqmc_status rs = rqmc_plan_batch(inst, n, M, seq, seed, prec, &pl);
    if (rs != RQMC_OK) return rs;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t nd = rqmc_plan_output_size(pl);
    double *theta_dev = nullptr;
    cudaError_t e = cudaMallocAsync(&theta_dev, sizeof(double) * nd, st);
    if (e != cudaSuccess) { destroy(pl, st); set_error("device allocation failed"); return RQMC_ENOMEM; }
    rs = rqmc_plan_execute(pl, theta_dev, stream);
    if (rs == RQMC_OK) {
        e = cudaMemcpyAsync(theta_host, theta_dev, sizeof(double) * nd, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rs = cuda_fail(e, "batch result copy");
    }
    cudaFreeAsync(theta_dev, st);
    destroy(pl, st);
    return rs;
}
