// batch.cu -- host side of the batched launch: instrument validation, per-instrument
// randomization tables and models, longest-first work lists (one per work class: LMM
// strips, MBS), CUDA-graph capture of [ticket reset -> the two persistent kernels as
// parallel branches -> per-instrument theta], and the tile autotuner.
//
// The autotuner times the captured launch for several tile sizes (paths per thread) on a
// copy of the batch with N capped at 8192 per instrument and keeps the fastest; the choice
// (and each candidate's time in microseconds, under "<key>|us_ppt<k>") is cached in a
// small JSON file keyed by GPU name, sequence and a hash of the batch
// (path: $RQMC_AUTOTUNE_CACHE, default ~/.cache/rqmc_gb300/autotune.json;
// RQMC_AUTOTUNE=0 skips tuning and uses 4 paths per thread).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <sys/stat.h>
#include <vector>

#include "k_batch.cuh"

namespace rqmc {

struct BatchPlan {
    std::vector<rqmc_instrument> desc;
    int M = 0, seq = 0, n = 0;
    uint64_t seed = 0;
    void *d_tables = nullptr;     // generator tables of every instrument + models + status
    void *d_work = nullptr;       // insts, items, counter, partials, theta
    BatchLaunch bl{};
    size_t theta_doubles = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;                             // capture stream (class 0)
    cudaStream_t side[kBatchClasses - 1] = {};              // classes 1.. (forked)
    cudaEvent_t fork = nullptr, join[kBatchClasses - 1] = {};
    std::vector<BatchInst> insts;   // host copy (device pointers filled)
    size_t smem_lmm_base = 0;
};

static const double kL2e = 1.4426950408889634;

static int lmm_bucket_of(int nf) { return nf <= 16 ? 16 : nf <= 40 ? 40 : nf <= 80 ? 80 : 160; }

static void fill_lmm_flat(LmmModel<float> &md, int nf, double rate, double vol, double K) {
    const double dl = 0.25, h = dl, sh = std::sqrt(dl);
    md = LmmModel<float>{};
    md.nf = nf;
    md.nK = 1;
    md.dl = (float)dl;
    md.inv_dl = (float)(1.0 / dl);
    md.disc0 = (float)(1.0 / (1.0 + dl * rate));
    md.hc = (float)(h * kL2e);
    md.sqhc = (float)(sh * kL2e);
    md.K[0] = (float)K;
    for (int slot = 0; slot < lmm_bucket_of(nf); ++slot) {
        const double sg = slot < nf ? vol : 0.0;
        md.sig[slot] = (float)sg;
        md.cc[slot] = (float)(-0.5 * sg * sg * h * kL2e);
        md.X0[slot] = (float)(std::log2(dl * rate));
    }
}

// shared memory of one item (must match batch_lmm / batch_mbs layouts)
static size_t item_smem(const BatchInst &bi, int threads) {
    const int nw = threads / 32;
    if (bi.kind == 0) {
        size_t a, b, c, d, e;
        switch (bi.bucket) {
            case 16: return lmm_smem_layout<16, float, batch_ilp<16>()>(bi.g, nw, 1, bi.nout, &a, &b, &c, &d, &e,
                                                                        batch_zg<16>() ? 2 : 1);
            case 40: return lmm_smem_layout<40, float, batch_ilp<40>()>(bi.g, nw, 1, bi.nout, &a, &b, &c, &d, &e,
                                                                        batch_zg<40>() ? 2 : 1);
            case 80: return lmm_smem_layout<80, float, batch_ilp<80>()>(bi.g, nw, 1, bi.nout, &a, &b, &c, &d, &e,
                                                                        batch_zg<80>() ? 2 : 1);
            default: return lmm_smem_layout<160, float, batch_ilp<160>()>(bi.g, nw, 1, bi.nout, &a, &b, &c, &d, &e,
                                                                          batch_zg<160>() ? 2 : 1);
        }
    }
    return stage_bytes(bi.g) + sizeof(float) * (2 * (size_t)nw + (size_t)bi.g.s + 1);
}

static double item_cost(const rqmc_instrument &d) {
    // forward updates per path for LMM; an MBS month costs about three updates
    return d.kind == 0 ? 0.5 * d.size * (d.size + 1.0) : 3.0 * d.size;
}

// Items of each work class (see BatchLaunch), each list longest first.
static rqmc_status build_work(BatchPlan &bp, int threads, int ppt, bool cap_n, std::vector<BatchInst> &insts,
                              std::vector<BatchItem> (&items)[kBatchClasses], size_t &part_doubles,
                              size_t &theta_doubles, size_t (&smem)[kBatchClasses]) {
    const uint32_t tile = (uint32_t)(threads * ppt);
    part_doubles = theta_doubles = 0;
    for (auto &x : smem) x = 0;
    std::vector<std::pair<double, BatchItem>> order[kBatchClasses];
    for (int i = 0; i < bp.n; ++i) {
        BatchInst &bi = insts[i];
        const uint64_t N = cap_n ? std::min<uint64_t>((uint64_t)bp.desc[i].N, 8192) : (uint64_t)bp.desc[i].N;
        bi.N = (uint32_t)N;
        bi.tiles_per_m = (uint32_t)((N + tile - 1) / tile);
        bi.part_off = part_doubles;
        bi.theta_off = theta_doubles;
        part_doubles += (size_t)bp.M * bi.tiles_per_m * bi.nout;
        theta_doubles += (size_t)bp.M * bi.nout;
        const int cls = batch_class(bi);
        smem[cls] = std::max(smem[cls], item_smem(bi, threads));
        const double c = item_cost(bp.desc[i]);
        for (int m = 0; m < bp.M; ++m)
            for (uint32_t t = 0; t < bi.tiles_per_m; ++t) {
                const uint32_t paths = std::min<uint64_t>(tile, N - (uint64_t)t * tile);
                order[cls].push_back({c * paths, BatchItem{(uint32_t)i, (uint32_t)m, t, 0u}});
            }
    }
    for (int cls = 0; cls < kBatchClasses; ++cls) {
        std::stable_sort(order[cls].begin(), order[cls].end(),
                         [](const std::pair<double, BatchItem> &a, const std::pair<double, BatchItem> &b) {
                             return a.first > b.first;
                         });
        items[cls].resize(order[cls].size());
        for (size_t k = 0; k < order[cls].size(); ++k) items[cls][k] = order[cls][k].second;
    }
    return RQMC_OK;
}

static void free_work(BatchPlan &bp) {
    if (bp.exec) cudaGraphExecDestroy(bp.exec);
    if (bp.graph) cudaGraphDestroy(bp.graph);
    bp.exec = nullptr;
    bp.graph = nullptr;
    if (bp.d_work) cudaFree(bp.d_work);
    bp.d_work = nullptr;
}

// Allocates the work buffers for one launch shape and captures the graph.
static rqmc_status setup_launch(BatchPlan &bp, int threads, int ppt, bool cap_n) {
    free_work(bp);
    std::vector<BatchInst> insts = bp.insts;
    std::vector<BatchItem> items[kBatchClasses];
    size_t part = 0, theta = 0, smem[kBatchClasses] = {};
    build_work(bp, threads, ppt, cap_n, insts, items, part, theta, smem);
    if (*std::max_element(smem, smem + kBatchClasses) > 227 * 1024) {
        set_error("batch: an instrument needs more shared memory than a CTA has");
        return RQMC_EUNSUPPORTED;
    }
    Carve cv;
    const size_t o_inst = cv.take(sizeof(BatchInst) * insts.size());
    size_t o_items[kBatchClasses];
    for (int k = 0; k < kBatchClasses; ++k) o_items[k] = cv.take(sizeof(BatchItem) * std::max<size_t>(items[k].size(), 1));
    const size_t o_cnt = cv.take(sizeof(uint32_t) * 4);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t stats_cap = 8u * (uint32_t)std::max(sms, 1);   // at most 8 CTAs of 256 threads per SM
    const size_t o_stats = cv.take(sizeof(unsigned long long) * 3 * kBatchClasses * stats_cap);
    const size_t o_part = cv.take(sizeof(double) * part);
    const size_t o_theta = cv.take(sizeof(double) * theta);
    // normals buffers of the strip classes: one per CTA of the persistent grid (one CTA per SM
    // in class 0, two in class 2: their register budgets), the class's largest bucket x the tile
    const uint32_t tile = (uint32_t)(threads * ppt);
    int zbucket[kBatchClasses] = {};
    for (const BatchInst &bi : insts)
        if (bi.kind == 0 && batch_zg_bucket(bi.bucket)) zbucket[batch_class(bi)] = std::max(zbucket[batch_class(bi)], bi.bucket);
    size_t o_z[kBatchClasses] = {}, zstride[kBatchClasses] = {};
    uint32_t zctas[kBatchClasses] = {};
    for (int k = 0; k < kBatchClasses; ++k) {
        if (!zbucket[k] || items[k].empty()) continue;
        zctas[k] = (uint32_t)std::max(sms, 1) * (k == 0 ? 1u : 2u);
        zstride[k] = (size_t)zbucket[k] * tile;
        o_z[k] = cv.take(sizeof(float) * zstride[k] * zctas[k]);
    }
    cudaError_t e = cudaMalloc(&bp.d_work, cv.off);
    if (e != cudaSuccess) { bp.d_work = nullptr; set_error("batch: work allocation failed"); return RQMC_ENOMEM; }
    unsigned char *d = static_cast<unsigned char *>(bp.d_work);
    bool up = cudaMemcpy(d + o_inst, insts.data(), sizeof(BatchInst) * insts.size(), cudaMemcpyHostToDevice) ==
              cudaSuccess;
    for (int k = 0; k < kBatchClasses; ++k)
        up = up && (items[k].empty() || cudaMemcpy(d + o_items[k], items[k].data(), sizeof(BatchItem) * items[k].size(),
                                                   cudaMemcpyHostToDevice) == cudaSuccess);
    if (!up) {
        set_error("batch: upload failed");
        return RQMC_ECUDA;
    }
    BatchLaunch &bl = bp.bl;
    bl.insts = reinterpret_cast<const BatchInst *>(d + o_inst);
    for (int k = 0; k < kBatchClasses; ++k) {
        bl.items[k] = reinterpret_cast<const BatchItem *>(d + o_items[k]);
        bl.n_items[k] = (uint32_t)items[k].size();
        bl.smem[k] = smem[k];
    }
    bl.n_inst = (uint32_t)insts.size();
    bl.counter = reinterpret_cast<uint32_t *>(d + o_cnt);
    bl.stats = reinterpret_cast<unsigned long long *>(d + o_stats);
    bl.stats_cap = stats_cap;
    bl.partials = reinterpret_cast<double *>(d + o_part);
    bl.theta = reinterpret_cast<double *>(d + o_theta);
    bl.threads = threads;
    bl.ppt = ppt;
    for (int k = 0; k < kBatchClasses; ++k) {
        bl.znorm[k] = zctas[k] ? reinterpret_cast<float *>(d + o_z[k]) : nullptr;
        bl.zstride[k] = zstride[k];
        bl.zctas[k] = zctas[k];
    }
    bl.fork = bp.fork;
    for (int k = 0; k + 1 < kBatchClasses; ++k) {
        bl.side[k] = bp.side[k];
        bl.join[k] = bp.join[k];
    }
    bp.theta_doubles = theta;
    // one direct launch sets kernel attributes outside the capture, then capture the graph
    if ((e = launch_batch(bl, bp.seq, bp.cap)) != cudaSuccess) return RQMC_ECUDA;
    if ((e = cudaStreamSynchronize(bp.cap)) != cudaSuccess) { set_error(cudaGetErrorString(e)); return RQMC_ECUDA; }
    if ((e = cudaStreamBeginCapture(bp.cap, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return RQMC_ECUDA;
    cudaError_t le = launch_batch(bl, bp.seq, bp.cap);
    e = cudaStreamEndCapture(bp.cap, &bp.graph);
    if (le != cudaSuccess || e != cudaSuccess) { set_error("batch: graph capture failed"); return RQMC_ECUDA; }
    if ((e = cudaGraphInstantiate(&bp.exec, bp.graph, 0)) != cudaSuccess) {
        set_error(std::string("batch: graph instantiation failed: ") + cudaGetErrorString(e));
        return RQMC_ECUDA;
    }
    return RQMC_OK;
}

// ------------------------------------------------------------------ autotuner cache
static std::string cache_path() {
    const char *p = std::getenv("RQMC_AUTOTUNE_CACHE");
    if (p && *p) return p;
    const char *home = std::getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/rqmc_gb300/autotune.json";
}

static std::map<std::string, int> cache_read() {
    std::map<std::string, int> out;
    std::ifstream f(cache_path());
    std::string line;
    while (std::getline(f, line)) {   // one `"key": value,` entry per line
        const size_t a = line.find('"'), b = line.rfind('"'), c = line.rfind(':');
        if (a == std::string::npos || b <= a || c == std::string::npos || c < b) continue;
        out[line.substr(a + 1, b - a - 1)] = std::atoi(line.c_str() + c + 1);
    }
    return out;
}

static void cache_write(const std::map<std::string, int> &kv) {
    const std::string p = cache_path();
    for (size_t i = 1; i < p.size(); ++i)
        if (p[i] == '/') mkdir(p.substr(0, i).c_str(), 0755);
    std::ofstream f(p + ".tmp");
    f << "{\n";
    size_t k = 0;
    for (const auto &e : kv) f << "  \"" << e.first << "\": " << e.second << (++k < kv.size() ? ",\n" : "\n");
    f << "}\n";
    f.close();
    std::rename((p + ".tmp").c_str(), p.c_str());
}

static std::string batch_key(const BatchPlan &bp) {
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    uint64_t h = 1469598103934665603ull;   // FNV-1a over the instrument list
    auto mix = [&h](const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    };
    for (const auto &d : bp.desc) {
        mix(&d.kind, sizeof d.kind);
        mix(&d.size, sizeof d.size);
        mix(&d.N, sizeof d.N);
    }
    mix(&bp.M, sizeof bp.M);
    std::ostringstream s;
    s << prop.name << "|seq" << bp.seq << "|" << std::hex << h;
    std::string k = s.str();
    for (auto &ch : k)
        if (ch == '"' || ch == '\\') ch = '_';
    return k;
}

static float time_launch(BatchPlan &bp) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaGraphLaunch(bp.exec, bp.cap);
    cudaEventRecord(a, bp.cap);
    cudaGraphLaunch(bp.exec, bp.cap);
    cudaEventRecord(b, bp.cap);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

static int autotune(BatchPlan &bp) {
    const char *env = std::getenv("RQMC_AUTOTUNE");
    if (env && std::strcmp(env, "0") == 0) return 4;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    const std::string key = batch_key(bp);
    auto kv = cache_read();
    auto it = kv.find(key);
    if (it != kv.end() && it->second >= 1 && it->second <= 16) return it->second;
    int best = 4;
    float best_ms = 1e30f;
    for (int ppt : {4, 8, 16}) {   // multiples of every bucket's paths per thread in lockstep
        if (setup_launch(bp, 256, ppt, true) != RQMC_OK) continue;
        const float ms = time_launch(bp);
        kv[key + "|us_ppt" + std::to_string(ppt)] = (int)std::lround(1000.0 * ms);   // the candidate's time
        if (ms < best_ms) { best_ms = ms; best = ppt; }
    }
    kv[key] = best;
    cache_write(kv);
    return best;
}

}  // namespace rqmc

using namespace rqmc;

struct rqmc_plan_s : public Plan {};

extern "C" rqmc_status rqmc_plan_batch(const rqmc_instrument *inst, int n, int M, rqmc_sequence seq, uint64_t seed,
                                       rqmc_precision prec, rqmc_plan **plan) {
    if (!inst || !plan || n < 1 || n > (1 << 20) || M < 1 || M > 65535 || seq < 0 || seq > 4) {
        set_error("batch: instruments, n in 1..2^20 and M in 1..65535 are required");
        return RQMC_EINVAL;
    }
    if (prec != RQMC_FP32) { set_error("batch: FP32 paths only"); return RQMC_EUNSUPPORTED; }
    for (int i = 0; i < n; ++i) {
        const rqmc_instrument &d = inst[i];
        const bool okN = d.N >= 1 && d.N <= (int64_t(1) << 31);
        bool ok = false;
        if (d.kind == 0)
            ok = d.size >= 1 && d.size <= kMaxFwd && d.rate > 0.0 && std::isfinite(d.rate) && d.vol >= 0.0 &&
                 std::isfinite(d.vol) && std::isfinite(d.strike);
        else if (d.kind == 1) {
            const double v[] = {d.mbs.i0, d.mbs.K1, d.mbs.K2, d.mbs.K3, d.mbs.K4, d.mbs.sigma, d.mbs.c};
            ok = d.size >= 1 && d.size <= kMaxDims && d.mbs.i0 > -1.0 && d.mbs.sigma >= 0.0;
            for (double x : v) ok = ok && std::isfinite(x);
        }
        if (!ok || !okN) {
            set_error("batch: instrument " + std::to_string(i) + " is invalid");
            return RQMC_EINVAL;
        }
    }
    auto *pl = new rqmc_plan_s();
    pl->kind = kBatch;
    pl->prec = prec;
    pl->seq = seq;
    pl->M = M;
    pl->seed = seed;
    cudaGetDevice(&pl->device);
    BatchPlan *bp = new BatchPlan();
    pl->batch = bp;
    bp->desc.assign(inst, inst + n);
    bp->M = M;
    bp->seq = seq;
    bp->n = n;
    bp->seed = seed;
    auto fail = [&](rqmc_status st) {
        rqmc_plan_destroy(pl);
        return st;
    };
    bool made = cudaStreamCreateWithFlags(&bp->cap, cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&bp->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k + 1 < kBatchClasses; ++k)
        made = made && cudaStreamCreateWithFlags(&bp->side[k], cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&bp->join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!made) return fail(RQMC_ECUDA);
    // generator tables of every instrument (instrument index i in the counters), models
    std::vector<Plan> sub(n);
    std::vector<GenLayout> gls(n);
    Carve cv;
    std::vector<size_t> base(n), model_off(n);
    int n_class[kBatchClasses] = {};
    for (int i = 0; i < n; ++i) {
        Plan &s = sub[i];
        s.kind = inst[i].kind == 0 ? kCaplets : kMbs;
        s.prec = RQMC_FP32;
        s.seq = seq;
        s.s = inst[i].size;
        s.M = M;
        s.N = (uint64_t)inst[i].N;
        s.offset = 0;
        s.seed = seed;
        s.inst = (uint32_t)i;
        Carve ci;
        rqmc_status rs = generator_layout(s, ci, gls[i]);
        if (rs != RQMC_OK) return fail(rs);
        base[i] = cv.take(ci.off);
        if (inst[i].kind == 0) {
            model_off[i] = cv.take(sizeof(LmmModel<float>));
            ++n_class[lmm_bucket_of(inst[i].size) == 160 ? 0 : 2];
        } else {
            model_off[i] = cv.take(sizeof(MbsModel<float>) + sizeof(float) * (inst[i].size + 1));
            ++n_class[1];
        }
    }
    const size_t status_off = cv.take(sizeof(uint32_t) * 4);
    cudaError_t e = cudaMalloc(&bp->d_tables, cv.off);
    if (e != cudaSuccess) { bp->d_tables = nullptr; set_error("batch: table allocation failed"); return fail(RQMC_ENOMEM); }
    unsigned char *d = static_cast<unsigned char *>(bp->d_tables);
    uint32_t *status = reinterpret_cast<uint32_t *>(d + status_off);
    cudaMemset(status, 0, sizeof(uint32_t) * 4);
    bp->insts.resize(n);
    for (int i = 0; i < n; ++i) {
        rqmc_status rs = generator_init(sub[i], gls[i], d + base[i], status, 0);
        if (rs != RQMC_OK) return fail(rs);
        if (!sub[i].gen.stage) {   // the batch kernels stage every instrument's tables
            set_error("batch: instrument " + std::to_string(i) + " has " + std::to_string(inst[i].size) +
                      " dimensions, more than the batch stages in shared memory; price it with its own plan");
            return fail(RQMC_EUNSUPPORTED);
        }
        BatchInst &bi = bp->insts[i];
        bi = BatchInst{};
        bi.g = sub[i].gen;
        bi.kind = inst[i].kind;
        unsigned char *mp = d + model_off[i];
        if (inst[i].kind == 0) {
            LmmModel<float> md;
            fill_lmm_flat(md, inst[i].size, inst[i].rate, inst[i].vol, inst[i].strike);
            if (cudaMemcpy(mp, &md, sizeof md, cudaMemcpyHostToDevice) != cudaSuccess) return fail(RQMC_ECUDA);
            bi.bucket = lmm_bucket_of(inst[i].size);
            bi.nout = inst[i].size;
            bi.lmm = reinterpret_cast<const LmmModel<float> *>(mp);
        } else {
            const rqmc_mbs_params &p = inst[i].mbs;
            const int Mm = inst[i].size;
            const double v = 1.0 / (1.0 + p.i0), s2 = p.sigma * p.sigma;
            std::vector<float> ck(Mm + 1, 0.f);
            for (int k = 1; k <= Mm; ++k) {
                double acc = 0.0, pw = 1.0;
                for (int j = 0; j <= Mm - k; ++j) { acc += pw; pw *= v; }
                ck[k] = (float)acc;
            }
            float *ckd = reinterpret_cast<float *>(mp + sizeof(MbsModel<float>));
            MbsModel<float> md{Mm, (float)p.i0, (float)p.K1, (float)p.K2, (float)p.K3, (float)p.K4, (float)p.c,
                               (float)v, (float)(-0.5 * s2 * kL2e), (float)(p.sigma * kL2e), ckd};
            if (cudaMemcpy(mp, &md, sizeof md, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(ckd, ck.data(), sizeof(float) * (Mm + 1), cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(RQMC_ECUDA);
            bi.bucket = 0;
            bi.nout = 1;
            bi.mbs = reinterpret_cast<const MbsModel<float> *>(mp);
        }
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) { set_error(cudaGetErrorString(e)); return fail(RQMC_ECUDA); }
    const int ppt = autotune(*bp);
    rqmc_status rs = setup_launch(*bp, 256, ppt, false);
    if (rs != RQMC_OK) return fail(rs);
    pl->threads = 256;
    pl->ppt = ppt;
    pl->nout = 0;
    pl->launches = 1;   // theta
    for (int k = 0; k < kBatchClasses; ++k) pl->launches += n_class[k] > 0 ? 1 : 0;
    *plan = pl;
    return RQMC_OK;
}

namespace rqmc {

rqmc_status batch_execute(Plan &pl, double *theta_dev, cudaStream_t st) {
    BatchPlan &bp = *pl.batch;
    cudaError_t e = cudaGraphLaunch(bp.exec, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(theta_dev, bp.bl.theta, sizeof(double) * bp.theta_doubles, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        set_error(std::string("batch launch failed: ") + cudaGetErrorString(e));
        return RQMC_ECUDA;
    }
    return RQMC_OK;
}

int64_t batch_output_size(const Plan &pl) { return (int64_t)pl.batch->theta_doubles; }

void batch_destroy(Plan &pl) {
    if (!pl.batch) return;
    BatchPlan &bp = *pl.batch;
    if (bp.cap) cudaStreamSynchronize(bp.cap);
    for (auto s : bp.side)
        if (s) cudaStreamSynchronize(s);
    free_work(bp);
    if (bp.d_tables) cudaFree(bp.d_tables);
    if (bp.cap) cudaStreamDestroy(bp.cap);
    for (auto s : bp.side)
        if (s) cudaStreamDestroy(s);
    if (bp.fork) cudaEventDestroy(bp.fork);
    for (auto ev : bp.join)
        if (ev) cudaEventDestroy(ev);
    delete pl.batch;
    pl.batch = nullptr;
}

int batch_ppt(const Plan &pl) { return pl.batch ? pl.batch->bl.ppt : 0; }

}  // namespace rqmc

using namespace rqmc;

// Timing of the last execute of a batch plan, from the CTA records of its persistent kernels
// (synchronises: one device-to-host copy).  An SM is busy from the first start to the last
// end of the CTAs it ran; out[0] = busiest SM / mean SM, out[1] = the span of all CTAs in ms,
// out[2..4] = the span of each work class in ms (0 when the class is empty).
extern "C" rqmc_status rqmc_plan_batch_stats(rqmc_plan *plan, double *out_host, int n) {
    if (!plan || !out_host || n < 5 || plan->kind != kBatch || !plan->batch) {
        set_error("rqmc_plan_batch_stats: a batch plan and 5 output values are required");
        return RQMC_EINVAL;
    }
    const BatchLaunch &bl = plan->batch->bl;
    std::vector<unsigned long long> h(3ull * kBatchClasses * bl.stats_cap);
    const cudaError_t e = cudaMemcpy(h.data(), bl.stats, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_error(std::string("rqmc_plan_batch_stats: ") + cudaGetErrorString(e));
        return RQMC_ECUDA;
    }
    std::map<unsigned long long, std::pair<unsigned long long, unsigned long long>> sm;   // SM -> (first start, last end)
    unsigned long long lo = ~0ull, hi = 0;
    for (int k = 0; k < kBatchClasses; ++k) {
        unsigned long long klo = ~0ull, khi = 0;
        for (uint32_t b = 0; b < bl.stats_cap; ++b) {
            const unsigned long long *r = h.data() + 3ull * ((unsigned long long)k * bl.stats_cap + b);
            if (r[2] == 0) continue;   // no record: CTA not launched
            auto it = sm.find(r[0]);
            if (it == sm.end()) sm[r[0]] = {r[1], r[2]};
            else it->second = {std::min(it->second.first, r[1]), std::max(it->second.second, r[2])};
            klo = std::min(klo, r[1]);
            khi = std::max(khi, r[2]);
        }
        out_host[2 + k] = khi > klo ? (double)(khi - klo) * 1e-6 : 0.0;
        lo = std::min(lo, klo);
        hi = std::max(hi, khi);
    }
    double busy_max = 0.0, busy_sum = 0.0;
    for (const auto &kv : sm) {
        const double b = (double)(kv.second.second - kv.second.first);
        busy_max = std::max(busy_max, b);
        busy_sum += b;
    }
    out_host[0] = sm.empty() || busy_sum <= 0.0 ? 0.0 : busy_max / (busy_sum / (double)sm.size());
    out_host[1] = hi > lo ? (double)(hi - lo) * 1e-6 : 0.0;
    return RQMC_OK;
}
