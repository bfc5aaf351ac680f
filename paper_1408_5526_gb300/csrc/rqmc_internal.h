// rqmc_internal.h -- library-internal plan layout and kernel launchers.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rqmc.h"
#include "rqmc_common.cuh"

namespace rqmc {

constexpr int kMaxFwd = 160;       // forwards per LMM instrument (register-resident buckets 16/40/80/160)
constexpr int kMaxDims = 4096;
constexpr int kMaxOutputs = 1280;  // nf * n_strikes per caplet plan

// Reduction layout: a unit is (replication m, tile of `tile` consecutive paths);
// each unit writes its own row of `nout` doubles, so the result does not depend on
// which CTA processed it.  theta[m][o] = sum_tiles partial / N in tile order.
struct RedParams {
    int nout;
    int ppt;                 // paths per thread per unit
    uint32_t tile;           // threads * ppt
    uint32_t tiles_per_m;
    uint32_t units;          // M * tiles_per_m
    uint32_t N;
    double *partials;        // [units][nout]
    uint32_t *status;        // device status word (0 = ok)
};

// One-factor LMM.  Log-Euler: X_n = log(delta L_n) (FP32: log2), so that
// delta L/(1 + delta L) = 1/(1 + b^-X) and one step is
// X_n += sigma_n (h S_n + sqrt(h) Z) - sigma_n^2 h / 2 (times log2 e in FP32).
// Euler: X_n = delta L_n itself and one step is X_n *= 1 + sigma_n (h S_n + sqrt(h) Z)
// (hc = h, sqhc = sqrt(h), cc unused).
template <typename T>
struct LmmModel {
    int nf, nK;
    T dl, inv_dl, disc0;     // delta, 1/delta, 1/(1 + delta L_0(0))
    T hc, sqhc;              // h, sqrt(h)               (FP32: times log2 e)
    T K[kMaxStrikes];
    T sig[kMaxFwd];          // sigma_n at slot n-1 (zero beyond nf)
    T cc[kMaxFwd];           // -sigma_n^2 h / 2         (FP32: times log2 e)
    T X0[kMaxFwd];           // log(delta L_n(0))        (FP32: log2)
};

template <typename T>
struct MbsModel {
    int months;
    T i0, K1, K2, K3, K4, c;
    T u1;                    // u_1 = 1 / (1 + i_0)
    T lk0;                   // log K0 = -sigma^2/2        (FP32: log2 K0)
    T sz;                    // sigma                      (FP32: sigma log2 e)
    const T *ck;             // [months + 1] remaining-annuity factors c_k (device)
};

template <typename T>
struct ProductModel {
    int s;
    const T *a;              // [s] (device)
    const T *inv1pa;         // [s] 1/(1+a_j) (device)
};

// Per-base constants computed on the host; the device setup kernel completes the
// per-(m, j) HaltonDim from the Philox draws.
struct BaseConst {
    uint32_t p, K, L, pL;
    unsigned long long P, D, pK;
    uint32_t magic, sig_off;
    float inv_pL;
    double invD;
};

constexpr int kMaxAdjFwd = 80;   // forwards of an adjoint strip (register buckets 40/80)

// Two-factor-capable LMM for the pathwise adjoint (FP32 paths).
struct AdjModel {
    int nf, nK, d;
    int reverse;                         // 0: prices only (all weights zero)
    float dl, inv_dl, disc0;
    float h, sqh;                        // h = delta, sqrt(h)
    float K[kMaxStrikes];
    float w[kMaxAdjFwd][kMaxStrikes];    // caplet weights w_{n,k} (row n-1)
    float sg[kMaxAdjFwd][2];             // sigma_n = vol_n b_n (zero beyond nf)
    float b[kMaxAdjFwd][2];              // unit loadings b_n
    float cc[kMaxAdjFwd];                // -h |sigma_n|^2 / 2 times log2 e
    float X0[kMaxAdjFwd];                // log2(delta L_n(0))
    float invL0ln2[kMaxAdjFwd];          // 1 / (L_n(0) ln 2)
};

// Per-thread global columns of the adjoint kernel (column stride T = threads in the grid).
struct AdjScratch {
    float *store;   // forward-sweep records: per step the prefix total A as float2 [nf][T]
    float *xb;      // adjoints dV/dX_n as float4 chunks [NF/4][T]
    float *acc;     // vega as float4 chunks [NF/4][T], then value, dV/dL_n(0) [NF], caplet prices [nf nK]
    uint32_t T;
};

// One instrument of a batched launch (device copy).
struct BatchInst {
    GenParams g;                      // its randomization tables (instrument index in the counters)
    int kind;                         // 0 LMM caplet strip, 1 MBS
    int bucket;                       // LMM register bucket
    int nout;                         // outputs per replication
    uint32_t N, tiles_per_m;
    unsigned long long part_off;      // first partial row, in doubles
    unsigned long long theta_off;     // first theta value, in doubles
    const LmmModel<float> *lmm;
    const MbsModel<float> *mbs;
};

struct BatchItem {
    uint32_t inst, m, tile, pad;
};

// Work classes, each with its own persistent kernel, register budget and ticket queue:
// 0 = LMM strips of the 160-forward bucket (one 256-thread CTA per SM), 1 = MBS (up to 4
// CTAs per SM), 2 = LMM strips of the 16/40/80-forward buckets (2 CTAs per SM).
constexpr int kBatchClasses = 3;
struct BatchLaunch {
    const BatchInst *insts;
    const BatchItem *items[kBatchClasses];
    uint32_t n_items[kBatchClasses], n_inst;
    uint32_t *counter;            // [kBatchClasses] ticket counters
    double *partials, *theta;
    unsigned long long *stats;    // [kBatchClasses][stats_cap] CTA records: SM id, start, end (ns)
    uint32_t stats_cap;
    int threads, ppt;
    size_t smem[kBatchClasses];
    // per-CTA normals buffers of the strip classes (0 and 2): zctas CTAs of zstride floats
    // (the largest bucket of the class x the tile); the class's grid never exceeds zctas
    float *znorm[kBatchClasses];
    size_t zstride[kBatchClasses];
    uint32_t zctas[kBatchClasses];
    cudaStream_t side[kBatchClasses - 1];   // classes 1.. run on forked streams
    cudaEvent_t fork, join[kBatchClasses - 1];
};

enum PlanKind { kPoints = 0, kProduct = 1, kCaplets = 2, kMbs = 3, kAdjoint = 4, kBatch = 5 };

struct BatchPlan;

struct Plan {
    PlanKind kind;
    int prec;                // RQMC_FP64 / RQMC_FP32
    int seq;
    int s, M;
    uint64_t N, offset, seed;
    uint32_t inst;
    int nout;
    GenParams gen{};
    RedParams red{};
    int threads = 256, ppt = 4, grid = 0;
    int nf_bucket = 0;
    int scheme = RQMC_LOG_EULER;   // caplet plans: rqmc_lmm_scheme
    int transform = 0;       // point-stream plans: RQMC_UNIFORM / RQMC_NORMAL / RQMC_RAW
    int launches = 0;
    // device memory (one allocation)
    void *d_buf = nullptr;
    size_t d_bytes = 0;
    // FP32 caplet plans: the paths' normals [M][n_fwd][N], written by the point-stream run
    // kernel before the caplet kernel reads them (null: the caplet kernel generates them)
    void *znorm = nullptr;
    // models
    LmmModel<float> lmm32{};
    LmmModel<double> lmm64{};
    MbsModel<float> mbs32{};
    MbsModel<double> mbs64{};
    ProductModel<float> prod32{};
    ProductModel<double> prod64{};
    // adjoint
    int checkpoint = 0;
    AdjModel *adjm = nullptr;
    AdjScratch adjs{};
    void *adj_buf = nullptr;          // per-thread scratch columns (cudaMalloc)
    BatchPlan *batch = nullptr;
    int device = 0;
};

// ---- device memory carve-up helper
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes, size_t align = 256) {
        off = (off + align - 1) / align * align;
        size_t r = off;
        off += bytes;
        return r;
    }
};

// ---- setup (setup.cu)
struct GenLayout {
    size_t hdim_off = 0, sigma_off = 0, base_off = 0, sobV_off = 0, shift_off = 0, scr_off = 0;
    unsigned long long sig_len = 0;
    std::vector<BaseConst> bases;
};
rqmc_status generator_layout(Plan &pl, Carve &cv, GenLayout &gl);
rqmc_status generator_init(Plan &pl, const GenLayout &gl, unsigned char *d, uint32_t *d_status, cudaStream_t st);
std::vector<uint32_t> first_primes(int s);
bool sobol_table_ready(int s);
const std::vector<uint32_t> &sobol_directions();

// ---- launchers (k_*.cu); all asynchronous on `st`
cudaError_t launch_points(const Plan &pl, int tr, void *out, cudaStream_t st);
// the point stream of pl takes the run kernels (N a multiple of 8, and so is the offset except for Philox)
bool points_runs_eligible(const Plan &pl);
cudaError_t launch_product(const Plan &pl, cudaStream_t st);
cudaError_t launch_caplets(const Plan &pl, cudaStream_t st);
cudaError_t launch_mbs(const Plan &pl, cudaStream_t st);
cudaError_t launch_theta(const Plan &pl, double *theta_dev, cudaStream_t st);
cudaError_t launch_adjoint(const Plan &pl, cudaStream_t st);
cudaError_t launch_batch(const BatchLaunch &bl, int seq, cudaStream_t st);
rqmc_status batch_execute(Plan &pl, double *theta_dev, cudaStream_t st);
int64_t batch_output_size(const Plan &pl);
void batch_destroy(Plan &pl);
int batch_ppt(const Plan &pl);
int adjoint_grid(const Plan &pl);
// Paths per thread in lockstep in the FP32 MBS kernels (the MBS plans' paths per thread per
// unit): four for Sobol' (the three extra points cost a few XORs of direction numbers each),
// two for Halton, Rasrap and Philox.  Measured on the MBS workload (360 months, N = 65536,
// M = 64): four lockstep paths took Sobol' from 5.50 to 4.68 ms but Rasrap from 6.18 to 6.69 ms.
__host__ __device__ constexpr int mbs_paths32(int seq) { return seq == 2 || seq == 4 ? 4 : 2; }   // kSobolDS, kSobolLMS

// CTA size of the adjoint kernel: 128 threads, so that five CTAs (20 warps) fit the shared
// memory of an SM with the per-thread state columns of an 80-forward strip.
constexpr int kAdjointThreads = 128;
int occupancy_blocks(const Plan &pl);

// ---- the caller's initial curve as forwards (eq. BL for bond prices); p points into itself
struct LmmCurve {
    rqmc_lmm_params p;
    std::vector<double> L0;
};
rqmc_status lmm_curve(const rqmc_lmm_params *in, LmmCurve &c);

// ---- argument checks and model constants shared by the caplet entry points (api.cu)
rqmc_status common_checks(int s, int64_t N, int64_t offset, int M, int seq, int prec);
rqmc_status check_lmm(const rqmc_lmm_params *p, const double *K, int nK, bool adjoint);
template <typename T>
void fill_lmm(LmmModel<T> &md, const rqmc_lmm_params *p, const double *K, int nK, int bucket);
void set_reduction(Plan &pl, int nout, int threads, int ppt);
int lmm_bucket(int nf);

// ---- errors
void set_error(const std::string &msg);

}  // namespace rqmc
