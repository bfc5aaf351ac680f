/*
 * rqmc.h -- C ABI of librqmc.so, the GB300 (sm_103a) data-parallel hot path of
 * randomized quasi-Monte Carlo financial simulation after Xu & Okten, "High
 * Performance Financial Simulation Using Randomized Quasi-Monte Carlo
 * Methods" (arXiv:1408.5526).
 *
 * The estimator (Sec. 1): for replication m = 0..M-1 the library computes
 *     theta_N^m = (1/N) sum_{i=0}^{N-1} f(q_i^m),     RQ_{M,N} = (1/M) sum_m theta_N^m,
 * where q_i^m is point i of the m-th independent randomization of an
 * s-dimensional sequence and f is a discounted payoff.  Sequences:
 *   RQMC_HALTON_RS  random-start Halton (Sec. 3.1, Algorithm 3, identity permutations)
 *   RQMC_RASRAP     random-start randomly permuted Halton "Rasrap" (Sec. 3.1, eq. perm,
 *                   Algorithm 3; a new start and new permutations for every replication)
 *   RQMC_SOBOL_DS   Sobol' in binary counter order (Sec. 3.2), digitally shifted per replication
 *   RQMC_PHILOX     the counter-based pseudorandom stream Philox4x32-10 (Sec. 2)
 *   RQMC_SOBOL_LMS  Sobol' with Matousek's random linear scrambling (Sec. 3.2): per replication
 *                   and dimension a random unit lower-triangular binary matrix acts on the
 *                   binary digits of every coordinate, followed by a digital shift
 * Randomizations are drawn from Philox4x32-10 keyed by `seed`, so a call is
 * reproducible bit for bit from (seq, s, M, seed).
 *
 * Conventions shared by every entry point:
 *   - Coordinates: the raw state of coordinate j of point n is an integer
 *     `num` over a denominator D (Halton: D = p_j^(K+1) with K the largest
 *     integer such that p_j^(K+1) < 2^64, num exact in 64 bits; Sobol'/Philox:
 *     D = 2^32).  The uniform is u = (num + 1/2) / D and the normal is
 *     z = -/+ Phi^-1(q) with q = (min(num, D-1-num) + 1/2) / D, so 1 - u is never
 *     formed in floating point.
 *   - Dimension of factor f at time step t is t*d + f; point n of a call with
 *     point offset `offset` is the sequence element offset + i.
 *   - Precision: RQMC_FP64 runs every path in double.  RQMC_FP32 runs paths in
 *     float with compensated (Kahan) payoff sums; integer digit arithmetic stays
 *     exact and the replication reduction is done in double in both modes.
 *   - Host pointers are named *_host or documented "host"; device pointers are
 *     documented "device" and must be device (or managed) memory on the
 *     current CUDA device.  `stream` is a cudaStream_t (NULL = legacy default
 *     stream).  The caller owns every buffer it passes; the library owns its
 *     internal workspace and the plans it creates.
 *   - Errors: every function returns an rqmc_status and never aborts or throws.
 *     Arguments are validated before any launch; on RQMC_EINVAL nothing was
 *     launched.  Device-side failures are reported through a status word read
 *     after synchronisation (RQMC_ETIMEOUT, RQMC_ECUDA).  The one-shot entry
 *     points (rqmc_integrate_product, price_*) synchronise `stream` before they
 *     return and serialise with one another through an internal lock.
 *
 * Limits: s <= 4096 dimensions; N >= 1 with offset + N <= 2^32 for Sobol',
 * <= 2^48 for Philox, and for Halton that every base p_j (j < s) has p_j^L <= 2^31
 * for the smallest L with p_j^L >= N (the largest N: 2^31 at s = 1, 214358881 = 11^8 at
 * s = 8, 38950081 = 79^4 at s = 40, 11089567 = 223^3 at s = 160, 1666681 = 1291^2 at
 * s = 360); M <= 65535.
 */
#ifndef RQMC_H
#define RQMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RQMC_OK = 0,
    RQMC_EINVAL = 1,        /* bad argument; nothing launched */
    RQMC_ENOMEM = 2,        /* device or pinned-host allocation failed */
    RQMC_ECUDA = 3,         /* a CUDA runtime call failed (see rqmc_last_error) */
    RQMC_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    RQMC_EUNSUPPORTED = 5,  /* valid request outside this build's limits */
    RQMC_ENOTABLE = 6       /* Sobol' requested before rqmc_set_sobol_table covered s dims */
} rqmc_status;

typedef enum {
    RQMC_HALTON_RS = 0,
    RQMC_RASRAP = 1,
    RQMC_SOBOL_DS = 2,
    RQMC_PHILOX = 3,
    RQMC_SOBOL_LMS = 4
} rqmc_sequence;
typedef enum { RQMC_FP64 = 0, RQMC_FP32 = 1 } rqmc_precision;
typedef enum { RQMC_UNIFORM = 0, RQMC_NORMAL = 1, RQMC_RAW = 2 } rqmc_transform;
typedef enum { RQMC_LOG_EULER = 0, RQMC_EULER = 1 } rqmc_lmm_scheme;

/* LIBOR market model (Sec. 5): forwards L_1..L_nf over [T_n, T_{n+1}], T_n = n*delta,
 * simulated on the grid t_i = T_i under the spot measure; L_0 is fixed at t = 0.
 * sigma_n = vol[n-1] * b_n with unit loading rows b_n (d = n_factors).  Schemes:
 * RQMC_EULER is eq. (L_n_discrete) as printed, L_n += mu_n L_n h + L_n sqrt(h) sigma_n.Z;
 * RQMC_LOG_EULER applies the same drift and noise to log L_n with the Ito correction,
 * log L_n += (mu_n - |sigma_n|^2 / 2) h + sqrt(h) sigma_n.Z.  price_caplets and the caplet
 * plans run both; the adjoint and the batch run log-Euler.  All arrays are host memory,
 * read during the call. */
typedef struct {
    int n_fwd;               /* nf >= 1 */
    int n_factors;           /* d in {1, 2} */
    int scheme;              /* rqmc_lmm_scheme */
    int init;                /* what L0 points to: 0 = forwards, 1 = bond prices (see L0) */
    double delta;            /* accrual period = time step, > 0 */
    const double *L0;        /* init 0: [nf+1] forwards L_0(0), L_1(0), ..., L_nf(0);
                              * init 1: [nf+2] bond prices B_0(0), ..., B_{nf+1}(0) > 0, converted
                              * by eq. BL, L_n(0) = (B_n(0) - B_{n+1}(0)) / (delta B_{n+1}(0)) */
    const double *vol;       /* [nf]: |sigma_n|, n = 1..nf */
    const double *loadings;  /* [nf][d] unit rows b_n; may be NULL when d == 1 */
} rqmc_lmm_params;

/* Mortgage-backed security (Sec. 6, Caflisch's model):
 *   PV = E sum_{k=1}^{months} u_k m_k, u_k = prod_{j<k}(1+i_j)^-1, m_k = c r_k((1-w_k) + w_k c_k),
 *   r_k = prod_{0<j<k}(1-w_j), c_k = sum_{j=0}^{months-k}(1+i_0)^-j,
 *   i_k = K0 exp(sigma z_k) i_{k-1}, K0 = exp(-sigma^2/2), w_k = K1 + K2 atan(K3 i_k + K4). */
typedef struct {
    int months;              /* M of the paper, = s */
    int reserved;
    double i0, K1, K2, K3, K4;
    double sigma;            /* standard deviation of xi_k */
    double c;                /* monthly payment */
} rqmc_mbs_params;

/* One instrument of a batch: kind 0 = LMM caplet strip with `size` forwards (one
 * factor, flat initial curve `rate`, flat vol `vol`, strike `strike`, delta = 0.25),
 * outputs `size` caplet values; kind 1 = MBS with `size` months and the model
 * constants in `mbs`, one output.  N points per replication. */
typedef struct {
    int kind;
    int size;
    int64_t N;
    double rate, vol, strike;
    rqmc_mbs_params mbs;
} rqmc_instrument;

/* Opaque device-resident plan: randomization tables, model constants and
 * workspace for repeated launches. */
typedef struct rqmc_plan_s rqmc_plan;

/* ---------------------------------------------------------------- setup */

/* Joe-Kuo primitive polynomials and initial direction numbers (Sec. 3.2):
 * poly[j] holds the whole polynomial of dimension j as bits (degree = bit
 * length - 1; row 0 is ignored and stands for van der Corput in base 2);
 * vinit[j*max_deg + k] = m_{k+1}.  The library derives the 32-bit direction
 * numbers with the recurrence of Sec. 3.2 and keeps them for the process.
 * Host arrays.  EINVAL if a row is malformed. */
rqmc_status rqmc_set_sobol_table(const int64_t *poly, const int64_t *vinit, int n_dims, int max_deg);

/* ---------------------------------------------------------------- point stream */

/* Writes coordinate j of point offset+i of replication m to out[(m*s + j)*N + i]
 * (device memory; float for RQMC_FP32, double for RQMC_FP64, uint64 for
 * RQMC_RAW whatever prec).  Transform: uniform u, normal z, or the raw integer
 * state num (see conventions).  Asynchronous on `stream`.  The analogue of
 * Table 2's generator throughput (Sec. 4). */
rqmc_status rqmc_points(int s, int64_t N, int M, rqmc_sequence seq, uint64_t seed, int64_t offset,
                        rqmc_precision prec, rqmc_transform tr, void *out, void *stream);

/* ---------------------------------------------------------------- one-shot estimators (synchronous) */

/* Product test integrand f(x) = prod_j (|4 x_j - 2| + a_j)/(1 + a_j) (exact integral 1).
 * theta_host[M], rq_host[1], sd_host[1] (sample standard deviation over m) are host
 * outputs; rq/sd may be NULL.  a_host[s]. */
rqmc_status rqmc_integrate_product(int s, int64_t N, int M, rqmc_sequence seq, uint64_t seed,
                                   const double *a_host, rqmc_precision prec,
                                   double *theta_host, double *rq_host, double *sd_host, void *stream);

/* Caplets on every forward (Sec. 5): output o = (n-1)*n_strikes + k holds the value of
 * the caplet on L_n with strike K_k, E[delta (L_n(T_n)-K_k)^+ / prod_{j<=n}(1+delta L_j(T_j))].
 * theta_host[M][nf*n_strikes]; rq_host, sd_host [nf*n_strikes] (may be NULL).
 * s = nf*d dimensions.  n_strikes in 1..8. */
rqmc_status price_caplets(const rqmc_lmm_params *p, const double *strikes_host, int n_strikes, int64_t N,
                          int M, rqmc_sequence seq, uint64_t seed, rqmc_precision prec,
                          double *theta_host, double *rq_host, double *sd_host, void *stream);

/* MBS present value (Sec. 6): theta_host[M], rq_host[1], sd_host[1]. s = months. */
rqmc_status price_mbs(const rqmc_mbs_params *p, int64_t N, int M, rqmc_sequence seq, uint64_t seed,
                      rqmc_precision prec, double *theta_host, double *rq_host, double *sd_host, void *stream);

/* Pathwise adjoint of the caplet strip V = sum_{n,k} w_{n,k} caplet_{n,k} (not in the
 * paper; the model and estimator are Sec. 5's): value_host[M], delta_host[M][nf] =
 * dV/dL_n(0), vega_host[M][nf] = dV/dvol_n with the loadings b_n fixed, per replication.
 * weights_host[nf*n_strikes].  FP32 paths, nf <= 80, d in {1, 2}.  The forward sweep
 * records every step's drift factors in per-thread device scratch (`checkpoint` must be
 * 0 or 1); the reverse sweep regenerates the normals from the counter. */
rqmc_status price_adjoint(const rqmc_lmm_params *p, const double *strikes_host, int n_strikes,
                          const double *weights_host, int64_t N, int M, rqmc_sequence seq, uint64_t seed,
                          rqmc_precision prec, int checkpoint, double *value_host, double *delta_host,
                          double *vega_host, void *stream);

/* Batch of n instruments in one CUDA graph (not in the paper): one persistent kernel per
 * work class (160-forward strips, smaller strips, MBS), each with a longest-first ticket
 * queue, as parallel branches; tiles picked by an autotuner whose choice is cached in
 * $RQMC_AUTOTUNE_CACHE (default ~/.cache/rqmc_gb300/autotune.json; RQMC_AUTOTUNE=0 skips it).
 * Instrument i uses instrument index i in its Philox counters.  Output
 * theta_host holds, instrument after instrument, an [M][n_out_i] block with n_out_i =
 * size (LMM) or 1 (MBS). */
rqmc_status price_batch(const rqmc_instrument *inst, int n, int M, rqmc_sequence seq, uint64_t seed,
                        rqmc_precision prec, double *theta_host, void *stream);

/* ---------------------------------------------------------------- pricing without allocation */

/* The caplet values of price_caplets written to theta_dev [M][nf*n_strikes] (device
 * memory), asynchronously on `stream`, WITHOUT allocating anything.  The paper has no
 * counterpart: this entry point serves callers that cannot allocate device memory at the
 * moment they price (a callback running inside another framework's device allocator, a
 * process whose device memory a pool reserved entirely at start-up, or a service whose
 * policy forbids allocation after start-up).  Its scratch space is one 16 MiB array built
 * into the library, created on every GPU that loads the library and held until the process
 * exits; a request whose tables and partial sums need more returns RQMC_EINVAL with the
 * size in rqmc_last_error().  The first call on each device looks up that array's device
 * address (cudaGetSymbolAddress) and caches it.  All calls share the array, so calls whose
 * work overlaps on the GPU race and must be serialised by the caller.  Same argument checks
 * and error codes as price_caplets (one factor).  A device-side status (a randomized point
 * range beyond a Halton start's digits, which cannot happen within these limits) makes every
 * theta value of the call NaN. */
rqmc_status rqmc_price_caplets_noalloc(const rqmc_lmm_params *p, const double *strikes_host, int n_strikes,
                                       int64_t N, int M, rqmc_sequence seq, uint64_t seed, rqmc_precision prec,
                                       double *theta_dev, void *stream);

/* ---------------------------------------------------------------- plans (device resident) */

/* Build randomization tables and model constants on the device once; every
 * rqmc_plan_execute then runs only the kernels and writes theta [M][n_out] doubles
 * to device memory `theta_dev` (asynchronous on `stream`).  `offset` shifts the point
 * range to offset..offset+N-1 (shards of one estimate add up exactly).  A plan owns its
 * workspace: executes of one plan must be ordered (one stream, or synchronised), while
 * different plans may run concurrently. */
rqmc_status rqmc_plan_product(int s, int64_t N, int64_t offset, int M, rqmc_sequence seq, uint64_t seed,
                              const double *a_host, rqmc_precision prec, rqmc_plan **plan);
rqmc_status rqmc_plan_caplets(const rqmc_lmm_params *p, const double *strikes_host, int n_strikes, int64_t N,
                              int64_t offset, int M, rqmc_sequence seq, uint64_t seed, rqmc_precision prec,
                              rqmc_plan **plan);
rqmc_status rqmc_plan_mbs(const rqmc_mbs_params *p, int64_t N, int64_t offset, int M, rqmc_sequence seq,
                          uint64_t seed, rqmc_precision prec, rqmc_plan **plan);
rqmc_status rqmc_plan_adjoint(const rqmc_lmm_params *p, const double *strikes_host, int n_strikes,
                              const double *weights_host, int64_t N, int64_t offset, int M, rqmc_sequence seq,
                              uint64_t seed, rqmc_precision prec, int checkpoint, rqmc_plan **plan);
rqmc_status rqmc_plan_batch(const rqmc_instrument *inst, int n, int M, rqmc_sequence seq, uint64_t seed,
                            rqmc_precision prec, rqmc_plan **plan);
/* Point stream as a plan (the tables of rqmc_points built once): each execute writes the
 * M*s*N coordinates of points offset..offset+N-1 to the device buffer passed as
 * `theta_dev`, laid out [M][s][N] with the element type of rqmc_points (float for FP32,
 * double for FP64, int64 numerators for RQMC_RAW) -- the pointer is only reinterpreted.
 * Same argument rules and errors as rqmc_points. */
rqmc_status rqmc_plan_points(int s, int64_t N, int64_t offset, int M, rqmc_sequence seq, uint64_t seed,
                             rqmc_precision prec, rqmc_transform tr, rqmc_plan **plan);
/* Number of values the plan writes per execute: M*s*N coordinates for point-stream plans,
 * otherwise M*n_out doubles.  Adjoint plans write per
 * replication [value, dV/dL_n(0) (nf), dV/dvol_n (nf), unweighted caplet values (nf*n_strikes)];
 * with all weights zero they skip the reverse sweep and act as a d-factor caplet pricer. */
int64_t rqmc_plan_output_size(const rqmc_plan *plan);
/* Timing of the last execute of a batch plan (not in the paper), from per-CTA records of its
 * persistent kernels (global timer): an SM counts as busy from the first start to the last end
 * of the CTAs it ran.  out_host[0] = busiest SM / mean SM (1 = perfectly balanced), [1] = span of
 * all CTAs in ms, [2], [3], [4] = span of the 160-forward, MBS and smaller-strip classes in ms
 * (0 when empty).  Synchronous (one copy); n must be at least 5; EINVAL for other plans. */
rqmc_status rqmc_plan_batch_stats(rqmc_plan *plan, double *out_host, int n);
/* Kernel launches one execute performs (for launch accounting). */
int rqmc_plan_launches(const rqmc_plan *plan);
/* Tuning knobs of a plan: threads per block and paths per thread (0 = keep). */
rqmc_status rqmc_plan_set_launch(rqmc_plan *plan, int threads, int paths_per_thread);
/* The plan's launch shape (not in the paper): threads per block and paths per thread, for a
 * batch plan the tile its autotuner chose or read from its cache.  Host-only, no GPU work;
 * RQMC_EINVAL for a NULL argument. */
rqmc_status rqmc_plan_get_launch(const rqmc_plan *plan, int *threads, int *paths_per_thread);
/* Launch the plan's kernels on `stream` (asynchronous), writing rqmc_plan_output_size(plan)
 * values to device memory `theta_dev`, which the caller owns and must size; the device the
 * plan was built on must be current (RQMC_EINVAL otherwise, nothing launched). */
rqmc_status rqmc_plan_execute(rqmc_plan *plan, double *theta_dev, void *stream);
/* Status word of the plan's last execute (synchronises `stream`). */
rqmc_status rqmc_plan_check(rqmc_plan *plan, void *stream);
rqmc_status rqmc_plan_destroy(rqmc_plan *plan);

/* ---------------------------------------------------------------- diagnostics */

/* Measured issue rates of this GPU's pipes (not in the paper), as operations per SM per
 * clock, written to rates_host[0..]: [0] ex2.approx, [1] rcp.approx, [2] lg2.approx, [3] the
 * forward update's pair rcp(1 + ex2(-x)) (counted once), [4] FP32 FMA, and when n allows
 * [5] FP64 FMA, [6] the FP64 update pair 1/(1 + exp(-x)) (counted once), [7] the SM clock in
 * MHz that the probes ran at, measured inside them (cycle counter against the global
 * nanosecond timer) and used as the clock of every rate.  Synchronous on the current device
 * (a few milliseconds); n must be at least 5. */
rqmc_status rqmc_probe_pipes(double *rates_host, int n);
const char *rqmc_status_string(rqmc_status st);
/* Text of the last error raised on the calling thread ("" if none). */
const char *rqmc_last_error(void);
/* ABI version, currently 1. */
int rqmc_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RQMC_H */
