/*
 * oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * A plain, slow FP64 CPU restatement of the randomized quasi-Monte Carlo
 * method of Xu & Okten, "High Performance Financial Simulation Using
 * Randomized Quasi-Monte Carlo Methods" (arXiv:1408.5526).  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may
 * load this library.  It shares no code, header or table with the CUDA
 * library: primes, Philox, digit expansions, Sobol' direction numbers and
 * the inverse normal CDF are all re-derived here from their definitions.
 *
 * Every function follows the paper's definitions in the paper's order, with
 * no blocking, caching or reordering:
 *   - estimator theta_N^m and RQ_{M,N}                      Sec. 1
 *   - van der Corput / permuted van der Corput              Sec. 3.1, eqs. (vdcp), (perm)
 *   - counter-based random-start permuted vdC (Rasrap)      Sec. 3.1, Algorithm 3
 *   - Sobol' in binary counter order                        Sec. 3.2
 *   - Philox4x32-10 (Salmon et al., SC'11)                  Sec. 2
 *   - LIBOR market model, Euler / log-Euler, caplets        Sec. 5, eqs. (L_n_discrete), (BL)
 *   - mortgage-backed security (Caflisch model)             Sec. 6
 * Where the paper is silent the oracle takes the reading listed as c1..c19
 * in the design notes (random start = K truncated digits, permutation of all
 * K start positions, digital shift for Sobol', uniform u = (num+1/2)/D,
 * spot-measure discounting, ...).
 *
 * Parity status: every function here is pinned by a `-m "not gpu"` test
 * against something other than itself (known-answer vectors, library
 * routines, exact rational arithmetic, closed forms), except the stochastic
 * MBS present value for paper parameters, which is pinned only through its
 * special cases (sigma = 0, two- and three-month quadrature).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 orc_u128;

/* ------------------------------------------------------------------ */
/* Philox4x32-10: ten rounds of the Philox S-P network with the round  */
/* multipliers 0xD2511F53, 0xCD9E8D57 and the Weyl key increments      */
/* 0x9E3779B9, 0xBB67AE85 (Salmon, Moraes, Dror, Shaw, SC'11).         */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod1;
        uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Counter layout (reading c17): key = (seed_lo, seed_hi); word 3 of the
 * counter carries a tag in its low 8 bits and the instrument index above. */
enum { ORC_TAG_PATH = 0, ORC_TAG_START = 1, ORC_TAG_PERM = 2, ORC_TAG_SHIFT = 3, ORC_TAG_SCRAMBLE = 4 };

static void orc_philox_call(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                            uint32_t tag, uint32_t inst, uint32_t out[4])
{
    uint32_t ctr[4] = { c0, c1, c2, tag | (inst << 8) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

/* Pseudorandom comparison stream: word (j mod 4) of one Philox call whose
 * counter holds the point index n (48 bits) and the dimension block j/4. */
uint32_t orc_philox_path_word(uint64_t seed, uint32_t inst, int m, int j, uint64_t n)
{
    uint32_t w[4];
    orc_philox_call(seed, (uint32_t)n,
                    (uint32_t)((n >> 32) & 0xFFFFu) | ((uint32_t)(j >> 2) << 16),
                    (uint32_t)m, ORC_TAG_PATH, inst, w);
    return w[j & 3];
}

/* ------------------------------------------------------------------ */
/* Primes: the Halton bases are the first s primes (Sec. 3.1).         */
/* ------------------------------------------------------------------ */
int orc_first_primes(int s, uint32_t *out)
{
    int found = 0;
    for (uint32_t c = 2; found < s; ++c) {
        int prime = 1;
        for (uint32_t d = 2; d * d <= c; ++d)
            if (c % d == 0) { prime = 0; break; }
        if (prime) out[found++] = c;
    }
    return found;
}

/* Number K of random-start digits in base p (reading c1): the largest K
 * with p^(K+1) <= 2^64 - 1, so one carry digit past the start still fits. */
int orc_halton_K(uint32_t p)
{
    uint64_t pw = p;           /* p^(k+1) */
    int k = 0;
    while (pw <= UINT64_MAX / p) { pw *= p; ++k; }
    return k;
}

uint64_t orc_ipow(uint32_t p, int e)
{
    uint64_t r = 1;
    for (int i = 0; i < e; ++i) r *= p;
    return r;
}

/* Algorithm 3, step (1): draw omega ~ U[0,1) as a 64-bit Philox word
 * U/2^64 and find n with |phi_p(n) - omega| < eps = p^-K.  Truncating
 * omega to its first K base-p digits d_0 d_1 ... d_{K-1} and reversing them
 * gives n = sum_t d_t p^t, for which phi_p(n) is that truncation. */
uint64_t orc_halton_start(uint64_t seed, uint32_t inst, int m, int j, uint32_t p, int K)
{
    uint32_t w[4];
    orc_philox_call(seed, (uint32_t)j, 0u, (uint32_t)m, ORC_TAG_START, inst, w);
    uint64_t U = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    uint64_t pK = orc_ipow(p, K);
    uint64_t lead = (uint64_t)(((orc_u128)U * (orc_u128)pK) >> 64); /* floor(omega p^K) */
    /* lead = d_0 p^(K-1) + ... + d_{K-1}: peel digits from the right. */
    uint64_t n = 0;
    for (int t = K - 1; t >= 0; --t) {
        uint64_t dt = lead % p;     /* digit d_t */
        lead /= p;
        n += dt * orc_ipow(p, t);
    }
    return n;
}

/* Random digit permutation sigma on {0..p-1} (Sec. 3.1, following the
 * random choice of Okten-Shah-Goncharov; reading c4): Fisher-Yates from the
 * identity, swap position k with floor(u (k+1) / 2^32) for k = p-1 .. 1,
 * the t-th draw being word (t mod 4) of Philox call t/4. */
void orc_halton_perm(uint64_t seed, uint32_t inst, int m, int j, uint32_t p,
                     int identity, uint16_t *sigma)
{
    for (uint32_t a = 0; a < p; ++a) sigma[a] = (uint16_t)a;
    if (identity) return;
    uint32_t w[4];
    for (uint32_t k = p - 1, t = 0; k >= 1; --k, ++t) {
        if ((t & 3u) == 0)
            orc_philox_call(seed, (uint32_t)j, t >> 2, (uint32_t)m, ORC_TAG_PERM, inst, w);
        uint32_t r = (uint32_t)(((uint64_t)w[t & 3u] * (uint64_t)(k + 1)) >> 32);
        uint16_t tmp = sigma[k]; sigma[k] = sigma[r]; sigma[r] = tmp;
    }
}

/* Permuted van der Corput, eq. (perm), as the integer numerator over
 * D = p^(K+1): expand n = (a_K ... a_1 a_0)_p and sum sigma(a_k) p^(K-k).
 * Reading c2: all K start positions k < K are permuted (zeros included);
 * position K contributes sigma(a_K) only when a carry has made a_K nonzero.
 * Returns UINT64_MAX when n >= p^(K+1) (outside the representable range). */
uint64_t orc_permuted_vdc_numerator(uint32_t p, int K, const uint16_t *sigma, uint64_t n)
{
    uint64_t D = orc_ipow(p, K + 1);
    if (n >= D) return UINT64_MAX;
    uint64_t num = 0, rest = n;
    for (int k = 0; k <= K; ++k) {
        uint64_t a = rest % p;
        rest /= p;
        uint64_t weight = orc_ipow(p, K - k);
        if (k < K) num += (uint64_t)sigma[a] * weight;
        else if (a != 0) num += (uint64_t)sigma[a];
    }
    return num;
}

/* ------------------------------------------------------------------ */
/* Sobol' (Sec. 3.2).  Direction numbers v_k = m_k / 2^k from the      */
/* primitive-polynomial recurrence; stored as 32-bit integers          */
/* V[k-1] = m_k 2^(32-k).  Dimension 0 is van der Corput in base 2     */
/* (all m_k = 1).  poly[j] holds the whole polynomial as bits (degree  */
/* = bit length - 1), vinit[j][0..deg-1] the free initial m's.         */
/* ------------------------------------------------------------------ */
int orc_sobol_directions(int s, const int64_t *poly, const int64_t *vinit, int maxdeg, uint32_t *V)
{
    for (int j = 0; j < s; ++j) {
        uint64_t mk[33];
        if (j == 0) {
            for (int k = 1; k <= 32; ++k) mk[k] = 1;
        } else {
            uint64_t P = (uint64_t)poly[j];
            int deg = 0;
            while ((P >> (deg + 1)) != 0) ++deg;
            if (deg < 1 || deg > maxdeg) return -1;
            for (int k = 1; k <= deg && k <= 32; ++k) mk[k] = (uint64_t)vinit[j * maxdeg + (k - 1)];
            for (int k = deg + 1; k <= 32; ++k) {
                /* m_k = 2 a_1 m_{k-1} ^ 4 a_2 m_{k-2} ^ ... ^ 2^(deg-1) a_{deg-1} m_{k-deg+1}
                 *       ^ 2^deg m_{k-deg} ^ m_{k-deg},
                 * polynomial x^deg + a_1 x^(deg-1) + ... + a_{deg-1} x + 1. */
                uint64_t v = (mk[k - deg] << deg) ^ mk[k - deg];
                for (int i = 1; i <= deg - 1; ++i) {
                    uint64_t a_i = (P >> (deg - i)) & 1u;
                    if (a_i) v ^= mk[k - i] << i;
                }
                mk[k] = v;
            }
        }
        for (int k = 1; k <= 32; ++k) {
            if ((mk[k] & 1u) == 0 || mk[k] >= ((uint64_t)1 << k)) return -2;
            V[j * 32 + (k - 1)] = (uint32_t)(mk[k] << (32 - k));
        }
    }
    return 0;
}

/* x_n = n_1 v_1 xor n_2 v_2 xor ... over the binary digits of n. */
uint32_t orc_sobol_binary(const uint32_t *Vj, uint64_t n)
{
    uint32_t x = 0;
    for (int k = 0; k < 32; ++k)
        if ((n >> k) & 1u) x ^= Vj[k];
    return x;
}

/* Digital shift D_{m,j} (reading c5): word 0 of one Philox call. */
uint32_t orc_sobol_shift(uint64_t seed, uint32_t inst, int m, int j)
{
    uint32_t w[4];
    orc_philox_call(seed, (uint32_t)j, 0u, (uint32_t)m, ORC_TAG_SHIFT, inst, w);
    return w[0];
}

/* Matousek's random linear scrambling (Sec. 3.2; reading c23): a random  */
/* nonsingular lower-triangular binary matrix L_{m,j} acts on the binary  */
/* digits (most significant first) of every coordinate, y = L x, before   */
/* the digital shift.  Row r (output digit r, r = 0..31) is stored as a   */
/* 32-bit mask over the input digits (digit l = bit 31 - l): the diagonal */
/* is 1, and the r entries left of it are the top r bits of Philox word   */
/* r - 1 of the counters (j, (r-1)/4, m, tag 4).                          */
void orc_sobol_lms_rows(uint64_t seed, uint32_t inst, int m, int j, uint32_t rows[32])
{
    rows[0] = 0x80000000u;
    for (int r = 1; r < 32; ++r) {
        uint32_t w[4];
        orc_philox_call(seed, (uint32_t)j, (uint32_t)((r - 1) >> 2), (uint32_t)m, ORC_TAG_SCRAMBLE, inst, w);
        const uint32_t word = w[(r - 1) & 3];
        rows[r] = ((word >> (32 - r)) << (32 - r)) | (0x80000000u >> r);
    }
}

/* y = L x over GF(2): output digit r is the parity of row r and x. */
uint32_t orc_sobol_lms_apply(const uint32_t rows[32], uint32_t x)
{
    uint32_t y = 0;
    for (int r = 0; r < 32; ++r) {
        uint32_t t = rows[r] & x, par = 0;
        while (t) { par ^= 1u; t &= t - 1u; }
        y |= par << (31 - r);
    }
    return y;
}

/* ------------------------------------------------------------------ */
/* Sequence object: randomization of every (m, j) for one call.        */
/* ------------------------------------------------------------------ */
enum { ORC_HALTON_RS = 0, ORC_RASRAP = 1, ORC_SOBOL_DS = 2, ORC_PHILOX = 3, ORC_SOBOL_LMS = 4 };

typedef struct {
    int seq, s, M;
    uint64_t seed;
    uint32_t inst;
    uint32_t *p;        /* [s] bases */
    int *K;             /* [s] start digits */
    uint64_t *D;        /* [s] denominators */
    uint64_t *n0;       /* [M][s] random starts */
    uint64_t *sig_off;  /* [s] offsets into one replication's permutations */
    uint64_t sig_len;   /* sum_j p_j */
    uint16_t *sigma;    /* [M][sig_len] */
    uint32_t *V;        /* [s][32] */
    uint32_t *shift;    /* [M][s] */
    uint32_t *lms;      /* [M][s][32] scrambling rows (ORC_SOBOL_LMS) */
} orc_seq;

void orc_seq_destroy(orc_seq *q)
{
    if (!q) return;
    free(q->p); free(q->K); free(q->D); free(q->n0); free(q->sig_off);
    free(q->sigma); free(q->V); free(q->shift); free(q->lms); free(q);
}

orc_seq *orc_seq_create(int seq, int s, int M, uint64_t seed, uint32_t inst,
                        const int64_t *poly, const int64_t *vinit, int maxdeg)
{
    if (s < 1 || M < 1 || seq < 0 || seq > 4) return NULL;
    orc_seq *q = (orc_seq *)calloc(1, sizeof(orc_seq));
    q->seq = seq; q->s = s; q->M = M; q->seed = seed; q->inst = inst;
    q->D = (uint64_t *)calloc((size_t)s, sizeof(uint64_t));
    if (seq == ORC_HALTON_RS || seq == ORC_RASRAP) {
        q->p = (uint32_t *)calloc((size_t)s, sizeof(uint32_t));
        q->K = (int *)calloc((size_t)s, sizeof(int));
        q->sig_off = (uint64_t *)calloc((size_t)s, sizeof(uint64_t));
        orc_first_primes(s, q->p);
        q->sig_len = 0;
        for (int j = 0; j < s; ++j) {
            q->K[j] = orc_halton_K(q->p[j]);
            q->D[j] = orc_ipow(q->p[j], q->K[j] + 1);
            q->sig_off[j] = q->sig_len;
            q->sig_len += q->p[j];
        }
        q->n0 = (uint64_t *)calloc((size_t)M * s, sizeof(uint64_t));
        q->sigma = (uint16_t *)calloc((size_t)M * q->sig_len, sizeof(uint16_t));
        for (int m = 0; m < M; ++m)
            for (int j = 0; j < s; ++j) {
                q->n0[(size_t)m * s + j] = orc_halton_start(seed, inst, m, j, q->p[j], q->K[j]);
                orc_halton_perm(seed, inst, m, j, q->p[j], seq == ORC_HALTON_RS,
                                q->sigma + (size_t)m * q->sig_len + q->sig_off[j]);
            }
    } else if (seq == ORC_SOBOL_DS || seq == ORC_SOBOL_LMS) {
        if (!poly || !vinit) { orc_seq_destroy(q); return NULL; }
        q->V = (uint32_t *)calloc((size_t)s * 32, sizeof(uint32_t));
        if (orc_sobol_directions(s, poly, vinit, maxdeg, q->V) != 0) { orc_seq_destroy(q); return NULL; }
        q->shift = (uint32_t *)calloc((size_t)M * s, sizeof(uint32_t));
        for (int m = 0; m < M; ++m)
            for (int j = 0; j < s; ++j)
                q->shift[(size_t)m * s + j] = orc_sobol_shift(seed, inst, m, j);
        if (seq == ORC_SOBOL_LMS) {
            q->lms = (uint32_t *)calloc((size_t)M * s * 32, sizeof(uint32_t));
            for (int m = 0; m < M; ++m)
                for (int j = 0; j < s; ++j) orc_sobol_lms_rows(seed, inst, m, j, q->lms + ((size_t)m * s + j) * 32);
        }
        for (int j = 0; j < s; ++j) q->D[j] = (uint64_t)1 << 32;
    } else {
        for (int j = 0; j < s; ++j) q->D[j] = (uint64_t)1 << 32;
    }
    return q;
}

/* Raw integer state of coordinate j of point n in replication m, and its
 * denominator: u = (raw + 1/2) / D (reading c6). */
uint64_t orc_coord_raw(const orc_seq *q, int m, int j, uint64_t n, uint64_t *D)
{
    *D = q->D[j];
    switch (q->seq) {
    case ORC_HALTON_RS:
    case ORC_RASRAP: {
        /* Algorithm 3, steps (2)-(3): the point for counter n is phi^sigma(n0 + n). */
        uint64_t start = q->n0[(size_t)m * q->s + j];
        const uint16_t *sg = q->sigma + (size_t)m * q->sig_len + q->sig_off[j];
        return orc_permuted_vdc_numerator(q->p[j], q->K[j], sg, start + n);
    }
    case ORC_SOBOL_DS:
        return (uint64_t)(orc_sobol_binary(q->V + (size_t)j * 32, n) ^ q->shift[(size_t)m * q->s + j]);
    case ORC_SOBOL_LMS:
        return (uint64_t)(orc_sobol_lms_apply(q->lms + ((size_t)m * q->s + j) * 32,
                                              orc_sobol_binary(q->V + (size_t)j * 32, n)) ^
                          q->shift[(size_t)m * q->s + j]);
    default:
        return (uint64_t)orc_philox_path_word(q->seed, q->inst, m, j, n);
    }
}

/* ------------------------------------------------------------------ */
/* Recursive CPU generators of Table 1 (Sec. 4), for the CPU timing      */
/* baselines: count consecutive raw states of row (m, j) from point      */
/* n_start on.                                                           */
/*  - Halton / Rasrap: Algorithm 2, an odometer on the digits a_0..a_K   */
/*    of n0 + n with the suffix sums S_k = sum_{i >= k} of the permuted  */
/*    digit terms cached, so one step touches only the digits the carry  */
/*    changed (same numerators as the counter-based form, reading c2).   */
/*  - Sobol' (shifted or scrambled): Antonov-Saleev Gray-code order:     */
/*    element c is the point of index g(n_start + c), g(n) = n ^ (n>>1); */
/*    the next one is one XOR with the direction number of the lowest    */
/*    zero bit of n (scrambling applied to the direction numbers, which  */
/*    is the same map by linearity).                                     */
/*  - Philox: counter-based.                                             */
/* ------------------------------------------------------------------ */
int orc_stream_raw(const orc_seq *q, int m, int j, uint64_t n_start, uint64_t count, uint64_t *out)
{
    if (q->seq == ORC_HALTON_RS || q->seq == ORC_RASRAP) {
        const uint32_t p = q->p[j];
        const int K = q->K[j];
        const uint16_t *sg = q->sigma + (size_t)m * q->sig_len + q->sig_off[j];
        uint64_t idx = q->n0[(size_t)m * q->s + j] + n_start;
        if (idx + count > q->D[j]) return -1;
        uint64_t a[64], w[64], S[65];
        for (int k = 0; k <= K; ++k) {
            a[k] = idx % p;
            idx /= p;
            w[k] = orc_ipow(p, K - k);
        }
#define ORC_TERM(k, d) ((k) < K ? (uint64_t)sg[d] * w[k] : ((d) ? (uint64_t)sg[d] : 0u))
        S[K + 1] = 0;
        for (int k = K; k >= 0; --k) S[k] = S[k + 1] + ORC_TERM(k, a[k]);
        for (uint64_t c = 0; c < count; ++c) {
            out[c] = S[0];
            int k = 0;
            while (k <= K && a[k] == p - 1) { a[k] = 0; ++k; }
            if (k > K) { if (c + 1 < count) return -1; break; }
            a[k] += 1;
            S[k] = S[k + 1] + ORC_TERM(k, a[k]);
            for (int i = k - 1; i >= 0; --i) S[i] = S[i + 1] + ORC_TERM(i, 0);
        }
#undef ORC_TERM
        return 0;
    }
    if (q->seq == ORC_SOBOL_DS || q->seq == ORC_SOBOL_LMS) {
        uint32_t V[32];
        for (int k = 0; k < 32; ++k) {
            const uint32_t v = q->V[(size_t)j * 32 + k];
            V[k] = q->seq == ORC_SOBOL_LMS ? orc_sobol_lms_apply(q->lms + ((size_t)m * q->s + j) * 32, v) : v;
        }
        const uint32_t e = q->shift[(size_t)m * q->s + j];
        uint64_t n = n_start;
        uint32_t x = 0;
        const uint64_t g = n ^ (n >> 1);
        for (int k = 0; k < 32; ++k)
            if ((g >> k) & 1u) x ^= V[k];
        for (uint64_t c = 0; c < count; ++c, ++n) {
            out[c] = (uint64_t)(x ^ e);
            int z = 0;
            while ((n >> z) & 1u) ++z;   /* lowest zero bit of n: g(n+1) = g(n) ^ 2^z */
            if (z < 32) x ^= V[z];
        }
        return 0;
    }
    for (uint64_t c = 0; c < count; ++c)
        out[c] = (uint64_t)orc_philox_path_word(q->seed, q->inst, m, j, n_start + c);
    return 0;
}

/* All rows [M][s][count] of the stream, OpenMP over rows. */
int orc_stream_rows(const orc_seq *q, uint64_t n_start, uint64_t count, int threads, uint64_t *out)
{
    int bad = 0;
    const int rows = q->M * q->s;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads) reduction(| : bad)
    for (int r = 0; r < rows; ++r)
        bad |= orc_stream_raw(q, r / q->s, r % q->s, n_start, count, out + (size_t)r * count) != 0;
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Inverse normal CDF (paper silent; reading c7): Newton's method on   */
/* Phi(x) = erfc(-x / sqrt 2) / 2 with a bisection safeguard, for the  */
/* lower half q in (0, 1/2].                                           */
/* ------------------------------------------------------------------ */
double orc_ndtri_lower(double q)
{
    if (!(q < 0.5)) return 0.0;
    double lo = -40.0, hi = 0.0;
    double x = -sqrt(-2.0 * log(q));
    if (x < lo) x = lo;
    for (int it = 0; it < 200; ++it) {
        double F = 0.5 * erfc(-x / sqrt(2.0)) - q;
        if (F > 0.0) hi = x; else lo = x;
        double dens = exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
        double xn = x - F / dens;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        int done = fabs(xn - x) <= 1e-15 * fmax(1.0, fabs(x));
        x = xn;
        if (done) break;
    }
    return x;
}

/* Uniform and normal value of one coordinate (reading c6): with
 * q = (min(raw, D-1-raw) + 1/2)/D the normal is -/+ Phi^-1(q), so 1 - u is
 * never formed in floating point. */
void orc_coord(const orc_seq *q, int m, int j, uint64_t n, double *u, double *z)
{
    uint64_t D;
    uint64_t raw = orc_coord_raw(q, m, j, n, &D);
    uint64_t comp = D - 1 - raw;
    if (u) *u = ((double)raw + 0.5) / (double)D;
    if (z) {
        int lower = raw <= comp;
        double qq = ((double)(lower ? raw : comp) + 0.5) / (double)D;
        double x = orc_ndtri_lower(qq);
        *z = lower ? x : -x;
    }
}

/* Point-stream output, layout [M][s][N]: transform 0 = uniform (double),
 * 1 = normal (double), 2 = raw integer numerators (uint64). */
int orc_points(const orc_seq *q, int64_t N, int64_t offset, int transform, void *out, int nthreads)
{
    int M = q->M, s = q->s;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int m = 0; m < M; ++m)
        for (int j = 0; j < s; ++j)
            for (int64_t i = 0; i < N; ++i) {
                size_t idx = ((size_t)m * s + j) * (size_t)N + (size_t)i;
                uint64_t n = (uint64_t)(offset + i);
                if (transform == 2) {
                    uint64_t D;
                    ((uint64_t *)out)[idx] = orc_coord_raw(q, m, j, n, &D);
                } else if (transform == 0) {
                    orc_coord(q, m, j, n, &((double *)out)[idx], NULL);
                } else {
                    orc_coord(q, m, j, n, NULL, &((double *)out)[idx]);
                }
            }
    (void)nthreads;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Estimator (Sec. 1): theta_N^m = (1/N) sum_i f(q_i^m).               */
/* Product test integrand f(x) = prod_j (|4 x_j - 2| + a_j)/(1 + a_j). */
/* ------------------------------------------------------------------ */
int orc_product_theta(const orc_seq *q, int64_t N, int64_t offset, const double *a,
                      int m_lo, int m_hi, double *theta, int nthreads)
{
    int s = q->s;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int m = m_lo; m < m_hi; ++m) {
        double sum = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double f = 1.0;
            for (int j = 0; j < s; ++j) {
                double u;
                orc_coord(q, m, j, (uint64_t)(offset + i), &u, NULL);
                f *= (fabs(4.0 * u - 2.0) + a[j]) / (1.0 + a[j]);
            }
            sum += f;
        }
        theta[m] = sum / (double)N;
    }
    (void)nthreads;
    return 0;
}

/* ------------------------------------------------------------------ */
/* LIBOR market model (Sec. 5).  Forwards L_1..L_nf over [T_n, T_n+1]  */
/* with T_n = n delta; L_0 is fixed at t = 0.  Steps t_i = T_i, split  */
/* into `substeps` equal sub-steps (substeps = 1 is the paper's grid). */
/* Dimension of factor f at global step g is g d + f (reading c8).     */
/* Caplet n pays delta (L_n(T_n) - K)^+ at T_{n+1}; under the spot     */
/* measure its value is E[delta (L_n(T_n)-K)^+ / prod_{j<=n}           */
/* (1 + delta L_j(T_j))] (reading c10).                                */
/* ------------------------------------------------------------------ */
typedef struct {
    int n_fwd;          /* forwards L_1..L_nf */
    int d;              /* factors */
    int scheme;         /* 0 = log-Euler, 1 = Euler (eq. L_n_discrete) */
    int substeps;       /* time steps per accrual period */
    double delta;
    const double *L0;   /* [nf+1]: L_0(0), L_1(0), .., L_nf(0) */
    const double *vol;  /* [nf]: |sigma_n| for n = 1..nf */
    const double *load; /* [nf][d] unit loadings b_n (sigma_n = vol_n b_n); NULL when d = 1 */
} orc_lmm;

static double orc_lmm_dot(const orc_lmm *lm, int n, int j)   /* sigma_n . sigma_j, 1-based n, j */
{
    double b = 0.0;
    if (lm->d == 1 || !lm->load) b = 1.0;
    else
        for (int f = 0; f < lm->d; ++f)
            b += lm->load[(size_t)(n - 1) * lm->d + f] * lm->load[(size_t)(j - 1) * lm->d + f];
    return lm->vol[n - 1] * lm->vol[j - 1] * b;
}

/* One path of the LMM; pay[(n-1) nK + k] receives the discounted payoff of
 * caplet n at strike K[k]. */
static void orc_lmm_path(const orc_seq *q, const orc_lmm *lm, const double *K, int nK,
                         int m, uint64_t n_pt, double *L, double *Lnew, double *Z, double *pay)
{
    int nf = lm->n_fwd, d = lm->d, S = lm->substeps;
    double dl = lm->delta, h = dl / S;
    for (int n = 0; n <= nf; ++n) L[n] = lm->L0[n];
    double disc = 1.0 / (1.0 + dl * L[0]);
    for (int t = 0; t < nf; ++t) {              /* period [T_t, T_{t+1}]; eta = t + 1 */
        for (int sub = 0; sub < S; ++sub) {
            int g = t * S + sub;
            for (int f = 0; f < d; ++f) orc_coord(q, m, g * d + f, n_pt, NULL, &Z[f]);
            for (int n = t + 1; n <= nf; ++n) {
                double mu = 0.0;               /* mu_n = sum_{j=eta}^{n} delta L_j sigma_n.sigma_j/(1+delta L_j) */
                for (int j = t + 1; j <= n; ++j)
                    mu += dl * L[j] * orc_lmm_dot(lm, n, j) / (1.0 + dl * L[j]);
                double sz = 0.0;               /* sigma_n . Z */
                for (int f = 0; f < d; ++f) {
                    double b = (d == 1 || !lm->load) ? 1.0 : lm->load[(size_t)(n - 1) * d + f];
                    sz += lm->vol[n - 1] * b * Z[f];
                }
                double s2 = orc_lmm_dot(lm, n, n);
                if (lm->scheme == 0)
                    Lnew[n] = L[n] * exp((mu - 0.5 * s2) * h + sqrt(h) * sz);
                else
                    Lnew[n] = L[n] + mu * L[n] * h + L[n] * sqrt(h) * sz;
            }
            for (int n = t + 1; n <= nf; ++n) L[n] = Lnew[n];
        }
        int n = t + 1;                          /* L_n is fixed at T_n */
        disc /= (1.0 + dl * L[n]);
        for (int k = 0; k < nK; ++k) {
            double x = L[n] - K[k];
            pay[(size_t)(n - 1) * nK + k] = dl * (x > 0.0 ? x : 0.0) * disc;
        }
    }
}

int orc_lmm_caplets(const orc_seq *q, const orc_lmm *lm, const double *K, int nK,
                    int64_t N, int64_t offset, int m_lo, int m_hi, double *theta, int nthreads)
{
    int nf = lm->n_fwd, nout = nf * nK;
    if (q->s < nf * lm->d * lm->substeps) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int m = m_lo; m < m_hi; ++m) {
        double *L = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *Lnew = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *Z = (double *)malloc(sizeof(double) * (size_t)lm->d);
        double *pay = (double *)malloc(sizeof(double) * (size_t)nout);
        double *sum = (double *)calloc((size_t)nout, sizeof(double));
        for (int64_t i = 0; i < N; ++i) {
            orc_lmm_path(q, lm, K, nK, m, (uint64_t)(offset + i), L, Lnew, Z, pay);
            for (int o = 0; o < nout; ++o) sum[o] += pay[o];
        }
        for (int o = 0; o < nout; ++o) theta[(size_t)m * nout + o] = sum[o] / (double)N;
        free(L); free(Lnew); free(Z); free(pay); free(sum);
    }
    (void)nthreads;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Pathwise adjoint of the caplet strip (not in the paper).            */
/* Objective per path: V = sum_n sum_k w_{n,k} delta (L_n(T_n)-K_k)^+  */
/* D_n with D_n = prod_{j=0}^{n} (1 + delta L_j(T_j))^-1, on the       */
/* paper's grid (one log-Euler step per period).  Reverse-mode chain   */
/* rule over the stored path gives dV/dL_n(0) and dV/dvol_n with the   */
/* unit loadings b_n held fixed.  Outputs are replication means.       */
/* ------------------------------------------------------------------ */
int orc_lmm_adjoint(const orc_seq *q, const orc_lmm *lm, const double *K, int nK, const double *wts,
                    int64_t N, int64_t offset, int m_lo, int m_hi,
                    double *value, double *delta, double *vega, int nthreads)
{
    int nf = lm->n_fwd, d = lm->d;
    if (lm->substeps != 1 || lm->scheme != 0) return -2;
    if (q->s < nf * d) return -1;
    double dl = lm->delta, h = dl, sh = sqrt(dl);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int m = m_lo; m < m_hi; ++m) {
        double *Lh = (double *)malloc(sizeof(double) * (size_t)nf * (nf + 1)); /* pre-step L per step */
        double *Zh = (double *)malloc(sizeof(double) * (size_t)nf * d);
        double *L = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *Lnew = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *Lfix = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *Dn = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *P = (double *)malloc(sizeof(double) * (size_t)(nf + 2));
        double *G = (double *)malloc(sizeof(double) * (size_t)(nf + 2));
        double *Lbar = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *Lbar2 = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *vbar = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *a = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *A = (double *)malloc(sizeof(double) * (size_t)(nf + 1) * d);
        double *X = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *Xbar = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
        double *B = (double *)malloc(sizeof(double) * (size_t)(nf + 1) * d);
        double *sg = (double *)malloc(sizeof(double) * (size_t)(nf + 1) * d);  /* sigma_n vectors */
        double vsum = 0.0;
        double *dsum = (double *)calloc((size_t)nf, sizeof(double));
        double *gsum = (double *)calloc((size_t)nf, sizeof(double));
        for (int n = 1; n <= nf; ++n)
            for (int f = 0; f < d; ++f)
                sg[(size_t)n * d + f] = lm->vol[n - 1] * ((d == 1 || !lm->load) ? 1.0 : lm->load[(size_t)(n - 1) * d + f]);
        for (int64_t i = 0; i < N; ++i) {
            uint64_t n_pt = (uint64_t)(offset + i);
            /* forward sweep, storing the state before every step */
            for (int n = 0; n <= nf; ++n) L[n] = lm->L0[n];
            double disc = 1.0 / (1.0 + dl * L[0]);
            for (int t = 0; t < nf; ++t) {
                for (int n = 0; n <= nf; ++n) Lh[(size_t)t * (nf + 1) + n] = L[n];
                for (int f = 0; f < d; ++f) orc_coord(q, m, t * d + f, n_pt, NULL, &Zh[(size_t)t * d + f]);
                for (int n = t + 1; n <= nf; ++n) {
                    double mu = 0.0, sz = 0.0;
                    for (int j = t + 1; j <= n; ++j)
                        mu += dl * L[j] * orc_lmm_dot(lm, n, j) / (1.0 + dl * L[j]);
                    for (int f = 0; f < d; ++f) sz += sg[(size_t)n * d + f] * Zh[(size_t)t * d + f];
                    Lnew[n] = L[n] * exp((mu - 0.5 * orc_lmm_dot(lm, n, n)) * h + sh * sz);
                }
                for (int n = t + 1; n <= nf; ++n) L[n] = Lnew[n];
                int n = t + 1;
                Lfix[n] = L[n];
                disc /= (1.0 + dl * L[n]);
                Dn[n] = disc;
                double pn = 0.0;
                for (int k = 0; k < nK; ++k) {
                    double x = L[n] - K[k];
                    pn += wts[(size_t)(n - 1) * nK + k] * dl * (x > 0.0 ? x : 0.0) * disc;
                }
                P[n] = pn;
            }
            G[nf + 1] = 0.0;
            for (int n = nf; n >= 1; --n) G[n] = G[n + 1] + P[n];
            vsum += G[1];
            /* reverse sweep */
            for (int n = 0; n <= nf; ++n) { Lbar[n] = 0.0; vbar[n] = 0.0; }
            for (int t = nf - 1; t >= 0; --t) {
                int jf = t + 1;   /* forward fixed at the end of this step */
                double lb = 0.0;
                for (int k = 0; k < nK; ++k)
                    if (Lfix[jf] > K[k]) lb += wts[(size_t)(jf - 1) * nK + k] * dl * Dn[jf];
                lb -= dl / (1.0 + dl * Lfix[jf]) * G[jf];
                Lbar[jf] += lb;
                const double *Lp = Lh + (size_t)t * (nf + 1);
                const double *Zt = Zh + (size_t)t * d;
                /* recompute the step: a_j, prefix vectors A_n, exponents X_n */
                for (int f = 0; f < d; ++f) A[(size_t)t * d + f] = 0.0;
                for (int n = t + 1; n <= nf; ++n) {
                    a[n] = dl * Lp[n] / (1.0 + dl * Lp[n]);
                    double xs = 0.0, sz = 0.0, s2 = 0.0;
                    for (int f = 0; f < d; ++f) {
                        A[(size_t)n * d + f] = A[(size_t)(n - 1) * d + f] + a[n] * sg[(size_t)n * d + f];
                        xs += sg[(size_t)n * d + f] * A[(size_t)n * d + f];
                        sz += sg[(size_t)n * d + f] * Zt[f];
                        s2 += sg[(size_t)n * d + f] * sg[(size_t)n * d + f];
                    }
                    X[n] = (xs - 0.5 * s2) * h + sh * sz;
                }
                for (int n = t + 1; n <= nf; ++n) Xbar[n] = Lbar[n] * Lp[n] * exp(X[n]);
                /* suffix vectors B_j = sum_{n >= j} Xbar_n sigma_n */
                for (int f = 0; f < d; ++f) B[(size_t)nf * d + f] = Xbar[nf] * sg[(size_t)nf * d + f];
                for (int n = nf - 1; n >= t + 1; --n)
                    for (int f = 0; f < d; ++f)
                        B[(size_t)n * d + f] = B[(size_t)(n + 1) * d + f] + Xbar[n] * sg[(size_t)n * d + f];
                for (int n = t + 1; n <= nf; ++n) {
                    double sB = 0.0, gv = 0.0;
                    for (int f = 0; f < d; ++f) {
                        double bnf = (d == 1 || !lm->load) ? 1.0 : lm->load[(size_t)(n - 1) * d + f];
                        double sgbar = Xbar[n] * (h * A[(size_t)n * d + f] - h * sg[(size_t)n * d + f] + sh * Zt[f])
                                       + h * a[n] * B[(size_t)n * d + f];
                        gv += sgbar * bnf;
                        sB += sg[(size_t)n * d + f] * B[(size_t)n * d + f];
                    }
                    double den = 1.0 + dl * Lp[n];
                    Lbar2[n] = Lbar[n] * exp(X[n]) + h * sB * dl / (den * den);
                    vbar[n] += gv;
                }
                for (int n = t + 1; n <= nf; ++n) Lbar[n] = Lbar2[n];
            }
            for (int n = 1; n <= nf; ++n) { dsum[n - 1] += Lbar[n]; gsum[n - 1] += vbar[n]; }
        }
        value[m] = vsum / (double)N;
        for (int n = 0; n < nf; ++n) {
            delta[(size_t)m * nf + n] = dsum[n] / (double)N;
            vega[(size_t)m * nf + n] = gsum[n] / (double)N;
        }
        free(Lh); free(Zh); free(L); free(Lnew); free(Lfix); free(Dn); free(P); free(G);
        free(Lbar); free(Lbar2); free(vbar); free(a); free(A); free(X); free(Xbar); free(B); free(sg);
        free(dsum); free(gsum);
    }
    (void)nthreads;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Mortgage-backed security (Sec. 6, Caflisch's model).                */
/*   PV = E sum_{k=1}^{Mm} u_k m_k,  u_k = prod_{j=0}^{k-1} (1+i_j)^-1, */
/*   m_k = c r_k ((1 - w_k) + w_k c_k),  r_k = prod_{j=1}^{k-1}(1-w_j), */
/*   c_k = sum_{j=0}^{Mm-k} (1+i_0)^-j,                                 */
/*   i_k = K0 e^{xi_k} i_{k-1},  w_k = K1 + K2 atan(K3 i_k + K4),       */
/*   K0 = exp(-sigma^2/2),  xi_k = sigma z_k (reading c13, c14).       */
/* ------------------------------------------------------------------ */
typedef struct {
    int months;
    double i0, K1, K2, K3, K4, sigma, c;
} orc_mbs;

int orc_mbs_theta(const orc_seq *q, const orc_mbs *mb, int64_t N, int64_t offset,
                  int m_lo, int m_hi, double *theta, int nthreads)
{
    int Mm = mb->months;
    if (q->s < Mm) return -1;
    double *ck = (double *)malloc(sizeof(double) * (size_t)(Mm + 1));
    for (int k = 1; k <= Mm; ++k) {
        double acc = 0.0;
        for (int j = 0; j <= Mm - k; ++j) acc += pow(1.0 + mb->i0, -(double)j);
        ck[k] = acc;
    }
    double K0 = exp(-0.5 * mb->sigma * mb->sigma);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int m = m_lo; m < m_hi; ++m) {
        double sum = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            uint64_t n_pt = (uint64_t)(offset + i);
            double i_prev = mb->i0;            /* i_{k-1} */
            double u = 1.0 / (1.0 + mb->i0);   /* u_1 */
            double r = 1.0;                    /* r_1 */
            double v = 0.0;
            for (int k = 1; k <= Mm; ++k) {
                double z;
                orc_coord(q, m, k - 1, n_pt, NULL, &z);
                double xi = mb->sigma * z;
                double ik = K0 * exp(xi) * i_prev;
                double w = mb->K1 + mb->K2 * atan(mb->K3 * ik + mb->K4);
                double mk = mb->c * r * ((1.0 - w) + w * ck[k]);
                v += u * mk;
                u = u / (1.0 + ik);            /* u_{k+1} */
                r = r * (1.0 - w);             /* r_{k+1} */
                i_prev = ik;
            }
            sum += v;
        }
        theta[m] = sum / (double)N;
    }
    free(ck);
    (void)nthreads;
    return 0;
}

/* ------------------------------------------------------------------ */
/* RQ_{M,N} and the sample standard deviation over replications.       */
/* ------------------------------------------------------------------ */
void orc_rq_stats(const double *theta, int M, int nout, double *rq, double *sd)
{
    for (int o = 0; o < nout; ++o) {
        double mean = 0.0;
        for (int m = 0; m < M; ++m) mean += theta[(size_t)m * nout + o];
        mean /= M;
        double ss = 0.0;
        for (int m = 0; m < M; ++m) {
            double e = theta[(size_t)m * nout + o] - mean;
            ss += e * e;
        }
        rq[o] = mean;
        sd[o] = M > 1 ? sqrt(ss / (M - 1)) : 0.0;
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
