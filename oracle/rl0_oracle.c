/*
 * rl0_oracle.c -- plain, slow FP64 CPU oracle for Robust-l0 decoding
 * (Mendoza-Smith, Tanner, Wechsung, "A robust parallel algorithm for
 * combinatorial compressed sensing", arXiv 1704.09012).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * (the CUDA library) never calls it and shares no code, header, table or
 * constant generator with it.
 *
 * Everything here is written for a reader checking it against the paper:
 * loops follow the paper's statement, all arithmetic is double precision,
 * and nothing is blocked, fused or reordered beyond what the paper states.
 *
 * Readings of the paper where it is silent, ambiguous or garbled are marked
 * "reading:" next to the code they shape.
 *
 * Parity status of each function (what pins it) is listed in the test-suite;
 * every function below has at least one pin that does not go through this file.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXQ 512

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Written from the published round function:     */
/* two 32x32->64 multiplies per round, key schedule bumped by the Weyl       */
/* constants between rounds, ten rounds.                                     */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A sequential stream of 32-bit words drawn from Philox blocks.  The counter
 * layout is part of the generator's definition (the CUDA side implements the
 * same definition independently):
 *   key     = (seed low 32 bits, seed high 32 bits)
 *   counter = (block index, id low 32 bits, id high 32 bits, stream tag)    */
typedef struct {
    uint32_t key[2];
    uint32_t id_lo, id_hi, tag;
    uint32_t block;
    uint32_t buf[4];
    int used;
} orc_stream;

static void orc_stream_init(orc_stream *s, uint64_t seed, uint64_t id, uint32_t tag)
{
    s->key[0] = (uint32_t)seed; s->key[1] = (uint32_t)(seed >> 32);
    s->id_lo = (uint32_t)id; s->id_hi = (uint32_t)(id >> 32); s->tag = tag;
    s->block = 0; s->used = 4;
}

static uint32_t orc_stream_next(orc_stream *s)
{
    if (s->used == 4) {
        uint32_t ctr[4] = { s->block, s->id_lo, s->id_hi, s->tag };
        orc_philox4x32_10(ctr, s->key, s->buf);
        s->block++;
        s->used = 0;
    }
    return s->buf[s->used++];
}

/* Uniform integer in [0, m) from 32-bit words, by Lemire's multiply-shift
 * with rejection ("Fast random integer generation in an interval", 2019),
 * which is exactly uniform.                                                 */
static uint32_t orc_uniform_below(orc_stream *s, uint32_t m)
{
    uint64_t prod = (uint64_t)orc_stream_next(s) * (uint64_t)m;
    uint32_t low = (uint32_t)prod;
    if (low < m) {
        uint32_t thresh = (uint32_t)(0u - m) % m;
        while (low < thresh) {
            prod = (uint64_t)orc_stream_next(s) * (uint64_t)m;
            low = (uint32_t)prod;
        }
    }
    return (uint32_t)(prod >> 32);
}

#define ORC_TAG_EXPANDER 0x41u  /* 'A' */
#define ORC_TAG_NOISE    0x4Eu  /* 'N' */

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Def. "Generating model GM(n,m,k,d,mu,nu)", item 1: the support of every
 * column of A is drawn uniformly from the d-subsets of [m].  Draw words in
 * order, keep the first d distinct rows, then sort them ascending (reading:
 * N(j) is listed in ascending row order).  rows is column-major: column j
 * owns rows[j*d .. j*d+d-1].                                                */
int orc_make_expander(int64_t n, int64_t m, int d, uint64_t seed, int32_t *rows)
{
    if (n < 1 || m < 1 || d < 1 || d > m || m > 0x7fffffffLL) return ORC_EINVAL;
    for (int64_t j = 0; j < n; ++j) {
        orc_stream s;
        orc_stream_init(&s, seed, (uint64_t)j, ORC_TAG_EXPANDER);
        int32_t *col = rows + j * d;
        int got = 0;
        while (got < d) {
            int32_t cand = (int32_t)orc_uniform_below(&s, (uint32_t)m);
            int dup = 0;
            for (int q = 0; q < got; ++q) if (col[q] == cand) { dup = 1; break; }
            if (!dup) col[got++] = cand;
        }
        qsort(col, (size_t)d, sizeof(int32_t), cmp_i32);
    }
    return ORC_OK;
}

/* Def. GM, items 4 and 6: yhat = A x + eta with eta_i i.i.d. N(0, sigma_n^2).
 * The standard normal deviate of row i comes from one Philox block with
 * id = i, by the Box-Muller transform (Box and Muller, 1958):
 *   u1 = (w0 + 1) / 2^32 in (0,1],  u2 = w1 / 2^32,
 *   z  = sqrt(-2 ln u1) cos(2 pi u2).                                       */
void orc_noise(int64_t m, double sigma_n, uint64_t noise_seed, double *eta)
{
    for (int64_t i = 0; i < m; ++i) {
        uint32_t ctr[4] = { 0u, (uint32_t)i, (uint32_t)((uint64_t)i >> 32), ORC_TAG_NOISE };
        uint32_t key[2] = { (uint32_t)noise_seed, (uint32_t)(noise_seed >> 32) };
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        double u1 = ((double)w[0] + 1.0) / 4294967296.0;
        double u2 = (double)w[1] / 4294967296.0;
        double z = sqrt(-2.0 * log(u1)) * cos(2.0 * ORC_PI * u2);
        eta[i] = sigma_n * z;
    }
}

/* y = A x (no noise), straight from the definition y_i = sum_j A_ij x_j.    */
void orc_matvec(int64_t n, int64_t m, int d, const int32_t *rows, const double *x, double *y)
{
    for (int64_t i = 0; i < m; ++i) y[i] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (x[j] == 0.0) continue;
        for (int s = 0; s < d; ++s) y[rows[j * d + s]] += x[j];
    }
}

/* yhat = A x + eta (Def. GM item 6), eta from orc_noise (sigma_n = 0: none). */
void orc_sketch(int64_t n, int64_t m, int d, const int32_t *rows, const double *x,
                double sigma_n, uint64_t noise_seed, double *yhat)
{
    orc_matvec(n, m, d, rows, x, yhat);
    if (sigma_n > 0.0) {
        double *eta = (double *)malloc((size_t)m * sizeof(double));
        orc_noise(m, sigma_n, noise_seed, eta);
        for (int64_t i = 0; i < m; ++i) yhat[i] += eta[i];
        free(eta);
    }
}

/* ------------------------------------------------------------------------ */
/* Posteriors for centred Gaussian signal and noise.                         */
/*                                                                          */
/* Eq. (pz_gaussian) / (pe_gaussian): with mu = N(0, s_s^2), nu = N(0, s_n^2)*/
/*   p_z(w) = phi(w|s_n^2)  / sum_q (d rho)^q/q!  phi(w| q s_s^2 +   s_n^2)   */
/*   p_e(w) = phi(w|2s_n^2) / sum_q (2d rho)^q/q! phi(w| q s_s^2 + 2 s_n^2)   */
/* Eq. (pz_approx) / (pe_approx) keep q = 0..ell and replace the remaining   */
/* terms by one Gaussian of weight R(ell) = sum_{q>ell} lam^q/q! and the     */
/* variance-matched tail variance (Lemma "sums of centred density functions"):*/
/*   v_tail = (s_s^2 lam R(ell-1) + v_noise R(ell)) / R(ell).                */
/* One structure serves both: lam = d rho, v_noise = s_n^2 for p_z, and      */
/* lam = 2 d rho, v_noise = 2 s_n^2 for p_e.                                 */
/* readings: the printed sigma_q^2 = q s_s^2 + s_n (no square) is read as    */
/* q s_s^2 + s_n^2, as in Eq. (pz_gaussian); the printed sigma_{q,e}^2 is    */
/* read as q s_s^2 + 2 s_n^2 and R_e's terms as (2 d rho)^q/q!, as in        */
/* Eq. (pe_gaussian); the tail sum "q = ell+1..ell" is read as ell+1..inf.   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nterms;               /* explicit terms q = 0..nterms-1 (= ell+1)   */
    double lam;               /* Poisson rate: d rho or 2 d rho             */
    double v_noise;           /* s_n^2 or 2 s_n^2                           */
    double s2;                /* s_s^2                                      */
    double w[ORC_MAXQ];       /* lam^q / q!                                 */
    double v[ORC_MAXQ];       /* q s_s^2 + v_noise                          */
    double R;                 /* tail weight R(ell)                         */
    double v_tail;            /* tail variance                              */
    int use_tail;
    double logp0;             /* log p(0): the maximum of p, see below      */
    int noiseless;            /* v_noise == 0                               */
    double tol;               /* noiseless equality tolerance               */
} orc_series;

/* R(ell) = sum_{q > ell} lam^q / q!, summed term by term until the terms no
 * longer change the sum (R(-1) = e^lam).                                    */
static double orc_poisson_tail(double lam, int ell)
{
    int q0 = (ell + 1 < 0) ? 0 : ell + 1;
    double term = 1.0;                       /* lam^0 / 0! */
    for (int q = 1; q <= q0; ++q) term *= lam / q;
    double sum = 0.0;
    for (int q = q0; q < q0 + 4000; ++q) {
        sum += term;
        term *= lam / (q + 1);
        if (term == 0.0 || (q + 1 > lam && term < sum * 1e-18)) break;
    }
    return sum;
}

static double log_phi(double w, double var)
{
    return -0.5 * log(2.0 * ORC_PI * var) - 0.5 * w * w / var;
}

/* log of the unnormalised posterior p(w) of Eq. (pz_approx)/(pe_approx),
 * evaluated as log(numerator) - log(denominator) with the denominator's sum
 * taken by log-sum-exp so that no term underflows to 0/0.                   */
static double orc_series_logp(const orc_series *S, double w)
{
    double lt[ORC_MAXQ + 1] = { 0.0 };
    int nt = 0;
    for (int q = 0; q < S->nterms; ++q) {
        if (S->w[q] <= 0.0) continue;
        lt[nt++] = log(S->w[q]) + log_phi(w, S->v[q]);
    }
    if (S->use_tail) lt[nt++] = log(S->R) + log_phi(w, S->v_tail);
    double mx = (nt > 0) ? lt[0] : -INFINITY;
    for (int q = 1; q < nt; ++q) if (lt[q] > mx) mx = lt[q];
    double acc = 0.0;
    for (int q = 0; q < nt; ++q) acc += exp(lt[q] - mx);
    double logden = mx + log(acc);
    return log_phi(w, S->v_noise) - logden;
}

/* Build the series.  ell = number of explicit terms beyond q = 0 (the paper's
 * ell).  exact != 0 keeps ell explicit terms and drops the tail, which with a
 * large ell is the untruncated series of Eq. (pz_gaussian)/(pe_gaussian).   */
static int orc_series_init(orc_series *S, double lam, double s2, double v_noise, int ell,
                           int exact, double tol)
{
    if (ell < 0 || ell + 1 > ORC_MAXQ) return ORC_EINVAL;
    memset(S, 0, sizeof(*S));
    S->lam = lam; S->s2 = s2; S->v_noise = v_noise; S->nterms = ell + 1;
    S->noiseless = (v_noise <= 0.0);
    S->tol = tol;
    double term = 1.0;
    for (int q = 0; q <= ell; ++q) {
        if (q > 0) term *= lam / q;
        S->w[q] = term;
        S->v[q] = q * s2 + v_noise;
    }
    S->use_tail = 0;
    if (!exact) {
        double R_l = orc_poisson_tail(lam, ell);          /* R(ell)   */
        double R_lm1 = orc_poisson_tail(lam, ell - 1);    /* R(ell-1) */
        if (R_l > 0.0) {
            S->R = R_l;
            S->v_tail = (s2 * lam * R_lm1 + v_noise * R_l) / R_l;
            S->use_tail = 1;
        }
    }
    /* reading: the maximiser of p in Eq. (breve) is w = 0.  With every term a
     * centred Gaussian of variance >= v_noise, 1/p(w) is a positive mixture of
     * exp(c w^2) with c >= 0, which is smallest at w = 0.                    */
    if (!S->noiseless) S->logp0 = orc_series_logp(S, 0.0);
    return ORC_OK;
}

/* The two posteriors' series: which = 0, p_z of a row, Eq. (pz_gaussian):
 * rate d rho, noise variance sigma_n^2; which = 1, p_e of a row pair,
 * Eq. (pe_gaussian): rate 2 d rho, noise variance 2 sigma_n^2.  The decoder,
 * log_posterior and tail_constants all build them here.                     */
static int orc_posterior_series(orc_series *S, int which, int d, double rho, double sigma_s, double sigma_n,
                                int ell, int exact, double tol)
{
    double s2 = sigma_s * sigma_s, n2 = sigma_n * sigma_n;
    double lam = (which == 0) ? d * rho : 2.0 * d * rho;
    double vn = (which == 0) ? n2 : 2.0 * n2;
    return orc_series_init(S, lam, s2, vn, ell, exact, tol);
}

/* log of the normalised posterior of Eq. (breve): log(p(w) / max_s p(s)).
 * Noiseless (v_noise = 0) reading: p is the indicator of w = 0, taken with
 * the tolerance tol, so log p_breve is 0 or -inf.                           */
static double orc_log_pbreve(const orc_series *S, double w)
{
    if (S->noiseless) return (fabs(w) <= S->tol) ? 0.0 : -INFINITY;
    return orc_series_logp(S, w) - S->logp0;
}

/* ------------------------------------------------------------------------ */
/* Decoder parameters and the posterior pair used by one decode.             */
/* ------------------------------------------------------------------------ */
typedef struct {
    double sigma_s;       /* signal std (mu = N(0, sigma_s^2))               */
    double sigma_n;       /* noise std  (nu = N(0, sigma_n^2)); 0 = noiseless */
    int quantised;        /* Table "scores": quantised (1) or continuous (0) */
    int adaptive_k;       /* Alg. 2's adaptive_k flag (analytic scores only) */
    double c;             /* sweep step; 0 = Eq. (finetune_c_*) rule         */
    double alpha;         /* consensus threshold; 0 = floor(d/2)+1           */
    int ell;              /* explicit series terms; 0 = 4                    */
    int max_rounds;       /* 0 = all rounds with t > 0                       */
    double noiseless_tol; /* 0 = 1e-5 (equality tolerance when sigma_n = 0)  */
    int literal_ei_test;  /* 1: the printed |r_i - w| <= |r_i| test          */
    int learned;          /* 1: the learned column scorer replaces n_e - n_z >= alpha */
    const uint16_t *mlp;  /* its parameters as BF16 bit patterns (1633 values)   */
    double mlp_threshold; /* accept when sigmoid(logit) >= this; 0 = 0.5        */
    int best_anchor;      /* 1: of a column's passing anchors, the one with the
                             largest n_e - n_z (ties: the lower row) gives the
                             update; 0: the last passing one in row order     */
} orc_params;

typedef struct {
    int rounds;            /* rounds executed                                */
    int accepted_rounds;   /* rounds whose candidate was accepted            */
    int converged;         /* ||r_hat||_1 <= stopping level at exit          */
    int64_t support_size;  /* |supp x_hat|                                   */
    double final_l1;       /* ||r_hat||_1 at exit                            */
    double c, alpha, stop_level;
    int ell, nrounds_max;
    int analytic_rounds;   /* learned decodes: rounds of the analytic continuation */
} orc_stats;

typedef struct {
    double t;              /* sweep value of the round                       */
    double l1_candidate;   /* ||y - A x'||_1                                 */
    double l1_hat;         /* ||r_hat||_1 after the round                    */
    int accepted;
    int64_t updated;       /* columns that received an update                */
    int64_t support;       /* |supp x'| after H_k                            */
    double k_prior;        /* the sparsity k of the posteriors this round used */
} orc_round_log;

/* ---- Learned column scorer (not in the paper: an addition whose
 * definition is fixed by the CUDA library's header) -------------------------
 * Features of a candidate, in order: the 7 smallest |r_l - w| / sigma_n
 * (clipped at 8, padded with 8), n_e/d, n_z/d, log(1 + |w|/sigma_n)/5, the
 * relative l1 gain (sum|r_l| - sum|r_l - w|) / sum|r_l| clipped to [-1, 1],
 * t, d k/m, (n_e - n_z)/d, 0, 0.  Network: 16 -> 32 -> 32 -> 1, ReLU hidden
 * layers, parameters W1 (16x32, input-major), b1, W2 (32x32), b2, w3, b3.    */
#define ORC_NFEAT 16
#define ORC_HID 32
#define ORC_MLP_PARAMS (ORC_NFEAT * ORC_HID + ORC_HID + ORC_HID * ORC_HID + ORC_HID + ORC_HID + 1)

double orc_bf16_to_double(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, sizeof(f));
    return (double)f;
}

void orc_features(int d, const double *rl, double w, double ne, double nz, double lhs, double rhs,
                  double sigma_n, double t, double drho, double *f)
{
    double dev[64];
    int used[64];
    for (int l = 0; l < d; ++l) {
        double v = fabs(rl[l] - w) / sigma_n;
        dev[l] = v < 8.0 ? v : 8.0;
        used[l] = 0;
    }
    for (int q = 0; q < 7; ++q) {          /* the 7 smallest, padded with 8 */
        double best = 8.0;
        int bi = -1;
        for (int l = 0; l < d; ++l)
            if (!used[l] && dev[l] < best) { best = dev[l]; bi = l; }
        if (bi >= 0) used[bi] = 1;
        f[q] = best;
    }
    f[7] = ne / d;
    f[8] = nz / d;
    f[9] = log1p(fabs(w) / sigma_n) / 5.0;
    double g = (rhs - lhs) / (rhs > 1e-30 ? rhs : 1e-30);
    f[10] = g < -1.0 ? -1.0 : (g > 1.0 ? 1.0 : g);
    f[11] = t;
    f[12] = drho;
    f[13] = (ne - nz) / d;
    f[14] = 0.0;
    f[15] = 0.0;
}

double orc_mlp_logit(const double *W, const double *f)
{
    const double *W1 = W, *b1 = W1 + ORC_NFEAT * ORC_HID, *W2 = b1 + ORC_HID, *b2 = W2 + ORC_HID * ORC_HID;
    const double *w3 = b2 + ORC_HID, *b3 = w3 + ORC_HID;
    double h1[ORC_HID], out = b3[0];
    for (int o = 0; o < ORC_HID; ++o) {
        double a = b1[o];
        for (int i = 0; i < ORC_NFEAT; ++i) a += f[i] * W1[i * ORC_HID + o];
        h1[o] = a > 0.0 ? a : 0.0;
    }
    for (int o = 0; o < ORC_HID; ++o) {
        double a = b2[o];
        for (int i = 0; i < ORC_HID; ++i) a += h1[i] * W2[i * ORC_HID + o];
        out += (a > 0.0 ? a : 0.0) * w3[o];
    }
    return out;
}

typedef struct {
    orc_series pz, pe;
    double drho;                     /* d k / m, a feature of the learned scorer */
    double mlp[ORC_MLP_PARAMS];      /* its parameters, decoded from BF16        */
} orc_post;

/* Eq. (finetune_c_quant) and Eq. (finetune_c_cont).                         */
double orc_default_c(int quantised, double delta, double rho)
{
    if (quantised) {
        if (delta <= 0.05) return 0.01;
        if (rho <= 0.1) return 0.05;
        if (rho <= 0.2) return 0.075;
        return 0.1;
    }
    return (delta <= 0.05) ? 0.01 : 0.025;
}

/* reading: t starts at 1 and drops by c while t > 0; the number of rounds is
 * the number of r >= 0 with 1 - r c > 0, counted with a tolerance so that
 * e.g. c = 0.025 gives exactly 40 rounds; round r uses t_r = 1 - r c.       */
int orc_num_rounds(double c)
{
    return (int)ceil(1.0 / c - 1e-9);
}

static void orc_resolve(const orc_params *in, int d, int64_t n, int64_t m, int64_t k, orc_params *p)
{
    *p = *in;
    if (p->c <= 0.0) p->c = orc_default_c(p->quantised, (double)m / (double)n, (double)k / (double)m);
    /* reading: the consensus test "more than d/2 rows agree" gives alpha =
     * floor(d/2)+1 for the integer counts of the quantised scores; for the
     * soft counts of the continuous scores it is alpha = d/2, the limit
     * alpha = (1-2 eps) d, eps = 1/4, of the convergence theorem.          */
    if (p->alpha <= 0.0) p->alpha = p->quantised ? (double)(d / 2 + 1) : 0.5 * d;
    if (p->ell <= 0) p->ell = 4;
    if (p->noiseless_tol <= 0.0) p->noiseless_tol = 1e-5;
}

static int orc_post_init(orc_post *P, int d, double rho, const orc_params *p)
{
    P->drho = d * rho;
    if (p->learned) {
        if (!p->mlp || !(p->sigma_n > 0.0)) return ORC_EINVAL;
        for (int q = 0; q < ORC_MLP_PARAMS; ++q) P->mlp[q] = orc_bf16_to_double(p->mlp[q]);
    }
    int rc = orc_posterior_series(&P->pz, 0, d, rho, p->sigma_s, p->sigma_n, p->ell, 0, p->noiseless_tol);
    if (rc) return rc;
    return orc_posterior_series(&P->pe, 1, d, rho, p->sigma_s, p->sigma_n, p->ell, 0, p->noiseless_tol);
}

/* Table "scores".  All three take the decision in exact-math form:
 *   anchor:  1 - p_z(r) >= t      <=>  log p_z(r) <= log(1 - t)
 *   q_z:     continuous p_z(r);   quantised 1{p_z(r) >= 1 - t}
 *   q_e:     continuous p_e(D);   quantised 1{p_e(D) >= t}
 * (p meaning the normalised p_breve).  Taking logs keeps the test exact where
 * p underflows: at t = 1 the anchor test needs p_z = 0, which never holds for
 * sigma_n > 0 (reading: round t = 1 then updates nothing).                 */
static int orc_is_anchor(const orc_post *P, double r, double t)
{
    double lp = orc_log_pbreve(&P->pz, r);
    double lim = (t >= 1.0) ? -INFINITY : log(1.0 - t);
    if (t <= 0.0) return 1;
    return lp <= lim;
}

static double orc_qz(const orc_post *P, int quantised, double r, double t)
{
    double lp = orc_log_pbreve(&P->pz, r);
    if (!quantised) return exp(lp);
    double lim = (t >= 1.0) ? -INFINITY : log(1.0 - t);
    return (lp >= lim) ? 1.0 : 0.0;
}

static double orc_qe(const orc_post *P, int quantised, double D, double t)
{
    double lp = orc_log_pbreve(&P->pe, D);
    if (!quantised) return exp(lp);
    return (lp >= log(t)) ? 1.0 : 0.0;
}

/* H_k of Alg. 2: keep the k entries of largest magnitude.
 * reading: ties in magnitude go to the smaller index; with at most k
 * nonzeros H_k is the identity.                                             */
typedef struct { double a; int64_t j; } orc_mag;
static int cmp_mag(const void *x, const void *y)
{
    const orc_mag *u = (const orc_mag *)x, *v = (const orc_mag *)y;
    if (u->a > v->a) return -1;
    if (u->a < v->a) return 1;
    return (u->j > v->j) - (u->j < v->j);
}

int orc_hard_threshold(int64_t n, int64_t k, double *x)
{
    int64_t nz = 0;
    for (int64_t j = 0; j < n; ++j) if (x[j] != 0.0) nz++;
    if (nz <= k) return ORC_OK;
    orc_mag *L = (orc_mag *)malloc((size_t)nz * sizeof(orc_mag));
    if (!L) return ORC_ENOMEM;
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) if (x[j] != 0.0) { L[c].a = fabs(x[j]); L[c].j = j; c++; }
    qsort(L, (size_t)nz, sizeof(orc_mag), cmp_mag);
    for (int64_t q = k; q < nz; ++q) x[L[q].j] = 0.0;
    free(L);
    return ORC_OK;
}

static double l1norm(int64_t m, const double *r)
{
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += fabs(r[i]);
    return s;
}

/* Per-column record of one round, for tests that compare decisions.        */
typedef struct {
    int32_t passed;        /* column received an update                      */
    int32_t best_slot;     /* slot (0..d-1) of the chosen anchor, -1 if none */
    double omega;          /* the chosen consensus value                     */
    double score;          /* n_e - n_z of the chosen anchor                 */
    double nz;             /* n_z of the column                              */
    double min_margin;     /* smallest |decision margin| met in the column   */
} orc_col_rec;

/* One synchronous round of Alg. 2 (the body of its while-loop, up to and
 * including the residual rebuild) from the state (xh, rh) at sweep value t.
 * Every column reads only rh (Jacobi: updates of this round are not seen).
 *
 * readings:
 *  - the update x'_j <- x'_j + w is applied once per column, because every
 *    member of a consensus group passes the test and would otherwise add w up
 *    to d times; the value is that of the last passing anchor in row order,
 *    the overwrite semantics of Alg. 1's u_j <- r_i (best_anchor = 1: the
 *    passing anchor with the largest n_e - n_z, the lower row on ties);
 *  - ||r - w e_i||_1 <= ||r||_1 is read over the column's rows N(j):
 *    sum_l |r_l - w| <= sum_l |r_l|, the l1 change that adding w to x_j
 *    alone would cause (literal_ei_test = 1 keeps the printed |r_i - w| <= |r_i|);
 *  - the self term l = i is part of n_e, so n_e >= 1.                       */
int orc_round_step(int64_t n, int64_t m, int d, const int32_t *rows, const double *yhat,
                   int64_t k, const orc_post *P, const orc_params *p, double t,
                   const double *xh, const double *rh,
                   double *xp, double *rp, int64_t *updated, orc_col_rec *rec)
{
    int64_t upd = 0;
    int nomem = 0;
    for (int64_t j = 0; j < n; ++j) xp[j] = xh[j];
    /* Every column reads only rh and writes only xp[j] and rec[j], so the
     * columns may be scored in any order: the OpenMP build of this file
     * shares them among threads and gives the serial build's results. */
#pragma omp parallel reduction(+ : upd, nomem)
    {
    double *rl = (double *)malloc((size_t)d * sizeof(double));
    if (!rl) nomem = 1;
#pragma omp for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        if (!rl) continue;
        const int32_t *N = rows + j * d;
        for (int l = 0; l < d; ++l) rl[l] = rh[N[l]];
        double nz = 0.0;
        for (int l = 0; l < d; ++l) nz += orc_qz(P, p->quantised, rl[l], t);
        int best = -1;
        double best_score = 0.0, best_w = 0.0;
        double margin = INFINITY;
        for (int s = 0; s < d; ++s) {
            double ri = rl[s];
            if (!orc_is_anchor(P, ri, t)) continue;
            double ne = 0.0, num = 0.0;
            for (int l = 0; l < d; ++l) {
                double q = orc_qe(P, p->quantised, ri - rl[l], t);
                ne += q;
                num += rl[l] * q;
            }
            double w = num / ne;
            double lhs = 0.0, rhs = 0.0;
            if (p->literal_ei_test) {
                lhs = fabs(ri - w); rhs = fabs(ri);
            } else {
                for (int l = 0; l < d; ++l) { lhs += fabs(rl[l] - w); rhs += fabs(rl[l]); }
            }
            double score = ne - nz;
            /* Diagnostic only: how far this anchor's pass/fail decision is from
             * flipping under rounding.  The decision is (score >= alpha) and
             * (lhs <= rhs).  Continuous scores are soft, so the slack is the
             * smaller of the two slacks.  Quantised counts are exact integers:
             * only the l1 test (when the count test passes) and the q_e
             * threshold comparisons of the pairs are rounding-sensitive.       */
            double m1 = score - p->alpha;
            double m2 = (rhs - lhs) / (rhs > 0.0 ? rhs : 1.0);
            double slack;
            if (p->quantised) {
                slack = (m1 >= 0.0) ? fabs(m2) : INFINITY;
                for (int l = 0; l < d; ++l) {
                    if (l == s) continue;
                    double g = fabs(orc_log_pbreve(&P->pe, ri - rl[l]) - log(t));
                    if (g < slack) slack = g;
                }
            } else {
                slack = fabs(m1 < m2 ? m1 : m2);
            }
            if (slack < margin) margin = slack;
            if (p->learned) {
                /* learned rule: l1 test, n_e - n_z >= 1.5, logit >= logit(threshold) */
                if (lhs <= rhs && score >= 1.5) {
                    double f[ORC_NFEAT];
                    orc_features(d, rl, w, ne, nz, lhs, rhs, p->sigma_n, t, P->drho, f);
                    double lg = orc_mlp_logit(P->mlp, f);
                    double th = p->mlp_threshold > 0.0 ? p->mlp_threshold : 0.5;
                    double lt = log(th / (1.0 - th));
                    double ml = fabs(lg - lt);
                    if (ml < margin) margin = ml;
                    double m3 = fabs(score - 1.5);
                    if (m3 < margin) margin = m3;
                    if (lg >= lt) { best = s; best_score = lg; best_w = w; }
                }
            } else if (lhs <= rhs && score >= p->alpha) {
                /* rows come in ascending order: the last passing anchor, or
                 * (best_anchor) the first of the largest score */
                if (!p->best_anchor || best < 0 || score > best_score) {
                    best = s; best_score = score; best_w = w;
                }
            }
        }
        if (best >= 0) { xp[j] = xh[j] + best_w; upd++; }
        if (rec) {
            rec[j].passed = (best >= 0);
            rec[j].best_slot = best;
            rec[j].omega = best_w;
            rec[j].score = best_score;
            rec[j].nz = nz;
            rec[j].min_margin = margin;
        }
    }
    free(rl);
    }
    if (nomem) return ORC_ENOMEM;
    int rc = orc_hard_threshold(n, k, xp);
    if (rc) return rc;
    /* r <- y - A x'  (Alg. 2 uses the measured y-hat as y; reading) */
    orc_matvec(n, m, d, rows, xp, rp);
    for (int64_t i = 0; i < m; ++i) rp[i] = yhat[i] - rp[i];
    if (updated) *updated = upd;
    return ORC_OK;
}

/* Stopping level of Section "Stopping conditions": ||r||_1 <= E||eta||_1 =
 * m sigma_n sqrt(2/pi).  reading: noiseless runs stop at
 * ||r||_1 <= noiseless_tol * ||y||_1.                                       */
static double orc_stop_level(int64_t m, const orc_params *p, const double *yhat)
{
    if (p->sigma_n > 0.0) return (double)m * p->sigma_n * sqrt(2.0 / ORC_PI);
    return p->noiseless_tol * l1norm(m, yhat);
}

/* Alg. 2's adaptive_k step, after an accepted round: the sparsity left in
 * the residual, k0 = k - sum_j (1 - p_z(x_hat_j)), floored at m/100; the
 * posteriors are then rebuilt with rho = k0/m.  reading: the printed
 * k - sum_j p_z(x_hat_j) would count nearly every one of the n zero entries
 * (p_z(0) = 1); the sum is of the probability that x_hat_j is nonzero, so
 * k0 is k less the support found so far, as the text of Section "Adaptive
 * k" describes (an update leaves a (k-1)-sparse problem).                  */
double orc_adaptive_k0(int64_t n, int64_t m, int64_t k, const orc_post *P, const double *xhat)
{
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j)
        if (xhat[j] != 0.0) s += 1.0 - exp(orc_log_pbreve(&P->pz, xhat[j]));
    double k0 = (double)k - s;
    double floor_k = floor((double)m / 100.0);
    return (k0 > floor_k) ? k0 : floor_k;
}

/* Alg. 2 (Robust-l0): all four variants of Table "variants".                */
int orc_decode(int64_t n, int64_t m, int d, const int32_t *rows, const double *yhat, int64_t k,
               const orc_params *pin, double *xhat, orc_stats *st,
               orc_round_log *log_out, int log_cap)
{
    if (n < 1 || m < 1 || d < 1 || d > m || k < 1 || k > n || !rows || !yhat || !xhat || !pin)
        return ORC_EINVAL;
    if (pin->adaptive_k && pin->learned) return ORC_EINVAL;
    orc_params p;
    orc_resolve(pin, d, n, m, k, &p);
    orc_post *PP = (orc_post *)malloc(sizeof(orc_post));
    if (!PP) return ORC_ENOMEM;
    int rc = orc_post_init(PP, d, (double)k / (double)m, &p);
    if (rc) { free(PP); return rc; }
    int R = orc_num_rounds(p.c);
    if (p.max_rounds > 0 && p.max_rounds < R) R = p.max_rounds;

    double *rh = (double *)malloc((size_t)m * sizeof(double));
    double *xp = (double *)malloc((size_t)n * sizeof(double));
    double *rp = (double *)malloc((size_t)m * sizeof(double));
    if (!rh || !xp || !rp) { free(rh); free(xp); free(rp); free(PP); return ORC_ENOMEM; }

    for (int64_t j = 0; j < n; ++j) xhat[j] = 0.0;        /* x_hat <- 0 */
    for (int64_t i = 0; i < m; ++i) rh[i] = yhat[i];      /* r_hat <- y */
    double l1h = l1norm(m, rh);
    double stop = orc_stop_level(m, &p, yhat);
    int rounds = 0, acc_rounds = 0;
    double k_prior = (double)k;
    for (int r = 0; r < R; ++r) {
        if (l1h <= stop) break;                           /* converged */
        double t = 1.0 - r * p.c;
        int64_t upd = 0;
        rc = orc_round_step(n, m, d, rows, yhat, k, PP, &p, t, xhat, rh, xp, rp, &upd, NULL);
        if (rc) break;
        double l1 = l1norm(m, rp);
        int accepted = (l1 < l1h);                        /* strict, as printed */
        double k_used = k_prior;
        if (accepted) {
            memcpy(xhat, xp, (size_t)n * sizeof(double));
            memcpy(rh, rp, (size_t)m * sizeof(double));
            l1h = l1;
            acc_rounds++;
            if (p.adaptive_k) {
                k_prior = orc_adaptive_k0(n, m, k, PP, xhat);
                rc = orc_post_init(PP, d, k_prior / (double)m, &p);
                if (rc) break;
            }
        }
        if (log_out && r < log_cap) {
            int64_t supp = 0;
            for (int64_t j = 0; j < n; ++j) supp += (xp[j] != 0.0);
            log_out[r].t = t;
            log_out[r].l1_candidate = l1;
            log_out[r].l1_hat = l1h;
            log_out[r].accepted = accepted;
            log_out[r].updated = upd;
            log_out[r].support = supp;
            log_out[r].k_prior = k_used;
        }
        rounds++;
    }
    int analytic_rounds = 0;
    /* the learned decode is kept when its residual is consistent with the noise,
     * ||r||_1 <= E||eta||_1 + 3 sqrt(Var||eta||_1) (Section "Stopping conditions");
     * otherwise the analytic rule continues from x_hat with a fresh sweep */
    double keep_level = (double)m * p.sigma_n * sqrt(2.0 / ORC_PI) +
                        3.0 * sqrt((double)m * p.sigma_n * p.sigma_n * (1.0 - 2.0 / ORC_PI));
    if (!rc && p.learned && !(l1h <= keep_level)) {
        orc_params p2 = p;
        p2.learned = 0;
        orc_matvec(n, m, d, rows, xhat, rh);
        for (int64_t i = 0; i < m; ++i) rh[i] = yhat[i] - rh[i];
        l1h = l1norm(m, rh);
        for (int r = 0; r < R; ++r) {
            if (l1h <= stop) break;
            double t = 1.0 - r * p2.c;
            int64_t upd = 0;
            rc = orc_round_step(n, m, d, rows, yhat, k, PP, &p2, t, xhat, rh, xp, rp, &upd, NULL);
            if (rc) break;
            double l1 = l1norm(m, rp);
            if (l1 < l1h) {
                memcpy(xhat, xp, (size_t)n * sizeof(double));
                memcpy(rh, rp, (size_t)m * sizeof(double));
                l1h = l1;
                acc_rounds++;
            }
            rounds++;
            analytic_rounds++;
        }
    }
    if (st) {
        int64_t supp = 0;
        for (int64_t j = 0; j < n; ++j) supp += (xhat[j] != 0.0);
        st->rounds = rounds;
        st->analytic_rounds = analytic_rounds;
        st->accepted_rounds = acc_rounds;
        st->converged = (l1h <= stop);
        st->support_size = supp;
        st->final_l1 = l1h;
        st->c = p.c; st->alpha = p.alpha; st->stop_level = stop;
        st->ell = p.ell; st->nrounds_max = R;
    }
    free(rh); free(xp); free(rp); free(PP);
    return rc;
}

/* One round from an injected state, for per-round comparisons: resolves the
 * parameters like orc_decode and runs orc_round_step at t = 1 - r c.        */
int orc_round(int64_t n, int64_t m, int d, const int32_t *rows, const double *yhat, int64_t k,
              const orc_params *pin, int round_index, const double *xh, const double *rh,
              double *xp, double *rp, int64_t *updated, orc_col_rec *rec)
{
    orc_params p;
    orc_resolve(pin, d, n, m, k, &p);
    orc_post *P = (orc_post *)malloc(sizeof(orc_post));
    if (!P) return ORC_ENOMEM;
    int rc = orc_post_init(P, d, (double)k / (double)m, &p);
    if (rc) { free(P); return rc; }
    double t = 1.0 - round_index * p.c;
    rc = orc_round_step(n, m, d, rows, yhat, k, P, &p, t, xh, rh, xp, rp, updated, rec);
    free(P);
    return rc;
}

/* Alg. 1 (Parallel-l0), noiseless.  Equality and zero tests use the absolute
 * tolerance tol.  u_j takes the last passing anchor in loop order, as the
 * printed assignment does; reading: the residual update is r <- y - A x_hat.
 * Returns the number of iterations run.                                     */
int orc_parallel_l0(int64_t n, int64_t m, int d, const int32_t *rows, const double *y,
                    double alpha, double tol, int max_iter, double *xhat, double *xhist)
{
    double *r = (double *)malloc((size_t)m * sizeof(double));
    double *u = (double *)malloc((size_t)n * sizeof(double));
    if (!r || !u) { free(r); free(u); return ORC_ENOMEM; }
    for (int64_t j = 0; j < n; ++j) xhat[j] = 0.0;
    for (int64_t i = 0; i < m; ++i) r[i] = y[i];
    int it = 0;
    for (; it < max_iter; ++it) {
        int any_nonzero = 0;
        for (int64_t i = 0; i < m; ++i) if (fabs(r[i]) > tol) { any_nonzero = 1; break; }
        if (!any_nonzero) break;                                  /* converged */
        int64_t changed = 0;
        for (int64_t j = 0; j < n; ++j) {
            u[j] = 0.0;
            const int32_t *N = rows + j * d;
            for (int s = 0; s < d; ++s) {
                double ri = r[N[s]];
                if (!(fabs(ri) > tol)) continue;
                int ne = 0, nz = 0;
                for (int l = 0; l < d; ++l) {
                    if (fabs(ri - r[N[l]]) <= tol) ne++;
                    if (fabs(r[N[l]]) <= tol) nz++;
                }
                if (ne - nz >= alpha) u[j] = ri;
            }
            if (u[j] != 0.0) changed++;
        }
        if (!changed) break;
        for (int64_t j = 0; j < n; ++j) xhat[j] += u[j];
        orc_matvec(n, m, d, rows, xhat, r);
        for (int64_t i = 0; i < m; ++i) r[i] = y[i] - r[i];
        if (xhist) memcpy(xhist + (int64_t)it * n, xhat, (size_t)n * sizeof(double));
    }
    free(r); free(u);
    return it;
}

/* ------------------------------------------------------------------------ */
/* Exposed evaluations of the posteriors, for pins.                          */
/* which: 0 = p_z, 1 = p_e.  mode: 0 = Eq. (p*_approx) with ell terms + tail, */
/* 1 = the untruncated series of Eq. (p*_gaussian) (ell terms, no tail).      */
/* out[i] = log of the normalised posterior (Eq. (breve)) at w[i];            */
/* raw_out[i] (if non-null) = log of the unnormalised posterior.              */
/* ------------------------------------------------------------------------ */
int orc_log_posterior(int which, int mode, int d, double rho, double sigma_s, double sigma_n,
                      int ell, double tol, int64_t count, const double *w, double *out, double *raw_out)
{
    orc_series S;
    int rc = orc_posterior_series(&S, which, d, rho, sigma_s, sigma_n, ell, mode == 1, tol);
    if (rc) return rc;
    for (int64_t i = 0; i < count; ++i) {
        out[i] = orc_log_pbreve(&S, w[i]);
        if (raw_out) raw_out[i] = S.noiseless ? out[i] : orc_series_logp(&S, w[i]);
    }
    return ORC_OK;
}

/* The tail constants of Eq. (pz_approx)/(pe_approx): R(ell) and v_tail.    */
int orc_tail_constants(int which, int d, double rho, double sigma_s, double sigma_n, int ell,
                       double *R, double *v_tail)
{
    orc_series S;
    int rc = orc_posterior_series(&S, which, d, rho, sigma_s, sigma_n, ell, 0, 1e-5);
    if (rc) return rc;
    *R = S.R;
    *v_tail = S.v_tail;
    return ORC_OK;
}

/* Size of the parameter/stat structures, so the Python side can check its
 * mirror of them.                                                           */
int orc_sizeof(int which)
{
    switch (which) {
    case 0: return (int)sizeof(orc_params);
    case 1: return (int)sizeof(orc_stats);
    case 2: return (int)sizeof(orc_round_log);
    case 3: return (int)sizeof(orc_col_rec);
    default: return -1;
    }
}

/* Learned-scorer pieces exposed for pins: features of one candidate and the
 * network's logit for FP64 parameters (n rows of 16 features).            */
void orc_mlp_logits(const double *W, int64_t nrows, const double *F, double *out)
{
    for (int64_t s = 0; s < nrows; ++s) out[s] = orc_mlp_logit(W, F + s * ORC_NFEAT);
}
