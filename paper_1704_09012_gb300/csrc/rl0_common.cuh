// rl0_common.cuh -- internal declarations shared by the CUDA translation units of
// the Robust-l0 library (arXiv 1704.09012, Algorithm 2).  Not part of the ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rl0.h"

#define RL0_MAXQ 12          // explicit series terms + tail (ell <= 10)
#define RL0_BUCKET 8         // contributors per row held by the sparse rebuild
#define RL0_ROWS_CHUNK 256   // rows per l1 partial, one row per thread (fixed: defines the summation order)
#define RL0_MAX_D 32

// 16-bit residual codes read by the column kernel's bound (rl0_device.cuh):
// r rounded toward zero to FP16, magnitude clamped to the largest finite code.
// The p_z lower-bound table has one entry per 2^RL0_PZ_SHIFT magnitude codes.
#define RL0_PZ_SHIFT 5
#define RL0_PZ_BINS (0x7c00 >> RL0_PZ_SHIFT)

// Status codes a kernel can leave in DecodeState::status.
#define RL0_DEV_OK 0
#define RL0_DEV_TIMEOUT 1

// 1/p_breve(w) = sum_q a[q] exp(b[q] w^2), q = 0..nq-1 (Eq. (pz_approx) or
// (pe_approx) divided through by the noise density, Eq. (breve) normalisation);
// beyond |w| > cut the posterior is below 2^-40 and is taken as 0.
// When use_poly is set, the q >= 1 terms are evaluated in factored form:
//   sum_{q>=1} a_q exp(b_q u) = exp(b1 u) G(u),  u = w^2,
// with G(u) = sum_{q>=1} a_q exp((b_q - b1) u) a slowly varying function on
// [0, cut^2] held as a Chebyshev series (t = u * inv_u2 - 1), so one exp per
// evaluation replaces one per term.
#define RL0_MAXPOLY 16
struct Series {
    int nq;
    float a[RL0_MAXQ];
    float b[RL0_MAXQ];
    float cut;
    int use_poly;
    int npoly;
    float b1;
    float inv_u2;
    float poly[RL0_MAXPOLY];
};

// Per-round thresholds on magnitudes, FP64-derived and rounded outward so that
// comparing an FP32 value with them is the exact test on that value:
//   anchor  (1 - p_z(r) >= t)   <=> |r| >= ta
//   q_z = 1 (quantised/noiseless)<=> |r| <= tz
//   q_e = 1 (quantised/noiseless)<=> |D| <= te
struct RoundThr {
    float ta, tz, te, t;
};

struct RoundLog {
    double l1_candidate;
    double l1_hat;
    int accepted;
    int updated;
    int support;
    int hk_dropped;
};

// Mutable state of one decode, in device memory.
struct DecodeState {
    int done;
    int status;
    int round;
    int cur;                  // which rz buffer holds r_hat
    unsigned list_count;      // support + columns that became nonzero this round
    unsigned upd_count;       // updates this round (undo log length); with list_count one 8-byte
                              // word, so that a CTA takes slots in both with one atomic
    unsigned shat_count;      // |supp x_hat|: list[0 .. shat_count) is the support
    unsigned drop_count;      // entries H_k zeroed this round (undo log length)
    int overflow;             // a row's fresh bucket received more than RL0_BUCKET columns
    unsigned bflags;          // bit b: support bucket B[b] incomplete (a row with > RL0_BUCKET columns)
    int converged;            // ||r_hat||_1 <= stop level
    unsigned nnz;             // |supp x_hat|
    int nnz_delta;            // change of the nonzero count made by this round's updates
    unsigned zeroed;          // updates that made an entry exactly zero this round
    unsigned iters;           // accept invocations (bounds the graph's while loop)
    unsigned col_done;        // CTAs of the column kernel finished (last one applies H_k)
    unsigned rb_done;         // CTAs of the rebuild finished (last one accepts or undoes)
    unsigned big_hat;         // Alg. 1 mode: rows of r_hat with |r_i| > conv_tol
    unsigned big_cand;        // Alg. 1 mode: the same count for the candidate r
    int skipped;              // rounds recorded without running their kernels (the t = 1 round)
    int rounds_run;
    int accepted_rounds;
    int hk_rounds;
    int fallback_rounds;
    unsigned long long tick;  // resident-code column kernel: CTAs done (bits 48..63) and their
                              // changes of the nonzero count, each biased by 2^31 (bits 0..47)
    double l1_hat;
    double l1_new;
    double final_l1;          // ||y_hat - A x_hat||_1 in FP64 (epilogue)
};

// Per-call data the round kernels read from device memory.  The graph that
// replays the round loop captures only the address of this block, so one
// captured graph serves every call on the same expander.
struct DecodeCtx {
    const float *y;           // y_hat, float[m]
    float *x;                 // the working x (x_hat, updated in place), float[n]
    long long k;
    float alpha;
    int nrounds;
    int quantised;
    int indicator;            // quantised or noiseless: 0/1 scores
    double stop_level;        // absolute stop level (sigma_n > 0)
    double stop_rel;          // > 0: stop level = stop_rel * ||y_hat||_1 (noiseless)
    Series pz, pe;
    int scorer;               // 0 analytic, 1 learned
    const void *mlp;          // BF16 parameters of the learned scorer
    float mlp_threshold;
    float logit_thr;          // learned: accept when the logit >= log(thr / (1 - thr))
    float learned_need;       // learned: candidates need n_e - n_z bound >= this
    float inv_sn;             // 1 / sigma_n (0 when noiseless)
    float drho;               // d k / m
    float pe_b1, pe_c1;       // q_e(D) <= 1 / (1 + c1 (u + u^2/2)), u = b1 D^2 (fast-path bound)
    int32_t *passed;          // optional per-column pass flags (round_step)
    int want_log;
    int no_accept;            // round_step: stop after the rebuild (no accept, no undo)
    int always_accept;        // Alg. 1 (Parallel-l0): keep every iteration, stop when one changes nothing
    int skip_t1;              // sigma_n > 0: the round at t = 1 provably changes nothing; record it only
    float conv_tol;           // Alg. 1: converged when every |r_i| <= conv_tol (0: Alg. 2's stop level)
    int wait_test;            // 0: the column kernel's first bounded wait makes its built-in number
    unsigned wait_polls;      // of polls; 1: it makes wait_polls (rl0_expander_set_wait_polls)
    int anchor_rule;          // 0: a column takes its last passing anchor; 1: the largest n_e - n_z
};

struct UndoEntry {
    int j;
    float old;
};

// Device workspace owned by an expander.
struct Workspace {
    float2 *rz[2];            // (r_i, p_z(r_i)) for r_hat and the candidate r
    unsigned short *code[2];  // 16-bit codes of the same residuals, padded to a multiple of 8 rows
    float *pzlb;              // p_z lower bound per code bin, float[RL0_PZ_BINS]
    int *res_list;            // survivors of the column kernel's code bound, n entries of rl0_res_dmax + 2 ints
    int *list;                // support + new nonzeros, capacity n
    int *list_tmp;            // one int: a counter
    UndoEntry *ulog;          // updates of this round, capacity n
    UndoEntry *dlog;          // H_k drops of this round, capacity n
    int *bcnt;                // per-row fresh-bucket counts, int[m] (kept zero between rounds)
    int *bkt;                 // per-row fresh-bucket columns, int[m * RL0_BUCKET]
    int *sbcnt[2];            // per-row support-bucket counts B[0], B[1], int[m] each
    int *sbkt[2];             // per-row support-bucket columns, int[m * RL0_BUCKET] each
    double *l1part;           // per-chunk l1 partials
    unsigned long long *hk_scratch;  // H_k candidate keys, capacity n
    DecodeState *st;
    DecodeCtx *ctx;
    RoundThr *thr;            // per-round thresholds, capacity RL0_MAX_ROUNDS
    RoundLog *rlog;           // per-round log, capacity RL0_MAX_ROUNDS
    double *final_part;       // FP64 residual-norm partials, one set per rz buffer (2 x chunks)
    float *host_y, *host_x;   // rl0_decode_host's device copies of y_hat (m) and x_hat (n)
    int max_rounds;
};

struct rl0_expander {
    int64_t n, m;
    int d;
    int device;
    int32_t *rows_cm;         // column-major rows, int[n*d]
    int32_t *rows_sm;         // slot-major rows: rows_sm[s*n + j], int[d*n]
    int32_t *rowptr;          // CSR of A^T: int[m+1]
    int32_t *colidx;          // CSR of A^T: int[n*d], ascending within a row
    Workspace ws;
    void *graph_cache;        // captured round loops
    void *host_pinned;        // pinned staging (ctx, thresholds, stats)
    size_t host_pinned_bytes;
    int *dev_flag;            // validation flag
    int last_log_rounds;      // rounds recorded by the last rl0_decode
    void *events;             // CUDA events used to time decodes
    void *table_cache;        // host tables of the last parameter set
    int wait_test;            // rl0_expander_set_wait_polls: override the first bounded wait
    unsigned wait_polls;
};

#define RL0_MAX_ROUNDS 1024

// Size limits of rl0_decode_static (its workspace is a fixed array).
#define RL0_STATIC_MAX_N 65536
#define RL0_STATIC_MAX_M 32768

// ---- host tables (rl0_tables.cu) ------------------------------------------
namespace rl0 {
struct HostSeries {
    int nq;
    double a[RL0_MAXQ], b[RL0_MAXQ];
};
struct Resolved {
    rl0_params p;
    int nrounds;
    int indicator;
    double stop_level, stop_rel;
    double keep_level;        // learned decodes end without the analytic continuation below this
};
HostSeries make_series(double lam, double s2, double vn, int ell);
double series_F(const HostSeries &H, double w);
float series_threshold_up(const HostSeries &H, double T);
float series_threshold_down(const HostSeries &H, double T);
Series to_device_series(const HostSeries &H);
double default_c(int quantised, double delta, double rho);
int resolve(int64_t n, int64_t m, int d, int64_t k, const rl0_params *in, Resolved *R);
// k_prior > 0: the posteriors use sparsity k_prior instead of k (adaptive_k)
void fill_tables(int64_t m, int d, int64_t k, const Resolved &R, DecodeCtx *ctx, RoundThr *thr, int nthr,
                 double k_prior = 0.0);
void pz_lower_bounds(int64_t m, int d, int64_t k, const Resolved &R, float *out, double k_prior = 0.0);
double adaptive_k0(int64_t m, int d, int64_t k, const Resolved &R, double k_prior, const float *vals, int64_t count);
}  // namespace rl0

// ---- helpers shared by translation units -------------------------------
int rl0_set_device_of(const rl0_expander *A);
int rl0_cuda_err(cudaError_t e);

// Expander construction pieces (rl0_expander.cu).
int rl0_expander_finish(rl0_expander *A, cudaStream_t s);
void rl0_expander_release(rl0_expander *A);

// Decode workspace (rl0_decode.cu).
int rl0_workspace_alloc(rl0_expander *A);
void rl0_workspace_free(rl0_expander *A);
// Host tables of (k, R) for A, cached per expander (rl0_decode.cu).
void rl0_cached_tables(rl0_expander *A, int64_t k, const rl0::Resolved &R, DecodeCtx *ctx, RoundThr *thr);
bool rl0_tables_cached(const rl0_expander *A, int64_t k, const rl0::Resolved &R);

static inline unsigned rl0_div_up(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Rows of a residual-code buffer (a multiple of 8, so that its bytes are a
// multiple of 16 and one bulk copy moves it).
__host__ __device__ static inline long long rl0_code_rows(long long m) { return (m + 7) / 8 * 8; }
