/*
 * rl0.h -- C ABI of the GB300 (sm_103a) Robust-l0 decoding library.
 *
 * Robust-l0 (Mendoza-Smith, Tanner, Wechsung, arXiv 1704.09012, Algorithm 2)
 * recovers a k-sparse x in R^n from a noisy expander sketch y_hat = A x + eta,
 * where A in {0,1}^{m x n} has exactly d ones per column (Def. 1.1, expander
 * matrices) and the instance follows the generating model GM(n,m,k,d,mu,nu)
 * (Def. "Generating model") with mu = N(0, sigma_s^2) and nu = N(0, sigma_n^2).
 *
 * Conventions shared by every entry point:
 *  - Return value: RL0_OK (0) on success, a negative RL0_ERR_* code otherwise;
 *    rl0_strerror() gives a message.  Failing to converge is not an error: it
 *    is reported in rl0_stats.converged.
 *  - "device" pointers are CUDA device memory of the current device, owned by
 *    the caller; "host" pointers are ordinary (pageable or pinned) host memory.
 *  - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is ordered on that stream.  Calls that return
 *    statistics (rl0_decode*, rl0_round_step) synchronise the stream before
 *    returning; the others only enqueue work.
 *  - Element types: rows int32, values float (IEEE binary32), sizes int64.
 *  - An rl0_expander owns its device copies of A and a decode workspace.  It
 *    serves one decode at a time: calls that use the same expander must be
 *    ordered (same stream, or synchronised), or they race on the workspace.
 *  - No entry point falls back to the CPU: without a usable CUDA device every
 *    call that needs one returns RL0_ERR_CUDA.
 */
#ifndef RL0_H
#define RL0_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RL0_OK                 0
#define RL0_ERR_INVALID_ARG   -1   /* a size, pointer or parameter is out of range   */
#define RL0_ERR_CUDA          -2   /* a CUDA runtime call failed                      */
#define RL0_ERR_ALLOC         -3   /* device or host allocation failed                */
#define RL0_ERR_TIMEOUT       -4   /* a bounded device-side wait gave up              */
#define RL0_ERR_UNSUPPORTED   -5   /* valid request this build does not implement    */
#define RL0_ERR_INVALID_A     -6   /* rows out of range, duplicated or unsorted       */
#define RL0_ERR_INVALID_Y     -7   /* y_hat holds NaN or Inf                          */
#define RL0_ERR_TOO_LARGE     -8   /* instance exceeds rl0_decode_static's fixed workspace */

/* Opaque handle: device copy of A as column-major row lists (column j owns
 * rows[j*d .. j*d+d-1], ascending), its transpose in CSR form, and the decode
 * workspace sized for (n, m, d). */
typedef struct rl0_expander rl0_expander;

/* Decoder parameters (Algorithm 2's inputs besides A, y_hat and k).
 * Zero in a field selects the documented default. */
typedef struct {
    double sigma_s;        /* std of the nonzeros of x (mu); 0 = 1.0                          */
    double sigma_n;        /* std of the noise (nu); 0 = noiseless                            */
    int    quantised;      /* Table "scores": 1 = quantised scores, 0 = continuous            */
    int    adaptive_k;     /* the adaptive_k flag of Algorithm 2 (analytic scorer only)      */
    double c;              /* sweep step of t; 0 = Eqs. (finetune_c_quant)/(finetune_c_cont)  */
    double alpha;          /* consensus threshold on n_e - n_z; 0 = floor(d/2)+1 (quantised)  */
                           /* or d/2 (continuous)                                            */
    int    ell;            /* explicit terms of the posterior series, Eq. (pz_approx); 0 = 4  */
    int    scorer;         /* 0 = analytic scores (Algorithm 2), 1 = learned column scorer    */
    const void *mlp;       /* scorer = 1: device pointer to an rl0_mlp_weights block          */
    double mlp_threshold;  /* scorer = 1: accept a column when its score >= this; 0 = 0.5     */
    int    max_rounds;     /* cap on the number of rounds; 0 = every round with t > 0         */
    double noiseless_tol;  /* sigma_n = 0: |a - b| <= tol counts as equal; 0 = 1e-5           */
    int    profile;        /* 1: time each kernel group with CUDA events captured into the    */
                           /* round graph and report it in rl0_stats.ms_* (adds event nodes)  */
    int    anchor_rule;    /* the update a column takes when several of its anchors pass      */
                           /* Algorithm 2's test (the paper adds one per anchor; one update   */
                           /* per column is kept): 0 = the last passing anchor in row order   */
                           /* (Alg. 1's overwrite), 1 = the one with the largest n_e - n_z,   */
                           /* ties to the lower row.  1 is for comparing the two readings:    */
                           /* the batched decoder, the learned scorer and rl0_decode_static   */
                           /* return RL0_ERR_UNSUPPORTED with it                              */
} rl0_params;

/* Per-decode statistics (host structure filled by the library). */
typedef struct {
    int     rounds;            /* rounds of the sweep, including t = 1 (see skipped_rounds)  */
    int     accepted_rounds;   /* rounds whose candidate passed ||r||_1 < ||r_hat||_1        */
    int     converged;         /* 1 if ||r_hat||_1 <= m sigma_n sqrt(2/pi) at exit           */
    int     status;            /* RL0_OK, or the device-side error of this decode            */
    int64_t support_size;      /* |supp x_hat|                                               */
    double  final_l1;          /* ||y_hat - A x_hat||_1 at exit: rows without FP32 rounding  */
    float   ms;                /* device time of the decode (CUDA events), milliseconds      */
    int     hk_rounds;         /* rounds in which H_k had to drop entries                    */
    int     fallback_rounds;   /* rounds whose residual took the full CSR rebuild            */
    /* profile = 1 only: summed device time of each kernel group over the rounds the decode
     * ran (event nodes around the groups, so each interval includes the launch gap) */
    float   ms_score;          /* column scoring, with H_k in the kernel's last CTA          */
    float   ms_hk;             /* from the scoring kernel's end to the scatter's start       */
    float   ms_rebuild;        /* scatter + residual rebuild, with accept/undo in the        */
                               /* rebuild's last CTA                                         */
    float   ms_accept;         /* from the rebuild's end to the next round's start           */
    int     launches;          /* kernels launched by the decode (any mode)                  */
    int     analytic_rounds;   /* scorer = 1: rounds of the analytic continuation (0 if the  */
                               /* learned decode converged on its own)                       */
    int     skipped_rounds;    /* rounds counted in `rounds` that launched no kernels: with   */
                               /* sigma_n > 0 the round at t = 1 provably changes nothing    */
                               /* (its anchor test needs p_z = 0) and is only recorded       */
} rl0_stats;

/* Def. "Generating model", item 1: draw A with each column's support uniform
 * over the d-subsets of [m].  Counter-based: column j's rows come from
 * Philox4x32-10 (key = seed, counter = (block, j_lo, j_hi, 0x41)), words
 * mapped to [0, m) by Lemire's unbiased multiply-shift, duplicates skipped,
 * then sorted.  Requires 1 <= d <= 32, d <= m < 2^31, 1 <= n, n*d < 2^31.
 * On success *out owns new device memory; free it with rl0_free_expander. */
int rl0_make_expander(int64_t n, int64_t m, int d, uint64_t seed,
                      void *cuda_stream, rl0_expander **out);

/* Same, from caller-supplied column-major rows (device, n*d int32, each column
 * ascending and distinct, values in [0, m)).  The rows are copied and
 * validated on the device; bad rows give RL0_ERR_INVALID_A. */
int rl0_expander_from_rows(int64_t n, int64_t m, int d, const int32_t *rows_dev,
                           void *cuda_stream, rl0_expander **out);

/* Copy the expander's column-major rows (n*d int32) into rows_dev. */
int rl0_expander_rows(const rl0_expander *A, int32_t *rows_dev, void *cuda_stream);

/* Sizes of an expander (any out pointer may be NULL). */
int rl0_expander_shape(const rl0_expander *A, int64_t *n, int64_t *m, int *d);

void rl0_free_expander(rl0_expander *A);

/* Def. "Generating model", items 4 and 6: y_hat = A x + eta.
 * x_dev: device float[n]; y_dev: device float[m] (output, overwritten).
 * y_i sums x over the row's columns in ascending column order in FP64 and adds
 * eta_i = sigma_n * z_i, z_i a Box-Muller deviate of one Philox4x32-10 block
 * (key = noise_seed, counter = (0, i_lo, i_hi, 0x4E)); the sum is rounded to
 * FP32 once.  sigma_n = 0 gives the noiseless sketch. */
int rl0_sketch(const rl0_expander *A, const float *x_dev, double sigma_n, uint64_t noise_seed,
               float *y_dev, void *cuda_stream);

/* Algorithm 2 (Robust-l0) on one instance: the four variants of Table
 * "variants" (params->quantised, params->adaptive_k).
 * y_dev: device float[m]; xhat_dev: device float[n] (output, overwritten).
 * k in [1, n].  params may be NULL (all defaults with sigma_n = 0).
 * stats (host, may be NULL) is filled after the stream is synchronised.
 * adaptive_k (Section "Adaptive k"): after every accepted round the posteriors
 * are rebuilt for the sparsity left, k0 = k - sum_j (1 - p_z(x_hat_j)) floored
 * at m/100 (the sum in FP64 over the support in ascending j); H_k keeps k.
 * The rounds then run one launch group at a time with the host in the loop
 * (no captured graph).  With scorer = 1 it returns RL0_ERR_UNSUPPORTED. */
int rl0_decode(const rl0_expander *A, const float *y_dev, int64_t k, const rl0_params *params,
               float *xhat_dev, rl0_stats *stats, void *cuda_stream);

/* Algorithm 1 (Parallel-l0) on one instance of the noiseless model y = A x:
 * from x_hat = 0, every iteration gives each column j the last anchor r_i != 0
 * in row order with n_e - n_z >= alpha, n_e = #{l in N(j): r_l = r_i},
 * n_z = #{l in N(j): r_l = 0}; then x_hat += u and r = y - A x_hat.  Equality
 * and zero are |.| <= tol on the FP32 residuals.  It stops when an iteration
 * changes nothing; stats.converged = 1 when then every |r_i| <= tol, and
 * stats.accepted_rounds counts the iterations that changed x_hat.
 * It runs the round kernels of rl0_decode with the 0/1 scores, no H_k and no
 * acceptance test.  alpha: 0 gives floor(d/2) + 1; alpha < d/2 returns
 * RL0_ERR_UNSUPPORTED (the kernels apply the l1 test of Alg. 2, which
 * n_e - n_z >= alpha implies when alpha >= d/2).  tol: 0 gives 1e-5 (FP32
 * residuals carry rounding of about 1e-7 |y|).  max_iter: 0 gives 100, at
 * most 1024.  y_dev: device float[m]; xhat_dev: device float[n] (output). */
int rl0_parallel_l0(const rl0_expander *A, const float *y_dev, double alpha, double tol, int max_iter,
                    float *xhat_dev, rl0_stats *stats, void *cuda_stream);

/* Monte-Carlo check of the posteriors (Section "Comparison with empirical
 * probabilities", Fig. 3) with the decoder's own FP32 series for sparsity k
 * (rho = k/m), sigma_s, sigma_n > 0 and ell = 4.  y0_dev: the noiseless sketch
 * A x (device float[m]); yhat_dev: the noisy one, A x + eta.  nbins <= 1024.
 *  - rows: for every i with |yhat_i| < wz_max, bin b = floor(|yhat_i| nbins / wz_max);
 *    hz[3b] += 1, hz[3b+1] += [y0_i == 0], hz[3b+2] += round(2^32 p_breve_z(yhat_i));
 *  - row pairs: for every column j and rows s < l of N(j) with
 *    |D| = |yhat_s - yhat_l| < we_max, the same into he with [y0_s == y0_l] and
 *    p_breve_e(D).
 * hz_dev, he_dev: device uint64[3 nbins], accumulated into (not cleared), so
 * several instances add up.  The counts are exact integers. */
int rl0_posterior_mc(const rl0_expander *A, const float *y0_dev, const float *yhat_dev, int64_t k,
                     double sigma_s, double sigma_n, int nbins, double wz_max, double we_max,
                     uint64_t *hz_dev, uint64_t *he_dev, void *cuda_stream);

/* rl0_decode with host buffers: copies y_host (float[m]) to the device and
 * x_hat back to xhat_host (float[n]) on the stream, through device buffers the
 * expander holds (so calls on one expander must not overlap, as for every
 * entry point).  Pinned host memory gives asynchronous copies; pageable memory
 * works too. */
int rl0_decode_host(const rl0_expander *A, const float *y_host, int64_t k,
                    const rl0_params *params, float *xhat_host, rl0_stats *stats,
                    void *cuda_stream);

/* One round of Algorithm 2 from an injected state, for tests and tools:
 * reads x_hat (xhat_dev, float[n]) and r_hat (rhat_dev, float[m]) at sweep
 * value t = 1 - round_index * c, writes x' = H_k(x_hat + updates) to xp_dev
 * (float[n]) and r = y_hat - A x' to rp_dev (float[m]).  passed_dev (int32[n],
 * may be NULL) receives 1 for every column that received an update.  l1_out
 * (host, may be NULL) receives ||r||_1 in FP64. */
int rl0_round_step(const rl0_expander *A, const float *y_dev, int64_t k, const rl0_params *params,
                   int round_index, const float *xhat_dev, const float *rhat_dev,
                   float *xp_dev, float *rp_dev, int32_t *passed_dev, double *l1_out,
                   void *cuda_stream);

/* Algorithm 2 on `count` independent instances in one persistent launch
 * (instances may differ in n, m, k, d <= 32 and parameters).  A, y_dev,
 * xhat_dev and k point to `count` entries each (host arrays of device
 * pointers); params points to `count` entries or is NULL; stats (host) to
 * `count` entries or NULL.  Each instance's result equals what rl0_decode
 * gives for it alone.  The learned scorer and adaptive_k (a host step after
 * every accepted round) return RL0_ERR_UNSUPPORTED. */
int rl0_decode_batched(int count, const rl0_expander *const *A, const float *const *y_dev,
                       const int64_t *k, const rl0_params *params, float *const *xhat_dev,
                       rl0_stats *stats, void *cuda_stream);

/* rl0_decode for callers that cannot allocate memory.  (The paper has no
 * counterpart: this is a deployment variant of Algorithm 2's loop.)
 *
 * Who needs it: code that must not call cudaMalloc or any other allocator
 * while it runs -- a real-time loop whose memory budget is fixed at
 * start-up, or a host application whose own allocator already owns all free
 * device memory, where a new allocation fails or evicts someone else's data.
 * rl0_decode does not allocate per call either, but its first call for a
 * given round count builds and instantiates a graph, which allocates.
 *
 * This entry point allocates nothing: its scratch is one file-scope device
 * array of about 6 MB compiled into the library, held by every GPU that
 * loads the library until the process exits.  The caller passes y_dev and
 * xhat_dev as for rl0_decode and gets the same result (with scorer = 1 that
 * includes the analytic continuation described below); the kernels are
 * launched directly on the stream, and the stream is synchronised before the
 * call returns.  Limits: n <= 65536, m <= 32768 (larger instances return
 * RL0_ERR_TOO_LARGE); adaptive_k returns RL0_ERR_UNSUPPORTED; stats.ms and
 * the profile fields stay 0; the decode keeps no round log (rl0_decode_log
 * then reports 0 rounds).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  Every call reuses the
 * same array and clears the parts that must start at zero.  Calls that
 * overlap on the GPU (from other streams or host threads) race on the array,
 * and calls on one expander also share its pinned host staging block with
 * rl0_decode and rl0_round_step: serialise them. */
int rl0_decode_static(const rl0_expander *A, const float *y_dev, int64_t k,
                      const rl0_params *params, float *xhat_dev, rl0_stats *stats,
                      void *cuda_stream);

/* Failure-detection test hook.  The column kernel waits for the bulk copy of
 * the residual codes into shared memory with a bounded poll loop (2^22 polls
 * of mbarrier.try_wait).  polls >= 0 makes that first wait on this expander
 * give up after `polls` polls (0: at once); the kernel then records
 * RL0_ERR_TIMEOUT, waits for its copies in flight with the built-in limit,
 * scores nothing and returns, and rl0_decode returns RL0_ERR_TIMEOUT with the
 * device still usable.  polls < 0 restores the built-in limit.  Affects
 * rl0_decode calls made after it on this expander. */
int rl0_expander_set_wait_polls(rl0_expander *A, int64_t polls);

/* Per-round record of the last rl0_decode on this expander (host copy kept by
 * the library).  Writes min(cap, rounds) records and returns the number of
 * rounds of that decode. */
typedef struct {
    double t;              /* sweep value of the round                         */
    double l1_candidate;   /* ||y_hat - A x'||_1 of the round's candidate       */
    double l1_hat;         /* ||r_hat||_1 after the round                       */
    int    accepted;       /* candidate kept (||r||_1 < ||r_hat||_1)            */
    int    updated;        /* columns that received an update                   */
    int    support;        /* |supp x_hat| after the round                       */
    int    hk_dropped;     /* entries H_k zeroed                                 */
    double k_prior;        /* the sparsity k of the posteriors the round used
                              (k, or the adaptive_k prior k0)                    */
} rl0_round_record;

int rl0_decode_log(const rl0_expander *A, rl0_round_record *out, int cap);

/* ---- Learned column scorer (an addition to the paper's method) ------------------------
 * A 16 -> 32 -> 32 -> 1 MLP with ReLU hidden layers whose logit replaces Algorithm 2's
 * consensus test n_e - n_z >= alpha when rl0_params.scorer = 1: an anchor passes when
 * the l1 test holds, n_e - n_z >= 1.5 and logit >= log(mlp_threshold / (1 - mlp_threshold));
 * as with the analytic rule, the last passing anchor in row order gives the update.
 * Features, in this order: the 7 smallest |r_l - w| / sigma_n
 * (clipped at 8, padded with 8), n_e/d, n_z/d, log(1 + |w|/sigma_n)/5, the column's
 * relative l1 gain (clipped to [-1, 1]), t, d k/m, (n_e - n_z)/d, 0, 0.  If the learned
 * decode ends with ||r||_1 > E||eta||_1 + 3 sqrt(Var||eta||_1), the analytic decode
 * continues from its x_hat.
 * Parameters: RL0_MLP_PARAMS (= 1633) values, W1 (16x32, input-major), b1 (32),
 * W2 (32x32), b2 (32), w3 (32), b3; FP32 for training, BF16 for decoding. */
#define RL0_MLP_PARAMS 1633

/* Features of every learned-scorer candidate of one round from an injected state
 * (x_hat, r_hat: device, n and m floats) at t = 1 - round_index c: feat_dev
 * (cap x 16 floats), meta_dev (cap x 4 int32: column, slot, passes the analytic test,
 * passes the l1 test), omega_dev (cap floats: the consensus value w), in ascending
 * (column, slot) order.  *count_out (host) receives the number of candidates (only
 * min(count, cap) are written).
 * Requires sigma_n > 0 and d <= 16. */
int rl0_candidate_features(const rl0_expander *A, const float *y_dev, int64_t k,
                           const rl0_params *params, int round_index, const float *xhat_dev,
                           const float *rhat_dev, float *feat_dev, int32_t *meta_dev,
                           float *omega_dev, int cap, int *count_out, void *cuda_stream);

/* Training data for the scorer: runs Algorithm 2 with the analytic rule (params->scorer
 * must be 0, adaptive_k 0; sigma_n > 0) from x_hat = 0, r_hat = y, for rounds
 * 1 .. max_rounds - 1, each as rl0_round_step computes it, keeping the round's candidate
 * when ||r||_1 < ||r_hat||_1 and stopping once ||r_hat||_1 <= m sigma_n sqrt(2/pi) (the
 * expected l1 norm of the noise, Section 'Stopping conditions').  Before each round the
 * features of every candidate of that round (as rl0_candidate_features gives them, in
 * ascending (column, slot) order) are appended to feat_dev (rows of 16 floats), with
 * label_dev = 1 when x_hat_j + w lies within tol_sigma sigma_n of x_true_j != 0
 * (xtrue_dev: device, n floats), else 0.  At most cap rows are written (feat_dev and
 * label_dev may be NULL when cap = 0); *count_out (host) receives the number of
 * candidates met, which may exceed cap; *rounds_out (host, may be NULL) the rounds run.
 * Allocates its scratch per call; synchronises the stream.  2 <= max_rounds <= 1024,
 * tol_sigma > 0. */
int rl0_scorer_log(const rl0_expander *A, const float *y_dev, int64_t k, const rl0_params *params,
                   const float *xtrue_dev, float tol_sigma, int max_rounds, float *feat_dev,
                   float *label_dev, int64_t cap, int64_t *count_out, int *rounds_out,
                   void *cuda_stream);

/* FP32 parameters, He-normal weights and zero biases from a counter-based hash of seed. */
int rl0_mlp_init(uint64_t seed, float *w_dev, void *cuda_stream);

/* Mean binary cross-entropy (logits vs labels in {0,1}) of N feature rows and its
 * gradient w.r.t. the FP32 parameters; deterministic (fixed summation order).
 * loss_host may be NULL.  Synchronises the stream. */
int rl0_mlp_grad(const float *w_dev, const float *feat_dev, const float *label_dev, int64_t N,
                 float *grad_dev, double *loss_host, void *cuda_stream);

/* Adam on minibatches of `batch` consecutive rows, `epochs` passes, learning rate lr;
 * updates w_dev in place, writes the BF16 copy to wbf16_dev (may be NULL) and the final
 * full-set loss to loss_host (may be NULL).  Synchronises the stream. */
int rl0_mlp_train(float *w_dev, const float *feat_dev, const float *label_dev, int64_t N,
                  int epochs, int batch, float lr, void *wbf16_dev, double *loss_host,
                  void *cuda_stream);

/* BF16 copy (round to nearest even) of FP32 parameters, for rl0_params.mlp. */
int rl0_mlp_export(const float *w_dev, void *wbf16_dev, void *cuda_stream);

/* Logits of N feature rows with BF16 parameters (the decoder's arithmetic). */
int rl0_mlp_forward(const void *wbf16_dev, const float *feat_dev, int64_t N, float *logit_dev,
                    void *cuda_stream);

/* RL0_MLP_PARAMS, for bindings. */
int rl0_mlp_params(void);

const char *rl0_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* RL0_H */
