// rl0_decode.cu -- the synchronous round loop of Robust-l0 (arXiv 1704.09012,
// Algorithm 2) on one instance: per-round thresholds and posterior
// coefficients (host, FP64), the round kernels, and the captured CUDA graph
// that replays the loop.
//
// One round, as two or three kernels on one stream:
//   column score  every column j bounds, then scores, its anchors (Table
//                 "scores", Eqs. (ne_nz_1), (ne_nz_2)), applies the last
//                 passing update to x in place and logs it for undo
//                 (k_column_score_res in rl0_column_res.cu: residual codes in
//                 shared memory; k_column_score below: L2 gathers).  The
//                 launch's last CTA applies H_k (radix select on the 63-bit
//                 key (|x_j| bits, ~j): ties go to the smaller j);
//   scatter       the support's (row, column) pairs into per-row buckets
//                 (the resident-code column kernel does this itself);
//   rebuild       r_i = y_i - sum of x_j over row i in ascending j, FP32 (and
//                 the same sum in FP32 pairs, about 48 bits, for the final
//                 residual check), with p_z(r_i), the residual code, and l1
//                 partials over fixed 256-row chunks (a CSR(A^T) pass replaces
//                 it when a bucket overflows).  The launch's last CTA accepts the round if
//                 ||r||_1 < ||r_hat||_1 or undoes it, advances t and clears
//                 the graph's loop condition when the decode is done.
// No float atomics anywhere: every sum has a fixed order, so results do not
// depend on the launch configuration or on scheduling.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "rl0_common.cuh"
#include "rl0_device.cuh"
#include "rl0_mma.cuh"
#include "rl0_round.cuh"
#include <cuda_bf16.h>

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return rl0_cuda_err(e_);   \
    } while (0)


// r source -> rz[dst] = (r, p_z(r)), the l1 partial (FP32 pairs, stored in FP64) of each RL0_ROWS_CHUNK-row
// chunk (one row per thread, blockDim = RL0_ROWS_CHUNK); zero_x: the grid also
// zeroes the working x (a decode from x_hat = 0).
__global__ void __launch_bounds__(RL0_ROWS_CHUNK) k_rows_from(KArgs a, const float *src_override, int dst, int zero_x)
{
    __shared__ DF sh[RL0_ROWS_CHUNK];
    const DecodeCtx *ctx = a.ctx;
    if (zero_x) {
        float *x = ctx->x;
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += gridDim.x * blockDim.x) x[j] = 0.0f;
    }
    const float *src = src_override ? src_override : ctx->y;
    float2 *rz = dst ? a.rz1 : a.rz0;
    DF l1{0.0f, 0.0f};
    const int i = blockIdx.x * RL0_ROWS_CHUNK + threadIdx.x;
    if (i < a.m) {
        // a decode starts with empty row buckets (x_hat = 0, or an injected
        // x_hat whose support k_bucket_support adds next)
        a.sbcnt0[i] = 0;
        a.sbcnt1[i] = 0;
        a.bcnt[i] = 0;
        const float r = src[i];
        if (!isfinite(r)) atomicExch(&a.st->status, (int)RL0_ERR_INVALID_Y);
        const float z = ctx->indicator ? 0.0f : series_eval(ctx->pz, r);
        rz[i] = make_float2(r, z);
        if (a.res_ok) (dst ? a.code1 : a.code0)[i] = residual_code(r);
        l1 = DF{fabsf(r), 0.0f};
    }
    const double s = block_sum_df(l1, sh);
    if (threadIdx.x == 0) {
        a.l1part[blockIdx.x] = s;
        // r = y_hat with x_hat = 0: the final residual-norm partial is the same sum
        if (!src_override) a.final_part[(size_t)dst * a.nchunks + blockIdx.x] = s;
    }
    if (ctx->conv_tol > 0.0f) {                    // Alg. 1: rows not yet zero
        const int big = __syncthreads_count(i < a.m && !(fabsf(src[i < a.m ? i : 0]) <= ctx->conv_tol));
        if (threadIdx.x == 0 && big) atomicAdd(&a.st->big_hat, (unsigned)big);
    }
}

// Initial state: r_hat = the source, ||r_hat||_1 from the chunk partials
// (lane-strided, then a butterfly: the accept step's order).  One warp.  A
// decode that is done before its first round also takes the final residual
// norm here (x_hat = 0: the partials of y_hat).
__global__ void k_start(KArgs a, int round0, int empty_support)
{
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    double l1 = 0.0, fin = 0.0;
    for (int c = lane; c < a.nchunks; c += 32) {
        l1 += a.l1part[c];
        fin += a.final_part[c];
    }
    for (int off = 16; off > 0; off >>= 1) {
        l1 += __shfl_xor_sync(0xffffffffu, l1, off);
        fin += __shfl_xor_sync(0xffffffffu, fin, off);
    }
    if (lane != 0) return;
    DecodeState *st = a.st;
    const int status = st->status;
    st->round = round0;
    st->cur = 0;
    if (empty_support) { st->shat_count = 0; st->list_count = 0; }
    st->upd_count = 0;
    st->drop_count = 0;
    st->overflow = 0;
    st->rounds_run = 0;
    st->accepted_rounds = 0;
    st->hk_rounds = 0;
    st->fallback_rounds = 0;
    st->l1_hat = l1;
    st->l1_new = l1;
    double stop = a.ctx->stop_level;
    if (a.ctx->stop_rel > 0.0) stop = a.ctx->stop_rel * l1;
    a.ctx->stop_level = stop;
    st->converged = (a.ctx->conv_tol > 0.0f) ? (st->big_hat == 0) : (l1 <= stop);
    st->done = (status != 0) || st->converged || (round0 >= a.ctx->nrounds);
    st->nnz = st->shat_count;
    st->nnz_delta = 0;
    st->tick = 0ull;
    st->zeroed = 0;
    st->iters = 0;
    st->skipped = 0;
    if (!st->done && round0 == 0 && a.ctx->skip_t1) {
        // the round at t = 1 changes nothing (sigma_n > 0): record it as the
        // accept step records an empty round, and start at the next one
        if (a.ctx->want_log) {
            RoundLog L;
            L.l1_candidate = l1;
            L.l1_hat = l1;
            L.accepted = 0;
            L.updated = 0;
            L.support = (int)st->nnz;
            L.hk_dropped = 0;
            a.rlog[0] = L;
        }
        st->round = 1;
        st->rounds_run = 1;
        st->iters = 1;
        st->skipped = 1;
        st->done = (1 >= a.ctx->nrounds);
    }
    if (st->done) st->final_l1 = fin;
    if (a.has_cond) cudaGraphSetConditional(a.cond, st->done ? 0u : 1u);
}

// Support list of an injected x_hat (order irrelevant: every consumer sorts
// or selects by key).
__global__ void k_support_from_x(KArgs a)
{
    const float *x = a.ctx->x;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool nz = (j < a.n) && x[j] != 0.0f;
    const unsigned mask = __ballot_sync(0xffffffffu, nz);
    if (!mask) return;
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&a.st->shat_count, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (nz) a.list[base + __popc(mask & ((1u << lane) - 1u))] = j;
}

__global__ void k_list_count_from_support(KArgs a)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) a.st->list_count = a.st->shat_count;
}

// ---------------------------------------------------------------------------
// Column score: Algorithm 2's loop over j in [n] and i in N(j).
//
// One thread per column.  Fast path (registers only): the anchors
// (|r_i| >= ta) and, for every anchor, the mask of rows within reach of it --
// |r_i - r_l| <= te for the 0/1 scores, or <= the 2^-40 cut of p_e for the
// continuous scores, where n_e <= 1 + popc(mask).  An anchor whose bound
// cannot reach n_e - n_z >= alpha is dropped here; for the 0/1 scores the
// bound is n_e itself.  Slow path (rare): the surviving anchors get the exact
// n_e, omega and l1 test from residuals kept in shared memory, scored by the
// whole CTA from each column's highest slot down until one passes (that one is
// the last passing anchor in row order, whose omega the column takes).
// ---------------------------------------------------------------------------
template <int DMAX> struct ColBlock { static constexpr int value = DMAX <= 8 ? 256 : (DMAX <= 16 ? 128 : 64); };

// Shared memory of the column kernels.  H_k's scratch (used by the launch's
// last CTA after its tiles) shares the bytes of the candidate queue.
template <int DMAX, int NT, bool LEARNED>
struct ColShared {
    union {
        struct {
            float r[DMAX][NT];                 // residuals of columns with candidates
            float nz[NT], rhs[NT];
            unsigned short q[NT];              // this pass's queue: (column lane << 5) | slot
            float score[NT], w[NT];
            unsigned char ok[NT];
            float f[LEARNED ? RL0_NFEAT : 1][LEARNED ? NT : 1];   // features of the candidates that pass
            unsigned short fq[LEARNED ? NT : 1];                  // their queue positions
        } c;
        struct {
            HkShared hk;
            unsigned suf[NT];
        } h;
    };
    Series pe;
    int nq, nf;
    int last;
};

template <int DMAX, bool IND, bool LEARNED, int NT>
__device__ __forceinline__ void col_setup(const DecodeCtx *ctx, ColShared<DMAX, NT, LEARNED> &S)
{
    const int tid = threadIdx.x;
    if (tid == 0) {
        S.nq = 0;
        S.nf = 0;
        if (!IND) S.pe = ctx->pe;
    }
    // (these shared copies are first read after a barrier of the tile body)
}

// One tile of NT columns starting at j0.  gather(row) returns (r_row, p_z(r_row)).
template <int DMAX, bool IND, bool LEARNED, int NT, class Gather>
__device__ __forceinline__ void score_tile(const KArgs &a, const DecodeCtx *ctx, const RoundThr &th, int j0,
                                           Gather gather, ColShared<DMAX, NT, LEARNED> &S)
{
    const int tid = threadIdx.x;
    const int n = a.n, d = a.d;
    const int j = j0 + tid;
    const bool active = j < n;
    const float alpha = ctx->alpha;

    float r[DMAX];
    float nz = 0.0f, rhs = 0.0f;
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        r[s] = 0.0f;
        if (s < d && active) {
            const float2 v = gather(__ldg(a.rows_sm + (size_t)s * n + j));
            r[s] = v.x;
            nz += IND ? (fabsf(v.x) <= th.tz ? 1.0f : 0.0f) : v.y;
            rhs += fabsf(v.x);
        }
    }
    const float need = LEARNED ? (IND ? ctx->learned_need : ctx->learned_need - 1e-3f) : (IND ? alpha : alpha - 1e-3f);
    unsigned cand = active ? anchor_candidates<DMAX, IND>(r, d, th.ta, IND ? th.te : ctx->pe.cut, ctx->pe_b1,
                                                          ctx->pe_c1, nz, need) : 0u;
    if (cand) {
#pragma unroll
        for (int s = 0; s < DMAX; ++s) S.c.r[s][tid] = r[s];
        S.c.nz[tid] = nz;
        S.c.rhs[tid] = rhs;
    }
    int best = -1;
    float bw = 0.0f, bsc = 0.0f;
    while (__syncthreads_or(cand != 0u)) {
        int my = -1, ms = 0;
        if (cand) {
            ms = 31 - __clz(cand);                  // highest remaining slot first
            cand &= ~(1u << ms);
            my = atomicAdd(&S.nq, 1);
            S.c.q[my] = (unsigned short)((tid << 5) | ms);
        }
        __syncthreads();
        const int nq = S.nq;
        if (LEARNED) {
            // the learned scorer's logit replaces n_e - n_z >= alpha: each queued
            // candidate's exact l1 test and n_e - n_z >= 1.5 first; the features
            // of those that pass go to a compact list, whose logits the MLP takes
            // 16 per warp on the tensor cores (rl0_mma.cuh: the arithmetic of
            // rl0_mlp_forward); a candidate passes when its logit reaches the
            // threshold
            for (int e = tid; e < nq; e += NT) {
                const int owner = S.c.q[e] >> 5, s = S.c.q[e] & 31;
                const AnchorEval E = eval_anchor<IND>(&S.c.r[0][owner], NT, d, s, th.te, S.pe);
                S.c.ok[e] = 0;
                S.c.score[e] = 0.0f;
                S.c.w[e] = E.w;
                if (E.lhs <= S.c.rhs[owner] && E.ne - S.c.nz[owner] >= ctx->learned_need) {
                    const int p = atomicAdd(&S.nf, 1);
                    float f[RL0_NFEAT];
                    candidate_features(&S.c.r[0][owner], NT, d, E, S.c.nz[owner], S.c.rhs[owner], ctx->inv_sn,
                                       th.t, ctx->drho, f);
#pragma unroll
                    for (int q = 0; q < RL0_NFEAT; ++q) S.c.f[q][p] = f[q];
                    S.c.fq[p] = (unsigned short)e;
                }
            }
            __syncthreads();
            const int nf = S.nf;
            const __nv_bfloat16 *wb = (const __nv_bfloat16 *)ctx->mlp;
            for (int e0 = (tid >> 5) * 16; e0 < nf; e0 += (NT / 32) * 16) {
                auto f = [&](int r, int i) { return (e0 + r < nf) ? S.c.f[i][e0 + r] : 0.0f; };
                float lo, hi;
                warp_mlp_logits16(f, wb, &lo, &hi);
                if ((tid & 3) == 0) {
                    const int gr = (tid & 31) >> 2;
                    if (e0 + gr < nf) {
                        const int e = S.c.fq[e0 + gr];
                        S.c.score[e] = lo;
                        S.c.ok[e] = (lo >= ctx->logit_thr) ? 1 : 0;
                    }
                    if (e0 + gr + 8 < nf) {
                        const int e = S.c.fq[e0 + gr + 8];
                        S.c.score[e] = hi;
                        S.c.ok[e] = (hi >= ctx->logit_thr) ? 1 : 0;
                    }
                }
            }
        } else {
            for (int e = tid; e < nq; e += NT) {
                const int owner = S.c.q[e] >> 5, s = S.c.q[e] & 31;
                float sc, w;
                S.c.ok[e] = score_anchor<IND>(&S.c.r[0][owner], NT, d, s, th.te, S.pe, S.c.nz[owner], S.c.rhs[owner],
                                              alpha, &sc, &w) ? 1 : 0;
                S.c.score[e] = sc;
                S.c.w[e] = w;
            }
        }
        __syncthreads();
        if (my >= 0 && S.c.ok[my]) {
            if (ctx->anchor_rule == 0) {            // the first pass from the top is the last passing
                best = ms;                          // anchor in row order: it stands, the rest is moot
                bw = S.c.w[my];
                cand = 0u;
            } else if (best < 0 || S.c.score[my] >= bsc) {   // largest n_e - n_z; slots come highest
                best = ms;                                   // first, so >= leaves ties to the lower row
                bw = S.c.w[my];
                bsc = S.c.score[my];
            }
        }
        if (tid == 0) {
            S.nq = 0;
            S.nf = 0;
        }
    }
    commit_column(a, ctx, j, active, best, bw);
}

template <int DMAX, int NT, bool LEARNED>
__device__ __forceinline__ void col_last_cta(const KArgs &a, const DecodeCtx *ctx, ColShared<DMAX, NT, LEARNED> &S)
{
    last_cta_hk<NT>(a, ctx, S.h.hk, S.h.suf, &S.last);
}

template <int DMAX, bool IND, bool LEARNED>
__global__ void __launch_bounds__(ColBlock<DMAX>::value) k_column_score(KArgs a)
{
    constexpr int NT = ColBlock<DMAX>::value;
    __shared__ ColShared<DMAX, NT, LEARNED> S;
    const DecodeState *st = a.st;
    pdl_wait();                                    // the previous rebuild's r, x and state
    pdl_launch_dependents();
    if (st->done) return;
    const DecodeCtx *ctx = a.ctx;
    const float2 *__restrict__ rz = st->cur ? a.rz1 : a.rz0;
    const RoundThr th = a.thr[st->round];
    col_setup<DMAX, IND, LEARNED, NT>(ctx, S);
    score_tile<DMAX, IND, LEARNED, NT>(a, ctx, th, blockIdx.x * NT, [rz](int row) { return __ldg(rz + row); }, S);
    col_last_cta<DMAX, NT, LEARNED>(a, ctx, S);
}

// ---------------------------------------------------------------------------
// Residual rebuild r = y - A x'.
// ---------------------------------------------------------------------------
// An injected x_hat's support (list[0, shat_count)) into the support bucket
// B[0] (emptied by k_rows_from / k_rows_from_x).
__global__ void __launch_bounds__(256) k_bucket_support(KArgs a)
{
    bucket_support_items(a, a.st->shat_count, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                         (long long)gridDim.x * blockDim.x);
}


__global__ void __launch_bounds__(RL0_ROWS_CHUNK) k_rebuild(KArgs a)
{
    __shared__ DF sha[RL0_ROWS_CHUNK], shb[RL0_ROWS_CHUNK];
    __shared__ unsigned s_scan[RL0_ROWS_CHUNK];
    __shared__ int s_last;
    DecodeState *st = a.st;
    const DecodeCtx *ctx = a.ctx;
    const int i = blockIdx.x * RL0_ROWS_CHUNK + threadIdx.x;
    // y_i and the support buckets load while the column kernel finishes; the
    // fresh bucket and the state words after it has
    RowIn pre;
    if (i < a.m) load_row_support(a, ctx, i, pre);
    pdl_wait();
    if (i < a.m) load_row_fresh(a, i, pre);
    const int done = st->done, cur = st->cur, ovf = st->overflow;
    const unsigned upd = st->upd_count, bfl = st->bflags;
    pdl_launch_dependents();
    if (done) return;
    const int no_accept = ctx->no_accept;
    const float conv_tol = ctx->conv_tol;
    if (upd == 0) {                                // nothing changed: r = r_hat, only t advances
        if (blockIdx.x == 0 && !no_accept) accept_step<RL0_ROWS_CHUNK>(a, 0u, s_scan);
        return;
    }
    // a full fresh bucket, or an incomplete support bucket: CSR(A^T) pass
    const bool csr = ovf != 0 || ((bfl >> cur) & 1u);
    DF l1{0.0f, 0.0f}, f1{0.0f, 0.0f};
    bool fits = true;
    if (i < a.m) fits = rebuild_row(a, ctx, i, csr, cur, l1, f1, pre);
    if (__syncthreads_or(!fits) && threadIdx.x == 0) atomicOr(&st->bflags, 1u << (cur ^ 1));
    // ||r||_1 of the FP32 residual, and ||y_hat - A x'||_1 without FP32 rounding
    const double2 s2 = block_sum2_df(l1, f1, sha, shb);
    if (threadIdx.x == 0) {
        a.l1part[blockIdx.x] = s2.x;
        a.final_part[(size_t)(cur ? 0 : 1) * a.nchunks + blockIdx.x] = s2.y;
    }
    if (conv_tol > 0.0f) {                         // Alg. 1: rows of r' not yet zero
        const int big = __syncthreads_count(i < a.m && !(l1.hi <= conv_tol));
        if (threadIdx.x == 0 && big) atomicAdd(&st->big_cand, (unsigned)big);
    }
    if (no_accept) return;
    // ---- the launch's last CTA accepts or undoes the round
    __syncthreads();
    if (threadIdx.x == 0) s_last = (cta_ticket(&st->rb_done) == gridDim.x - 1u);
    __syncthreads();
    if (!s_last) return;
    if (threadIdx.x == 0) st->rb_done = 0u;
    accept_step<RL0_ROWS_CHUNK>(a, upd, s_scan);
}

// ||y_hat - A x_hat||_1 without FP32 rounding (the final residual-norm check):
// the chunk partials of r_hat, formed in FP32 pairs by the kernel that built
// it (rows summed in ascending column order, 256-row trees) and stored in
// FP64, summed in chunk order by one warp in FP64.
__global__ void k_final_sum(KArgs a)
{
    const double *part = a.final_part + (size_t)a.st->cur * a.nchunks;
    double v = 0.0;
    for (int c = threadIdx.x; c < a.nchunks; c += 32) v += part[c];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) a.st->final_l1 = v;
}

// r_hat = y - A x_hat for an arbitrary x_hat (CSR rows, ascending columns: the
// same FP32 sum as the rebuild) into rz[0], with the chunk l1 partials.
__global__ void __launch_bounds__(RL0_ROWS_CHUNK) k_rows_from_x(KArgs a)
{
    __shared__ DF sh[RL0_ROWS_CHUNK];
    const DecodeCtx *ctx = a.ctx;
    const float *x = ctx->x;
    DF l1{0.0f, 0.0f}, f1{0.0f, 0.0f};
    const int i = blockIdx.x * RL0_ROWS_CHUNK + threadIdx.x;
    if (i < a.m) {
        a.sbcnt0[i] = 0;                           // k_bucket_support fills B[0] next
        a.sbcnt1[i] = 0;
        a.bcnt[i] = 0;
        float sum = 0.0f;
        DF acc{ctx->y[i], 0.0f};
        for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) {
            const float xv = x[a.colidx[p]];
            sum += xv;
            acc = df_sub(acc, xv);
        }
        const float r = ctx->y[i] - sum;
        if (!isfinite(ctx->y[i])) atomicExch(&a.st->status, (int)RL0_ERR_INVALID_Y);
        a.rz0[i] = make_float2(r, ctx->indicator ? 0.0f : series_eval(ctx->pz, r));
        if (a.res_ok) a.code0[i] = residual_code(r);
        l1 = DF{fabsf(r), 0.0f};
        f1 = df_abs(acc);
    }
    const double s = block_sum_df(l1, sh);
    const double sf = block_sum_df(f1, sh);
    if (threadIdx.x == 0) {
        a.l1part[blockIdx.x] = s;
        a.final_part[blockIdx.x] = sf;
    }
}

// p_z(r_i) of r_hat under the posteriors now in ctx (after the adaptive_k
// step changed the prior; the rebuild stored p_z under the prior of its round).
__global__ void k_refresh_pz(KArgs a)
{
    const DecodeCtx *ctx = a.ctx;
    float2 *rz = a.st->cur ? a.rz1 : a.rz0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.m; i += gridDim.x * blockDim.x)
        rz[i].y = ctx->indicator ? 0.0f : series_eval(ctx->pz, rz[i].x);
}

// (column, FP32 bits of x_hat) of every support entry, for the host's
// adaptive_k step.
__global__ void k_support_pairs(KArgs a, int *out)
{
    const unsigned cnt = a.st->shat_count;
    const float *x = a.ctx->x;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
        const int j = a.list[e];
        out[2 * (size_t)e] = j;
        out[2 * (size_t)e + 1] = __float_as_int(x[j]);
    }
}

// Features of every learned-scorer candidate of one round (for training logs):
// feat[e*16..], meta[e*4..] = (column, slot, analytic pass, l1 test), omega[e],
// in ascending (column, slot) order.  Two passes over the same arithmetic:
// pass 0 writes each block's candidate count to bbase[block]; k_collect_scan
// turns the counts into block offsets; pass 1 writes each candidate at its
// block's offset plus its rank within the block.
template <int DMAX, bool IND>
__global__ void __launch_bounds__(ColBlock<DMAX>::value) k_collect(KArgs a, float *feat, int *meta, float *omega,
                                                                   int cap, int *bbase, int pass)
{
    constexpr int NT = ColBlock<DMAX>::value;
    __shared__ Series s_pe;
    __shared__ float s_r[DMAX][NT];
    __shared__ int s_wsum[NT / 32];
    const DecodeState *st = a.st;
    const DecodeCtx *ctx = a.ctx;
    const float2 *__restrict__ rz = st->cur ? a.rz1 : a.rz0;
    const RoundThr th = a.thr[st->round];
    const float alpha = ctx->alpha;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0 && !IND) s_pe = ctx->pe;
    __syncthreads();
    const int n = a.n, d = a.d;
    const int j = blockIdx.x * NT + tid;
    const bool active = j < n;
    float r[DMAX];
    float nz = 0.0f, rhs = 0.0f;
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        r[s] = 0.0f;
        if (s < d && active) {
            const float2 v = rz[a.rows_sm[(size_t)s * n + j]];
            r[s] = v.x;
            nz += IND ? (fabsf(v.x) <= th.tz ? 1.0f : 0.0f) : v.y;
            rhs += fabsf(v.x);
        }
    }
    const float need = IND ? ctx->learned_need : ctx->learned_need - 1e-3f;
    const unsigned cand0 = active ? anchor_candidates<DMAX, IND>(r, d, th.ta, IND ? th.te : s_pe.cut, ctx->pe_b1,
                                                                 ctx->pe_c1, nz, need) : 0u;
#pragma unroll
    for (int s = 0; s < DMAX; ++s) s_r[s][tid] = r[s];
    // this column's candidates (slots in ascending order)
    unsigned keep = 0u;
    for (unsigned cand = cand0; cand; cand &= cand - 1u) {
        const int s = __ffs(cand) - 1;
        const AnchorEval E = eval_anchor<IND>(&s_r[0][tid], NT, d, s, th.te, s_pe);
        if (E.ne - nz >= ctx->learned_need) keep |= 1u << s;
    }
    const int c = __popc(keep);
    // exclusive scan of c over the block
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_wsum[wid] = incl;
    __syncthreads();
    int wbase = 0, total = 0;
    for (int w = 0; w < NT / 32; ++w) {
        if (w < wid) wbase += s_wsum[w];
        total += s_wsum[w];
    }
    if (pass == 0) {
        if (tid == 0) bbase[blockIdx.x] = total;
        return;
    }
    int e = bbase[blockIdx.x] + wbase + incl - c;
    for (; keep; keep &= keep - 1u, ++e) {
        const int s = __ffs(keep) - 1;
        if (e >= cap) break;
        const AnchorEval E = eval_anchor<IND>(&s_r[0][tid], NT, d, s, th.te, s_pe);
        float f[RL0_NFEAT];
        candidate_features(&s_r[0][tid], NT, d, E, nz, rhs, ctx->inv_sn, th.t, ctx->drho, f);
#pragma unroll
        for (int q = 0; q < RL0_NFEAT; ++q) feat[(long long)e * RL0_NFEAT + q] = f[q];
        meta[4 * e + 0] = j;
        meta[4 * e + 1] = s;
        meta[4 * e + 2] = (E.lhs <= rhs && E.ne - nz >= alpha) ? 1 : 0;
        meta[4 * e + 3] = (E.lhs <= rhs) ? 1 : 0;
        omega[e] = E.w;
    }
}

// Exclusive scan of the nb block counts in place (one block); *total gets the sum.
__global__ void __launch_bounds__(1024) k_collect_scan(int *bbase, int nb, int *total)
{
    __shared__ int s_part[1024];
    const int t = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    const int b0 = min(nb, t * per), b1 = min(nb, b0 + per);
    int sum = 0;
    for (int b = b0; b < b1; ++b) sum += bbase[b];
    s_part[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {           // Hillis-Steele inclusive scan of the parts
        const int u = (t >= o) ? s_part[t - o] : 0;
        __syncthreads();
        s_part[t] += u;
        __syncthreads();
    }
    int run = s_part[t] - sum;
    for (int b = b0; b < b1; ++b) {
        const int v = bbase[b];
        bbase[b] = run;
        run += v;
    }
    if (t == 1023) *total = s_part[1023];
}

// round_step output: the candidate residual (or r_hat when nothing changed).
__global__ void k_extract_r(KArgs a, float *rp, int use_candidate_always)
{
    const DecodeState *st = a.st;
    const bool changed = use_candidate_always || st->upd_count > 0;
    const float2 *src = (st->cur ^ (changed ? 1 : 0)) ? a.rz1 : a.rz0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.m; i += gridDim.x * blockDim.x) rp[i] = src[i].x;
}

// ---------------------------------------------------------------------------
// Host: posterior coefficients and thresholds in FP64.
// ---------------------------------------------------------------------------
using rl0::Resolved;

namespace {

struct GraphEntry {
    int nrounds, dmax, indicator, profile, learned;
    cudaGraphExec_t exec;
    std::vector<cudaEvent_t> events;   // profile: 4 per round + 1, boundaries of the kernel groups
};

// Rounds per iteration of the graph's WHILE loop: one iteration of the
// conditional node costs about 4 us, a round whose kernels only see the done
// flag about 2 us per kernel; three rounds per iteration measured best on 5-,
// 6- and 39-round decodes (2 and 4 were slower).
#define RL0_ROUNDS_PER_ITER 3

// Kernels of one round: the column score and the rebuild.
int kernels_per_round(const KArgs &, int) { return 2; }

// Kernels one decode graph launches: prologue (2), kpr per round in whole loop
// iterations (the step that ends the decode takes the final residual norm).
int launches_per_decode(int nrounds, int kpr)
{
    const int iters = (nrounds + RL0_ROUNDS_PER_ITER - 1) / RL0_ROUNDS_PER_ITER;
    return 2 + kpr * RL0_ROUNDS_PER_ITER * iters;
}

// The same with every round launched on its own (profile graph).
int launches_unrolled(int nrounds, int kpr) { return 2 + kpr * nrounds; }

struct GraphCache {
    std::vector<GraphEntry> entries;
    cudaStream_t capture_stream = nullptr;
};

KArgs make_args(const rl0_expander *A)
{
    const Workspace &w = A->ws;
    KArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = (int)A->n;
    a.m = (int)A->m;
    a.d = A->d;
    a.nchunks = (int)rl0_div_up(A->m, RL0_ROWS_CHUNK);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, A->device);
    a.nsm = nsm > 0 ? nsm : 1;
    a.rows_sm = A->rows_sm;
    a.rows_cm = A->rows_cm;
    a.rowptr = A->rowptr;
    a.colidx = A->colidx;
    a.rz0 = w.rz[0];
    a.rz1 = w.rz[1];
    a.code0 = w.code[0];
    a.code1 = w.code[1];
    a.pzlb = w.pzlb;
    a.list = w.list;
    a.ulog = w.ulog;
    a.dlog = w.dlog;
    a.bcnt = w.bcnt;
    a.bkt = w.bkt;
    a.sbcnt0 = w.sbcnt[0];
    a.sbcnt1 = w.sbcnt[1];
    a.sbkt0 = w.sbkt[0];
    a.sbkt1 = w.sbkt[1];
    a.l1part = w.l1part;
    a.hkkey = w.hk_scratch;
    a.st = w.st;
    a.ctx = w.ctx;
    a.thr = w.thr;
    a.rlog = w.rlog;
    a.final_part = w.final_part;
    a.res_list = w.res_list;
    rl0_res_setup(A, &a);
    return a;
}

// Launches the column score (+ H_k in its last CTA).  Returns true when it is
// the resident-code kernel, which also fills the rebuild's buckets.
bool launch_column_score(const KArgs &a, int dmax, int indicator, int learned, cudaStream_t s)
{
    if (rl0_res_launch(a, indicator, learned, s)) return true;
#define RL0_CS(D, I, L) launch_pdl(k_column_score<D, I, L>, rl0_div_up(a.n, ColBlock<D>::value), ColBlock<D>::value, 0, s, a)
    if (learned) {
        if (dmax == 8) { if (indicator) RL0_CS(8, true, true); else RL0_CS(8, false, true); }
        else { if (indicator) RL0_CS(16, true, true); else RL0_CS(16, false, true); }
    } else if (dmax == 8) { if (indicator) RL0_CS(8, true, false); else RL0_CS(8, false, false); }
    else if (dmax == 16) { if (indicator) RL0_CS(16, true, false); else RL0_CS(16, false, false); }
    else { if (indicator) RL0_CS(32, true, false); else RL0_CS(32, false, false); }
#undef RL0_CS
    return false;
}

int dmax_of(int d) { return d <= 8 ? 8 : (d <= 16 ? 16 : 32); }

// The residual rebuild of a round (+ accept in the rebuild's last CTA).
void launch_rebuild(const KArgs &a, cudaStream_t s)
{
    launch_pdl(k_rebuild, a.nchunks, RL0_ROWS_CHUNK, 0, s, a);
}

// The kernels of one round (shared by the graph and by round_step).
void launch_round(const KArgs &a, int dmax, int indicator, int learned, cudaStream_t s)
{
    launch_column_score(a, dmax, indicator, learned, s);   // + H_k in its last CTA
    launch_rebuild(a, s);
}

// An injected x_hat's support into the support bucket B[0].
void launch_bucket_support(const KArgs &a, cudaStream_t s)
{
    k_bucket_support<<<2 * a.nsm, 256, 0, s>>>(a);
}

// The round loop as a graph.  Normal decodes: prologue kernels, then a WHILE
// conditional node whose body is RL0_ROUNDS_PER_ITER rounds (the rebuild's
// last CTA clears the condition once the decode is done; a round after that
// only sees the done flag); the step that ends the decode takes the final
// residual norm.  Profile decodes:
// the rounds unrolled, with event-record nodes around each kernel group (event
// nodes are not allowed in a conditional body).
int add_kernel_node(cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *dep, int ndep, void *func,
                    unsigned grid, unsigned block, KArgs *a, void **extra, int nextra)
{
    void *args[4] = {a, nullptr, nullptr, nullptr};
    for (int i = 0; i < nextra; ++i) args[1 + i] = extra[i];
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.func = func;
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.kernelParams = args;
    CK(cudaGraphAddKernelNode(node, g, dep, ndep, &kp));
    return RL0_OK;
}

int capture_decode_graph(rl0_expander *A, int nrounds, int dmax, int indicator, int profile, int learned,
                         GraphEntry *E)
{
    GraphCache *gc = (GraphCache *)A->graph_cache;
    KArgs a = make_args(A);
    cudaStream_t s = gc->capture_stream;
    E->nrounds = nrounds;
    E->dmax = dmax;
    E->indicator = indicator;
    E->profile = profile;
    E->learned = learned;
    cudaGraph_t g = nullptr;
    if (!profile) {
        CK(cudaGraphCreate(&g, 0));
        int rc = RL0_OK;
        do {
            cudaGraphConditionalHandle h;
            if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
                rc = RL0_ERR_CUDA;
                break;
            }
            a.cond = h;
            a.has_cond = 1;
            cudaGraphNode_t n1, n2, nw;
            const float *nullsrc = nullptr;
            int zero = 0, one = 1;
            void *ex_rows[3] = {&nullsrc, &zero, &one};
            void *ex_start[2] = {&zero, &one};
            if ((rc = add_kernel_node(g, &n1, nullptr, 0, (void *)k_rows_from, a.nchunks, RL0_ROWS_CHUNK, &a, ex_rows, 3)))
                break;
            if ((rc = add_kernel_node(g, &n2, &n1, 1, (void *)k_start, 1, 32, &a, ex_start, 2))) break;
            cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional, {0, 0, 0}, {}, 0};
            std::memset((void *)&cp, 0, sizeof(cp));
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            if (cudaGraphAddNode(&nw, g, &n2, nullptr, 1, &cp) != cudaSuccess) { rc = RL0_ERR_CUDA; break; }
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            if (cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
                cudaSuccess) { rc = RL0_ERR_CUDA; break; }
            for (int q = 0; q < RL0_ROUNDS_PER_ITER; ++q) launch_round(a, dmax, indicator, learned, s);
            cudaGraph_t body_out = nullptr;
            if (cudaStreamEndCapture(s, &body_out) != cudaSuccess) { rc = RL0_ERR_CUDA; break; }
            // the final residual norm is taken by the step that ends the
            // decode (k_start or the accept step): no epilogue kernel
        } while (0);
        if (rc) { cudaGetLastError(); cudaGraphDestroy(g); return rc; }
        cudaError_t e = cudaGraphInstantiate(&E->exec, g, 0);
        cudaGraphDestroy(g);
        return rl0_cuda_err(e);
    }
    E->events.resize(4 * nrounds + 1);
    for (auto &ev : E->events) CK(cudaEventCreate(&ev));
    auto mark = [&](int idx) -> cudaError_t {
        return cudaEventRecordWithFlags(E->events[idx], s, cudaEventRecordExternal);
    };
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    k_rows_from<<<a.nchunks, RL0_ROWS_CHUNK, 0, s>>>(a, nullptr, 0, 1);
    k_start<<<1, 32, 0, s>>>(a, 0, 1);
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < nrounds && e == cudaSuccess; ++r) {
        e = mark(4 * r);
        launch_column_score(a, dmax, indicator, learned, s);
        if (e == cudaSuccess) e = mark(4 * r + 1);
        if (e == cudaSuccess) e = mark(4 * r + 2);
        launch_rebuild(a, s);
        if (e == cudaSuccess) e = mark(4 * r + 3);
    }
    if (e == cudaSuccess) e = mark(4 * nrounds);
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return rl0_cuda_err(e); }
    if (e2 != cudaSuccess) return rl0_cuda_err(e2);
    e = cudaGraphInstantiate(&E->exec, g, 0);
    cudaGraphDestroy(g);
    return rl0_cuda_err(e);
}

// Pinned host staging: ctx, thresholds, state, final partials, log.
struct HostStage {
    DecodeCtx ctx;
    float pzlb[RL0_PZ_BINS];
    DecodeState st;
    RoundThr thr[RL0_MAX_ROUNDS];
    RoundLog log[RL0_MAX_ROUNDS];
    double kprior[RL0_MAX_ROUNDS];     // the posteriors' sparsity per round (adaptive_k)
};

// Host tables of the last parameter set, reused when a decode repeats it.
struct TableCache {
    bool valid = false;
    int64_t k = 0;
    rl0_params p;
    int nrounds = 0;
    DecodeCtx ctx;
    RoundThr thr[RL0_MAX_ROUNDS];
    bool pz_valid = false;
    float pzlb[RL0_PZ_BINS];
};

}  // namespace

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
int rl0_workspace_alloc(rl0_expander *A)
{
    Workspace &w = A->ws;
    const size_t n = (size_t)A->n, m = (size_t)A->m;
    const size_t nchunks = rl0_div_up(A->m, RL0_ROWS_CHUNK);
    w.max_rounds = RL0_MAX_ROUNDS;
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    al((void **)&w.rz[0], m * sizeof(float2));
    al((void **)&w.rz[1], m * sizeof(float2));
    al((void **)&w.code[0], (size_t)rl0_code_rows(A->m) * sizeof(unsigned short));
    al((void **)&w.code[1], (size_t)rl0_code_rows(A->m) * sizeof(unsigned short));
    al((void **)&w.pzlb, RL0_PZ_BINS * sizeof(float));
    al((void **)&w.res_list, n * (size_t)(rl0_res_dmax(A->d) + 2) * sizeof(int));
    al((void **)&w.list, n * sizeof(int));
    al((void **)&w.list_tmp, sizeof(int));
    al((void **)&w.ulog, n * sizeof(UndoEntry));
    al((void **)&w.dlog, n * sizeof(UndoEntry));
    al((void **)&w.bcnt, m * sizeof(int));
    al((void **)&w.bkt, m * RL0_BUCKET * sizeof(int));
    al((void **)&w.sbcnt[0], m * sizeof(int));
    al((void **)&w.sbcnt[1], m * sizeof(int));
    al((void **)&w.sbkt[0], m * RL0_BUCKET * sizeof(int));
    al((void **)&w.sbkt[1], m * RL0_BUCKET * sizeof(int));
    al((void **)&w.l1part, nchunks * sizeof(double));
    al((void **)&w.hk_scratch, n * sizeof(unsigned long long));
    al((void **)&w.st, sizeof(DecodeState));
    al((void **)&w.ctx, sizeof(DecodeCtx));
    al((void **)&w.thr, RL0_MAX_ROUNDS * sizeof(RoundThr));
    al((void **)&w.rlog, RL0_MAX_ROUNDS * sizeof(RoundLog));
    al((void **)&w.final_part, 2 * nchunks * sizeof(double));   // one set per rz buffer
    al((void **)&w.host_y, m * sizeof(float));
    al((void **)&w.host_x, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(w.bcnt, 0, m * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(w.sbcnt[0], 0, m * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(w.sbcnt[1], 0, m * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(w.st, 0, sizeof(DecodeState));
    if (e == cudaSuccess) e = cudaMallocHost(&A->host_pinned, sizeof(HostStage));
    if (e != cudaSuccess) { cudaGetLastError(); return rl0_cuda_err(e); }
    A->host_pinned_bytes = sizeof(HostStage);
    GraphCache *gc = new (std::nothrow) GraphCache;
    if (!gc) return RL0_ERR_ALLOC;
    A->graph_cache = gc;
    e = cudaStreamCreateWithFlags(&gc->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return rl0_cuda_err(e);
    cudaEvent_t *ev = new (std::nothrow) cudaEvent_t[2];
    if (!ev) return RL0_ERR_ALLOC;
    A->events = ev;
    e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e != cudaSuccess) return rl0_cuda_err(e);
    TableCache *tc = new (std::nothrow) TableCache;
    if (!tc) return RL0_ERR_ALLOC;
    A->table_cache = tc;
    return RL0_OK;
}

void rl0_workspace_free(rl0_expander *A)
{
    Workspace &w = A->ws;
    GraphCache *gc = (GraphCache *)A->graph_cache;
    if (gc) {
        for (auto &g : gc->entries) {
            cudaGraphExecDestroy(g.exec);
            for (auto ev : g.events) cudaEventDestroy(ev);
        }
        if (gc->capture_stream) cudaStreamDestroy(gc->capture_stream);
        delete gc;
        A->graph_cache = nullptr;
    }
    if (A->events) {
        cudaEvent_t *ev = (cudaEvent_t *)A->events;
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        delete[] ev;
        A->events = nullptr;
    }
    if (A->table_cache) {
        delete (TableCache *)A->table_cache;
        A->table_cache = nullptr;
    }
    void *ptrs[] = {w.rz[0], w.rz[1], w.code[0], w.code[1], w.pzlb, w.res_list, w.list, w.list_tmp, w.ulog, w.dlog, w.bcnt, w.bkt,
                    w.sbcnt[0], w.sbcnt[1], w.sbkt[0], w.sbkt[1], w.l1part, w.hk_scratch, w.st, w.ctx, w.thr, w.rlog,
                    w.final_part, w.host_y, w.host_x};
    for (void *p : ptrs) if (p) cudaFree(p);
    std::memset(&w, 0, sizeof(w));
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
static bool same_params(const rl0_params &a, const rl0_params &b)
{
    return a.sigma_s == b.sigma_s && a.sigma_n == b.sigma_n && a.quantised == b.quantised && a.c == b.c &&
           a.alpha == b.alpha && a.ell == b.ell && a.scorer == b.scorer && a.mlp == b.mlp &&
           a.mlp_threshold == b.mlp_threshold && a.max_rounds == b.max_rounds && a.noiseless_tol == b.noiseless_tol &&
           a.anchor_rule == b.anchor_rule;
}

static void cached_tables(rl0_expander *A, int64_t k, const Resolved &R, DecodeCtx *ctx, RoundThr *thr)
{
    TableCache *tc = (TableCache *)A->table_cache;
    if (tc && tc->valid && tc->k == k && tc->nrounds == R.nrounds && same_params(tc->p, R.p)) {
        *ctx = tc->ctx;
        std::memcpy(thr, tc->thr, R.nrounds * sizeof(RoundThr));
        return;
    }
    rl0::fill_tables(A->m, A->d, k, R, ctx, thr, R.nrounds);
    if (tc) {
        tc->pz_valid = false;
        tc->valid = true;
        tc->k = k;
        tc->p = R.p;
        tc->nrounds = R.nrounds;
        tc->ctx = *ctx;
        std::memcpy(tc->thr, thr, R.nrounds * sizeof(RoundThr));
    }
}

// The same for other translation units (the batched decoder): the tables of
// (k, R) for expander A, from its cache when they repeat the last call's.
// Calls for distinct expanders may run concurrently.
void rl0_cached_tables(rl0_expander *A, int64_t k, const Resolved &R, DecodeCtx *ctx, RoundThr *thr)
{
    cached_tables(A, k, R, ctx, thr);
}

// Whether A's cache holds the tables of (k, R).
bool rl0_tables_cached(const rl0_expander *A, int64_t k, const Resolved &R)
{
    const TableCache *tc = (const TableCache *)A->table_cache;
    return tc && tc->valid && tc->k == k && tc->nrounds == R.nrounds && same_params(tc->p, R.p);
}

// p_z lower bounds of the parameter set cached_tables just resolved.
static void cached_pz(rl0_expander *A, int64_t k, const Resolved &R, float *out)
{
    TableCache *tc = (TableCache *)A->table_cache;
    if (tc && tc->valid && tc->pz_valid) {
        std::memcpy(out, tc->pzlb, sizeof(tc->pzlb));
        return;
    }
    rl0::pz_lower_bounds(A->m, A->d, k, R, out);
    if (tc && tc->valid) {
        std::memcpy(tc->pzlb, out, sizeof(tc->pzlb));
        tc->pz_valid = true;
    }
}

// The captured round loop for this shape (captured on first use).
static int get_graph(rl0_expander *A, int nrounds, int dmax, int indicator, int prof, int learned, GraphEntry **out)
{
    GraphCache *gc = (GraphCache *)A->graph_cache;
    for (auto &g : gc->entries)
        if (g.nrounds == nrounds && g.dmax == dmax && g.indicator == indicator && g.profile == prof &&
            g.learned == learned) {
            *out = &g;
            return RL0_OK;
        }
    GraphEntry fresh;
    const int rc = capture_decode_graph(A, nrounds, dmax, indicator, prof, learned, &fresh);
    if (rc) {
        for (auto ev : fresh.events) if (ev) cudaEventDestroy(ev);
        return rc;
    }
    gc->entries.push_back(fresh);
    *out = &gc->entries.back();
    return RL0_OK;
}

// Alg. 2 with the analytic scores, continued from the x_hat a learned decode
// left (a fresh sweep): the analytic tables, the state rebuilt from x_hat, then
// every round of the sweep launched directly, and the final residual norm.
// `a` holds the buffers the kernels use (an expander's workspace or the static
// array).  When the kernels bound n_z with the residual codes (a.pzlb set),
// the analytic scores' p_z bound table is uploaded too: the learned decode
// does not upload one, and a table left by an earlier decode with other
// parameters would drop valid candidates.  *launches receives the kernels
// launched.  Enqueues only; the caller synchronises.
static int launch_analytic_continuation(rl0_expander *A, const KArgs &a, int64_t k, const Resolved &R,
                                        const float *y_dev, float *xhat_dev, int *launches, cudaStream_t s)
{
    HostStage *H = (HostStage *)A->host_pinned;
    Resolved R2 = R;
    R2.p.scorer = 0;
    R2.p.profile = 0;
    rl0::fill_tables(A->m, A->d, k, R2, &H->ctx, H->thr, R2.nrounds);
    H->ctx.y = y_dev;
    H->ctx.x = xhat_dev;
    H->ctx.want_log = 0;
    H->ctx.passed = nullptr;
    CK(cudaMemcpyAsync(a.ctx, &H->ctx, sizeof(DecodeCtx), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((void *)a.thr, H->thr, R2.nrounds * sizeof(RoundThr), cudaMemcpyHostToDevice, s));
    if (a.pzlb && !R2.indicator) {
        rl0::pz_lower_bounds(A->m, A->d, k, R2, H->pzlb);
        CK(cudaMemcpyAsync((void *)a.pzlb, H->pzlb, sizeof(H->pzlb), cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemsetAsync(a.st, 0, sizeof(DecodeState), s));
    const int dmax = dmax_of(A->d);
    k_support_from_x<<<rl0_div_up(a.n, 256), 256, 0, s>>>(a);
    k_rows_from_x<<<a.nchunks, RL0_ROWS_CHUNK, 0, s>>>(a);
    k_start<<<1, 32, 0, s>>>(a, 0, 0);
    k_list_count_from_support<<<1, 32, 0, s>>>(a);
    launch_bucket_support(a, s);
    for (int r = 0; r < R2.nrounds; ++r) launch_round(a, dmax, R2.indicator, 0, s);
    k_final_sum<<<1, 32, 0, s>>>(a);
    CK(cudaGetLastError());
    *launches = 5 + kernels_per_round(a, 0) * R2.nrounds + 1;
    return RL0_OK;
}

// Alg. 2 with the adaptive_k flag: the rounds of the captured graph, launched
// one round at a time; after each accepted round the host reads the support,
// takes the adaptive_k step in FP64 (ascending column order) and uploads the
// rebuilt posteriors and thresholds before the next round.
static int decode_adaptive(rl0_expander *A, const float *y_dev, int64_t k, const Resolved &R, float *xhat_dev,
                           rl0_stats *stats, cudaStream_t s)
{
    HostStage *H = (HostStage *)A->host_pinned;
    const Workspace &w = A->ws;
    const KArgs a = make_args(A);
    const int dmax = dmax_of(A->d);
    cudaEvent_t *ev = (cudaEvent_t *)A->events;
    if (stats) CK(cudaEventRecord(ev[0], s));
    k_rows_from<<<a.nchunks, RL0_ROWS_CHUNK, 0, s>>>(a, nullptr, 0, 1);
    k_start<<<1, 32, 0, s>>>(a, 0, 0);
    CK(cudaGetLastError());
    // the device set the stop level (noiseless: tol ||y_hat||_1); keep it
    CK(cudaMemcpyAsync(&H->ctx, w.ctx, sizeof(DecodeCtx), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&H->st, w.st, sizeof(DecodeState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double stop_level = H->ctx.stop_level;
    double kprior = (double)k;
    int accepted = H->st.accepted_rounds;
    std::vector<int> pairs;
    std::vector<std::pair<int, float>> supp;
    std::vector<float> vals;
    int launches = 2;
    for (int r = 0; r < H->st.round && r < RL0_MAX_ROUNDS; ++r) H->kprior[r] = kprior;   // recorded rounds
    for (int r = H->st.round; r < R.nrounds && !H->st.done; ++r) {
        H->kprior[r] = kprior;
        launch_round(a, dmax, R.indicator, 0, s);
        launches += kernels_per_round(a, 0);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&H->st, w.st, sizeof(DecodeState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (H->st.status) break;
        if (H->st.accepted_rounds == accepted) continue;
        accepted = H->st.accepted_rounds;
        if (H->st.done) break;
        // the adaptive_k step on the accepted x_hat
        const unsigned cnt = H->st.shat_count;
        pairs.resize(2 * (size_t)cnt);
        if (cnt) {
            k_support_pairs<<<2 * a.nsm, 256, 0, s>>>(a, a.res_list);
            launches += 1;
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(pairs.data(), a.res_list, 2 * (size_t)cnt * sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
        supp.resize(cnt);
        for (unsigned e = 0; e < cnt; ++e) {
            float v;
            std::memcpy(&v, &pairs[2 * (size_t)e + 1], sizeof(float));
            supp[e] = std::make_pair(pairs[2 * (size_t)e], v);
        }
        std::sort(supp.begin(), supp.end());
        vals.resize(cnt);
        for (unsigned e = 0; e < cnt; ++e) vals[e] = supp[e].second;
        kprior = rl0::adaptive_k0(A->m, A->d, k, R, kprior, vals.data(), (int64_t)cnt);
        rl0::fill_tables(A->m, A->d, k, R, &H->ctx, H->thr, R.nrounds, kprior);
        H->ctx.y = y_dev;
        H->ctx.x = xhat_dev;
        H->ctx.want_log = 1;
        H->ctx.passed = nullptr;
        H->ctx.stop_level = stop_level;
        H->ctx.wait_test = A->wait_test;
        H->ctx.wait_polls = A->wait_polls;
        CK(cudaMemcpyAsync(w.ctx, &H->ctx, sizeof(DecodeCtx), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(w.thr, H->thr, R.nrounds * sizeof(RoundThr), cudaMemcpyHostToDevice, s));
        if (!R.indicator) {
            rl0::pz_lower_bounds(A->m, A->d, k, R, H->pzlb, kprior);
            CK(cudaMemcpyAsync(w.pzlb, H->pzlb, sizeof(H->pzlb), cudaMemcpyHostToDevice, s));
            // n_z of the next round sums p_z(r_hat) under the new prior
            k_refresh_pz<<<2 * a.nsm, 256, 0, s>>>(a);
            launches += 1;
            CK(cudaGetLastError());
        }
    }
    k_final_sum<<<1, 32, 0, s>>>(a);
    launches += 1;
    CK(cudaGetLastError());
    if (stats) CK(cudaEventRecord(ev[1], s));
    CK(cudaMemcpyAsync(&H->st, w.st, sizeof(DecodeState), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(H->log, w.rlog, R.nrounds * sizeof(RoundLog), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // the next decode on this expander starts from the cached (non-adaptive) tables
    TableCache *tc = (TableCache *)A->table_cache;
    if (tc) tc->valid = false;
    if (H->st.status == RL0_ERR_INVALID_Y) return RL0_ERR_INVALID_Y;
    A->last_log_rounds = H->st.rounds_run;
    if (stats) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        std::memset(stats, 0, sizeof(*stats));
        stats->rounds = H->st.rounds_run;
        stats->accepted_rounds = H->st.accepted_rounds;
        stats->converged = H->st.converged;
        stats->status = H->st.status;
        stats->support_size = H->st.nnz;
        stats->final_l1 = H->st.final_l1;
        stats->ms = ms;
        stats->hk_rounds = H->st.hk_rounds;
        stats->fallback_rounds = H->st.fallback_rounds;
        stats->launches = launches;
        stats->skipped_rounds = H->st.skipped;
    }
    if (H->st.status) return H->st.status < 0 ? H->st.status : RL0_ERR_TIMEOUT;
    return RL0_OK;
}

// xhat_host (may be NULL): for the plain decode, x_hat is copied there right
// after the round graph, before the one synchronisation; *copied says whether
// that happened (the learned and adaptive decodes leave the copy to the caller).
static int decode_common(const rl0_expander *Ac, const float *y_dev, int64_t k, const rl0_params *params,
                         float *xhat_dev, rl0_stats *stats, cudaStream_t s, float *xhat_host = nullptr,
                         bool *copied = nullptr)
{
    rl0_expander *A = const_cast<rl0_expander *>(Ac);
    Resolved R;
    int rc = rl0::resolve(A->n, A->m, A->d, k, params, &R);
    if (rc) return rc;
    HostStage *H = (HostStage *)A->host_pinned;
    cached_tables(A, k, R, &H->ctx, H->thr);
    H->ctx.y = y_dev;
    H->ctx.x = xhat_dev;
    H->ctx.want_log = 1;
    H->ctx.passed = nullptr;
    H->ctx.wait_test = A->wait_test;
    H->ctx.wait_polls = A->wait_polls;
    const Workspace &w = A->ws;
    CK(cudaMemcpyAsync(w.ctx, &H->ctx, sizeof(DecodeCtx), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.thr, H->thr, R.nrounds * sizeof(RoundThr), cudaMemcpyHostToDevice, s));
    if (!R.indicator) {                           // the resident-code column kernel's n_z bound
        cached_pz(A, k, R, H->pzlb);
        CK(cudaMemcpyAsync(w.pzlb, H->pzlb, sizeof(H->pzlb), cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemsetAsync(w.st, 0, sizeof(DecodeState), s));
    if (R.p.adaptive_k) return decode_adaptive(A, y_dev, k, R, xhat_dev, stats, s);
    for (int r = 0; r < R.nrounds; ++r) H->kprior[r] = (double)k;
    const int dmax = dmax_of(A->d);
    const int prof = R.p.profile ? 1 : 0;
    const int learned = R.p.scorer == 1;
    GraphEntry *E = nullptr;
    rc = get_graph(A, R.nrounds, dmax, R.indicator, prof, learned, &E);
    if (rc) return rc;
    cudaEvent_t *ev = (cudaEvent_t *)A->events;
    if (stats) CK(cudaEventRecord(ev[0], s));
    CK(cudaGraphLaunch(E->exec, s));
    if (stats) CK(cudaEventRecord(ev[1], s));
    if (xhat_host && !learned) {
        CK(cudaMemcpyAsync(xhat_host, xhat_dev, (size_t)A->n * sizeof(float), cudaMemcpyDeviceToHost, s));
        if (copied) *copied = true;
    }
    CK(cudaMemcpyAsync(&H->st, w.st, sizeof(DecodeState), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(H->log, w.rlog, R.nrounds * sizeof(RoundLog), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (H->st.status == RL0_ERR_INVALID_Y) return RL0_ERR_INVALID_Y;
    if (stats) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        std::memset(stats, 0, sizeof(*stats));
        stats->rounds = H->st.rounds_run;
        stats->accepted_rounds = H->st.accepted_rounds;
        stats->converged = H->st.converged;
        stats->status = H->st.status;
        stats->support_size = H->st.nnz;
        stats->final_l1 = H->st.final_l1;
        stats->ms = ms;
        stats->hk_rounds = H->st.hk_rounds;
        stats->fallback_rounds = H->st.fallback_rounds;
        const int kpr = kernels_per_round(make_args(A), learned);
        stats->launches = prof ? launches_unrolled(R.nrounds, kpr)
                               : launches_per_decode(H->st.rounds_run - H->st.skipped, kpr);
        stats->skipped_rounds = H->st.skipped;
        if (prof) {
            float acc[4] = {0, 0, 0, 0};
            const int ran = H->st.rounds_run - H->st.skipped;   // launch groups that did a round
            const int active = ran < R.nrounds ? ran : R.nrounds;
            for (int r = 0; r < active; ++r)            // rounds after the decode finished only exit
                for (int q = 0; q < 4; ++q) {
                    float v = 0.0f;
                    if (cudaEventElapsedTime(&v, E->events[4 * r + q], E->events[4 * r + q + 1]) == cudaSuccess)
                        acc[q] += v;
                }
            stats->ms_score = acc[0];
            stats->ms_hk = acc[1];
            stats->ms_rebuild = acc[2];
            stats->ms_accept = acc[3];
        }
    }
    A->last_log_rounds = H->st.rounds_run;
    if (H->st.status) return H->st.status < 0 ? H->st.status : RL0_ERR_TIMEOUT;
    if (learned && !(H->st.l1_hat <= R.keep_level)) {
        // The learned decode's residual is not consistent with the noise
        // (||r||_1 > E||eta||_1 + 3 sqrt(Var||eta||_1)): Algorithm 2 with the
        // analytic scores continues from the learned x_hat (a fresh sweep).
        const DecodeState first = H->st;
        const KArgs a = make_args(A);
        int cont_launches = 0;
        rc = launch_analytic_continuation(A, a, k, R, y_dev, xhat_dev, &cont_launches, s);
        if (rc) return rc;
        if (stats) CK(cudaEventRecord(ev[1], s));
        CK(cudaMemcpyAsync(&H->st, w.st, sizeof(DecodeState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (H->st.status) return H->st.status < 0 ? H->st.status : RL0_ERR_TIMEOUT;
        if (stats) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            stats->rounds = first.rounds_run + H->st.rounds_run;
            stats->accepted_rounds = first.accepted_rounds + H->st.accepted_rounds;
            stats->converged = H->st.converged;
            stats->support_size = H->st.nnz;
            stats->final_l1 = H->st.final_l1;
            stats->ms = ms;
            stats->hk_rounds = first.hk_rounds + H->st.hk_rounds;
            stats->fallback_rounds = first.fallback_rounds + H->st.fallback_rounds;
            stats->analytic_rounds = H->st.rounds_run;
            stats->skipped_rounds = first.skipped + H->st.skipped;
            stats->launches += cont_launches;
        }
    }
    return RL0_OK;
}

extern "C" int rl0_decode_log(const rl0_expander *A, rl0_round_record *out, int cap)
{
    if (!A || (!out && cap > 0) || cap < 0) return RL0_ERR_INVALID_ARG;
    const HostStage *H = (const HostStage *)A->host_pinned;
    const int nr = A->last_log_rounds < cap ? A->last_log_rounds : cap;
    for (int r = 0; r < nr; ++r) {
        out[r].t = H->thr[r].t;
        out[r].l1_candidate = H->log[r].l1_candidate;
        out[r].l1_hat = H->log[r].l1_hat;
        out[r].accepted = H->log[r].accepted;
        out[r].updated = H->log[r].updated;
        out[r].support = H->log[r].support;
        out[r].hk_dropped = H->log[r].hk_dropped;
        out[r].k_prior = H->kprior[r];
    }
    return A->last_log_rounds;
}

extern "C" int rl0_expander_set_wait_polls(rl0_expander *A, int64_t polls)
{
    if (!A || polls > (int64_t)0xffffffffu) return RL0_ERR_INVALID_ARG;
    A->wait_test = polls >= 0 ? 1 : 0;
    A->wait_polls = polls >= 0 ? (unsigned)polls : 0u;
    return RL0_OK;
}

extern "C" int rl0_decode(const rl0_expander *A, const float *y_dev, int64_t k, const rl0_params *params,
                          float *xhat_dev, rl0_stats *stats, void *cuda_stream)
{
    if (!A || !y_dev || !xhat_dev) return RL0_ERR_INVALID_ARG;
    int rc = rl0_set_device_of(A);
    if (rc) return rc;
    return decode_common(A, y_dev, k, params, xhat_dev, stats, (cudaStream_t)cuda_stream);
}

extern "C" int rl0_decode_host(const rl0_expander *A, const float *y_host, int64_t k, const rl0_params *params,
                               float *xhat_host, rl0_stats *stats, void *cuda_stream)
{
    if (!A || !y_host || !xhat_host) return RL0_ERR_INVALID_ARG;
    int rc = rl0_set_device_of(A);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the expander's own device buffers (calls on one expander are serialised)
    float *yd = A->ws.host_y, *xd = A->ws.host_x;
    cudaError_t e = cudaMemcpyAsync(yd, y_host, (size_t)A->m * 4, cudaMemcpyHostToDevice, s);
    bool copied = false;
    if (e == cudaSuccess) rc = decode_common(A, yd, k, params, xd, stats, s, xhat_host, &copied);
    else rc = rl0_cuda_err(e);
    if (rc == RL0_OK && !copied) {
        e = cudaMemcpyAsync(xhat_host, xd, (size_t)A->n * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        rc = rl0_cuda_err(e);
    }
    return rc;
}

extern "C" int rl0_parallel_l0(const rl0_expander *Ac, const float *y_dev, double alpha, double tol, int max_iter,
                               float *xhat_dev, rl0_stats *stats, void *cuda_stream)
{
    rl0_expander *A = const_cast<rl0_expander *>(Ac);
    if (!A || !y_dev || !xhat_dev) return RL0_ERR_INVALID_ARG;
    if (alpha == 0.0) alpha = (double)(A->d / 2 + 1);
    if (!(alpha <= (double)A->d) || !(tol >= 0.0) || max_iter < 0 || max_iter > RL0_MAX_ROUNDS)
        return RL0_ERR_INVALID_ARG;
    // the kernels keep Alg. 2's l1 test: alpha >= d/2 implies it (n_e > d/2
    // rows move to zero, at most d - n_e rows grow, each by at most |omega|)
    if (alpha < 0.5 * A->d) return RL0_ERR_UNSUPPORTED;
    if (tol == 0.0) tol = 1e-5;
    if (max_iter == 0) max_iter = 100;
    int rc = rl0_set_device_of(A);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    rl0_params p;
    std::memset(&p, 0, sizeof(p));
    p.sigma_s = 1.0;
    p.quantised = 1;                               // 0/1 scores: q_e = 1{|D| <= tol}, q_z = 1{|r| <= tol}
    p.alpha = alpha;
    p.noiseless_tol = tol;
    p.c = 0.5;
    Resolved R;
    rc = rl0::resolve(A->n, A->m, A->d, A->n, &p, &R);
    if (rc) return rc;
    R.nrounds = max_iter;
    R.stop_level = -1.0;
    R.stop_rel = 0.0;
    HostStage *H = (HostStage *)A->host_pinned;
    rl0::fill_tables(A->m, A->d, A->n, R, &H->ctx, H->thr, 2);
    for (int r = 0; r < max_iter; ++r) {           // every iteration takes the t in (0, 1) thresholds
        H->thr[r] = H->thr[1];
        H->kprior[r] = (double)A->n;
    }
    H->ctx.y = y_dev;
    H->ctx.x = xhat_dev;
    H->ctx.want_log = 1;
    H->ctx.passed = nullptr;
    H->ctx.always_accept = 1;
    H->ctx.conv_tol = (float)tol;
    const Workspace &w = A->ws;
    CK(cudaMemcpyAsync(w.ctx, &H->ctx, sizeof(DecodeCtx), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.thr, H->thr, max_iter * sizeof(RoundThr), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(w.st, 0, sizeof(DecodeState), s));
    TableCache *tc = (TableCache *)A->table_cache;
    if (tc) tc->valid = false;                     // H->ctx no longer holds a decode's cached tables
    GraphEntry *E = nullptr;
    rc = get_graph(A, max_iter, dmax_of(A->d), 1, 0, 0, &E);
    if (rc) return rc;
    cudaEvent_t *ev = (cudaEvent_t *)A->events;
    if (stats) CK(cudaEventRecord(ev[0], s));
    CK(cudaGraphLaunch(E->exec, s));
    if (stats) CK(cudaEventRecord(ev[1], s));
    CK(cudaMemcpyAsync(&H->st, w.st, sizeof(DecodeState), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(H->log, w.rlog, max_iter * sizeof(RoundLog), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (H->st.status == RL0_ERR_INVALID_Y) return RL0_ERR_INVALID_Y;
    A->last_log_rounds = H->st.rounds_run;
    if (stats) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        std::memset(stats, 0, sizeof(*stats));
        stats->rounds = H->st.rounds_run;
        stats->accepted_rounds = H->st.accepted_rounds;
        stats->converged = H->st.converged;
        stats->status = H->st.status;
        stats->support_size = H->st.nnz;
        stats->final_l1 = H->st.final_l1;
        stats->ms = ms;
        stats->launches = launches_per_decode(H->st.rounds_run, kernels_per_round(make_args(A), 0));
    }
    if (H->st.status) return H->st.status < 0 ? H->st.status : RL0_ERR_TIMEOUT;
    return RL0_OK;
}

__global__ void k_copy_f(const float *src, float *dst, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

extern "C" int rl0_round_step(const rl0_expander *Ac, const float *y_dev, int64_t k, const rl0_params *params,
                              int round_index, const float *xhat_dev, const float *rhat_dev, float *xp_dev,
                              float *rp_dev, int32_t *passed_dev, double *l1_out, void *cuda_stream)
{
    rl0_expander *A = const_cast<rl0_expander *>(Ac);
    if (!A || !y_dev || !xhat_dev || !rhat_dev || !xp_dev || !rp_dev || round_index < 0) return RL0_ERR_INVALID_ARG;
    int rc = rl0_set_device_of(A);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Resolved R;
    rc = rl0::resolve(A->n, A->m, A->d, k, params, &R);
    if (rc) return rc;
    if (round_index >= RL0_MAX_ROUNDS) return RL0_ERR_INVALID_ARG;
    R.nrounds = round_index + 1;
    R.stop_level = -1.0;                          // never "converged" here
    R.stop_rel = 0.0;
    HostStage *H = (HostStage *)A->host_pinned;
    rl0::fill_tables(A->m, A->d, k, R, &H->ctx, H->thr, R.nrounds);
    H->ctx.y = y_dev;
    H->ctx.x = xp_dev;
    H->ctx.want_log = 0;
    H->ctx.passed = passed_dev;
    H->ctx.no_accept = 1;
    H->ctx.skip_t1 = 0;                            // run exactly the round asked for
    const Workspace &w = A->ws;
    CK(cudaMemcpyAsync(w.ctx, &H->ctx, sizeof(DecodeCtx), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.thr, H->thr, R.nrounds * sizeof(RoundThr), cudaMemcpyHostToDevice, s));
    if (!R.indicator) {
        rl0::pz_lower_bounds(A->m, A->d, k, R, H->pzlb);
        CK(cudaMemcpyAsync(w.pzlb, H->pzlb, sizeof(H->pzlb), cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemsetAsync(w.st, 0, sizeof(DecodeState), s));
    const KArgs a = make_args(A);
    k_copy_f<<<2 * a.nsm, 256, 0, s>>>(xhat_dev, xp_dev, a.n);
    k_rows_from<<<a.nchunks, RL0_ROWS_CHUNK, 0, s>>>(a, rhat_dev, 0, 0);
    k_support_from_x<<<rl0_div_up(a.n, 256), 256, 0, s>>>(a);
    k_start<<<1, 32, 0, s>>>(a, round_index, 0);
    k_list_count_from_support<<<1, 32, 0, s>>>(a);
    launch_bucket_support(a, s);
    launch_round(a, dmax_of(A->d), R.indicator, R.p.scorer == 1, s);
    k_extract_r<<<2 * a.nsm, 256, 0, s>>>(a, rp_dev, 0);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&H->st, w.st, sizeof(DecodeState), cudaMemcpyDeviceToHost, s));
    const int nchunks = a.nchunks;
    std::vector<double> part(nchunks);
    CK(cudaMemcpyAsync(part.data(), w.l1part, nchunks * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (H->st.status == RL0_ERR_INVALID_Y) return RL0_ERR_INVALID_Y;
    if (l1_out) {
        if (H->st.upd_count > 0) {
            double l1 = 0.0;
            for (int c = 0; c < nchunks; ++c) l1 += part[c];
            *l1_out = l1;
        } else {
            *l1_out = H->st.l1_hat;
        }
    }
    return RL0_OK;
}


// ---------------------------------------------------------------------------
// rl0_decode_static: the same decode with no allocation at all.
//
// Its working memory is one fixed array compiled into this library (below), so
// a call never asks the CUDA allocator (or any other allocator) for memory and
// never builds a graph (instantiating one allocates).  The price: instances are
// limited to n <= RL0_STATIC_MAX_N and m <= RL0_STATIC_MAX_M, every GPU that
// loads the library keeps the array (about 6 MB) until the process exits,
// and all calls share it, so calls that overlap on the GPU (other streams,
// other host threads) race and must be serialised by the caller.
// ---------------------------------------------------------------------------
#include <mutex>

#define RL0_STATIC_CHUNKS ((RL0_STATIC_MAX_M + RL0_ROWS_CHUNK - 1) / RL0_ROWS_CHUNK)
#define RL0_STATIC_ALIGN(x) (((x) + 255) & ~(size_t)255)

// Byte layout of the static workspace (each piece 256-byte aligned).
struct StaticLayout {
    size_t rz0, rz1, list, ulog, dlog, bcnt, bkt, sbcnt0, sbcnt1, sbkt0, sbkt1, l1part, final_part, hkkey, st, ctx, thr,
        rlog, total;
};

static constexpr StaticLayout static_layout()
{
    StaticLayout L{};
    size_t o = 0;
    L.rz0 = o; o += RL0_STATIC_ALIGN(sizeof(float2) * RL0_STATIC_MAX_M);
    L.rz1 = o; o += RL0_STATIC_ALIGN(sizeof(float2) * RL0_STATIC_MAX_M);
    L.list = o; o += RL0_STATIC_ALIGN(sizeof(int) * RL0_STATIC_MAX_N);
    L.ulog = o; o += RL0_STATIC_ALIGN(sizeof(UndoEntry) * RL0_STATIC_MAX_N);
    L.dlog = o; o += RL0_STATIC_ALIGN(sizeof(UndoEntry) * RL0_STATIC_MAX_N);
    L.bcnt = o; o += RL0_STATIC_ALIGN(sizeof(int) * RL0_STATIC_MAX_M);
    L.bkt = o; o += RL0_STATIC_ALIGN(sizeof(int) * RL0_STATIC_MAX_M * RL0_BUCKET);
    L.sbcnt0 = o; o += RL0_STATIC_ALIGN(sizeof(int) * RL0_STATIC_MAX_M);
    L.sbcnt1 = o; o += RL0_STATIC_ALIGN(sizeof(int) * RL0_STATIC_MAX_M);
    L.sbkt0 = o; o += RL0_STATIC_ALIGN(sizeof(int) * RL0_STATIC_MAX_M * RL0_BUCKET);
    L.sbkt1 = o; o += RL0_STATIC_ALIGN(sizeof(int) * RL0_STATIC_MAX_M * RL0_BUCKET);
    L.l1part = o; o += RL0_STATIC_ALIGN(sizeof(double) * RL0_STATIC_CHUNKS);
    L.final_part = o; o += RL0_STATIC_ALIGN(sizeof(double) * 2 * RL0_STATIC_CHUNKS);
    L.hkkey = o; o += RL0_STATIC_ALIGN(sizeof(unsigned long long) * RL0_STATIC_MAX_N);
    L.st = o; o += RL0_STATIC_ALIGN(sizeof(DecodeState));
    L.ctx = o; o += RL0_STATIC_ALIGN(sizeof(DecodeCtx));
    L.thr = o; o += RL0_STATIC_ALIGN(sizeof(RoundThr) * RL0_MAX_ROUNDS);
    L.rlog = o; o += RL0_STATIC_ALIGN(sizeof(RoundLog) * RL0_MAX_ROUNDS);
    L.total = o;
    return L;
}

static constexpr StaticLayout kStaticLayout = static_layout();

// The scratch array itself.  In host code this name is only a stand-in for
// the device object; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_rl0_static_scratch[kStaticLayout.total];

#define RL0_STATIC_MAX_DEVICES 64
static std::mutex g_static_mutex;
static void *g_static_base[RL0_STATIC_MAX_DEVICES];

// Device address of the scratch array on device `dev` (which must be current);
// looked up once per device, on the first call that runs there.
static int static_scratch_base(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= RL0_STATIC_MAX_DEVICES) return RL0_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rl0_static_scratch);
        if (e != cudaSuccess || !p) return rl0_cuda_err(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        g_static_base[dev] = p;
    }
    *out = (unsigned char *)g_static_base[dev];
    return RL0_OK;
}

extern "C" int rl0_decode_static(const rl0_expander *Ac, const float *y_dev, int64_t k, const rl0_params *params,
                                 float *xhat_dev, rl0_stats *stats, void *cuda_stream)
{
    rl0_expander *A = const_cast<rl0_expander *>(Ac);
    if (!A || !y_dev || !xhat_dev) return RL0_ERR_INVALID_ARG;
    if (A->n > RL0_STATIC_MAX_N || A->m > RL0_STATIC_MAX_M) return RL0_ERR_TOO_LARGE;
    int rc = rl0_set_device_of(A);
    if (rc) return rc;
    Resolved R;
    rc = rl0::resolve(A->n, A->m, A->d, k, params, &R);
    if (rc) return rc;
    if (R.p.adaptive_k || R.p.anchor_rule != 0) return RL0_ERR_UNSUPPORTED;
    unsigned char *base = nullptr;
    rc = static_scratch_base(A->device, &base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const StaticLayout &L = kStaticLayout;

    KArgs a = make_args(A);
    a.rz0 = (float2 *)(base + L.rz0);
    a.rz1 = (float2 *)(base + L.rz1);
    a.list = (int *)(base + L.list);
    a.ulog = (UndoEntry *)(base + L.ulog);
    a.dlog = (UndoEntry *)(base + L.dlog);
    a.bcnt = (int *)(base + L.bcnt);
    a.bkt = (int *)(base + L.bkt);
    a.sbcnt0 = (int *)(base + L.sbcnt0);
    a.sbcnt1 = (int *)(base + L.sbcnt1);
    a.sbkt0 = (int *)(base + L.sbkt0);
    a.sbkt1 = (int *)(base + L.sbkt1);
    a.l1part = (double *)(base + L.l1part);
    a.final_part = (double *)(base + L.final_part);
    a.hkkey = (unsigned long long *)(base + L.hkkey);
    a.st = (DecodeState *)(base + L.st);
    a.ctx = (DecodeCtx *)(base + L.ctx);
    a.thr = (const RoundThr *)(base + L.thr);
    a.rlog = (RoundLog *)(base + L.rlog);
    a.code0 = a.code1 = nullptr;                  // no residual codes: the L2 column kernel
    a.pzlb = nullptr;
    a.res_list = nullptr;
    a.res_ok = 0;

    // Per-call tables go through the expander's pinned staging block, which was
    // set up when the expander was created.
    HostStage *H = (HostStage *)A->host_pinned;
    rl0::fill_tables(A->m, A->d, k, R, &H->ctx, H->thr, R.nrounds);
    H->ctx.y = y_dev;
    H->ctx.x = xhat_dev;
    H->ctx.want_log = 0;
    H->ctx.passed = nullptr;
    CK(cudaMemcpyAsync(base + L.ctx, &H->ctx, sizeof(DecodeCtx), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(base + L.thr, H->thr, R.nrounds * sizeof(RoundThr), cudaMemcpyHostToDevice, s));
    // the array keeps the last call's contents: clear what must start at zero
    CK(cudaMemsetAsync(base + L.st, 0, sizeof(DecodeState), s));
    CK(cudaMemsetAsync(base + L.bcnt, 0, sizeof(int) * (size_t)A->m, s));

    const int dmax = dmax_of(A->d);
    k_rows_from<<<a.nchunks, RL0_ROWS_CHUNK, 0, s>>>(a, nullptr, 0, 1);
    k_start<<<1, 32, 0, s>>>(a, 0, 1);
    for (int r = 0; r < R.nrounds; ++r) {
        launch_round(a, dmax, R.indicator, R.p.scorer == 1, s);
    }
    k_final_sum<<<1, 32, 0, s>>>(a);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&H->st, base + L.st, sizeof(DecodeState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    A->last_log_rounds = 0;                       // this decode keeps no round log
    if (H->st.status == RL0_ERR_INVALID_Y) return RL0_ERR_INVALID_Y;
    const DecodeState first = H->st;
    int launches = launches_unrolled(R.nrounds, kernels_per_round(a, R.p.scorer == 1)) + 1;   // and k_final_sum
    int cont = 0;
    if (!first.status && R.p.scorer == 1 && !(first.l1_hat <= R.keep_level)) {
        // as rl0_decode: the learned result's residual is not noise-like, so
        // Alg. 2 with the analytic scores continues from its x_hat (the L2
        // column kernel here: the static array holds no residual codes)
        int nl = 0;
        rc = launch_analytic_continuation(A, a, k, R, y_dev, xhat_dev, &nl, s);
        if (rc) return rc;
        launches += nl;
        CK(cudaMemcpyAsync(&H->st, base + L.st, sizeof(DecodeState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        cont = 1;
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->rounds = (cont ? first.rounds_run : 0) + H->st.rounds_run;
        stats->accepted_rounds = (cont ? first.accepted_rounds : 0) + H->st.accepted_rounds;
        stats->converged = H->st.converged;
        stats->status = H->st.status;
        stats->support_size = H->st.nnz;
        stats->final_l1 = H->st.final_l1;
        stats->hk_rounds = (cont ? first.hk_rounds : 0) + H->st.hk_rounds;
        stats->fallback_rounds = (cont ? first.fallback_rounds : 0) + H->st.fallback_rounds;
        stats->launches = launches;
        stats->analytic_rounds = cont ? H->st.rounds_run : 0;
        stats->skipped_rounds = (cont ? first.skipped : 0) + H->st.skipped;
    }
    if (H->st.status) return H->st.status < 0 ? H->st.status : RL0_ERR_TIMEOUT;
    return RL0_OK;
}

extern "C" int rl0_candidate_features(const rl0_expander *Ac, const float *y_dev, int64_t k, const rl0_params *params,
                                      int round_index, const float *xhat_dev, const float *rhat_dev, float *feat_dev,
                                      int32_t *meta_dev, float *omega_dev, int cap, int *count_out, void *cuda_stream)
{
    rl0_expander *A = const_cast<rl0_expander *>(Ac);
    if (!A || !y_dev || !xhat_dev || !rhat_dev || !feat_dev || !meta_dev || !omega_dev || !count_out || cap < 0 ||
        round_index < 0 || round_index >= RL0_MAX_ROUNDS)
        return RL0_ERR_INVALID_ARG;
    if (A->d > 16) return RL0_ERR_UNSUPPORTED;
    int rc = rl0_set_device_of(A);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Resolved R;
    rc = rl0::resolve(A->n, A->m, A->d, k, params, &R);
    if (rc) return rc;
    if (!(R.p.sigma_n > 0.0)) return RL0_ERR_INVALID_ARG;
    R.nrounds = round_index + 1;
    HostStage *H = (HostStage *)A->host_pinned;
    rl0::fill_tables(A->m, A->d, k, R, &H->ctx, H->thr, R.nrounds);
    H->ctx.y = y_dev;
    H->ctx.x = const_cast<float *>(xhat_dev);
    H->ctx.want_log = 0;
    H->ctx.passed = nullptr;
    const Workspace &w = A->ws;
    CK(cudaMemcpyAsync(w.ctx, &H->ctx, sizeof(DecodeCtx), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.thr, H->thr, R.nrounds * sizeof(RoundThr), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(w.st, 0, sizeof(DecodeState), s));
    int *cnt = (int *)w.list_tmp;
    int *bbase = w.res_list;                       // free outside the column kernel; capacity >= n
    const KArgs a = make_args(A);
    k_rows_from<<<a.nchunks, RL0_ROWS_CHUNK, 0, s>>>(a, rhat_dev, 0, 0);
    k_start<<<1, 32, 0, s>>>(a, round_index, 0);
    for (int pass = 0; pass < 2; ++pass) {
        if (A->d <= 8) {
            const unsigned nb = rl0_div_up(a.n, 256);
            if (R.indicator) k_collect<8, true><<<nb, 256, 0, s>>>(a, feat_dev, meta_dev, omega_dev, cap, bbase, pass);
            else k_collect<8, false><<<nb, 256, 0, s>>>(a, feat_dev, meta_dev, omega_dev, cap, bbase, pass);
            if (pass == 0) k_collect_scan<<<1, 1024, 0, s>>>(bbase, (int)nb, cnt);
        } else {
            const unsigned nb = rl0_div_up(a.n, 128);
            if (R.indicator) k_collect<16, true><<<nb, 128, 0, s>>>(a, feat_dev, meta_dev, omega_dev, cap, bbase, pass);
            else k_collect<16, false><<<nb, 128, 0, s>>>(a, feat_dev, meta_dev, omega_dev, cap, bbase, pass);
            if (pass == 0) k_collect_scan<<<1, 1024, 0, s>>>(bbase, (int)nb, cnt);
        }
    }
    CK(cudaGetLastError());
    int c = 0;
    CK(cudaMemcpyAsync(&c, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *count_out = c;
    return RL0_OK;
}
