// rl0_round.cuh -- pieces of one Robust-l0 round (arXiv 1704.09012,
// Algorithm 2) shared by the translation units that launch round kernels:
// the kernel argument block, a column's commit, the last-CTA ticket and the
// H_k step run by the column kernel's last CTA, the scatter and the per-row
// rebuild, and the accept step run by the rebuild's last CTA.  Not part of
// the ABI.
#pragma once

#include "rl0_common.cuh"
#include "rl0_device.cuh"

// Fixed pointers and sizes of one expander's decode, passed by value.
struct KArgs {
    int n, m, d, nchunks, nsm;
    const int32_t *rows_sm, *rows_cm, *rowptr, *colidx;
    float2 *rz0, *rz1;
    unsigned short *code0, *code1;     // residual codes beside rz0 / rz1 (written when res_ok)
    const float *pzlb;                 // p_z lower bound per code bin
    int res_ok;                        // the column kernel holds every row's code in shared memory
    int res_grid;                      // its CTAs (one per SM)
    unsigned res_pz_off, res_s_off, res_q_off, res_smem;   // its dynamic shared-memory layout
    int res_qcap;                      // survivors per CTA staged in shared memory (FP32 residuals and x_j)
    int *res_list;                     // its other survivors: n entries of (j, candidate mask, DMAX row ids);
                                       // CTA b uses its column range
    int *list;
    UndoEntry *ulog, *dlog;
    int *bcnt, *bkt;
    double *l1part;
    unsigned long long *hkkey;
    DecodeState *st;
    DecodeCtx *ctx;
    const RoundThr *thr;
    RoundLog *rlog;
    double *final_part;
    cudaGraphConditionalHandle cond;   // while-loop condition of the round graph
    int has_cond;
};

// Column j's outcome: x_j += omega of its chosen anchor (best >= 0), with the
// undo log, the support list and the nonzero count kept in step.  Every lane
// of the warp calls it; the warp's leader takes its undo-log and list slots
// with two independent atomics.
__device__ __forceinline__ void commit_column(const KArgs &a, const DecodeCtx *ctx, int j, bool active, int best,
                                              float bw)
{
    const bool pass = best >= 0;
    float old = 0.0f, nv = 0.0f;
    if (pass) {
        float *x = ctx->x;
        old = x[j];
        nv = old + bw;
        x[j] = nv;
    }
    if (ctx->passed && active) ctx->passed[j] = pass ? 1 : 0;
    const int lane = threadIdx.x & 31;
    const unsigned mask = __ballot_sync(0xffffffffu, pass);
    if (mask) {
        const int leader = __ffs(mask) - 1;
        const int dn = __reduce_add_sync(0xffffffffu, pass ? (int)(nv != 0.0f) - (int)(old != 0.0f) : 0);
        const unsigned gone = __popc(__ballot_sync(0xffffffffu, pass && old != 0.0f && nv == 0.0f));
        const bool fresh = pass && old == 0.0f && nv != 0.0f;
        const unsigned fmask = __ballot_sync(0xffffffffu, fresh);
        unsigned base = 0, fbase = 0;
        if (lane == leader) {
            if (dn) atomicAdd(&a.st->nnz_delta, dn);
            if (gone) atomicAdd(&a.st->zeroed, gone);
            base = atomicAdd(&a.st->upd_count, (unsigned)__popc(mask));
            if (fmask) fbase = atomicAdd(&a.st->list_count, (unsigned)__popc(fmask));
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        fbase = __shfl_sync(0xffffffffu, fbase, leader);
        const unsigned below = (1u << lane) - 1u;
        if (pass) {
            UndoEntry e;
            e.j = j;
            e.old = old;
            a.ulog[base + __popc(mask & below)] = e;
        }
        if (fresh) a.list[fbase + __popc(fmask & below)] = j;
    }
}

// A CTA's ticket at the end of a launch: after the block barrier, thread 0
// adds one with release and acquire semantics at GPU scope, so the CTA's
// writes are visible to whichever CTA draws the last ticket, and that CTA
// (after its next block barrier) sees every other CTA's.  Returns the count
// before this CTA's ticket.
__device__ __forceinline__ unsigned cta_ticket(unsigned *ctr)
{
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
    return old;
}

// The launch's last CTA applies H_k when |supp x'| > k (state read past L1,
// since other CTAs updated it during this launch).  hk and suf are scratch of
// that CTA; *last is a shared flag.
template <int NT>
__device__ __forceinline__ void last_cta_hk(const KArgs &a, const DecodeCtx *ctx, HkShared &hk, unsigned *suf,
                                            int *last)
{
    __syncthreads();
    if (threadIdx.x == 0) *last = (cta_ticket(&a.st->col_done) == gridDim.x - 1u);
    __syncthreads();
    if (!*last) return;
    DecodeState *stw = a.st;
    const unsigned upd = __ldcg(&stw->upd_count);
    const long long nnz = (long long)__ldcg(&stw->nnz) + __ldcg(&stw->nnz_delta);
    if (threadIdx.x == 0) stw->col_done = 0u;
    if (upd == 0 || nnz <= ctx->k || __ldcg(&stw->status) != 0) return;
    cta_hk_select<NT>(a.list, __ldcg(&stw->list_count), ctx->x, ctx->k, a.hkkey, a.dlog, &stw->drop_count, hk, suf);
}

// ---------------------------------------------------------------------------
// Scatter: the support's (row, column) pairs into per-row buckets, work items
// w = e d + s (support entry e, slot s) from w0 in steps of ws.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void scatter_items(const KArgs &a, unsigned total, long long w0, long long ws)
{
    const float *x = a.ctx->x;
    const int d = a.d;
    const long long work = (long long)total * d;
    for (long long w = w0; w < work; w += ws) {
        const unsigned e = (unsigned)(w / d);
        const int s = (int)(w % d);
        const int j = a.list[e];
        // x_j and the row id in one L2 trip; entries that became zero add nothing
        const float xj = x[j];
        const int row = a.rows_cm[(long long)j * d + s];
        if (xj == 0.0f) continue;
        const int slot = atomicAdd(&a.bcnt[row], 1);
        if (slot < RL0_BUCKET) a.bkt[(long long)row * RL0_BUCKET + slot] = j;
        else a.st->overflow = 1;
    }
}

// A row's inputs to the rebuild that do not depend on the decode state: its
// bucket count, the bucket's 8 slots and y_i (loaded side by side, one L2 trip).
struct RowIn {
    int c;
    int4 b0, b1;
    float y;
};

__device__ __forceinline__ RowIn load_row_inputs(const KArgs &a, const DecodeCtx *ctx, int i)
{
    RowIn in;
    in.c = a.bcnt[i];
    const int4 *bq = (const int4 *)(a.bkt + (long long)i * RL0_BUCKET);
    in.b0 = bq[0];
    in.b1 = bq[1];
    in.y = ctx->y[i];
    return in;
}

// ---------------------------------------------------------------------------
// Rebuild of R rows i[0..R) (has[r]: row r exists): r_i = y_i - sum of x_j
// over the row in ascending j (FP32), the same sum in FP32 pairs for the final
// residual check, p_z(r_i) and the residual code into the candidate buffer
// (cur: the accepted one); l1 = |r_i|, f1 = |that pair sum|.  Every row's
// loads are issued before any row's stores, so R rows cost one chain of L2
// trips; pre, if not null, holds the rows' inputs already loaded.  csr: a
// bucket overflowed, take the rows from CSR(A^T).
// ---------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ void rebuild_rows(const KArgs &a, const DecodeCtx *ctx, const int *i, const bool *has,
                                             bool csr, int cur, DF *l1, DF *f1, const RowIn *pre = nullptr)
{
    static_assert(RL0_BUCKET == 8, "sorting network is for 8 entries");
    const float *x = ctx->x;
    float2 *rz = cur ? a.rz0 : a.rz1;              // the candidate buffer
    float sum[R], yv[R];
    DF acc[R];
    if (csr) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            sum[r] = 0.0f;
            yv[r] = has[r] ? ctx->y[i[r]] : 0.0f;
            acc[r] = DF{yv[r], 0.0f};
            if (!has[r]) continue;
            for (int p = a.rowptr[i[r]]; p < a.rowptr[i[r] + 1]; ++p) {
                const float xv = x[a.colidx[p]];
                sum[r] += xv;
                acc[r] = df_sub(acc[r], xv);
            }
            a.bcnt[i[r]] = 0;
        }
    } else {
        // each row's count and all 8 slots side by side (one L2 trip); slots
        // past the count are ignored
        int c[R], js[R][RL0_BUCKET];
        float xv[R][RL0_BUCKET];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            c[r] = 0;
            yv[r] = 0.0f;
            int4 b0 = make_int4(0, 0, 0, 0), b1 = b0;
            if (has[r]) {
                const RowIn in = pre ? pre[r] : load_row_inputs(a, ctx, i[r]);
                c[r] = in.c;
                b0 = in.b0;
                b1 = in.b1;
                yv[r] = in.y;
            }
            const int raw[RL0_BUCKET] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int q = 0; q < RL0_BUCKET; ++q) js[r][q] = (q < c[r]) ? raw[q] : 0x7fffffff;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (c[r] > 1) sort8(js[r]);             // ascending column order
#pragma unroll
            for (int q = 0; q < RL0_BUCKET; ++q) xv[r][q] = (q < c[r]) ? x[js[r][q]] : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            sum[r] = 0.0f;
            acc[r] = DF{yv[r], 0.0f};
#pragma unroll
            for (int q = 0; q < RL0_BUCKET; ++q)
                if (q < c[r]) {
                    sum[r] += xv[r][q];
                    acc[r] = df_sub(acc[r], xv[r][q]);
                }
            if (c[r] > 0) a.bcnt[i[r]] = 0;
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        l1[r] = DF{0.0f, 0.0f};
        f1[r] = DF{0.0f, 0.0f};
        if (!has[r]) continue;
        const float rr = yv[r] - sum[r];
        const float z = ctx->indicator ? 0.0f : series_eval(ctx->pz, rr);
        rz[i[r]] = make_float2(rr, z);
        if (a.res_ok) (cur ? a.code0 : a.code1)[i[r]] = residual_code(rr);
        l1[r] = DF{fabsf(rr), 0.0f};
        f1[r] = df_abs(acc[r]);
    }
}

__device__ __forceinline__ void rebuild_row(const KArgs &a, const DecodeCtx *ctx, int i, bool csr, int cur, DF &l1,
                                            DF &f1, const RowIn *pre = nullptr)
{
    const bool has = true;
    rebuild_rows<1>(a, ctx, &i, &has, csr, cur, &l1, &f1, pre);
}

// ---------------------------------------------------------------------------
// Accept / undo and round control, run by one CTA of NT threads: the rebuild's
// last CTA, or its CTA 0 when the round changed nothing.
// ---------------------------------------------------------------------------
template <int NT>
__device__ void accept_step(const KArgs &a, unsigned upd, unsigned *shu)
{
    // The state is read once into shared memory (warp 0, one word per lane,
    // through L2: other CTAs of this launch wrote to it), decided on there,
    // and written back once, so thread 0's decisions wait on no global loads.
    constexpr int SW = sizeof(DecodeState) / 4;
    static_assert(sizeof(DecodeState) % 4 == 0 && SW <= 32, "one word per lane of warp 0");
    __shared__ DecodeState S;
    __shared__ double s_l1;
    __shared__ int s_acc;
    DecodeState *st = a.st;
    const int t = threadIdx.x;
    const DecodeCtx *ctx = a.ctx;
    float *x = ctx->x;
    if (t < 32) {
        if (t < SW) ((unsigned *)&S)[t] = __ldcg((const unsigned *)st + t);
        double v = 0.0;
        // ||r||_1 of the candidate: chunk partials combined in a fixed order
        if (upd > 0) v = warp_sum_parts_l2(a.l1part, a.nchunks, t);
        __syncwarp();
        if (t == 0) {
            S.rb_done = 0u;                        // the rebuild's last-CTA count starts over
            s_l1 = v;
            s_acc = (upd > 0) ? (ctx->always_accept ? 1 : (v < S.l1_hat)) : 0;
        }
    }
    __syncthreads();
    if (upd > 0) {
        if (s_acc) {
            if (S.drop_count > 0 || S.zeroed > 0) {
                // entries became zero: stable in-place compaction of the list
                const unsigned total = S.list_count;
                unsigned out = 0;
                for (unsigned base = 0; base < total; base += NT) {
                    const unsigned e = base + t;
                    int j = -1;
                    unsigned keep = 0;
                    if (e < total) { j = a.list[e]; keep = (x[j] != 0.0f); }
                    shu[t] = keep;
                    __syncthreads();
                    for (int off = 1; off < NT; off <<= 1) {
                        const unsigned w = (t >= off) ? shu[t - off] : 0u;
                        __syncthreads();
                        shu[t] += w;
                        __syncthreads();
                    }
                    const unsigned incl = shu[t];
                    const unsigned blk = shu[NT - 1];
                    __syncthreads();
                    if (keep) a.list[out + incl - 1] = j;
                    out += blk;
                    __syncthreads();
                }
                if (t == 0) S.list_count = out;
            }
            if (t == 0) {
                S.shat_count = S.list_count;
                S.nnz = (unsigned)((int)S.nnz + S.nnz_delta - (int)S.drop_count);
                S.cur ^= 1;
                S.l1_hat = s_l1;
                S.accepted_rounds += 1;
            }
        } else {
            const unsigned nd = S.drop_count;
            for (unsigned e = t; e < nd; e += NT) x[a.dlog[e].j] = a.dlog[e].old;
            __syncthreads();
            for (unsigned e = t; e < upd; e += NT) x[a.ulog[e].j] = a.ulog[e].old;
            if (t == 0) S.list_count = S.shat_count;
        }
        __syncthreads();
    }
    if (t == 0) {
        const int round = S.round;
        const double l1n = (upd > 0) ? s_l1 : S.l1_hat;
        if (ctx->want_log && round < RL0_MAX_ROUNDS) {
            RoundLog L;
            L.l1_candidate = l1n;
            L.l1_hat = S.l1_hat;
            L.accepted = s_acc;
            L.updated = (int)upd;
            L.support = (int)S.nnz;
            L.hk_dropped = (int)S.drop_count;
            a.rlog[round] = L;
        }
        if (upd > 0 && S.drop_count > 0) S.hk_rounds += 1;
        if (upd > 0 && S.overflow) S.fallback_rounds += 1;
        S.upd_count = 0;
        S.drop_count = 0;
        S.overflow = 0;
        S.nnz_delta = 0;
        S.zeroed = 0;
        S.round = round + 1;
        S.rounds_run += 1;
        S.iters += 1;
        S.l1_new = l1n;
        if (ctx->always_accept) {
            // Alg. 1: every iteration is kept; it ends when one changes nothing
            if (upd > 0) S.big_hat = S.big_cand;
            S.converged = (S.big_hat == 0);
            if (upd == 0) S.done = 1;
        } else {
            S.converged = (S.l1_hat <= ctx->stop_level);
        }
        S.big_cand = 0;
        if (S.converged || S.round >= ctx->nrounds || S.iters > (unsigned)ctx->nrounds || S.status != 0)
            S.done = 1;
    }
    __syncthreads();
    if (S.done && t < 32) {
        // the decode ends here: ||y_hat - A x_hat||_1 from r_hat's chunk
        // partials, in k_final_sum's order
        const double v = warp_sum_parts_l2(a.final_part + (size_t)S.cur * a.nchunks, a.nchunks, t);
        if (t == 0) S.final_l1 = v;
        __syncwarp();
    }
    __syncthreads();
    if (t < SW) ((unsigned *)st)[t] = ((const unsigned *)&S)[t];
    if (t == 0 && a.has_cond) cudaGraphSetConditional(a.cond, S.done ? 0u : 1u);
}

// Column kernel with every row's residual code in shared memory
// (rl0_column_res.cu).  rl0_res_setup fills a's res_* fields for expander A
// (res_ok = 0 when the codes do not fit the device's shared memory or the
// workspace has no code buffers); rl0_res_launch launches it and returns false
// when a.res_ok is 0.
void rl0_res_setup(const rl0_expander *A, KArgs *a);
int rl0_res_dmax(int d);                     // slots per survivor-list entry for degree d
bool rl0_res_launch(const KArgs &a, int indicator, cudaStream_t s);
