// rl0_round.cuh -- pieces of one Robust-l0 round (arXiv 1704.09012,
// Algorithm 2) shared by the translation units that launch round kernels:
// the kernel argument block, a column's commit, the last-CTA ticket and the
// H_k step run by the column kernel's last CTA, the scatter and the per-row
// rebuild, and the accept step run by the rebuild's last CTA.  Not part of
// the ABI.
#pragma once

#include <cstddef>

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
    int *bcnt, *bkt;                   // fresh buckets F (see the rebuild's row buckets below)
    int *sbcnt0, *sbcnt1, *sbkt0, *sbkt1;   // support buckets B[0], B[1]
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

// ---------------------------------------------------------------------------
// Programmatic dependent launch between the round kernels.  A round kernel is
// launched so that it may start while the kernel before it on the stream is
// still running; before it touches anything that kernel writes it waits for
// that kernel's completion (griddepcontrol.wait, which also makes its writes
// visible), and only then lets the next kernel start early
// (griddepcontrol.launch_dependents).  So a kernel overlaps only the tail of
// its immediate predecessor, and what it reads before its wait (row ids, y,
// the support buckets of the previous round) no kernel still running writes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch of kernel k on stream s with programmatic stream serialization
// (errors are left for cudaGetLastError, as with <<< >>>).
template <typename... P, typename... A>
inline void launch_pdl(void (*k)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t s, A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

// Slots in the undo log (upd_count) and in the support list (list_count) for
// nupd updates and nfresh new nonzeros, taken with one 64-bit atomic on the
// two adjacent counters.  Returns the counters before: low word list_count,
// high word upd_count (list_count stays below 2^32, so no carry crosses).
__device__ __forceinline__ unsigned long long take_upd_list(DecodeState *st, unsigned nupd, unsigned nfresh)
{
    static_assert(offsetof(DecodeState, list_count) % 8 == 0 &&
                  offsetof(DecodeState, upd_count) == offsetof(DecodeState, list_count) + 4, "counter pair layout");
    return atomicAdd((unsigned long long *)&st->list_count, ((unsigned long long)nupd << 32) | nfresh);
}

// Column j, which became nonzero this round, into the fresh bucket of each of
// its d rows (RL0_BUCKET per row; a fuller row sets the overflow flag, and
// the rebuild then takes every row from CSR(A^T)), in two halves: the slots
// (d <= DM atomics, issued before any store, so they overlap) and the stores.
template <int DM>
__device__ __forceinline__ void bucket_slots(const KArgs &a, const int *rid, int d, int *slot)
{
#pragma unroll
    for (int s = 0; s < DM; ++s) slot[s] = (s < d) ? atomicAdd(&a.bcnt[rid[s]], 1) : 0;
}

template <int DM>
__device__ __forceinline__ void bucket_store(const KArgs &a, int j, const int *rid, int d, const int *slot)
{
#pragma unroll
    for (int s = 0; s < DM; ++s)
        if (s < d) {
            if (slot[s] < RL0_BUCKET) a.bkt[(long long)rid[s] * RL0_BUCKET + slot[s]] = j;
            else a.st->overflow = 1;
        }
}

template <int DM>
__device__ __forceinline__ void bucket_column(const KArgs &a, int j, const int *rid, int d)
{
    int slot[DM];
    bucket_slots<DM>(a, rid, d, slot);
    bucket_store<DM>(a, j, rid, d, slot);
}

// Column j's outcome: x_j += omega of its chosen anchor (best >= 0), with the
// undo log, the support list and the nonzero count kept in step.  Every lane
// of the warp calls it; the warp's leader takes its undo-log and list slots
// with one atomic (take_upd_list).
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
        // d <= 8: a fresh column's row ids and bucket slots, before (and so in
        // flight with) the leader's atomic below
        int rid[8], slot[8];
        const bool early = fresh && a.d <= 8;
        if (early) {
#pragma unroll
            for (int q = 0; q < 8; ++q) rid[q] = (q < a.d) ? __ldg(a.rows_sm + (size_t)q * a.n + j) : 0;
            bucket_slots<8>(a, rid, a.d, slot);
        }
        unsigned base = 0, fbase = 0;
        if (lane == leader) {
            if (dn) atomicAdd(&a.st->nnz_delta, dn);
            if (gone) atomicAdd(&a.st->zeroed, gone);
            const unsigned long long old2 = take_upd_list(a.st, (unsigned)__popc(mask), (unsigned)__popc(fmask));
            base = (unsigned)(old2 >> 32);
            fbase = (unsigned)old2;
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
        if (early) {
            a.list[fbase + __popc(fmask & below)] = j;
            bucket_store<8>(a, j, rid, a.d, slot);
        } else if (fresh) {
            a.list[fbase + __popc(fmask & below)] = j;
            // into the rebuild's fresh buckets, up to 8 rows at a time
            for (int s0 = 0; s0 < a.d; s0 += 8) {
                int rid[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) rid[q] = (s0 + q < a.d) ? __ldg(a.rows_sm + (size_t)(s0 + q) * a.n + j) : 0;
                bucket_column<8>(a, j, rid, min(8, a.d - s0));
            }
        }
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

// The resident-code kernel's ticket: one acquire-release atomic per CTA adds 1
// to the CTA count (bits 48..63 of DecodeState::tick) and the CTA's change of
// the nonzero count plus 2^31 to bits 0..47 (at most 2^16 CTAs, so the biased
// sum stays below 2^47), so that the last CTA learns |supp x'| = nnz0 + the
// changes from the atomic's own return value and reads more state only when
// H_k has to run.  That CTA stores the round's change in nnz_delta (read by the
// accept step) and clears the ticket.  nnz0: |supp x_hat| at the round's start.
#define RL0_TICK_BIAS (1ull << 31)

__device__ __forceinline__ unsigned long long cta_ticket64(unsigned long long *ctr, unsigned long long add)
{
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(ctr), "l"(add) : "memory");
    return old;
}

template <int NT>
__device__ __forceinline__ void last_cta_hk_tick(const KArgs &a, const DecodeCtx *ctx, HkShared &hk, unsigned *suf,
                                                 int *go, int cta_dn, unsigned nnz0)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long k = ctx->k;                 // loaded before the ticket's round trip
        const unsigned long long mine = (1ull << 48) + (unsigned long long)((long long)cta_dn + (long long)RL0_TICK_BIAS);
        const unsigned long long v = cta_ticket64(&a.st->tick, mine) + mine;
        int run = 0;
        if ((unsigned)(v >> 48) == gridDim.x) {
            DecodeState *stw = a.st;
            const long long dn = (long long)(v & ((1ull << 48) - 1ull)) - (long long)gridDim.x * (long long)RL0_TICK_BIAS;
            stw->tick = 0ull;
            stw->nnz_delta = (int)dn;
            run = ((long long)nnz0 + dn > k) && __ldcg(&stw->upd_count) != 0u && __ldcg(&stw->status) == 0;
        }
        *go = run;
    }
    __syncthreads();
    if (!*go) return;
    cta_hk_select<NT>(a.list, __ldcg(&a.st->list_count), ctx->x, ctx->k, a.hkkey, a.dlog, &a.st->drop_count, hk, suf);
}

// ---------------------------------------------------------------------------
// The rebuild's row buckets.  Row i's contributors to r = y - A x' are kept in
// two kinds of buckets of RL0_BUCKET column ids:
//   support  B[b] (sbcnt_b, sbkt_b), b = 0, 1: the columns j of row i with
//            x_hat_j != 0, for the x_hat whose residual is in rz[b] (so B[cur]
//            describes r_hat); the rebuild writes B[cur ^ 1] for the candidate
//            x', and accepting the round (cur ^= 1) makes it current;
//   fresh    F (bcnt, bkt): columns that became nonzero this round, added by
//            the column kernel as they commit; the rebuild empties it.
// A support bucket that would need more than RL0_BUCKET entries sets bit b of
// DecodeState::bflags (bucket b incomplete), a full fresh bucket sets
// DecodeState::overflow, and either makes the rebuild take every row from
// CSR(A^T).  Columns that H_k or an update set to zero stay in the buckets
// until the next compaction and add an exact 0 to the sums.
// ---------------------------------------------------------------------------

// x_hat's support (list[0, total)) into B[0], which must be empty: work items
// w = e d + s (support entry e, slot s) from w0 in steps of ws.  Used where a
// decode starts from an injected x_hat.
__device__ __forceinline__ void bucket_support_items(const KArgs &a, unsigned total, long long w0, long long ws)
{
    const int d = a.d;
    const long long work = (long long)total * d;
    for (long long w = w0; w < work; w += ws) {
        const unsigned e = (unsigned)(w / d);
        const int s = (int)(w % d);
        const int j = a.list[e];
        const int row = a.rows_cm[(long long)j * d + s];
        const int slot = atomicAdd(&a.sbcnt0[row], 1);
        if (slot < RL0_BUCKET) a.sbkt0[(long long)row * RL0_BUCKET + slot] = j;
        else atomicOr(&a.st->bflags, 1u);
    }
}

// A row's inputs to the rebuild: both support buckets, the fresh bucket and
// y_i (both support buckets are loaded before the state says which one is
// current, so that the loads do not wait on the state).
struct RowIn {
    int c0, c1, cf;
    int4 b00, b01, b10, b11, f0, f1;
    float y;
};

// The inputs no kernel of this round writes (y_i and both support buckets):
// loaded before the rebuild waits for the column kernel.
__device__ __forceinline__ void load_row_support(const KArgs &a, const DecodeCtx *ctx, int i, RowIn &in)
{
    in.c0 = a.sbcnt0[i];
    in.c1 = a.sbcnt1[i];
    const int4 *q0 = (const int4 *)(a.sbkt0 + (long long)i * RL0_BUCKET);
    const int4 *q1 = (const int4 *)(a.sbkt1 + (long long)i * RL0_BUCKET);
    in.b00 = q0[0];
    in.b01 = q0[1];
    in.b10 = q1[0];
    in.b11 = q1[1];
    in.y = ctx->y[i];
}

// The fresh bucket, written by this round's column kernel.
__device__ __forceinline__ void load_row_fresh(const KArgs &a, int i, RowIn &in)
{
    in.cf = a.bcnt[i];
    const int4 *qf = (const int4 *)(a.bkt + (long long)i * RL0_BUCKET);
    in.f0 = qf[0];
    in.f1 = qf[1];
}

// Merge of two ascending runs js[0..8) and js[8..16) into one ascending run of
// 16 (the second run reversed makes the sequence bitonic; then Batcher's
// half-cleaners at strides 8, 4, 2, 1).
#define RL0_CSWAP16(i, j) { const int lo_ = min(js[i], js[j]), hi_ = max(js[i], js[j]); js[i] = lo_; js[j] = hi_; }
__device__ __forceinline__ void merge8x2(int *js)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) { const int t = js[8 + q]; js[8 + q] = js[15 - q]; js[15 - q] = t; }
#pragma unroll
    for (int st = 8; st >= 1; st >>= 1) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if ((q & st) == 0) RL0_CSWAP16(q, q + st)
    }
}
#undef RL0_CSWAP16

// ---------------------------------------------------------------------------
// Row i of the candidate: r_i = y_i - sum of x'_j over the row in ascending j
// (FP32), the same sum in FP32 pairs for the final residual check, p_z(r_i)
// and the residual code into the candidate buffer (cur: the accepted one);
// l1 = |r_i|, f1 = |that pair sum|.  The contributors are the support bucket
// B[cur] and the fresh bucket merged into ascending order, or, when csr is
// set, the row of CSR(A^T).  The row's entries with x'_j != 0 become the
// candidate's support bucket B[cur ^ 1]; returns false when they do not fit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool rebuild_row(const KArgs &a, const DecodeCtx *ctx, int i, bool csr, int cur, DF &l1,
                                            DF &f1, const RowIn &in)
{
    static_assert(RL0_BUCKET == 8, "sorting networks are for 8 entries");
    const float *x = ctx->x;
    float2 *rz = cur ? a.rz0 : a.rz1;              // the candidate buffer
    int *ncnt = cur ? a.sbcnt0 : a.sbcnt1;         // the candidate's support bucket
    int *nbkt = (cur ? a.sbkt0 : a.sbkt1) + (long long)i * RL0_BUCKET;
    float sum = 0.0f;
    DF acc{in.y, 0.0f};
    int kept = 0;
    if (csr) {
        for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) {
            const int j = a.colidx[p];
            const float xv = x[j];
            sum += xv;
            acc = df_sub(acc, xv);
            if (xv != 0.0f) {
                if (kept < RL0_BUCKET) nbkt[kept] = j;
                ++kept;
            }
        }
        if (in.cf != 0) a.bcnt[i] = 0;
    } else {
        const int cb = cur ? in.c1 : in.c0;
        const int4 b0 = cur ? in.b10 : in.b00, b1 = cur ? in.b11 : in.b01;
        const int rb[RL0_BUCKET] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
        const int rf[RL0_BUCKET] = {in.f0.x, in.f0.y, in.f0.z, in.f0.w, in.f1.x, in.f1.y, in.f1.z, in.f1.w};
        int js[2 * RL0_BUCKET];
#pragma unroll
        for (int q = 0; q < RL0_BUCKET; ++q) {
            js[q] = (q < cb) ? rb[q] : 0x7fffffff;
            js[RL0_BUCKET + q] = (q < in.cf) ? rf[q] : 0x7fffffff;
        }
        if (cb > 1) sort8(js);                      // ascending column order
        if (in.cf > 0) {
            if (in.cf > 1) sort8(js + RL0_BUCKET);
            merge8x2(js);
        }
        float xv[2 * RL0_BUCKET];
#pragma unroll
        for (int q = 0; q < 2 * RL0_BUCKET; ++q) xv[q] = (js[q] != 0x7fffffff) ? x[js[q]] : 0.0f;
#pragma unroll
        for (int q = 0; q < 2 * RL0_BUCKET; ++q)
            if (js[q] != 0x7fffffff) {
                sum += xv[q];
                acc = df_sub(acc, xv[q]);
                if (xv[q] != 0.0f) {
                    if (kept < RL0_BUCKET) nbkt[kept] = js[q];
                    ++kept;
                }
            }
        if (in.cf != 0) a.bcnt[i] = 0;
    }
    ncnt[i] = kept < RL0_BUCKET ? kept : RL0_BUCKET;
    const float rr = in.y - sum;
    const float z = ctx->indicator ? 0.0f : series_eval(ctx->pz, rr);
    rz[i] = make_float2(rr, z);
    if (a.res_ok) (cur ? a.code0 : a.code1)[i] = residual_code(rr);
    l1 = DF{fabsf(rr), 0.0f};
    f1 = df_abs(acc);
    return kept <= RL0_BUCKET;
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
    __shared__ double s_parts[4 * NT];
    DecodeState *st = a.st;
    const int t = threadIdx.x;
    const DecodeCtx *ctx = a.ctx;
    float *x = ctx->x;
    if (t < SW) ((unsigned *)&S)[t] = __ldcg((const unsigned *)st + t);
    // the per-call settings thread 0 decides with, loaded beside the state
    // words (read later, after stores to global memory, each would be a
    // dependent L2 trip of its own)
    int c_always = 0, c_log = 0, c_nrounds = 0;
    double c_stop = 0.0;
    if (t == 0) {
        c_always = ctx->always_accept;
        c_log = ctx->want_log;
        c_nrounds = ctx->nrounds;
        c_stop = ctx->stop_level;
    }
    // ||r||_1 of the candidate: chunk partials combined in a fixed order
    const double v = (upd > 0) ? cta_sum_parts_l2<NT>(a.l1part, a.nchunks, s_parts) : 0.0;
    __syncthreads();
    if (t == 0) {
        S.rb_done = 0u;                            // the rebuild's last-CTA count starts over
        s_l1 = v;
        s_acc = (upd > 0) ? (c_always ? 1 : (v < S.l1_hat)) : 0;
    }
    __syncthreads();
    const int cur0 = S.cur;                        // r_hat's buffer during this round
    if (upd > 0) {
        if (s_acc) {
            if (S.drop_count > 0 || S.zeroed > 0) {
                // entries became zero: stable in-place compaction of the list,
                // 4 NT entries at a time (each thread 4 consecutive ones; a warp
                // scan of the per-thread counts, then one over the warps).
                // Reading block b and writing its survivors below position
                // 4 NT b cannot overwrite an unread entry.
                constexpr int NW = NT / 32;
                unsigned *wsum = shu;                 // NW words of scratch
                const unsigned total = S.list_count;
                const int lane = t & 31, warp = t >> 5;
                unsigned out = 0;
                for (unsigned base = 0; base < total; base += 4 * NT) {
                    int j[4];
                    unsigned keep = 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const unsigned e = base + 4 * t + q;
                        j[q] = (e < total) ? __ldcg(a.list + e) : -1;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (j[q] >= 0 && __ldcg(x + j[q]) != 0.0f) keep |= 1u << q;
                    const unsigned cnt = __popc(keep);
                    unsigned incl = cnt;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned w = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += w;
                    }
                    if (lane == 31) wsum[warp] = incl;
                    __syncthreads();
                    unsigned before = 0, blk = 0;
                    for (int w = 0; w < NW; ++w) {
                        const unsigned sw = wsum[w];
                        if (w < warp) before += sw;
                        blk += sw;
                    }
                    unsigned pos = out + before + incl - cnt;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if ((keep >> q) & 1u) a.list[pos++] = j[q];
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
        if (c_log && round < RL0_MAX_ROUNDS) {
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
        if (upd > 0 && (S.overflow || ((S.bflags >> cur0) & 1u))) S.fallback_rounds += 1;
        // the next round's candidate support bucket starts out complete
        S.bflags &= ~(1u << (S.cur ^ 1));
        S.upd_count = 0;
        S.drop_count = 0;
        S.overflow = 0;
        S.nnz_delta = 0;
        S.zeroed = 0;
        S.round = round + 1;
        S.rounds_run += 1;
        S.iters += 1;
        S.l1_new = l1n;
        if (c_always) {
            // Alg. 1: every iteration is kept; it ends when one changes nothing
            if (upd > 0) S.big_hat = S.big_cand;
            S.converged = (S.big_hat == 0);
            if (upd == 0) S.done = 1;
        } else {
            S.converged = (S.l1_hat <= c_stop);
        }
        S.big_cand = 0;
        if (S.converged || S.round >= c_nrounds || S.iters > (unsigned)c_nrounds || S.status != 0)
            S.done = 1;
    }
    __syncthreads();
    if (S.done) {
        // the decode ends here: ||y_hat - A x_hat||_1 from r_hat's chunk
        // partials, in k_final_sum's order
        const double fv = cta_sum_parts_l2<NT>(a.final_part + (size_t)S.cur * a.nchunks, a.nchunks, s_parts);
        if (t == 0) S.final_l1 = fv;
    }
    __syncthreads();
    if (t < SW) ((unsigned *)st)[t] = ((const unsigned *)&S)[t];
    if (t == 0 && a.has_cond) cudaGraphSetConditional(a.cond, S.done ? 0u : 1u);
}

// Column kernel with every row's residual code in shared memory
// (rl0_column_res.cu).  rl0_res_setup fills a's res_* fields for expander A
// (res_ok = 0 when the codes do not fit the device's shared memory or the
// workspace has no code buffers); rl0_res_launch launches it (the learned
// scorer's variant when learned is set) and returns false when a.res_ok is 0.
void rl0_res_setup(const rl0_expander *A, KArgs *a);
int rl0_res_dmax(int d);                     // slots per survivor-list entry for degree d
bool rl0_res_launch(const KArgs &a, int indicator, int learned, cudaStream_t s);
