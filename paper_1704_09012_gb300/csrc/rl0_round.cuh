// rl0_round.cuh -- pieces of one Robust-l0 round (arXiv 1704.09012,
// Algorithm 2) shared by the translation units that launch round kernels:
// the kernel argument block, a column's commit, and the H_k step run by the
// column kernel's last CTA.  Not part of the ABI.
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

// The launch's last CTA applies H_k when |supp x'| > k (state read past L1,
// since other CTAs updated it during this launch).  hk and suf are scratch of
// that CTA; *last is a shared flag.
template <int NT>
__device__ __forceinline__ void last_cta_hk(const KArgs &a, const DecodeCtx *ctx, HkShared &hk, unsigned *suf,
                                            int *last)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *last = (atomicAdd(&a.st->col_done, 1u) == gridDim.x - 1u);
    __syncthreads();
    if (!*last) return;
    __threadfence();
    DecodeState *stw = a.st;
    const unsigned upd = __ldcg(&stw->upd_count);
    const long long nnz = (long long)__ldcg(&stw->nnz) + __ldcg(&stw->nnz_delta);
    if (threadIdx.x == 0) stw->col_done = 0u;
    if (upd == 0 || nnz <= ctx->k || __ldcg(&stw->status) != 0) return;
    cta_hk_select<NT>(a.list, __ldcg(&stw->list_count), ctx->x, ctx->k, a.hkkey, a.dlog, &stw->drop_count, hk, suf);
}

// Column kernel with every row's residual code in shared memory
// (rl0_column_res.cu).  rl0_res_setup fills a's res_* fields for expander A
// (res_ok = 0 when the codes do not fit the device's shared memory or the
// workspace has no code buffers); rl0_res_launch launches it and returns false
// when a.res_ok is 0.
void rl0_res_setup(const rl0_expander *A, KArgs *a);
int rl0_res_dmax(int d);                     // slots per survivor-list entry for degree d
bool rl0_res_launch(const KArgs &a, int indicator, cudaStream_t s);
