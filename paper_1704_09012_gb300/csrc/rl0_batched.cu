// rl0_batched.cu -- many independent Robust-l0 decodes (arXiv 1704.09012,
// Algorithm 2) in one persistent launch.
//
// One CTA decodes one instance at a time and pulls the next instance from an
// atomic work queue (instances ordered by decreasing work).  The instance's
// residual r_hat and p_z(r_hat) live in shared memory for the whole decode, so
// the d gathers of every column hit shared memory instead of L2; the round loop
// runs inside the kernel with CTA barriers only (no grid-wide waits, nothing
// that can spin).  Every step uses the same device functions, summation trees
// and chunking as the single-instance kernels, so each instance's x_hat is
// bitwise what rl0_decode returns for it alone, whatever the schedule.
//
// Schedule: threads per CTA (NT) and CTAs per SM come from a small autotuner
// that times the candidates on a sample of the batch the first time a
// (max d, score kind, shared-memory bucket) combination is seen.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "rl0_common.cuh"
#include "rl0_device.cuh"

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return rl0_cuda_err(e_);   \
    } while (0)

#define RL0_BATCH_MAX_M 22528                       // rows held in shared memory (88 chunks)
#define RL0_BATCH_MAX_CHUNKS (RL0_BATCH_MAX_M / RL0_ROWS_CHUNK)
#define RL0_BATCH_QCAP 2048                         // queued columns held in shared memory

struct BatchItem {
    int n, m, d, nrounds, nchunks, indicator;
    long long k;
    float alpha;
    double stop_level, stop_rel;
    Series pz, pe;
    float pe_b1, pe_c1;                             // fast-path bound of q_e (see anchor_candidates)
    const RoundThr *thr;
    const int32_t *rows_sm, *rows_cm, *rowptr, *colidx;
    const float *y;
    float *x;
    float2 *rzc;                                    // candidate residual
    int *list;
    UndoEntry *ulog, *dlog;
    int *bcnt, *bkt;
    unsigned long long *hkkey;
    int *spill;                                     // queued columns beyond the shared queue: 2 ints each
};

struct BatchResult {
    int rounds, accepted_rounds, converged, status, hk_rounds, fallback_rounds;
    unsigned nnz;
    double l1_hat, final_l1;
};

struct BatchState {
    int item, done, round, converged, status, overflow, nq;
    int accepted_rounds, hk_rounds, fallback_rounds, rounds_run, nnz_delta, acc;
    unsigned upd, list_count, shat_count, drop_count, nnz, zeroed;
    double l1_hat, l1n, stop;
};

// The column bound of the single-instance column kernel (code_candidates2 in
// rl0_device.cuh: two columns side by side in the FP16 lanes of half2
// registers, every anchor and pair test taken on the residuals' 16-bit codes)
// for columns a and b of exactly D rows, with the codes formed from r_hat
// held in shared memory (code(r) = FP16(r) rounded toward zero; no clamp is
// needed for finite r, since rounding toward zero never overflows) and n_z
// exact: the p_z(r) values beside r_hat (0/1 scores: the count of |r| <= t_z)
// summed in slot order, so the count test needs no lower-bound table.
// Returns a superset of each column's anchors that pass Alg. 2's test.
template <int D, bool IND>
__device__ __forceinline__ void smem_candidates2(const float2 *s_rz, const int *ra, const int *rb, bool act_a,
                                                 bool act_b, const CodeThr2 &ct, float tz, unsigned &ma,
                                                 unsigned &mb)
{
    __half2 v[D];
    __half2 vmax = __float2half2_rn(0.0f);
    float nza = 0.0f, nzb = 0.0f;
#pragma unroll
    for (int s = 0; s < D; ++s) {
        const float2 pa = s_rz[ra[s]], pb = s_rz[rb[s]];
        v[s] = __halves2half2(__float2half_rz(pa.x), __float2half_rz(pb.x));
        vmax = __hmax2(vmax, __habs2(v[s]));
        nza += IND ? (fabsf(pa.x) <= tz ? 1.0f : 0.0f) : pa.y;
        nzb += IND ? (fabsf(pb.x) <= tz ? 1.0f : 0.0f) : pb.y;
    }
    ma = mb = 0u;
    const float va = __low2float(vmax), vb = __high2float(vmax);
    const float ta = __low2float(ct.ta);
    const bool any_a = act_a && va >= ta, any_b = act_b && vb >= ta;
    if (!(any_a || any_b)) return;
    const __half2 thr = __halves2half2(__float2half_ru(fmaf(va, ct.c1, ct.c0)), __float2half_ru(fmaf(vb, ct.c1, ct.c0)));
    __half2 cnt[D];
#pragma unroll
    for (int s = 0; s < D; ++s) cnt[s] = __float2half2_rn(0.0f);
#pragma unroll
    for (int s = 0; s < D; ++s) {
#pragma unroll
        for (int l = s + 1; l < D; ++l) {
            const __half2 q = __hle2(__habs2(__hsub2(v[s], v[l])), thr);
            cnt[s] = __hadd2(cnt[s], q);
            cnt[l] = __hadd2(cnt[l], q);
        }
    }
    // candidate: near count >= need - 1 + n_z (rounded up to FP16: the count is exact)
    const __half2 kneed = __halves2half2(__float2half_ru(ct.need1 + nza), __float2half_ru(ct.need1 + nzb));
    unsigned anc = 0u, acc = 0u;
#pragma unroll
    for (int s = 0; s < D; ++s) {
        const unsigned a = h2bits(__hge2(__habs2(v[s]), ct.ta)) & 0x04000400u;
        const unsigned c = h2bits(__hge2(cnt[s], kneed));
        anc |= a >> (10 - s);
        acc |= (a & c) >> (10 - s);
    }
    // a saturated code (|v| = 65504 stands for every larger |r|): no bound
    const unsigned fa = (va >= 65504.0f) ? anc : acc, fb = (vb >= 65504.0f) ? anc : acc;
    ma = any_a ? (fa & 0xffffu) : 0u;
    mb = any_b ? (fb >> 16) : 0u;
}

// Queue position q of a column that may pass: the shared queue, else the
// instance's spill list (at most one entry per column, so it never fills).
__device__ __forceinline__ void queue_push(int *qj, unsigned *qm, int *spill, int q, int j, unsigned mask)
{
    if (q < RL0_BATCH_QCAP) {
        qj[q] = j;
        qm[q] = mask;
    } else {
        spill[2 * (size_t)(q - RL0_BATCH_QCAP)] = j;
        spill[2 * (size_t)(q - RL0_BATCH_QCAP) + 1] = (int)mask;
    }
}

// __launch_bounds__(NT, 1): up to 65536/NT registers per thread.  With the
// compiler's default target the column loop's row-id prefetch spilled; with
// this bound no variant spills and a 2048-instance batch ran 19% faster.
template <int DMAX, bool IND, bool EXACT, int NT>
__global__ void __launch_bounds__(NT, 1) k_decode_batched(const BatchItem *__restrict__ items, BatchResult *results,
                                                       int count, int *queue)
{
    constexpr int G = NT / RL0_ROWS_CHUNK;          // 256-row chunk groups per CTA
    // exact d <= 8: two columns per thread per tile, bounded in FP16 lanes
    constexpr bool PAIRED = EXACT && DMAX <= 8;
    constexpr int CPT = PAIRED ? 2 : 1;             // columns per thread per tile
    extern __shared__ float2 s_rz[];                // r_hat, p_z(r_hat) of the current instance
    __shared__ BatchState S;
    __shared__ BatchItem I;
    __shared__ int s_qj[RL0_BATCH_QCAP];            // the round's queued columns
    __shared__ unsigned s_qm[RL0_BATCH_QCAP];       // and their candidate slots
    __shared__ unsigned s_scan[NT];
    __shared__ DF s_red[NT];
    __shared__ double s_parts[RL0_BATCH_MAX_CHUNKS];
    __shared__ double s_fpart[RL0_BATCH_MAX_CHUNKS];     // ||y - A x_hat||_1 chunk partials (FP32 pairs)
    __shared__ double s_fcand[RL0_BATCH_MAX_CHUNKS];     // the same for the candidate x'
    __shared__ DF s_red2[NT];
    __shared__ HkShared s_hk;
    __shared__ RoundThr s_th;

    const int tid = threadIdx.x, lane = tid & 31;
    const int grp = tid / RL0_ROWS_CHUNK, gl = tid % RL0_ROWS_CHUNK;

    for (;;) {
        if (tid == 0) S.item = atomicAdd(queue, 1);
        __syncthreads();
        const int it = S.item;
        if (it >= count) return;
        {   // descriptor -> shared memory, word by word
            const int *src = (const int *)(items + it);
            int *dst = (int *)&I;
            for (int w = tid; w < (int)(sizeof(BatchItem) / sizeof(int)); w += NT) dst[w] = src[w];
        }
        __syncthreads();
        const int n = I.n, m = I.m, d = I.d, nchunks = I.nchunks;
        float *x = I.x;

        // ---- start: x_hat = 0, r_hat = y_hat (Alg. 2), ||r_hat||_1 by chunks
        for (int j = tid; j < n; j += NT) x[j] = 0.0f;
        int bad = 0;
        for (int cb = 0; cb < nchunks; cb += G) {
            const int c = cb + grp, i = c * RL0_ROWS_CHUNK + gl;
            DF v{0.0f, 0.0f};
            if (c < nchunks && i < m) {
                const float r = I.y[i];
                bad |= !isfinite(r);
                s_rz[i] = make_float2(r, I.indicator ? 0.0f : series_eval(I.pz, r));
                v = DF{fabsf(r), 0.0f};
            }
            const double sum = group_sum_df(v, s_red + grp * RL0_ROWS_CHUNK, gl, RL0_ROWS_CHUNK);
            if (gl == 0 && c < nchunks) s_parts[c] = s_fpart[c] = sum;   // x_hat = 0: both are ||y||_1's
        }
        bad = __syncthreads_or(bad);
        // ||r_hat||_1 in k_start's order (lane-strided, then a butterfly)
        double l1w = 0.0;
        if (tid < 32) l1w = warp_sum_parts(s_parts, nchunks, lane);
        if (tid == 0) {
            const double l1 = l1w;
            S.l1_hat = l1;
            S.stop = (I.stop_rel > 0.0) ? I.stop_rel * l1 : I.stop_level;
            S.status = bad ? RL0_ERR_INVALID_Y : 0;
            S.converged = (l1 <= S.stop);
            S.done = bad || S.converged || I.nrounds <= 0;
            S.round = 0;
            S.upd = S.list_count = S.shat_count = S.drop_count = S.nnz = S.zeroed = 0;
            S.nnz_delta = S.overflow = 0;
            S.nq = 0;
            S.accepted_rounds = S.hk_rounds = S.fallback_rounds = S.rounds_run = 0;
        }
        __syncthreads();

        while (!S.done) {
            if (tid == 0) s_th = I.thr[S.round];
            __syncthreads();
            const RoundThr th = s_th;
            const float alpha = I.alpha;

            // ---- column scores.
            // Stream: each thread bounds its columns' anchors (smem_candidates2
            // for exact d <= 8, else anchor_candidates on the FP32 residuals)
            // and queues the columns that may pass (a few in a thousand: the
            // first RL0_BATCH_QCAP in shared memory, the rest in the
            // instance's spill list); the row ids of the next tile load while
            // a tile is bounded; no thread waits on another.
            // Resolve, once per round: one thread per queued column scores its
            // candidate slots exactly, highest first (score_anchor's arithmetic:
            // the first to pass is the last passing anchor in row order), and
            // commits.
            const CodeThr2 ct2 = code_thresholds2(code_thresholds(th.ta, th.tz, IND ? th.te : I.pe.cut),
                                                  IND ? alpha : alpha - 1e-3f);
            int nxa[DMAX], nxb[PAIRED ? DMAX : 1];
#pragma unroll
            for (int s = 0; s < DMAX; ++s) {
                nxa[s] = (s < d && tid < n) ? __ldg(I.rows_sm + (size_t)s * n + tid) : 0;
                if constexpr (PAIRED) nxb[s] = (tid + NT < n) ? __ldg(I.rows_sm + (size_t)s * n + tid + NT) : 0;
            }
            {
                for (int base = 0; base < n; base += NT * CPT) {
                    const int ja = base + tid, jb = ja + NT;
                    int ra[DMAX], rb[PAIRED ? DMAX : 1];
#pragma unroll
                    for (int s = 0; s < DMAX; ++s) {
                        ra[s] = nxa[s];
                        if constexpr (PAIRED) rb[s] = nxb[s];
                    }
                    {
                        const int jn = base + NT * CPT + tid;
#pragma unroll
                        for (int s = 0; s < DMAX; ++s) {
                            if (s < d && jn < n) nxa[s] = __ldg(I.rows_sm + (size_t)s * n + jn);
                            if constexpr (PAIRED)
                                if (jn + NT < n) nxb[s] = __ldg(I.rows_sm + (size_t)s * n + jn + NT);
                        }
                    }
                    unsigned ma = 0u, mb = 0u;
                    if constexpr (PAIRED) {
                        smem_candidates2<DMAX, IND>(s_rz, ra, rb, ja < n, jb < n, ct2, th.tz, ma, mb);
                    } else if (ja < n) {
                        float r[DMAX];
                        float nz = 0.0f;
#pragma unroll
                        for (int s = 0; s < DMAX; ++s) {
                            r[s] = 0.0f;
                            if (s < d) {
                                const float2 v = s_rz[ra[s]];
                                r[s] = v.x;
                                nz += IND ? (fabsf(v.x) <= th.tz ? 1.0f : 0.0f) : v.y;
                            }
                        }
                        ma = anchor_candidates<DMAX, IND>(r, d, th.ta, IND ? th.te : I.pe.cut, I.pe_b1, I.pe_c1, nz,
                                                          IND ? alpha : alpha - 1e-3f);
                    }
                    const unsigned ba = __ballot_sync(0xffffffffu, ma != 0u);
                    const unsigned bb = PAIRED ? __ballot_sync(0xffffffffu, mb != 0u) : 0u;
                    if (ba | bb) {
                        const int leader = __ffs(ba | bb) - 1;
                        int q0 = 0;
                        if (lane == leader) q0 = atomicAdd(&S.nq, __popc(ba) + __popc(bb));
                        q0 = __shfl_sync(0xffffffffu, q0, leader);
                        const unsigned lt = (1u << lane) - 1u;
                        if (ma) queue_push(s_qj, s_qm, I.spill, q0 + __popc(ba & lt), ja, ma);
                        if (PAIRED && mb) queue_push(s_qj, s_qm, I.spill, q0 + __popc(ba) + __popc(bb & lt), jb, mb);
                    }
                }
                __syncthreads();
                const int nq = S.nq;
                for (int e = tid; e < nq; e += NT) {
                    int j;
                    unsigned cm;
                    if (e < RL0_BATCH_QCAP) {
                        j = s_qj[e];
                        cm = s_qm[e];
                    } else {
                        j = __ldcg(I.spill + 2 * (size_t)(e - RL0_BATCH_QCAP));
                        cm = (unsigned)__ldcg(I.spill + 2 * (size_t)(e - RL0_BATCH_QCAP) + 1);
                    }
                    float r[DMAX];
                    float nz = 0.0f, rhs = 0.0f;
                    unsigned cand = 0u;
#pragma unroll
                    for (int s = 0; s < DMAX; ++s) {
                        r[s] = 0.0f;
                        if (s < d) {
                            const float2 v = s_rz[__ldg(I.rows_sm + (size_t)s * n + j)];
                            r[s] = v.x;
                            nz += IND ? (fabsf(v.x) <= th.tz ? 1.0f : 0.0f) : v.y;
                            rhs += fabsf(v.x);
                            if (((cm >> s) & 1u) && fabsf(v.x) >= th.ta) cand |= 1u << s;
                        }
                    }
                    // the FP32 bound (exact near counts; continuous scores: an upper
                    // bound of each q_e) before the exact evaluation
                    if (cand)
                        cand &= anchor_candidates<DMAX, IND>(r, d, th.ta, IND ? th.te : I.pe.cut, I.pe_b1, I.pe_c1,
                                                             nz, IND ? alpha : alpha - 1e-3f);
                    int best = -1;
                    float bw = 0.0f;
                    while (cand) {
                        const int s = 31 - __clz(cand);
                        cand &= ~(1u << s);
                        const AnchorEval E = eval_anchor_regs<DMAX, IND>(r, d, s, th.te, I.pe);
                        if (E.lhs <= rhs && E.ne - nz >= alpha) {
                            best = s;
                            bw = E.w;
                            break;
                        }
                    }
                    if (best >= 0) {
                        const float old = x[j];
                        const float nv = old + bw;
                        x[j] = nv;
                        const int dn = (int)(nv != 0.0f) - (int)(old != 0.0f);
                        if (dn) atomicAdd(&S.nnz_delta, dn);
                        if (old != 0.0f && nv == 0.0f) atomicAdd(&S.zeroed, 1u);
                        UndoEntry u;
                        u.j = j;
                        u.old = old;
                        I.ulog[atomicAdd(&S.upd, 1u)] = u;
                        if (old == 0.0f && nv != 0.0f) I.list[atomicAdd(&S.list_count, 1u)] = j;
                    }
                }
                __syncthreads();
                if (tid == 0) S.nq = 0;                 // next read after the round's later barriers
            }
            __syncthreads();
            const unsigned upd = S.upd;
            if (tid == 0) S.acc = 0;
            if (upd > 0) {
                // ---- H_k
                if ((long long)S.nnz + S.nnz_delta > I.k)
                    cta_hk_select<NT>(I.list, S.list_count, x, I.k, I.hkkey, I.dlog, &S.drop_count, s_hk, s_scan);
                // ---- scatter the support into per-row buckets
                const unsigned total = S.list_count;
                for (long long w = tid; w < (long long)total * d; w += NT) {
                    const unsigned e = (unsigned)(w / d);
                    const int s = (int)(w % d);
                    const int j = I.list[e];
                    if (x[j] == 0.0f) continue;
                    const int row = I.rows_cm[(long long)j * d + s];
                    const int slot = atomicAdd(&I.bcnt[row], 1);
                    if (slot < RL0_BUCKET) I.bkt[(long long)row * RL0_BUCKET + slot] = j;
                    else S.overflow = 1;
                }
                __syncthreads();
                // ---- rebuild r = y - A x' (k_rebuild's arithmetic): one warp per
                // 256-row chunk, lane l taking rows l + 32 q (q < 8); the chunk's
                // two sums are the tree of group_sum2_df, formed inside the warp
                // (the same additions in the same order), so no CTA barrier waits
                // on the slowest row
                const bool csr = S.overflow != 0;
                for (int c = tid >> 5; c < nchunks; c += NT / 32) {
                    DF v[8], v2[8];
                    // four rows at a time: their loads are all issued before
                    // any of their stores
#pragma unroll
                    for (int h = 0; h < 8; h += 4) {
                        int cnt[4];
                        int4 b0[4], b1[4];
                        float yv[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int i = c * RL0_ROWS_CHUNK + lane + 32 * (h + q);
                            cnt[q] = 0;
                            yv[q] = 0.0f;
                            b0[q] = b1[q] = make_int4(0, 0, 0, 0);
                            if (i < m) {
                                yv[q] = I.y[i];
                                if (!csr) {
                                    cnt[q] = I.bcnt[i];
                                    const int4 *bq = (const int4 *)(I.bkt + (long long)i * RL0_BUCKET);
                                    b0[q] = bq[0];
                                    b1[q] = bq[1];
                                }
                            }
                        }
                        float sum[4];
                        DF acc[4];
                        if (csr) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int i = c * RL0_ROWS_CHUNK + lane + 32 * (h + q);
                                sum[q] = 0.0f;
                                acc[q] = DF{yv[q], 0.0f};
                                if (i < m)
                                    for (int p = I.rowptr[i]; p < I.rowptr[i + 1]; ++p) {
                                        const float xv = x[I.colidx[p]];
                                        sum[q] += xv;
                                        acc[q] = df_sub(acc[q], xv);
                                    }
                            }
                        } else {
                            float xs[4][RL0_BUCKET];
                            int js[4][RL0_BUCKET];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int raw[RL0_BUCKET] = {b0[q].x, b0[q].y, b0[q].z, b0[q].w,
                                                             b1[q].x, b1[q].y, b1[q].z, b1[q].w};
#pragma unroll
                                for (int u = 0; u < RL0_BUCKET; ++u) js[q][u] = (u < cnt[q]) ? raw[u] : 0x7fffffff;
                                if (cnt[q] > 1) sort8(js[q]);
#pragma unroll
                                for (int u = 0; u < RL0_BUCKET; ++u) xs[q][u] = (u < cnt[q]) ? x[js[q][u]] : 0.0f;
                            }
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                sum[q] = 0.0f;
                                acc[q] = DF{yv[q], 0.0f};
#pragma unroll
                                for (int u = 0; u < RL0_BUCKET; ++u)
                                    if (u < cnt[q]) {
                                        sum[q] += xs[q][u];
                                        acc[q] = df_sub(acc[q], xs[q][u]);
                                    }
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int i = c * RL0_ROWS_CHUNK + lane + 32 * (h + q);
                            v[h + q] = DF{0.0f, 0.0f};
                            v2[h + q] = DF{0.0f, 0.0f};
                            if (i < m) {
                                if (csr || cnt[q] > 0) I.bcnt[i] = 0;
                                const float r = yv[q] - sum[q];
                                I.rzc[i] = make_float2(r, I.indicator ? 0.0f : series_eval(I.pz, r));
                                v[h + q] = DF{fabsf(r), 0.0f};
                                v2[h + q] = df_abs(acc[q]);
                            }
                        }
                    }
                    // levels 128, 64, 32 of the chunk's tree, then its warp shuffles
                    DF a0 = df_add(v[0], v[4]), a1 = df_add(v[1], v[5]), a2 = df_add(v[2], v[6]), a3 = df_add(v[3], v[7]);
                    DF e0 = df_add(v2[0], v2[4]), e1 = df_add(v2[1], v2[5]), e2 = df_add(v2[2], v2[6]),
                       e3 = df_add(v2[3], v2[7]);
                    a0 = df_add(a0, a2);
                    a1 = df_add(a1, a3);
                    e0 = df_add(e0, e2);
                    e1 = df_add(e1, e3);
                    DF ra = df_add(a0, a1), rb = df_add(e0, e1);
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        const DF ua = df_shfl_down(ra, off), ub = df_shfl_down(rb, off);
                        if (lane < off) {
                            ra = df_add(ra, ua);
                            rb = df_add(rb, ub);
                        }
                    }
                    if (lane == 0) {
                        s_parts[c] = df_to_double(ra);
                        s_fcand[c] = df_to_double(rb);
                    }
                }
                __syncthreads();
                // ---- accept: ||r||_1 < ||r_hat||_1 (same combination as k_accept)
                if (tid < 32) {
                    const double l1n = warp_sum_parts(s_parts, nchunks, lane);
                    if (tid == 0) { S.l1n = l1n; S.acc = (l1n < S.l1_hat); }
                }
                __syncthreads();
                if (S.acc) {
                    if (S.drop_count > 0 || S.zeroed > 0) {
                        // stable compaction of the list to the new support
                        const unsigned tot = S.list_count;
                        unsigned out = 0;
                        for (unsigned b0 = 0; b0 < tot; b0 += NT) {
                            const unsigned e = b0 + tid;
                            int j = -1;
                            unsigned keep = 0;
                            if (e < tot) { j = I.list[e]; keep = (x[j] != 0.0f); }
                            s_scan[tid] = keep;
                            __syncthreads();
                            for (int off = 1; off < NT; off <<= 1) {
                                const unsigned w = (tid >= off) ? s_scan[tid - off] : 0u;
                                __syncthreads();
                                s_scan[tid] += w;
                                __syncthreads();
                            }
                            const unsigned incl = s_scan[tid], blk = s_scan[NT - 1];
                            __syncthreads();
                            if (keep) I.list[out + incl - 1] = j;
                            out += blk;
                            __syncthreads();
                        }
                        if (tid == 0) S.list_count = out;
                    }
                    for (int i = tid; i < m; i += NT) s_rz[i] = I.rzc[i];
                    for (int c = tid; c < nchunks; c += NT) s_fpart[c] = s_fcand[c];
                    if (tid == 0) {
                        S.shat_count = S.list_count;
                        S.nnz = (unsigned)((int)S.nnz + S.nnz_delta - (int)S.drop_count);
                        S.l1_hat = S.l1n;
                        S.accepted_rounds += 1;
                    }
                } else {
                    const unsigned nd = S.drop_count;
                    for (unsigned e = tid; e < nd; e += NT) x[I.dlog[e].j] = I.dlog[e].old;
                    __syncthreads();
                    for (unsigned e = tid; e < upd; e += NT) x[I.ulog[e].j] = I.ulog[e].old;
                    if (tid == 0) S.list_count = S.shat_count;
                }
                __syncthreads();
            }
            if (tid == 0) {
                if (upd > 0 && S.drop_count > 0) S.hk_rounds += 1;
                if (upd > 0 && S.overflow) S.fallback_rounds += 1;
                S.upd = 0;
                S.drop_count = 0;
                S.overflow = 0;
                S.nnz_delta = 0;
                S.zeroed = 0;
                S.round += 1;
                S.rounds_run += 1;
                S.converged = (S.l1_hat <= S.stop);
                if (S.converged || S.round >= I.nrounds) S.done = 1;
            }
            __syncthreads();
        }

        // ---- ||y - A x_hat||_1 in FP32 pairs: the accepted rebuild's chunk partials
        // (same chunks and combination as the single decode)
        __syncthreads();
        if (tid < 32) {
            const double fl = warp_sum_parts(s_fpart, nchunks, lane);
            if (tid == 0) {
                BatchResult R;
                R.rounds = S.rounds_run;
                R.accepted_rounds = S.accepted_rounds;
                R.converged = S.converged;
                R.status = S.status;
                R.hk_rounds = S.hk_rounds;
                R.fallback_rounds = S.fallback_rounds;
                R.nnz = S.nnz;
                R.l1_hat = S.l1_hat;
                R.final_l1 = fl;
                results[it] = R;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

typedef void (*BatchKernel)(const BatchItem *, BatchResult *, int, int *);

struct Variant {
    BatchKernel fn;
    int nt;
};

template <int DMAX, bool IND, bool EXACT, int NT>
Variant variant() { return Variant{k_decode_batched<DMAX, IND, EXACT, NT>, NT}; }

// Kernel group of column degree d: the exact-d kernels (two columns per thread
// in FP16 lanes) for 6 <= d <= 8, else the smallest DMAX >= d.
int batch_group(int d) { return (d >= 6 && d <= 8) ? d : (d < 6 ? 9 : (d <= 16 ? 16 : 32)); }

// Candidate schedules for a (group, score kind): threads per CTA.
std::vector<Variant> variants(int grp, int ind)
{
    std::vector<Variant> v;
#define RL0_V(D, I, E) { v.push_back(variant<D, I, E, 256>()); v.push_back(variant<D, I, E, 512>()); }
    switch (grp) {
    case 6: if (ind) RL0_V(6, true, true) else RL0_V(6, false, true) break;
    case 7: if (ind) RL0_V(7, true, true) else RL0_V(7, false, true) break;
    case 8: if (ind) RL0_V(8, true, true) else RL0_V(8, false, true) break;
    case 9: if (ind) RL0_V(8, true, false) else RL0_V(8, false, false) break;
    case 16: if (ind) RL0_V(16, true, false) else RL0_V(16, false, false) break;
    default:
        if (ind) v.push_back(variant<32, true, false, 256>()); else v.push_back(variant<32, false, false, 256>());
    }
#undef RL0_V
    return v;
}

struct Schedule {
    int variant, ctas_per_sm;
};

std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int>, Schedule> g_tuned;   // (device, dmax, ind, smem bucket)

struct BatchBuffers {
    int device = -1;
    size_t cap_items = 0, cap_thr = 0;
    BatchItem *d_items = nullptr;
    RoundThr *d_thr = nullptr;
    BatchResult *d_res = nullptr;
    int *d_queue = nullptr;
    BatchItem *h_items = nullptr;
    RoundThr *h_thr = nullptr;
    BatchResult *h_res = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};
std::mutex g_buf_mutex;
BatchBuffers g_buf[64];

int ensure_buffers(BatchBuffers &B, int dev, size_t nitems, size_t nthr)
{
    if (B.device < 0) {
        B.device = dev;
        CK(cudaEventCreate(&B.ev0));
        CK(cudaEventCreate(&B.ev1));
        CK(cudaMalloc(&B.d_queue, 16 * sizeof(int)));
    }
    if (nitems > B.cap_items) {
        cudaFree(B.d_items); cudaFree(B.d_res); cudaFreeHost(B.h_items); cudaFreeHost(B.h_res);
        B.d_items = nullptr; B.d_res = nullptr; B.h_items = nullptr; B.h_res = nullptr;
        B.cap_items = 0;
        CK(cudaMalloc(&B.d_items, nitems * sizeof(BatchItem)));
        CK(cudaMalloc(&B.d_res, nitems * sizeof(BatchResult)));
        CK(cudaMallocHost(&B.h_items, nitems * sizeof(BatchItem)));
        CK(cudaMallocHost(&B.h_res, nitems * sizeof(BatchResult)));
        B.cap_items = nitems;
    }
    if (nthr > B.cap_thr) {
        cudaFree(B.d_thr); cudaFreeHost(B.h_thr);
        B.d_thr = nullptr; B.h_thr = nullptr; B.cap_thr = 0;
        CK(cudaMalloc(&B.d_thr, nthr * sizeof(RoundThr)));
        CK(cudaMallocHost(&B.h_thr, nthr * sizeof(RoundThr)));
        B.cap_thr = nthr;
    }
    return RL0_OK;
}

// Launch one persistent decode of items[lo, hi) with a schedule.
int launch_group(const Variant &V, int ctas_per_sm, int nsm, size_t dyn, const BatchItem *d_items,
                 BatchResult *d_res, int cnt, int *d_queue, cudaStream_t s)
{
    CK(cudaFuncSetAttribute((const void *)V.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    CK(cudaMemsetAsync(d_queue, 0, sizeof(int), s));
    const int grid = std::min(cnt, nsm * ctas_per_sm);
    V.fn<<<grid, V.nt, dyn, s>>>(d_items, d_res, cnt, d_queue);
    CK(cudaGetLastError());
    return RL0_OK;
}

// CTAs per SM that fit the shared memory, registers and threads of an SM.
int max_ctas_per_sm(const Variant &V, size_t dyn)
{
    int nb = 0;
    if (cudaFuncSetAttribute((const void *)V.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)V.fn, V.nt, dyn) != cudaSuccess) return 0;
    return nb;
}

}  // namespace

extern "C" int rl0_decode_batched(int count, const rl0_expander *const *A, const float *const *y_dev,
                                  const int64_t *k, const rl0_params *params, float *const *xhat_dev,
                                  rl0_stats *stats, void *cuda_stream)
{
    if (count < 1 || !A || !y_dev || !k || !xhat_dev) return RL0_ERR_INVALID_ARG;
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return RL0_ERR_UNSUPPORTED;
    for (int i = 0; i < count; ++i) {
        if (!A[i] || !y_dev[i] || !xhat_dev[i]) return RL0_ERR_INVALID_ARG;
        if (A[i]->device != dev) return RL0_ERR_INVALID_ARG;
        if (A[i]->m > RL0_BATCH_MAX_M) return RL0_ERR_UNSUPPORTED;
    }
    {   // every instance needs its own workspace: no expander twice
        std::vector<const rl0_expander *> u(A, A + count);
        std::sort(u.begin(), u.end());
        if (std::adjacent_find(u.begin(), u.end()) != u.end()) return RL0_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // ---- host tables, in parallel over instances
    std::vector<rl0::Resolved> R(count);
    std::vector<int> rc(count, 0);
    std::vector<size_t> thr_off(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        rc[i] = rl0::resolve(A[i]->n, A[i]->m, A[i]->d, k[i], params ? params + i : nullptr, &R[i]);
        if (rc[i]) return rc[i];
        // the learned scorer and adaptive_k (a host step after every accepted
        // round) do not fit one persistent launch
        if (R[i].p.scorer == 1 || R[i].p.adaptive_k || R[i].p.anchor_rule != 0) return RL0_ERR_UNSUPPORTED;
        thr_off[i + 1] = thr_off[i] + R[i].nrounds;
    }
    std::lock_guard<std::mutex> lock(g_buf_mutex);
    BatchBuffers &B = g_buf[dev];
    int e = ensure_buffers(B, dev, count, thr_off[count]);
    if (e) return e;
    std::vector<DecodeCtx> ctx(count);
    {
        // tables each expander's cache does not hold are built by a pool of
        // host threads (a few tens of microseconds each); the rest are copies
        std::vector<int> miss;
        std::vector<char> is_miss(count, 0);
        for (int i = 0; i < count; ++i)
            if (!rl0_tables_cached(A[i], k[i], R[i])) {
                miss.push_back(i);
                is_miss[i] = 1;
            }
        const unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
        const int nth = (int)std::min<unsigned>(hw, (unsigned)std::max<size_t>(1, miss.size() / 16));
        auto work = [&](int t0) {
            for (size_t q = t0; q < miss.size(); q += nth) {
                const int i = miss[q];
                rl0_cached_tables(const_cast<rl0_expander *>(A[i]), k[i], R[i], &ctx[i], B.h_thr + thr_off[i]);
            }
            if (t0 == 0)
                for (int i = 0; i < count; ++i)
                    if (!is_miss[i])
                        rl0_cached_tables(const_cast<rl0_expander *>(A[i]), k[i], R[i], &ctx[i], B.h_thr + thr_off[i]);
        };
        std::vector<std::thread> pool;
        for (int t = 1; t < nth; ++t) pool.emplace_back(work, t);
        work(0);
        for (auto &th : pool) th.join();
    }
    // ---- descriptors, grouped by (DMAX, score kind), largest work first
    auto dmax_of = batch_group;
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        const int ga = dmax_of(A[a]->d) * 2 + R[a].indicator, gb = dmax_of(A[b]->d) * 2 + R[b].indicator;
        if (ga != gb) return ga < gb;
        const double wa = (double)A[a]->n * A[a]->d * R[a].nrounds, wb = (double)A[b]->n * A[b]->d * R[b].nrounds;
        if (wa != wb) return wa > wb;
        return a < b;
    });
    for (int q = 0; q < count; ++q) {
        const int i = order[q];
        const rl0_expander *X = A[i];
        BatchItem &It = B.h_items[q];
        std::memset(&It, 0, sizeof(It));
        It.n = (int)X->n;
        It.m = (int)X->m;
        It.d = X->d;
        It.nrounds = R[i].nrounds;
        It.nchunks = (int)rl0_div_up(X->m, RL0_ROWS_CHUNK);
        It.indicator = R[i].indicator;
        It.k = k[i];
        It.alpha = ctx[i].alpha;
        It.stop_level = ctx[i].stop_level;
        It.stop_rel = ctx[i].stop_rel;
        It.pz = ctx[i].pz;
        It.pe = ctx[i].pe;
        It.pe_b1 = ctx[i].pe_b1;
        It.pe_c1 = ctx[i].pe_c1;
        It.thr = B.d_thr + thr_off[i];
        It.rows_sm = X->rows_sm;
        It.rows_cm = X->rows_cm;
        It.rowptr = X->rowptr;
        It.colidx = X->colidx;
        It.y = y_dev[i];
        It.x = xhat_dev[i];
        It.rzc = X->ws.rz[1];
        It.list = X->ws.list;
        It.ulog = X->ws.ulog;
        It.dlog = X->ws.dlog;
        It.bcnt = X->ws.bcnt;
        It.bkt = X->ws.bkt;
        It.hkkey = X->ws.hk_scratch;
        It.spill = X->ws.res_list;                  // n entries of at least 2 ints
    }
    CK(cudaMemcpyAsync(B.d_items, B.h_items, count * sizeof(BatchItem), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.d_thr, B.h_thr, thr_off[count] * sizeof(RoundThr), cudaMemcpyHostToDevice, s));
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (stats) CK(cudaEventRecord(B.ev0, s));
    // ---- one persistent launch per group
    for (int g0 = 0; g0 < count;) {
        const int i0 = order[g0];
        const int dm = dmax_of(A[i0]->d), ind = R[i0].indicator;
        int g1 = g0;
        int64_t mmax = 0;
        while (g1 < count && dmax_of(A[order[g1]]->d) == dm && R[order[g1]].indicator == ind) {
            mmax = std::max<int64_t>(mmax, A[order[g1]]->m);
            ++g1;
        }
        const size_t dyn = ((size_t)mmax * sizeof(float2) + 1023) & ~(size_t)1023;
        std::vector<Variant> V = variants(dm, ind);
        const auto key = std::make_tuple(dev, dm, ind, (int)(dyn / 16384));
        Schedule sch{-1, 0};
        {
            std::lock_guard<std::mutex> tl(g_tune_mutex);
            auto f = g_tuned.find(key);
            if (f != g_tuned.end()) sch = f->second;
        }
        if (sch.variant < 0) {
            // autotune on a sample of this group: every (threads per CTA, CTAs per SM) that fits
            const int sample = std::min(g1 - g0, 2 * nsm);
            float best_ms = INFINITY;
            for (int v = 0; v < (int)V.size(); ++v) {
                const int cmax = max_ctas_per_sm(V[v], dyn);
                for (int c = 1; c <= cmax && c <= 4; ++c) {
                    float ms = 0.0f;
                    for (int rep = 0; rep < 2; ++rep) {           // first run warms up
                        CK(cudaEventRecord(B.ev1, s));
                        e = launch_group(V[v], c, nsm, dyn, B.d_items + g0, B.d_res + g0, sample, B.d_queue, s);
                        if (e) return e;
                        cudaEvent_t t1;
                        CK(cudaEventCreate(&t1));
                        CK(cudaEventRecord(t1, s));
                        CK(cudaEventSynchronize(t1));
                        CK(cudaEventElapsedTime(&ms, B.ev1, t1));
                        cudaEventDestroy(t1);
                    }
                    if (ms < best_ms) { best_ms = ms; sch = Schedule{v, c}; }
                }
            }
            if (sch.variant < 0) return RL0_ERR_UNSUPPORTED;
            std::lock_guard<std::mutex> tl(g_tune_mutex);
            g_tuned[key] = sch;
            if (stats) CK(cudaEventRecord(B.ev0, s));
        }
        e = launch_group(V[sch.variant], sch.ctas_per_sm, nsm, dyn, B.d_items + g0, B.d_res + g0, g1 - g0,
                         B.d_queue, s);
        if (e) return e;
        g0 = g1;
    }
    if (stats) CK(cudaEventRecord(B.ev1, s));
    CK(cudaMemcpyAsync(B.h_res, B.d_res, count * sizeof(BatchResult), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.0f;
    if (stats) cudaEventElapsedTime(&ms, B.ev0, B.ev1);
    int status = RL0_OK;
    for (int q = 0; q < count; ++q) {
        const int i = order[q];
        const BatchResult &Rr = B.h_res[q];
        if (Rr.status == RL0_ERR_INVALID_Y) status = RL0_ERR_INVALID_Y;
        if (stats) {
            rl0_stats &S = stats[i];
            std::memset(&S, 0, sizeof(S));
            S.rounds = Rr.rounds;
            S.accepted_rounds = Rr.accepted_rounds;
            S.converged = Rr.converged;
            S.status = Rr.status;
            S.support_size = Rr.nnz;
            S.final_l1 = Rr.final_l1;
            S.ms = ms;
            S.hk_rounds = Rr.hk_rounds;
            S.fallback_rounds = Rr.fallback_rounds;
            S.launches = (q == 0) ? 1 : 0;
        }
    }
    return status;
}
