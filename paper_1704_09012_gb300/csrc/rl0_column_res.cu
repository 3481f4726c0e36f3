// rl0_column_res.cu -- the column score of Robust-l0 (arXiv 1704.09012,
// Algorithm 2, the loop over j in [n] and i in N(j)) with every row's
// residual code resident in shared memory.
//
// One CTA per SM; CTA b owns the contiguous columns [b n / G, (b + 1) n / G).
//   load     the CTA copies the 16-bit codes of all m rows (and the p_z bound
//            table) into shared memory with bulk asynchronous copies
//            (cp.async.bulk + mbarrier), 2 bytes per row;
//   stream   each thread takes one column per tile of NT columns (two, j and
//            j + NT, per tile of 2 NT for exact d <= 8), reads their d row ids
//            (one coalesced 4-byte load per slot; the next tile's are
//            prefetched) and their codes from shared memory, and bounds their
//            anchors with code_candidates (code_candidates2: both columns in
//            the FP16 lanes of half2 registers); no thread waits on another;
//            a column that survives (about 1%) is listed
//            with its candidate slots: the first res_qcap of a CTA in shared
//            memory, where asynchronous copies (cp.async) fetch its FP32
//            (r, p_z) and x_j while the stream goes on, the rest in the CTA's
//            slice [lo, hi) of a list in global memory;
//   resolve  with the codes no longer needed, their shared memory stages the
//            survivors, NT at a time: one thread per column takes its FP32
//            (r, p_z) and keeps the candidate slots that are anchors
//            (|r_s| >= t_a); the candidates' posteriors q_e(r_s - r_l) are
//            evaluated one per thread, then one thread per candidate (column,
//            slot) sums them, and each column takes its highest passing slot
//            (the last passing anchor in row order); the CTA then commits with
//            one global atomic per counter, and the columns that became
//            nonzero go into the rebuild's fresh row buckets;
//   H_k      the launch's last CTA (a 64-bit acquire-release ticket that also
//            sums the CTAs' changes of the nonzero count) applies H_k
//            when |supp x'| > k, its scratch in the bytes that held the codes.
// The resolve runs the arithmetic of k_column_score in the same order, so
// both kernels give the same x'.
#include <algorithm>

#include "rl0_common.cuh"
#include "rl0_device.cuh"
#include "rl0_mma.cuh"
#include "rl0_round.cuh"

#define RL0_RES_CHUNK 32768u            // bytes per bulk copy
#define RL0_RES_WAIT_LIMIT (1u << 22)   // try_wait polls before a copy counts as lost
#define RL0_RES_MAX_NT 1024

namespace {

struct ResShared {
    Series pe;
    unsigned long long bar;             // completion of the bulk copies
    int count, last;
    unsigned total, ubase, fbase;
    int dn;                             // this CTA's change of the nonzero count
    unsigned nnz0;                      // |supp x_hat| at the round's start
};

// A survivor staged in shared memory: its column, candidate slots, x_j, the
// (r, p_z) of its rows (x_j and (r, p_z) copied with cp.async) and its row ids
// (for the fresh-bucket insert if it becomes nonzero).
template <int DMAX>
struct ResEntry {
    int j;
    unsigned mask;
    float old, pad;
    float2 rz[DMAX];
    int rid[DMAX + (DMAX & 1)];
};
__host__ __device__ constexpr unsigned res_entry_bytes(int d) { return 16u + 8u * d + 4u * (d + (d & 1)); }
static_assert(sizeof(ResEntry<7>) == res_entry_bytes(7) && sizeof(ResEntry<32>) == res_entry_bytes(32),
              "entry layout");

__device__ __forceinline__ void cp_async_4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                 :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
                 :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

// Bytes of the code region, which later holds the resolve scratch and, in
// the last CTA, H_k's scratch.
unsigned res_region_bytes(long long m, int nt, size_t scratch)
{
    const size_t codes = 2 * (size_t)rl0_code_rows(m);
    const size_t hk = ((sizeof(HkShared) + 15) & ~(size_t)15) + 4 * (size_t)nt;
    return (unsigned)((std::max(std::max(codes, hk), scratch) + 15) & ~(size_t)15);
}

__device__ __forceinline__ bool mbar_try_wait_bounded(unsigned bar, unsigned parity, unsigned polls)
{
    for (unsigned it = 0; it < polls; ++it) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// Resolve scratch, laid over the code region once the stream is done: a
// batch of NT listed columns and their candidate items (at most DMAX each).
template <int DMAX, int NT, bool LEARNED = false>
struct ResScratch {
    float r[DMAX][NT];                   // FP32 residuals of the batch's columns
    float nz[NT], rhs[NT];
    unsigned off[NT];                    // first item of each column
    unsigned short it_e[NT * DMAX];      // item -> column in the batch
    unsigned char it_s[NT * DMAX];       // item -> slot (descending within a column)
    unsigned char it_ok[NT * DMAX];
    float it_w[NT * DMAX];
    float it_sc[NT * DMAX];              // n_e - n_z of the item
    float feat[LEARNED ? NT : 1][RL0_NFEAT];   // learned scorer: features of the items that pass the
    unsigned short fidx[LEARNED ? NT : 1];     // exact tests (compact, NT items at a time) and their items
    float q[NT][DMAX];                   // q_e of (item, slot l), NT items at a time
    unsigned wsum[NT / 32];
    int nf;
};

// Exclusive prefix over the CTA of v (NT threads, all of them call it);
// *total (shared) gets the sum.  wsum: NT / 32 shared words.
template <int NT>
__device__ __forceinline__ unsigned cta_exclusive_scan(unsigned v, unsigned *wsum, unsigned *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned w = (lane < NT / 32) ? wsum[lane] : 0u;
        unsigned wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NT / 32) wsum[lane] = wi - w;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    const unsigned r = wsum[warp] + incl - v;
    __syncthreads();
    return r;
}

// One round's column score up to the CTA's commit (load, stream, resolve).
// DMAX slots per column; EXACT: d == DMAX (the slot guards fold away).
// cur, round: the decode state's accepted buffer and round (read by the caller).
template <int DMAX, bool IND, bool EXACT, int NT, bool LEARNED>
__device__ __forceinline__ bool column_phase(const KArgs &a, unsigned char *dsm)
{
    // exact d <= 8: two columns per thread in FP16 lanes (code_candidates2)
    constexpr bool PAIRED = EXACT && DMAX <= 8;
    DecodeState *st = a.st;
    const DecodeCtx *ctx = a.ctx;
    const int n = a.n, tid = threadIdx.x;
    const int d = EXACT ? DMAX : a.d;
    const unsigned short *s_code = (const unsigned short *)dsm;
    const float *s_pz = (const float *)(dsm + a.res_pz_off);
    ResShared &S = *(ResShared *)(dsm + a.res_s_off);
    // this CTA's columns: [lo, hi), equal shares of n
    const int lo = (int)(((long long)blockIdx.x * n) / gridDim.x);
    const int hi = (int)(((long long)(blockIdx.x + 1) * n) / gridDim.x);
    int j0 = lo;
    // row ids of this thread's first column(s): j0 + tid (and j0 + NT + tid
    // when paired), loaded while the previous kernel finishes (A never changes)
    // paired with even n: the two columns of a thread are adjacent (j, j + 1
    // from the even column below lo), so that each slot's two row ids come in
    // one 8-byte load; otherwise they are j and j + NT
    const bool vec = PAIRED && (n & 1) == 0;
    int nxt[DMAX], nxb[PAIRED ? DMAX : 1];
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        if constexpr (PAIRED) {
            if (vec) {
                const int j = (lo & ~1) + 2 * tid;
                const int2 v = (j < hi) ? __ldg(reinterpret_cast<const int2 *>(a.rows_sm + (size_t)s * n + j))
                                        : make_int2(0, 0);
                nxt[s] = v.x;
                nxb[s] = v.y;
            } else {
                const int j = j0 + tid;
                nxt[s] = (j < hi) ? __ldg(a.rows_sm + (size_t)s * n + j) : 0;
                nxb[s] = (j + NT < hi) ? __ldg(a.rows_sm + (size_t)s * n + j + NT) : 0;
            }
        } else {
            const int j = j0 + tid;
            nxt[s] = (s < d && j < hi) ? __ldg(a.rows_sm + (size_t)s * n + j) : 0;
        }
    }
    pdl_wait();                                    // the previous rebuild's r, codes, x and state
    // done, cur and round in one L2 trip (the code copy waits on cur)
    const int done = st->done, cur = st->cur, round = st->round;
    const unsigned nnz0 = st->nnz;
    pdl_launch_dependents();
    if (done) return false;
    const float2 *__restrict__ rz = cur ? a.rz1 : a.rz0;
    const RoundThr th = a.thr[round];
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&S.bar);
    if (tid == 0) {
        S.count = 0;
        S.dn = 0;
        S.nnz0 = nnz0;
        if (!IND) S.pe = ctx->pe;
        const unsigned code_bytes = 2u * (unsigned)rl0_code_rows(a.m);
        const unsigned bytes = code_bytes + (IND ? 0u : 4u * RL0_PZ_BINS);
        const unsigned char *src = (const unsigned char *)(cur ? a.code1 : a.code0);
        const unsigned dst = (unsigned)__cvta_generic_to_shared(dsm);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (((dst | (unsigned)(size_t)src | (unsigned)(size_t)a.pzlb) & 15u) != 0u) {
            // bulk copies need 16-byte alignment: report it, complete the phase, copy nothing
            atomicExch(&st->status, (int)RL0_ERR_CUDA);
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
        } else {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
            for (unsigned o = 0; o < code_bytes; o += RL0_RES_CHUNK) {
                const unsigned sz = (code_bytes - o < RL0_RES_CHUNK) ? code_bytes - o : RL0_RES_CHUNK;
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             :: "r"(dst + o), "l"(src + o), "r"(sz), "r"(bar) : "memory");
            }
            if (!IND)
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             :: "r"(dst + a.res_pz_off), "l"(a.pzlb), "r"(4u * RL0_PZ_BINS), "r"(bar) : "memory");
        }
    }
    // polls of the first wait: the built-in limit, or the expander's test
    // setting (rl0_expander_set_wait_polls), which may make it give up at once
    const unsigned polls = ctx->wait_test ? ctx->wait_polls : RL0_RES_WAIT_LIMIT;
    __syncthreads();                               // the barrier is initialised
    const bool arrived = mbar_try_wait_bounded(bar, 0u, polls);
    if (__syncthreads_or(!arrived || __ldcg(&st->status) == (int)RL0_ERR_CUDA)) {
        // a copy did not complete in time: record it, wait for the copies in
        // flight once more (with the built-in limit) before this CTA's shared
        // memory is reused, skip the columns (the last-CTA count below still runs)
        if (tid == 0 && !arrived) {
            atomicCAS(&st->status, 0, (int)RL0_ERR_TIMEOUT);
            mbar_try_wait_bounded(bar, 0u, RL0_RES_WAIT_LIMIT);
        }
        j0 = hi;
    }
    const CodeThr ct = code_thresholds(th.ta, th.tz, IND ? th.te : S.pe.cut);
    // the count the code bound must allow: Alg. 2's alpha, or the learned
    // scorer's candidate threshold (the slack covers FP32 rounding of n_e)
    const float need0 = LEARNED ? ctx->learned_need : ctx->alpha;
    const int rule = ctx->anchor_rule;            // read by the resolve; loaded here, off its path
    const float need = IND ? need0 : need0 - 1e-3f;
    int32_t *passed = ctx->passed;
    const int lane = tid & 31;
    // this CTA's survivors: the first qcap in shared memory, the others in its
    // slice of the global list, entries (j, candidate mask, its d row ids)
    ResEntry<DMAX> *sq = (ResEntry<DMAX> *)(dsm + a.res_q_off);
    const int qcap = a.res_qcap;
    int *seg = a.res_list + (size_t)lo * (size_t)(DMAX + 2);
    const float *xg = ctx->x;
    // list column j (candidate mask cm, row ids rid) at position pos
    auto emit = [&](int j, unsigned cm, int pos, const int *rid) {
        if (pos < qcap) {
            ResEntry<DMAX> &q = sq[pos];
            q.j = j;
            q.mask = cm;
            cp_async_4(&q.old, xg + j);
#pragma unroll
            for (int s = 0; s < DMAX; ++s)
                if (s < d) {
                    cp_async_8(&q.rz[s], rz + rid[s]);
                    q.rid[s] = rid[s];
                }
        } else if (pos < hi - lo) {                 // pos < hi - lo always: one entry per column
            int *ent = seg + (size_t)pos * (DMAX + 2);
            ent[0] = j;
            ent[1] = (int)cm;
#pragma unroll
            for (int s = 0; s < DMAX; ++s)
                if (s < d) ent[2 + s] = rid[s];
        }
    };
    if constexpr (PAIRED) {
        // two columns per thread bounded side by side in FP16 lanes; a listed
        // column reads its row ids again (from L2)
        const CodeThr2 ct2 = code_thresholds2(ct, need);
        auto pair_body = [&](const int *ra, const int *rb, int ja, int jb, bool aa, bool ab) {
            unsigned ma, mb;
            code_candidates2<DMAX, IND>(s_code, s_pz, ra, rb, aa, ab, ct2, ma, mb);
            const unsigned ba = __ballot_sync(0xffffffffu, ma != 0u), bb = __ballot_sync(0xffffffffu, mb != 0u);
            if (ba | bb) {
                const int leader = __ffs(ba | bb) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(&S.count, __popc(ba) + __popc(bb));
                base = __shfl_sync(0xffffffffu, base, leader);
                const unsigned lt = (1u << lane) - 1u;
                int rr[DMAX];
                if (ma) {
#pragma unroll
                    for (int s = 0; s < DMAX; ++s) rr[s] = __ldg(a.rows_sm + (size_t)s * n + ja);
                    emit(ja, ma, base + __popc(ba & lt), rr);
                }
                if (mb) {
#pragma unroll
                    for (int s = 0; s < DMAX; ++s) rr[s] = __ldg(a.rows_sm + (size_t)s * n + jb);
                    emit(jb, mb, base + __popc(ba) + __popc(bb & lt), rr);
                }
            }
            if (passed) {
                if (aa && !ma) passed[ja] = 0;
                if (ab && !mb) passed[jb] = 0;
            }
        };
        if (vec) {
            // columns jp + 2 tid and jp + 2 tid + 1; the one below lo (when lo is
            // odd) belongs to the previous CTA and is masked
            for (int jp = (j0 < hi) ? (lo & ~1) : hi; jp < hi; jp += 2 * NT) {
                int ra[DMAX], rb[DMAX];
#pragma unroll
                for (int s = 0; s < DMAX; ++s) {
                    ra[s] = nxt[s];
                    rb[s] = nxb[s];
                }
                {
                    const int jn = jp + 2 * NT + 2 * tid;
#pragma unroll
                    for (int s = 0; s < DMAX; ++s) {
                        if (jn < hi) {
                            const int2 v = __ldg(reinterpret_cast<const int2 *>(a.rows_sm + (size_t)s * n + jn));
                            nxt[s] = v.x;
                            nxb[s] = v.y;
                        }
                    }
                }
                const int ja = jp + 2 * tid;
                pair_body(ra, rb, ja, ja + 1, ja >= lo && ja < hi, ja + 1 < hi);
            }
            j0 = hi;
        }
        for (; j0 < hi; j0 += 2 * NT) {
            int ra[DMAX], rb[DMAX];
#pragma unroll
            for (int s = 0; s < DMAX; ++s) {
                ra[s] = nxt[s];
                rb[s] = nxb[s];
            }
            {
                const int jn = j0 + 2 * NT + tid;
#pragma unroll
                for (int s = 0; s < DMAX; ++s) {
                    if (jn < hi) nxt[s] = __ldg(a.rows_sm + (size_t)s * n + jn);
                    if (jn + NT < hi) nxb[s] = __ldg(a.rows_sm + (size_t)s * n + jn + NT);
                }
            }
            const int ja = j0 + tid, jb = ja + NT;
            pair_body(ra, rb, ja, jb, ja < hi, jb < hi);
        }
    }
    for (; j0 < hi; j0 += NT) {
        int rid[DMAX];
#pragma unroll
        for (int s = 0; s < DMAX; ++s) rid[s] = nxt[s];
        {
            const int jn = j0 + NT + tid;
#pragma unroll
            for (int s = 0; s < DMAX; ++s)
                if (s < d && jn < hi) nxt[s] = __ldg(a.rows_sm + (size_t)s * n + jn);
        }
        const int j = j0 + tid;
        const bool active = j < hi;
        const unsigned cm = active ? code_candidates<DMAX, IND>(s_code, s_pz, rid, d, ct, need) : 0u;
        const bool cand = cm != 0u;
        const unsigned m = __ballot_sync(0xffffffffu, cand);
        if (m) {
            const int leader = __ffs(m) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&S.count, __popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (cand) emit(j, cm, base + __popc(m & ((1u << lane) - 1u)), rid);
        }
        if (passed && active && !cand) passed[j] = 0;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();                               // the stream is done: the codes' bytes become scratch
    const int count = min(S.count, hi - lo);
    ResScratch<DMAX, NT, LEARNED> &R = *(ResScratch<DMAX, NT, LEARNED> *)dsm;
    if (LEARNED && tid == 0) R.nf = 0;              // first read after the batch's barriers
    const float alpha = ctx->alpha;
    for (int b0 = 0; b0 < count; b0 += NT) {
        // one thread per listed column: FP32 residuals, exact candidates
        const int e = b0 + tid;
        const bool act = e < count;
        int j = 0;
        unsigned cand = 0u;
        float old = 0.0f;
        if (act) {
            float2 v[DMAX];
            unsigned cm;
            if (e < qcap) {
                const ResEntry<DMAX> &q = sq[e];
                j = q.j;
                cm = q.mask;
                old = q.old;
#pragma unroll
                for (int s = 0; s < DMAX; ++s) v[s] = (s < d) ? q.rz[s] : make_float2(0.0f, 0.0f);
            } else {
                const int *ent = seg + (size_t)e * (DMAX + 2);
                j = __ldcg(ent);
                cm = (unsigned)__ldcg(ent + 1);
                old = xg[j];
#pragma unroll
                for (int s = 0; s < DMAX; ++s) v[s] = (s < d) ? __ldg(rz + __ldcg(ent + 2 + s)) : make_float2(0.0f, 0.0f);
            }
            float nz = 0.0f, rhs = 0.0f;
#pragma unroll
            for (int s = 0; s < DMAX; ++s) {
                if (s < d) {
                    nz += IND ? (fabsf(v[s].x) <= th.tz ? 1.0f : 0.0f) : v[s].y;
                    rhs += fabsf(v[s].x);
                    // the code bound's candidates that are anchors: a superset of
                    // the passing anchors, each then tested exactly below
                    if (((cm >> s) & 1u) && fabsf(v[s].x) >= th.ta) cand |= 1u << s;
                }
                R.r[s][tid] = (s < d) ? v[s].x : 0.0f;
            }
            R.nz[tid] = nz;
            R.rhs[tid] = rhs;
        }
        // one item per candidate (column, slot), a column's slots in descending order
        const unsigned nc = (unsigned)__popc(cand);
        const unsigned off = cta_exclusive_scan<NT>(nc, R.wsum, &S.total);
        const unsigned nitems = S.total;
        {
            unsigned c = cand, q = off;
            while (c) {
                const int sl = 31 - __clz(c);
                c &= ~(1u << sl);
                R.it_e[q] = (unsigned short)tid;
                R.it_s[q] = (unsigned char)sl;
                ++q;
            }
        }
        __syncthreads();
        // eval_anchor's arithmetic in two steps, so that an item's d posteriors
        // are evaluated side by side (one per thread) rather than one after
        // another: q_e of every (item, l), then each item's sums in slot order
        for (unsigned k0 = 0; k0 < nitems; k0 += NT) {
            const unsigned kn = min(nitems - k0, (unsigned)NT);
            for (unsigned p = tid; p < kn * (unsigned)d; p += NT) {
                const unsigned kk = p / (unsigned)d, l = p % (unsigned)d;
                const int ee = R.it_e[k0 + kk], sl = R.it_s[k0 + kk];
                const float rs = R.r[sl][ee], rl = R.r[l][ee];
                R.q[kk][l] = IND ? (fabsf(rs - rl) <= th.te ? 1.0f : 0.0f) : series_eval(S.pe, rs - rl);
            }
            __syncthreads();
            for (unsigned kk = tid; kk < kn; kk += NT) {
                const unsigned k = k0 + kk;
                const int ee = R.it_e[k];
                float ne = 0.0f, num = 0.0f;
                for (int l = 0; l < d; ++l) {
                    const float rl = R.r[l][ee];
                    const float q = R.q[kk][l];
                    ne += q;
                    num += rl * q;
                }
                const float w = num / ne;
                float lhs = 0.0f;
                for (int l = 0; l < d; ++l) lhs += fabsf(R.r[l][ee] - w);
                if constexpr (LEARNED) {
                    // the learned scorer: the l1 test and n_e - n_z >= 1.5 here; the
                    // features of the items that pass go to a compact list, whose
                    // logits the network takes below
                    const bool ok = lhs <= R.rhs[ee] && ne - R.nz[ee] >= ctx->learned_need;
                    R.it_ok[k] = ok ? 1 : 0;
                    if (ok) {
                        AnchorEval E;
                        E.ne = ne;
                        E.w = w;
                        E.lhs = lhs;
                        float f[RL0_NFEAT];
                        candidate_features(&R.r[0][ee], NT, d, E, R.nz[ee], R.rhs[ee], ctx->inv_sn, th.t, ctx->drho,
                                           f);
                        const int p = atomicAdd(&R.nf, 1);
#pragma unroll
                        for (int q = 0; q < RL0_NFEAT; ++q) R.feat[p][q] = f[q];
                        R.fidx[p] = (unsigned short)kk;
                    }
                } else {
                    R.it_ok[k] = (lhs <= R.rhs[ee] && ne - R.nz[ee] >= alpha) ? 1 : 0;
                }
                R.it_w[k] = w;
                R.it_sc[k] = ne - R.nz[ee];
            }
            __syncthreads();
            if constexpr (LEARNED) {
                // the passing items' logits, 16 per warp on the tensor cores
                const unsigned nf = (unsigned)R.nf;
                const __nv_bfloat16 *wb = (const __nv_bfloat16 *)ctx->mlp;
                for (unsigned t0 = (unsigned)(tid >> 5) * 16u; t0 < nf; t0 += (NT / 32) * 16u) {
                    auto f = [&](int r, int i) { return (t0 + r < nf) ? R.feat[t0 + r][i] : 0.0f; };
                    float lo, hi;
                    warp_mlp_logits16(f, wb, &lo, &hi);
                    if ((tid & 3) == 0) {
                        const unsigned gr = (unsigned)((tid & 31) >> 2);
                        if (t0 + gr < nf && !(lo >= ctx->logit_thr)) R.it_ok[k0 + R.fidx[t0 + gr]] = 0;
                        if (t0 + gr + 8 < nf && !(hi >= ctx->logit_thr)) R.it_ok[k0 + R.fidx[t0 + gr + 8]] = 0;
                    }
                }
                __syncthreads();
                if (tid == 0) R.nf = 0;                // read again only after the next batch's barriers
            }
        }
        // each column: its first passing item is its highest passing slot (the
        // last passing anchor in row order); with anchor_rule 1 the passing item
        // of largest n_e - n_z, ties to the lower slot (items come highest first)
        int best = -1;
        float bw = 0.0f, bsc = 0.0f;
        for (unsigned q = 0; q < nc; ++q)
            if (R.it_ok[off + q]) {
                if (rule == 0) {
                    best = R.it_s[off + q];
                    bw = R.it_w[off + q];
                    break;
                }
                if (best < 0 || R.it_sc[off + q] >= bsc) {
                    best = R.it_s[off + q];
                    bw = R.it_w[off + q];
                    bsc = R.it_sc[off + q];
                }
            }
        const bool pass = best >= 0;
        float nv = old;
        if (pass) {
            nv = old + bw;
            ctx->x[j] = nv;
        }
        if (passed && act) passed[j] = pass ? 1 : 0;
        // a column that became nonzero takes its rows' fresh-bucket slots now,
        // so that those atomics travel with the commit's below
        const bool fresh = pass && old == 0.0f && nv != 0.0f;
        int rid[DMAX], slot[DMAX];
        if (fresh) {
            if (e < qcap) {
#pragma unroll
                for (int s2 = 0; s2 < DMAX; ++s2) rid[s2] = (s2 < d) ? sq[e].rid[s2] : 0;
            } else {
                const int *ent = seg + (size_t)e * (DMAX + 2);
#pragma unroll
                for (int s2 = 0; s2 < DMAX; ++s2) rid[s2] = (s2 < d) ? __ldcg(ent + 2 + s2) : 0;
            }
            bucket_slots<DMAX>(a, rid, d, slot);
        }
        // the batch's commit: one global atomic per counter
        const unsigned pf = cta_exclusive_scan<NT>((pass ? 0x10000u : 0u) | (fresh ? 1u : 0u), R.wsum, &S.total);
        const unsigned tpf = S.total;
        // entries that became zero; the fresh ones are the scan's low field
        const int ngone = __syncthreads_count(pass && old != 0.0f && nv == 0.0f);
        if (tid == 0) {
            const int nup = (int)(tpf & 0xffffu);
            S.dn += nup - ngone;                   // added to the ticket at the end
            if (ngone) atomicAdd(&st->zeroed, (unsigned)ngone);
            const unsigned long long old2 = (tpf != 0u) ? take_upd_list(st, tpf >> 16, tpf & 0xffffu) : 0ull;
            S.ubase = (unsigned)(old2 >> 32);
            S.fbase = (unsigned)old2;
        }
        __syncthreads();
        if (pass) {
            UndoEntry u;
            u.j = j;
            u.old = old;
            a.ulog[S.ubase + (pf >> 16)] = u;
        }
        if (fresh) {
            a.list[S.fbase + (pf & 0xffffu)] = j;
            bucket_store<DMAX>(a, j, rid, d, slot);
        }
        __syncthreads();                           // the scratch is reused by the next batch
    }
    return true;
}

template <int DMAX, bool IND, bool EXACT, int NT, bool LEARNED>
__global__ void __launch_bounds__(NT, 1) k_column_score_res(KArgs a)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    if (!column_phase<DMAX, IND, EXACT, NT, LEARNED>(a, dsm)) return;     // the decode is done
    // the codes are no longer needed: their bytes become H_k's scratch
    ResShared &S = *(ResShared *)(dsm + a.res_s_off);
    HkShared &hk = *(HkShared *)dsm;
    unsigned *suf = (unsigned *)(dsm + ((sizeof(HkShared) + 15) & ~(size_t)15));
    last_cta_hk_tick<NT>(a, a.ctx, hk, suf, &S.last, S.dn, S.nnz0);
}

// Threads per CTA of each variant: 512 up to 16 slots (the paired exact
// variants hold two columns' codes and counts in up to 128 registers; at 64
// registers the compiler reloads them from shared memory), 256 beyond.
template <int DMAX, bool EXACT> struct ResNT {
    static constexpr int value = DMAX <= 16 ? 512 : 256;
};

template <int DMAX, bool EXACT>
bool res_attr(unsigned smem)
{
    constexpr int NT = ResNT<DMAX, EXACT>::value;
    const int sm = (int)smem;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (cudaFuncSetAttribute(k_column_score_res<DMAX, false, EXACT, NT, false>, at, sm) != cudaSuccess ||
        cudaFuncSetAttribute(k_column_score_res<DMAX, true, EXACT, NT, false>, at, sm) != cudaSuccess ||
        cudaFuncSetAttribute(k_column_score_res<DMAX, false, EXACT, NT, true>, at, sm) != cudaSuccess ||
        cudaFuncSetAttribute(k_column_score_res<DMAX, true, EXACT, NT, true>, at, sm) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Variant for column degree d: exact for 6 <= d <= 8, else the smallest DMAX >= d.
int res_variant(int d) { return (d >= 6 && d <= 8) ? d : (d < 6 ? 8 : (d <= 16 ? 16 : 32)); }
// (the learned variant's scratch, which adds the features of NT items, is the larger)
size_t res_scratch_bytes(int d)
{
    switch (res_variant(d)) {
    case 6: return sizeof(ResScratch<6, ResNT<6, true>::value, true>);
    case 7: return sizeof(ResScratch<7, ResNT<7, true>::value, true>);
    case 8: return d == 8 ? sizeof(ResScratch<8, ResNT<8, true>::value, true>)
                          : sizeof(ResScratch<8, ResNT<8, false>::value, true>);
    case 16: return sizeof(ResScratch<16, ResNT<16, false>::value, true>);
    default: return sizeof(ResScratch<32, ResNT<32, false>::value, true>);
    }
}

int res_nt(int d)
{
    switch (res_variant(d)) {
    case 6: return ResNT<6, true>::value;
    case 7: return ResNT<7, true>::value;
    case 8: return d == 8 ? ResNT<8, true>::value : ResNT<8, false>::value;
    case 16: return ResNT<16, false>::value;
    default: return ResNT<32, false>::value;
    }
}

}  // namespace

int rl0_res_dmax(int d) { return res_variant(d); }

void rl0_res_setup(const rl0_expander *A, KArgs *a)
{
    a->res_ok = 0;
    if (!A->ws.code[0] || !A->ws.code[1] || !A->ws.pzlb || !A->ws.res_list) return;
    const int nt = res_nt(A->d);
    const unsigned region = res_region_bytes(A->m, nt, res_scratch_bytes(A->d));
    a->res_pz_off = region;
    a->res_s_off = region + 4u * RL0_PZ_BINS;
    a->res_q_off = (a->res_s_off + (unsigned)sizeof(ResShared) + 15u) & ~15u;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, A->device) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (a->res_q_off > (unsigned)optin) return;
    // the shared memory left over stages survivors (one CTA per SM: nothing
    // else competes for it); the others go to the global list
    const unsigned eb = res_entry_bytes(res_variant(A->d));
    a->res_qcap = (int)std::min<unsigned>(((unsigned)optin - a->res_q_off) / eb, 4096u);
    a->res_smem = a->res_q_off + (unsigned)a->res_qcap * eb;
    bool ok = false;
    switch (res_variant(A->d)) {
    case 6: ok = res_attr<6, true>(a->res_smem); break;
    case 7: ok = res_attr<7, true>(a->res_smem); break;
    case 8: ok = (A->d == 8) ? res_attr<8, true>(a->res_smem) : res_attr<8, false>(a->res_smem); break;
    case 16: ok = res_attr<16, false>(a->res_smem); break;
    default: ok = res_attr<32, false>(a->res_smem); break;
    }
    if (!ok) return;
    const long long ntiles = rl0_div_up(A->n, nt);
    a->res_grid = (int)(ntiles < a->nsm ? ntiles : a->nsm);
    a->res_ok = 1;
}

bool rl0_res_launch(const KArgs &a, int indicator, int learned, cudaStream_t s)
{
    if (!a.res_ok || (learned && a.d > 16)) return false;
#define RL0_CR(D, E) do {                                                                                        \
        constexpr int NT_ = ResNT<D, E>::value;                                                                   \
        if (learned) {                                                                                            \
            if (indicator) launch_pdl(k_column_score_res<D, true, E, NT_, true>, a.res_grid, NT_, a.res_smem, s, a); \
            else launch_pdl(k_column_score_res<D, false, E, NT_, true>, a.res_grid, NT_, a.res_smem, s, a);      \
        } else if (indicator) {                                                                                   \
            launch_pdl(k_column_score_res<D, true, E, NT_, false>, a.res_grid, NT_, a.res_smem, s, a);            \
        } else {                                                                                                  \
            launch_pdl(k_column_score_res<D, false, E, NT_, false>, a.res_grid, NT_, a.res_smem, s, a);           \
        }                                                                                                         \
    } while (0)
    switch (res_variant(a.d)) {
    case 6: RL0_CR(6, true); break;
    case 7: RL0_CR(7, true); break;
    case 8: if (a.d == 8) RL0_CR(8, true); else RL0_CR(8, false); break;
    case 16: RL0_CR(16, false); break;
    default: RL0_CR(32, false); break;
    }
#undef RL0_CR
    return true;
}
