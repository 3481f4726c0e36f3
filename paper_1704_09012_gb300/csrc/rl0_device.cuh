// rl0_device.cuh -- device building blocks shared by the single-instance round
// kernels and the batched decoder, so both run the same arithmetic in the same
// order (Robust-l0, arXiv 1704.09012, Algorithm 2).
#pragma once

#include <cuda_fp16.h>

#include "rl0_common.cuh"

// ---------------------------------------------------------------------------
// Posterior evaluation in FP32: 1/p_breve(w) = sum_q a_q exp(b_q w^2)
// (Eqs. (pz_approx)/(pe_approx) normalised per Eq. (breve)).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float series_eval(const Series &S, float w)
{
    // branch-free: the sum is formed for every w and the two special cases
    // are selected at the end (same values as returning early)
    const float u = w * w;
    float acc;
    if (S.use_poly) {
        const float t = fmaf(u, S.inv_u2, -1.0f);
        const float t2 = 2.0f * t;
        float b1 = 0.0f, b2 = 0.0f;
#pragma unroll
        for (int k = RL0_MAXPOLY - 1; k >= 1; --k) {   // Clenshaw recurrence over k < npoly
            if (k < S.npoly) {
                const float b0 = fmaf(t2, b1, S.poly[k] - b2);
                b2 = b1;
                b1 = b0;
            }
        }
        const float G = fmaf(t, b1, S.poly[0] - b2);
        acc = fmaf(expf(S.b1 * u), G, S.a[0]);
    } else {
        acc = S.a[0];
#pragma unroll
        for (int q = 1; q < RL0_MAXQ; ++q)
            if (q < S.nq) acc += S.a[q] * expf(S.b[q] * u);
    }
    const float p = __frcp_rn(acc);             // = 1 / acc, correctly rounded
    return (w == 0.0f) ? 1.0f                   // p_breve(0) = 1 exactly
                       : (fabsf(w) > S.cut ? 0.0f : p);   // below 2^-40 beyond the cut
}

// ---------------------------------------------------------------------------
// Residual norms in FP32 pairs.  A value is hi + lo with |lo| <= ulp(hi)/2
// (about 48 significant bits), added with error-free transformations: TwoSum
// (Knuth, TAOCP vol. 2, 4.2.2) makes s + e = a + b exactly.  Everything runs
// on the FP32 pipes (this GPU's FP64 rate is a small fraction of its FP32
// rate); a sum is converted to FP64 once, exactly, as (double)hi + (double)lo.
// The compiler keeps these steps as written: no FMA pattern, no reassociation.
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return DF{s, (a - (s - bb)) + (b - bb)};
}

// a + b, both normalised
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const DF s = df_two_sum(a.hi, b.hi);
    return df_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

// a - x for an FP32 x
__device__ __forceinline__ DF df_sub(DF a, float x)
{
    const DF s = df_two_sum(a.hi, -x);
    return df_two_sum(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ DF df_abs(DF a) { return (a.hi < 0.0f) ? DF{-a.hi, -a.lo} : a; }
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ DF df_shfl_down(DF v, int off)
{
    return DF{__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off)};
}

// Fixed-shape tree over `n` consecutive threads (n a power of two, 64 <= n):
// sh[t] += sh[t + off] for off = n/2 .. 1, the levels off >= 32 through shared
// memory, the last five through warp shuffles in the group's first warp: the
// same additions in the same order wherever it runs.  Every thread of the
// block must call it (it synchronises the block).  Returns the sum in FP64.
__device__ __forceinline__ double group_sum_df(DF v, DF *sh, int lane, int n)
{
    sh[lane] = v;
    __syncthreads();
    for (int off = n >> 1; off >= 32; off >>= 1) {
        if (lane < off) sh[lane] = df_add(sh[lane], sh[lane + off]);
        __syncthreads();
    }
    DF r{0.0f, 0.0f};
    if (lane < 32) {
        r = sh[lane];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const DF u = df_shfl_down(r, off);
            if (lane < off) r = df_add(r, u);
        }
        if (lane == 0) sh[0] = r;
    }
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return df_to_double(r);
}

__device__ __forceinline__ double block_sum_df(DF v, DF *sh)
{
    return group_sum_df(v, sh, threadIdx.x, blockDim.x);
}

// Two group_sum_df trees in one pass (the same additions in the same order),
// over groups of n consecutive threads; sha/shb point at the group's n slots.
__device__ __forceinline__ double2 group_sum2_df(DF a, DF b, DF *sha, DF *shb, int lane, int n)
{
    sha[lane] = a;
    shb[lane] = b;
    __syncthreads();
    for (int off = n >> 1; off >= 32; off >>= 1) {
        if (lane < off) {
            sha[lane] = df_add(sha[lane], sha[lane + off]);
            shb[lane] = df_add(shb[lane], shb[lane + off]);
        }
        __syncthreads();
    }
    DF ra{0.0f, 0.0f}, rb{0.0f, 0.0f};
    if (lane < 32) {
        ra = sha[lane];
        rb = shb[lane];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const DF ua = df_shfl_down(ra, off), ub = df_shfl_down(rb, off);
            if (lane < off) {
                ra = df_add(ra, ua);
                rb = df_add(rb, ub);
            }
        }
        if (lane == 0) {
            sha[0] = ra;
            shb[0] = rb;
        }
    }
    __syncthreads();
    const double2 r = make_double2(df_to_double(sha[0]), df_to_double(shb[0]));
    __syncthreads();
    return r;
}

__device__ __forceinline__ double2 block_sum2_df(DF a, DF b, DF *sha, DF *shb)
{
    return group_sum2_df(a, b, sha, shb, threadIdx.x, blockDim.x);
}

// The same tree in FP64 (the MLP's training loss).
__device__ __forceinline__ double group_sum_f64(double v, double *sh, int lane, int n)
{
    sh[lane] = v;
    __syncthreads();
    for (int off = n >> 1; off >= 32; off >>= 1) {
        if (lane < off) sh[lane] += sh[lane + off];
        __syncthreads();
    }
    double r = 0.0;
    if (lane < 32) {
        r = sh[lane];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double u = __shfl_down_sync(0xffffffffu, r, off);
            if (lane < off) r += u;
        }
        if (lane == 0) sh[0] = r;
    }
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

// Chunk partials combined in a fixed order by one warp: lane l sums chunks
// l, l+32, ... then an xor-butterfly.  Call with all 32 lanes of one warp.
__device__ __forceinline__ double warp_sum_parts(const double *parts, int nparts, int lane)
{
    double v = 0.0;
    for (int c = lane; c < nparts; c += 32) v += parts[c];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// The same sum over chunk partials in global memory written in this launch
// (read through L2), four loads in flight per lane; the additions are those
// of warp_sum_parts, in the same order.
__device__ __forceinline__ double warp_sum_parts_l2(const double *parts, int nparts, int lane)
{
    double v = 0.0;
    int c = lane;
    for (; c + 96 < nparts; c += 128) {
        const double p0 = __ldcg(parts + c), p1 = __ldcg(parts + c + 32), p2 = __ldcg(parts + c + 64),
                     p3 = __ldcg(parts + c + 96);
        v += p0;
        v += p1;
        v += p2;
        v += p3;
    }
    for (; c < nparts; c += 32) v += __ldcg(parts + c);
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// The same sum (warp_sum_parts's order: lane l of warp 0 adds chunks l,
// l + 32, ... in turn, then the xor butterfly) over partials written in this
// launch, with all NT threads of the CTA first bringing 4 NT partials at a
// time into shared memory sh (4 NT doubles): one L2 trip per 4 NT chunks
// rather than one per four chunks of a lane.  Every thread of the CTA calls
// it; the sum is valid in warp 0.
template <int NT>
__device__ __forceinline__ double cta_sum_parts_l2(const double *parts, int nparts, double *sh)
{
    static_assert((4 * NT) % 32 == 0, "blocks keep each chunk on its lane");
    const int t = threadIdx.x;
    double v = 0.0;
    for (int c0 = 0; c0 < nparts; c0 += 4 * NT) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = c0 + q * NT + t;
            if (c < nparts) sh[q * NT + t] = __ldcg(parts + c);
        }
        __syncthreads();
        if (t < 32) {
            const int lim = min(4 * NT, nparts - c0);
            for (int c = t; c < lim; c += 32) v += sh[c];
        }
        __syncthreads();
    }
    if (t < 32)
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Sort 8 column ids ascending (Batcher's 19-comparator network).
#define RL0_CSWAP(i, j) { const int lo_ = min(js[i], js[j]), hi_ = max(js[i], js[j]); js[i] = lo_; js[j] = hi_; }
__device__ __forceinline__ void sort8(int *js)
{
    RL0_CSWAP(0, 1) RL0_CSWAP(2, 3) RL0_CSWAP(4, 5) RL0_CSWAP(6, 7)
    RL0_CSWAP(0, 2) RL0_CSWAP(1, 3) RL0_CSWAP(4, 6) RL0_CSWAP(5, 7)
    RL0_CSWAP(1, 2) RL0_CSWAP(5, 6) RL0_CSWAP(0, 4) RL0_CSWAP(1, 5)
    RL0_CSWAP(2, 6) RL0_CSWAP(3, 7) RL0_CSWAP(2, 4) RL0_CSWAP(3, 5)
    RL0_CSWAP(1, 2) RL0_CSWAP(3, 4) RL0_CSWAP(5, 6)
}
#undef RL0_CSWAP

// Exact quantities of one anchor s of one column (Alg. 2's inner test):
//   n_e = sum_l q_e(r_s - r_l), w = sum_l r_l q_e(r_s - r_l) / n_e,
//   lhs = sum_l |r_l - w|  (compared with rhs = sum_l |r_l|).
// The column's residuals are rc[l * stride], l < d, in slot order.
struct AnchorEval {
    float ne, w, lhs;
};

template <bool IND>
__device__ __forceinline__ AnchorEval eval_anchor(const float *rc, int stride, int d, int s, float te, const Series &pe)
{
    const float rs = rc[s * stride];
    float ne = 0.0f, num = 0.0f;
#pragma unroll 1
    for (int l = 0; l < d; ++l) {
        const float rl = rc[l * stride];
        const float q = IND ? (fabsf(rs - rl) <= te ? 1.0f : 0.0f) : series_eval(pe, rs - rl);
        ne += q;
        num += rl * q;
    }
    AnchorEval E;
    E.ne = ne;
    E.w = num / ne;
    float lhs = 0.0f;
#pragma unroll 1
    for (int l = 0; l < d; ++l) lhs += fabsf(rc[l * stride] - E.w);
    E.lhs = lhs;
    return E;
}

// eval_anchor on a column held in registers (r[l], l < d): the same FP32
// operations in the same order, so the results are bitwise those of eval_anchor.
template <int DMAX, bool IND>
__device__ __forceinline__ AnchorEval eval_anchor_regs(const float *r, int d, int s, float te, const Series &pe)
{
    float rs = 0.0f;
#pragma unroll
    for (int l = 0; l < DMAX; ++l)
        if (l == s) rs = r[l];
    float ne = 0.0f, num = 0.0f;
#pragma unroll
    for (int l = 0; l < DMAX; ++l) {
        if (l < d) {
            const float rl = r[l];
            const float q = IND ? (fabsf(rs - rl) <= te ? 1.0f : 0.0f) : series_eval(pe, rs - rl);
            ne += q;
            num += rl * q;
        }
    }
    AnchorEval E;
    E.ne = ne;
    E.w = num / ne;
    float lhs = 0.0f;
#pragma unroll
    for (int l = 0; l < DMAX; ++l)
        if (l < d) lhs += fabsf(r[l] - E.w);
    E.lhs = lhs;
    return E;
}

// Alg. 2's pass test: l1 decrease over the column and n_e - n_z >= alpha.
template <bool IND>
__device__ __forceinline__ bool score_anchor(const float *rc, int stride, int d, int s, float te,
                                             const Series &pe, float nz, float rhs, float alpha,
                                             float *score_out, float *w_out)
{
    const AnchorEval E = eval_anchor<IND>(rc, stride, d, s, te, pe);
    const float score = E.ne - nz;
    *score_out = score;
    *w_out = E.w;
    return E.lhs <= rhs && score >= alpha;
}

// ---------------------------------------------------------------------------
// Learned column scorer: a 16 -> 32 -> 32 -> 1 MLP (ReLU) on per-candidate
// features; its logit replaces the test n_e - n_z >= alpha.  Parameters, in
// this order: W1[i*32+o] (16x32), b1[32], W2[i*32+o] (32x32), b2[32], w3[32], b3.
// ---------------------------------------------------------------------------
#define RL0_NFEAT 16
#define RL0_HID 32
#define RL0_OFF_W1 0
#define RL0_OFF_B1 (RL0_OFF_W1 + RL0_NFEAT * RL0_HID)
#define RL0_OFF_W2 (RL0_OFF_B1 + RL0_HID)
#define RL0_OFF_B2 (RL0_OFF_W2 + RL0_HID * RL0_HID)
#define RL0_OFF_W3 (RL0_OFF_B2 + RL0_HID)
#define RL0_OFF_B3 (RL0_OFF_W3 + RL0_HID)
static_assert(RL0_OFF_B3 + 1 == RL0_MLP_PARAMS, "parameter layout");
#define RL0_DEV_CLIP 8.0f

// Features of a candidate (column residuals rc, anchor evaluation E, n_z, rhs):
//  f0..f6  the 7 smallest |r_l - w| / sigma_n, clipped at 8 (8 pads d < 7)
//  f7 n_e/d, f8 n_z/d, f9 log(1 + |w|/sigma_n)/5, f10 l1 gain (rhs - lhs)/rhs in [-1, 1],
//  f11 t, f12 d rho, f13 (n_e - n_z)/d, f14 = f15 = 0.
__device__ __forceinline__ void candidate_features(const float *rc, int stride, int d, const AnchorEval &E, float nz,
                                                   float rhs, float inv_sn, float t, float drho, float *f)
{
    unsigned used = 0u;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        float best = RL0_DEV_CLIP;
        int bi = -1;
#pragma unroll 1
        for (int l = 0; l < d; ++l) {
            if ((used >> l) & 1u) continue;
            const float v = fminf(fabsf(rc[l * stride] - E.w) * inv_sn, RL0_DEV_CLIP);
            if (v < best) { best = v; bi = l; }
        }
        if (bi >= 0) used |= 1u << bi;
        f[q] = best;
    }
    const float invd = 1.0f / (float)d;
    f[7] = E.ne * invd;
    f[8] = nz * invd;
    f[9] = log1pf(fabsf(E.w) * inv_sn) * 0.2f;
    f[10] = fminf(fmaxf((rhs - E.lhs) / fmaxf(rhs, 1e-30f), -1.0f), 1.0f);
    f[11] = t;
    f[12] = drho;
    f[13] = (E.ne - nz) * invd;
    f[14] = 0.0f;
    f[15] = 0.0f;
}

// Logit of the MLP with parameters W (FP32 copies of the BF16 weights).
__device__ __forceinline__ float mlp_logit(const float *W, const float *f)
{
    float h1[RL0_HID];
#pragma unroll
    for (int o = 0; o < RL0_HID; ++o) {
        float acc = W[RL0_OFF_B1 + o];
#pragma unroll
        for (int i = 0; i < RL0_NFEAT; ++i) acc = fmaf(f[i], W[RL0_OFF_W1 + i * RL0_HID + o], acc);
        h1[o] = fmaxf(acc, 0.0f);
    }
    float out = W[RL0_OFF_B3];
#pragma unroll 4
    for (int o = 0; o < RL0_HID; ++o) {
        float acc = W[RL0_OFF_B2 + o];
#pragma unroll
        for (int i = 0; i < RL0_HID; ++i) acc = fmaf(h1[i], W[RL0_OFF_W2 + i * RL0_HID + o], acc);
        out = fmaf(fmaxf(acc, 0.0f), W[RL0_OFF_W3 + o], out);
    }
    return out;
}

// Fast-path bound of Alg. 2's test for every anchor of a column held in
// registers: the anchors (|r_i| >= ta) whose n_e can still reach n_z + need.
// First level, both score kinds: n_e <= 1 + #{l != i : |r_i - r_l| <= reach}
// (exact for the 0/1 scores, where reach = te).  Second level, continuous
// scores, only for the anchors that survive the first: q_e(D) <=
// 1 / (1 + c1 (u + u^2/2)), u = b1 D^2 (b1 the smallest b_q of the q >= 1
// terms, c1 = 1 - a_0, from e^x >= 1 + x + x^2/2), so n_e <= 1 + the sum of
// these bounds over the near partners.  Callers pass need = alpha for the 0/1
// scores and alpha - 1e-3 for the continuous ones (the slack covers FP32
// rounding in the bound, the approximate reciprocal and n_e itself).
template <int DMAX, bool IND>
__device__ __forceinline__ unsigned anchor_candidates(const float *r, int d, float ta, float reach, float b1,
                                                      float c1, float nz, float need)
{
    unsigned amask = 0;
#pragma unroll
    for (int s = 0; s < DMAX; ++s)
        if (s < d && fabsf(r[s]) >= ta) amask |= 1u << s;
    if (!amask) return 0u;
    unsigned nm[DMAX];
#pragma unroll
    for (int s = 0; s < DMAX; ++s) nm[s] = 0u;
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
#pragma unroll
        for (int l = s + 1; l < DMAX; ++l) {
            if (l < d && fabsf(r[s] - r[l]) <= reach) {
                nm[s] |= 1u << l;
                nm[l] |= 1u << s;
            }
        }
    }
    unsigned cand = 0;
#pragma unroll
    for (int s = 0; s < DMAX; ++s)
        if (((amask >> s) & 1u) && (1.0f + (float)__popc(nm[s])) - nz >= need) cand |= 1u << s;
    if (IND || !cand) return cand;
    unsigned out = 0;
    for (unsigned rest = cand; rest; rest &= rest - 1) {
        const int s = __ffs(rest) - 1;
        float rs = 0.0f;
        unsigned ns = 0u;
#pragma unroll
        for (int l = 0; l < DMAX; ++l)
            if (l == s) {
                rs = r[l];
                ns = nm[l];
            }
        float ub = 1.0f;
#pragma unroll
        for (int l = 0; l < DMAX; ++l) {
            if ((ns >> l) & 1u) {
                const float u = b1 * ((rs - r[l]) * (rs - r[l]));
                ub += __fdividef(1.0f, fmaf(c1, fmaf(0.5f * u, u, u), 1.0f));
            }
        }
        if (ub - nz >= need) out |= 1u << s;
    }
    return out;
}

// ---------------------------------------------------------------------------
// 16-bit residual codes.  code(r) = FP16(r) rounded toward zero, its magnitude
// clamped to 0x7bff.  For v = the code's FP16 value, |r| lies in
// [|v|, |v| + ulp(v)) with ulp(v) <= |v| 2^-10 + 2^-24, and r has v's sign
// (or |r| < 2^-24), so |r - v| < e(v) = |v| 2^-10 + 2^-24.  Magnitude 0x7bff
// (65504) also stands for every larger |r|: a column holding one gets no
// bound.  The column kernel keeps every row's code in shared memory and bounds
// Alg. 2's test from them; only the columns that survive read the FP32
// residuals.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned short residual_code(float r)
{
    unsigned b = __half_as_ushort(__float2half_rz(r));
    if ((b & 0x7fffu) > 0x7bffu) b = (b & 0x8000u) | 0x7bffu;
    return (unsigned short)b;
}

#define RL0_CODE_WIDEN 1.00000095367431640625f    // 1 + 2^-20
#define RL0_CODE_NARROW 0.99999904632568359375f   // 1 - 2^-20
#define RL0_CODE_EREL 9.7656343132257461548e-4f   // 2^-10 (1 + 2^-20), rounded up
#define RL0_CODE_EABS 5.9604701102204882773e-8f   // 2^-24 (1 + 2^-20), rounded up

// Per-launch thresholds of the code bound, from the round's FP32 thresholds:
// an anchor (|r| >= ta) needs |v| >= ta_lo, a row with |v| <= tz_in has
// |r| <= tz, and reach1 = reach widened by 2^-20 (covers the FP32 rounding of
// the near test here and in the exact path).
struct CodeThr {
    float ta_lo, tz_in, reach1;
};

__device__ __forceinline__ CodeThr code_thresholds(float ta, float tz, float reach)
{
    // |r| < |v| (1 + 2^-10) + 2^-24 and 1 / (1 + 2^-10) >= 1 - 2^-10
    CodeThr c;
    c.ta_lo = (ta - 5.9604644775390625e-8f) * 0.9990224838256836f * RL0_CODE_NARROW;
    c.tz_in = (tz - 5.9604644775390625e-8f) * 0.9990224838256836f * RL0_CODE_NARROW;
    c.reach1 = reach * RL0_CODE_WIDEN;
    return c;
}

// The bound of anchor_candidates taken over every residual the codes allow:
//  - anchor possible when |v| >= ta_lo;
//  - near possible when |v_s - v_l| <= reach1 + 2 max_l e_l;
//  - n_z at least the sum of pzlb over the rows' bins (0/1 scores: the count
//    of rows with |v| <= tz_in);
//  - n_e at most 1 + the number of rows that can be near (q_e <= 1).
// Returns a superset of the anchors that pass Alg. 2's test on the FP32
// residuals; the resolve keeps those that are anchors on the FP32 residuals
// and tests them exactly.
template <int DMAX, bool IND>
__device__ __forceinline__ unsigned code_candidates(const unsigned short *codes, const float *pzlb, const int *rid,
                                                    int d, const CodeThr &ct, float need)
{
    float v[DMAX], e[DMAX];
    unsigned amask = 0, bmax = 0;
    float nzlb = 0.0f;
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
        v[s] = 0.0f;
        e[s] = 0.0f;
        if (s < d) {
            const unsigned c = codes[rid[s]];
            const float vv = __half2float(__ushort_as_half((unsigned short)c));
            const float av = fabsf(vv);
            v[s] = vv;
            e[s] = fmaf(av, RL0_CODE_EREL, RL0_CODE_EABS);
            bmax = max(bmax, c & 0x7fffu);
            if (av >= ct.ta_lo) amask |= 1u << s;
            nzlb += IND ? (av <= ct.tz_in ? 1.0f : 0.0f) : pzlb[(c & 0x7fffu) >> RL0_PZ_SHIFT];
        }
    }
    if (!amask) return 0u;
    if (bmax >= 0x7bffu) return amask;            // a saturated code: no bound
    // near possible: |v_s - v_l| <= reach1 + 2 max_l e_l (>= reach1 + e_s + e_l).
    // Counted on the FMA pipe: q = sat((thr - |v_s - v_l|) 2^100 + 2^10) is 1
    // when the pair can be near, 0 when thr - |v_s - v_l| < -2^-90, and in
    // between only within 2^-90 of the test (an over-count, still a bound).
    float emax = 0.0f;
#pragma unroll
    for (int s = 0; s < DMAX; ++s) emax = fmaxf(emax, e[s]);
    const float thr = fmaf(2.0f, emax, ct.reach1);
    float cnt[DMAX];
#pragma unroll
    for (int s = 0; s < DMAX; ++s) cnt[s] = 0.0f;
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
#pragma unroll
        for (int l = s + 1; l < DMAX; ++l) {
            if (l < d) {
                const float q = __saturatef(fmaf(thr - fabsf(v[s] - v[l]), 0x1p100f, 0x1p10f));
                cnt[s] += q;
                cnt[l] += q;
            }
        }
    }
    // candidate: 1 + near count - n_z >= need
    const float kneed = need - 1.0f + nzlb;
    unsigned cand = 0;
#pragma unroll
    for (int s = 0; s < DMAX; ++s)
        if (((amask >> s) & 1u) && cnt[s] >= kneed) cand |= 1u << s;
    return cand;
}

// code_candidates for two columns at once, d = D rows each, in the two FP16
// lanes of half2 registers (lane 0: column a, lane 1: column b).  The codes
// are FP16 values, so the anchor, n_z and count comparisons against a float
// threshold T are exact when T is first rounded to FP16 in the direction that
// keeps the test (|v| >= T iff |v| >= RU(T); |v| <= T iff |v| <= RD(T)); the
// pair test is the one inexact step: |v_s - v_l| is rounded to FP16 (relative
// error <= 2^-11, absolute <= 2^-25 below 2^-14) and compared with a reach
// rounded up with that margin, so a pair that can be near always counts.
// The near count is exact (each pair adds 0 or 1).  Returns the two columns'
// candidate masks (0 for an inactive column).
struct CodeThr2 {
    __half2 ta, tz;                 // RU(ta_lo), RD(tz_in) in both lanes
    float c1, c0;                   // reach of a column: RU16(c1 vmax + c0)
    float need1;                    // need - 1
};

__device__ __forceinline__ CodeThr2 code_thresholds2(const CodeThr &ct, float need)
{
    CodeThr2 c;
    c.ta = __half2half2(__float2half_ru(ct.ta_lo));
    c.tz = __half2half2(__float2half_rd(ct.tz_in));
    // reach1 + 2 e(vmax), e(v) = v EREL + EABS, widened by 2^-10 for the FP16
    // difference and by 2^-20 for this FP32 arithmetic
    c.c1 = 2.0f * RL0_CODE_EREL * 1.0009775161743164f;
    c.c0 = fmaf(ct.reach1 + 2.0f * RL0_CODE_EABS, 1.0009775161743164f, 5.9604644775390625e-8f) * RL0_CODE_WIDEN;
    c.need1 = need - 1.0f;
    return c;
}

__device__ __forceinline__ unsigned h2bits(__half2 h) { return *reinterpret_cast<const unsigned *>(&h); }

template <int D, bool IND>
__device__ __forceinline__ void code_candidates2(const unsigned short *codes, const float *pzlb, const int *ra,
                                                 const int *rb, bool act_a, bool act_b, const CodeThr2 &ct,
                                                 unsigned &ma, unsigned &mb)
{
    __half2 v[D];
    __half2 vmax = __float2half2_rn(0.0f), nzi = __float2half2_rn(0.0f);
#pragma unroll
    for (int s = 0; s < D; ++s) {
        const unsigned ca = codes[ra[s]], cb = codes[rb[s]];
        v[s] = __halves2half2(__ushort_as_half((unsigned short)ca), __ushort_as_half((unsigned short)cb));
        const __half2 av = __habs2(v[s]);
        vmax = __hmax2(vmax, av);
        if (IND) nzi = __hadd2(nzi, __hle2(av, ct.tz));
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
    // the test with the n_z bound: 0/1 scores count rows here; the continuous
    // scores first test with n_z >= 0 (no table) and look the bound up only
    // for the columns that pass that
    __half2 kneed;
    if (IND) {
        kneed = __halves2half2(__float2half_ru(ct.need1 + __low2float(nzi)), __float2half_ru(ct.need1 + __high2float(nzi)));
    } else {
        kneed = __halves2half2(__float2half_ru(ct.need1), __float2half_ru(ct.need1));
    }
    // bit 10 of each lane of a 1.0/0.0 result, moved to bit s (lane 0) and
    // bit 16 + s (lane 1)
    unsigned anc = 0u, acc = 0u;
#pragma unroll
    for (int s = 0; s < D; ++s) {
        const unsigned a = h2bits(__hge2(__habs2(v[s]), ct.ta)) & 0x04000400u;
        const unsigned c = h2bits(__hge2(cnt[s], kneed));
        anc |= a >> (10 - s);
        acc |= (a & c) >> (10 - s);
    }
    if (!IND && acc != 0u) {
        float nza = 0.0f, nzb = 0.0f;
#pragma unroll
        for (int s = 0; s < D; ++s) {
            const unsigned w = h2bits(v[s]);
            nza += pzlb[(w & 0x7fffu) >> RL0_PZ_SHIFT];
            nzb += pzlb[(w >> 16 & 0x7fffu) >> RL0_PZ_SHIFT];
        }
        kneed = __halves2half2(__float2half_ru(ct.need1 + nza), __float2half_ru(ct.need1 + nzb));
        acc = 0u;
#pragma unroll
        for (int s = 0; s < D; ++s) {
            const unsigned a = h2bits(__hge2(__habs2(v[s]), ct.ta)) & 0x04000400u;
            const unsigned c = h2bits(__hge2(cnt[s], kneed));
            acc |= (a & c) >> (10 - s);
        }
    }
    // a saturated code (|v| = 65504 stands for every larger |r|): no bound
    const unsigned fa = (va >= 65504.0f) ? anc : acc, fb = (vb >= 65504.0f) ? anc : acc;
    ma = any_a ? (fa & 0xffffu) : 0u;
    mb = any_b ? (fb >> 16) : 0u;
}

// ---------------------------------------------------------------------------
// H_k (Alg. 2): keep the k entries of largest |x_j|, ties to the smaller j.
// Radix select of the k-th largest 63-bit key (bits(|x|) << 32 | ~j) among the
// listed nonzero entries, six passes of at most 11 bits, by one CTA of NT
// threads; everything below the key is zeroed and logged for undo.
// ---------------------------------------------------------------------------
#define HK_BINS 2048

__device__ __forceinline__ unsigned long long hk_key(float v, int j)
{
    return ((unsigned long long)(__float_as_uint(v) & 0x7fffffffu) << 32) | (unsigned long long)(0xffffffffu - (unsigned)j);
}

struct HkShared {
    unsigned hist[HK_BINS];
    unsigned long long prefix;
    unsigned need;
};

template <int NT>
__device__ void cta_hk_select(const int *list, unsigned total, float *x, long long k, unsigned long long *keys,
                              UndoEntry *dlog, unsigned *drop_count, HkShared &sm, unsigned *suf)
{
    constexpr int BPT = HK_BINS / NT;          // bins per thread
    const int t = threadIdx.x;
    for (unsigned e = t; e < total; e += NT) {
        const int j = list[e];
        const float v = x[j];
        keys[e] = (v != 0.0f) ? hk_key(v, j) : 0ull;
    }
    if (t == 0) { sm.prefix = 0ull; sm.need = (unsigned)k; }
    __syncthreads();
    for (int p = 0; p < 6; ++p) {
        // digits of 11 bits from bit 63 down (shifts 52, 41, 30, 19, 8), then the last 8
        const int sh = (p < 5) ? 52 - 11 * p : 0, wd = (p < 5) ? 11 : 8;
        const int nb = 1 << wd;
        for (int b = t; b < HK_BINS; b += NT) sm.hist[b] = 0;
        const unsigned long long prefix = sm.prefix;
        const unsigned need = sm.need;
        __syncthreads();
        for (unsigned e = t; e < total; e += NT) {
            const unsigned long long key = keys[e];
            if (key != 0ull && (key >> (sh + wd)) == prefix) atomicAdd(&sm.hist[(unsigned)(key >> sh) & (nb - 1)], 1u);
        }
        __syncthreads();
        // thread t owns bins nb-1-BPT*t .. nb-BPT*(t+1) (highest first)
        unsigned own = 0;
#pragma unroll
        for (int q = 0; q < BPT; ++q) {
            const int b = nb - 1 - BPT * t - q;
            if (b >= 0) own += sm.hist[b];
        }
        suf[t] = own;
        __syncthreads();
        for (int off = 1; off < NT; off <<= 1) {
            const unsigned v = (t >= off) ? suf[t - off] : 0u;
            __syncthreads();
            suf[t] += v;
            __syncthreads();
        }
        unsigned run = suf[t] - own;               // count in bins above this thread's bins
#pragma unroll
        for (int q = 0; q < BPT; ++q) {
            const int b = nb - 1 - BPT * t - q;
            if (b >= 0) {
                const unsigned hb = sm.hist[b];
                if (run < need && run + hb >= need) {
                    sm.prefix = (prefix << wd) | (unsigned)b;
                    sm.need = need - run;
                }
                run += hb;
            }
        }
        __syncthreads();
    }
    const unsigned long long kth = sm.prefix;      // the k-th largest key
    for (unsigned e = t; e < total; e += NT) {
        const unsigned long long key = keys[e];
        if (key != 0ull && key < kth) {
            const int j = list[e];
            UndoEntry u;
            u.j = j;
            u.old = x[j];
            x[j] = 0.0f;
            dlog[atomicAdd(drop_count, 1u)] = u;
        }
    }
    __syncthreads();
}
