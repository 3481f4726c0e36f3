// rl0_mma.cuh -- the learned column scorer's network (16 -> 32 -> 32 -> 1, ReLU)
// on the tensor cores: warp-level mma.sync m16n8k16 with BF16 operands and FP32
// accumulation, 16 rows (candidates or training samples) per warp.  Not part of
// the ABI.
//
// Precision.  An FP32 value x is split into three BF16 parts, x1 = bf16(x),
// x2 = bf16(x - x1), x3 = bf16(x - x1 - x2), which together carry its 24-bit
// significand; x1 + x2 + x3 = x unless x is below the BF16 normal range.  A
// product of such a part with a BF16 weight is exact in FP32, so a layer
// computed as sum_parts (x_p . W) differs from the FP32 dot product only by
// the FP32 accumulation's rounding.  The decoder's weights are BF16 already;
// FP32 master weights (training) are split the same way and the six products
// of parts whose ranks add up to at most 4 are kept (the rest are below 2^-24
// relative).
//
// Fragment layouts of mma.sync.m16n8k16 (PTX ISA): with g = lane / 4 and
// q = lane % 4, A (16 x 16, row-major) holds rows g and g + 8, columns 2q, 2q+1,
// 2q+8, 2q+9; B (16 x 8) holds rows (k) 2q, 2q+1, 2q+8, 2q+9 of column (n) g;
// C/D (16 x 8) holds rows g and g + 8, columns 2q and 2q+1.  So layer 1's
// accumulators over hidden units 16kk .. 16kk+15 (two n-tiles) are, entry for
// entry, layer 2's A fragment for k-step kk: no data moves between layers.
#pragma once

#include <cuda_bf16.h>

#include "rl0_device.cuh"

__device__ __forceinline__ unsigned bf16x2_bits(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// x = p[0] + p[1] + p[2] in BF16 parts (round to nearest at each step)
__device__ __forceinline__ void split3(float x, __nv_bfloat16 *p)
{
    p[0] = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(p[0]);
    p[1] = __float2bfloat16_rn(r1);
    p[2] = __float2bfloat16_rn(r1 - __bfloat162float(p[1]));
}

// d += a . b, m16n8k16, BF16 x BF16 -> FP32
__device__ __forceinline__ void mma_bf16_16816(float *d, const unsigned *a, const unsigned *b)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragments (three parts) of a 16 x 16 FP32 tile given its values at this
// lane's positions: v[0..1] row g cols 2q..2q+1, v[2..3] row g+8 same cols,
// v[4..5] row g cols 2q+8..2q+9, v[6..7] row g+8 same cols.
__device__ __forceinline__ void a_frag_split3(const float *v, unsigned a[3][4])
{
    __nv_bfloat16 p[8][3];
#pragma unroll
    for (int e = 0; e < 8; ++e) split3(v[e], p[e]);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        a[s][0] = bf16x2_bits(p[0][s], p[1][s]);
        a[s][1] = bf16x2_bits(p[2][s], p[3][s]);
        a[s][2] = bf16x2_bits(p[4][s], p[5][s]);
        a[s][3] = bf16x2_bits(p[6][s], p[7][s]);
    }
}

// B fragment of the BF16 matrix W (row-major, ldw columns; rows k0 .., columns n0 ..)
__device__ __forceinline__ void b_frag_bf16(const __nv_bfloat16 *W, int ldw, int k0, int n0, unsigned b[2])
{
    const int g = (threadIdx.x & 31) >> 2, q = threadIdx.x & 3;
    b[0] = bf16x2_bits(W[(k0 + 2 * q) * ldw + n0 + g], W[(k0 + 2 * q + 1) * ldw + n0 + g]);
    b[1] = bf16x2_bits(W[(k0 + 2 * q + 8) * ldw + n0 + g], W[(k0 + 2 * q + 9) * ldw + n0 + g]);
}

// A fragments (three parts) of a 16 x 16 FP32 tile whose entry (r, c) is e(r, c).
template <class Fn>
__device__ __forceinline__ void a_frag_split3_fn(Fn e, unsigned a[3][4])
{
    const int g = (threadIdx.x & 31) >> 2, q = threadIdx.x & 3;
    float v[8];
    v[0] = e(g, 2 * q);
    v[1] = e(g, 2 * q + 1);
    v[2] = e(g + 8, 2 * q);
    v[3] = e(g + 8, 2 * q + 1);
    v[4] = e(g, 2 * q + 8);
    v[5] = e(g, 2 * q + 9);
    v[6] = e(g + 8, 2 * q + 8);
    v[7] = e(g + 8, 2 * q + 9);
    a_frag_split3(v, a);
}

// B fragments (three parts) of a 16 x 8 FP32 tile whose entry (k, n) is e(k, n).
template <class Fn>
__device__ __forceinline__ void b_frag_split3_fn(Fn e, unsigned b[3][2])
{
    const int g = (threadIdx.x & 31) >> 2, q = threadIdx.x & 3;
    __nv_bfloat16 p[4][3];
    split3(e(2 * q, g), p[0]);
    split3(e(2 * q + 1, g), p[1]);
    split3(e(2 * q + 8, g), p[2]);
    split3(e(2 * q + 9, g), p[3]);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        b[s][0] = bf16x2_bits(p[0][s], p[1][s]);
        b[s][1] = bf16x2_bits(p[2][s], p[3][s]);
    }
}

// d += a . b for two FP32 operands in three BF16 parts each: the six part
// products whose ranks add up to at most 4, smallest first.
__device__ __forceinline__ void mma_split3x3(float *d, const unsigned a[3][4], const unsigned b[3][2])
{
    mma_bf16_16816(d, a[2], b[0]);
    mma_bf16_16816(d, a[1], b[1]);
    mma_bf16_16816(d, a[0], b[2]);
    mma_bf16_16816(d, a[1], b[0]);
    mma_bf16_16816(d, a[0], b[1]);
    mma_bf16_16816(d, a[0], b[0]);
}

// Logits of 16 rows with the BF16 parameters wb (layout of rl0.h: W1 16x32
// input-major, b1, W2 32x32, b2, w3, b3).  f(r, i) gives feature i of row r
// (rows 0..15 of this warp's tile).  Every lane of the warp calls it; lane
// 4g + q returns in *lo / *hi the logits of rows g and g + 8 (the same in the
// four lanes of a quad).
template <class FeatFn>
__device__ __forceinline__ void warp_mlp_logits16(FeatFn f, const __nv_bfloat16 *wb, float *lo, float *hi)
{
    const int g = (threadIdx.x & 31) >> 2, q = threadIdx.x & 3;
    // layer 1: z1 = F W1 + b1 (K = 16, four n-tiles of 8 hidden units)
    unsigned a1[3][4];
    {
        float v[8];
        v[0] = f(g, 2 * q);
        v[1] = f(g, 2 * q + 1);
        v[2] = f(g + 8, 2 * q);
        v[3] = f(g + 8, 2 * q + 1);
        v[4] = f(g, 2 * q + 8);
        v[5] = f(g, 2 * q + 9);
        v[6] = f(g + 8, 2 * q + 8);
        v[7] = f(g + 8, 2 * q + 9);
        a_frag_split3(v, a1);
    }
    float c1[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float b0 = __bfloat162float(wb[RL0_OFF_B1 + 8 * nt + 2 * q]);
        const float b1 = __bfloat162float(wb[RL0_OFF_B1 + 8 * nt + 2 * q + 1]);
        c1[nt][0] = b0;
        c1[nt][1] = b1;
        c1[nt][2] = b0;
        c1[nt][3] = b1;
        unsigned bw[2];
        b_frag_bf16(wb + RL0_OFF_W1, RL0_HID, 0, 8 * nt, bw);
#pragma unroll
        for (int s = 0; s < 3; ++s) mma_bf16_16816(c1[nt], a1[s], bw);
    }
    // layer 2: z2 = relu(z1) W2 + b2 (K = 32 in two k-steps)
    float c2[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float b0 = __bfloat162float(wb[RL0_OFF_B2 + 8 * nt + 2 * q]);
        const float b1 = __bfloat162float(wb[RL0_OFF_B2 + 8 * nt + 2 * q + 1]);
        c2[nt][0] = b0;
        c2[nt][1] = b1;
        c2[nt][2] = b0;
        c2[nt][3] = b1;
    }
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            v[e] = fmaxf(c1[2 * kk][e], 0.0f);
            v[4 + e] = fmaxf(c1[2 * kk + 1][e], 0.0f);
        }
        unsigned a2[3][4];
        a_frag_split3(v, a2);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            unsigned bw[2];
            b_frag_bf16(wb + RL0_OFF_W2, RL0_HID, 16 * kk, 8 * nt, bw);
#pragma unroll
            for (int s = 0; s < 3; ++s) mma_bf16_16816(c2[nt], a2[s], bw);
        }
    }
    // layer 3: relu(z2) . w3 + b3, the quad's four column pairs added by shuffles
    float sl = 0.0f, sh = 0.0f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float w0 = __bfloat162float(wb[RL0_OFF_W3 + 8 * nt + 2 * q]);
        const float w1 = __bfloat162float(wb[RL0_OFF_W3 + 8 * nt + 2 * q + 1]);
        sl = fmaf(fmaxf(c2[nt][0], 0.0f), w0, sl);
        sl = fmaf(fmaxf(c2[nt][1], 0.0f), w1, sl);
        sh = fmaf(fmaxf(c2[nt][2], 0.0f), w0, sh);
        sh = fmaf(fmaxf(c2[nt][3], 0.0f), w1, sh);
    }
    sl += __shfl_xor_sync(0xffffffffu, sl, 1);
    sl += __shfl_xor_sync(0xffffffffu, sl, 2);
    sh += __shfl_xor_sync(0xffffffffu, sh, 1);
    sh += __shfl_xor_sync(0xffffffffu, sh, 2);
    const float b3 = __bfloat162float(wb[RL0_OFF_B3]);
    *lo = sl + b3;
    *hi = sh + b3;
}
