// rl0_mlp.cu -- the learned column scorer's network: a 16 -> 32 -> 32 -> 1 MLP
// with ReLU hidden layers and a logistic output, trained with binary
// cross-entropy on candidate features logged from analytic Robust-l0 decodes
// (labels: the candidate update x_j + w lands on the true x_j).  FP32 master
// weights train here; decodes use a BF16 copy with FP32 accumulation, on the
// tensor cores (rl0_mma.cuh).
//
// The gradient is deterministic: each block of RL0_MLP_BLOCK samples writes its
// own partial gradient (sums over its samples in index order), and a second
// kernel adds the block partials in block order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>

#include "rl0_common.cuh"
#include "rl0_device.cuh"
#include "rl0_mma.cuh"

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return rl0_cuda_err(e_);   \
    } while (0)

#define RL0_MLP_BLOCK 128

// He-normal initial weights (std sqrt(2 / fan_in)), zero biases.  Normal
// deviates by Box-Muller from a 64-bit mixing hash of (seed, index).
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_mlp_init(unsigned long long seed, float *w)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= RL0_MLP_PARAMS) return;
    float fan = 0.0f;
    if (p < RL0_OFF_B1) fan = RL0_NFEAT;
    else if (p >= RL0_OFF_W2 && p < RL0_OFF_B2) fan = RL0_HID;
    else if (p >= RL0_OFF_W3 && p < RL0_OFF_B3) fan = RL0_HID;
    if (fan == 0.0f) { w[p] = 0.0f; return; }
    const unsigned long long h = mix64(seed * 0x100000001B3ull + (unsigned long long)p);
    const double u1 = ((double)(h >> 40) + 1.0) / 16777216.0;
    const double u2 = (double)((h >> 16) & 0xFFFFFFull) / 16777216.0;
    const double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    w[p] = (float)(z * sqrt(2.0 / fan));
}

// Per-block loss and gradient of the mean binary cross-entropy
//   L = (1/N) sum_s softplus(o_s) - y_s o_s,   dL/do_s = (sigmoid(o_s) - y_s) / N,
// on the tensor cores.  Warp w takes samples 16w .. 16w+15 of the block through
// the forward pass (z1 = F W1 + b1, z2 = relu(z1) W2 + b2) and the backward pass
// (D2 = relu'(z2) dL/do w3^T, D1 = relu'(z1) (D2 W2^T)) as m16n8k16 tiles,
// keeping every activation in its accumulator fragment; then the block forms
// dW1 = F^T D1 and dW2 = H1^T D2 (K = the block's samples) as 12 output tiles of
// 16 x 8, and the vector terms (biases, w3) with FP32 sums in sample order.
// Both operands of every product are FP32 split into three BF16 parts.
#define RL0_MLP_WARPS (RL0_MLP_BLOCK / 16)
#define RL0_MLP_LDF 20                                     // row pitch of F in shared memory
#define RL0_MLP_LDH 36                                     // row pitch of H1, D1, H2, D2

__global__ void __launch_bounds__(RL0_MLP_WARPS * 32) k_mlp_grad_block(const float *__restrict__ w,
                                                                        const float *__restrict__ feat,
                                                                        const float *__restrict__ label,
                                                                        long long N, float *__restrict__ part,
                                                                        double *loss_part)
{
    extern __shared__ float sm[];
    float *W = sm;                                          // RL0_MLP_PARAMS (+3 pad)
    float *F = W + RL0_MLP_PARAMS + 3;                      // [B][LDF]
    float *H1 = F + RL0_MLP_BLOCK * RL0_MLP_LDF;            // [B][LDH] relu(z1)
    float *D1 = H1 + RL0_MLP_BLOCK * RL0_MLP_LDH;           // [B][LDH] dL/dz1
    float *H2 = D1 + RL0_MLP_BLOCK * RL0_MLP_LDH;           // [B][LDH] relu(z2)
    float *D2 = H2 + RL0_MLP_BLOCK * RL0_MLP_LDH;           // [B][LDH] dL/dz2
    float *DO = D2 + RL0_MLP_BLOCK * RL0_MLP_LDH;           // [B] dL/do
    __shared__ double s_loss[RL0_MLP_BLOCK];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int g = lane >> 2, q = lane & 3;
    const long long s0 = (long long)blockIdx.x * RL0_MLP_BLOCK;
    for (int p = t; p < RL0_MLP_PARAMS; p += blockDim.x) W[p] = w[p];
    for (int e = t; e < RL0_MLP_BLOCK * RL0_NFEAT; e += blockDim.x) {
        const int s = e / RL0_NFEAT, i = e % RL0_NFEAT;
        F[s * RL0_MLP_LDF + i] = (s0 + s < N) ? feat[s0 * RL0_NFEAT + e] : 0.0f;
    }
    __syncthreads();
    const int r0 = 16 * wid;                                // this warp's first sample in the block
    // ---- forward ----
    unsigned af[3][4];
    a_frag_split3_fn([&](int r, int c) { return F[(r0 + r) * RL0_MLP_LDF + c]; }, af);
    float c1[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float b0 = W[RL0_OFF_B1 + 8 * nt + 2 * q], b1 = W[RL0_OFF_B1 + 8 * nt + 2 * q + 1];
        c1[nt][0] = b0;
        c1[nt][1] = b1;
        c1[nt][2] = b0;
        c1[nt][3] = b1;
        unsigned bw[3][2];
        b_frag_split3_fn([&](int k, int n) { return W[RL0_OFF_W1 + k * RL0_HID + 8 * nt + n]; }, bw);
        mma_split3x3(c1[nt], af, bw);
    }
    float c2[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float b0 = W[RL0_OFF_B2 + 8 * nt + 2 * q], b1 = W[RL0_OFF_B2 + 8 * nt + 2 * q + 1];
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
            unsigned bw[3][2];
            b_frag_split3_fn([&](int k, int n) { return W[RL0_OFF_W2 + (16 * kk + k) * RL0_HID + 8 * nt + n]; }, bw);
            mma_split3x3(c2[nt], a2, bw);
        }
    }
    float ol = 0.0f, oh = 0.0f;                             // rows g and g + 8
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float w0 = W[RL0_OFF_W3 + 8 * nt + 2 * q], w1 = W[RL0_OFF_W3 + 8 * nt + 2 * q + 1];
        ol = fmaf(fmaxf(c2[nt][0], 0.0f), w0, ol);
        ol = fmaf(fmaxf(c2[nt][1], 0.0f), w1, ol);
        oh = fmaf(fmaxf(c2[nt][2], 0.0f), w0, oh);
        oh = fmaf(fmaxf(c2[nt][3], 0.0f), w1, oh);
    }
    ol += __shfl_xor_sync(0xffffffffu, ol, 1);
    ol += __shfl_xor_sync(0xffffffffu, ol, 2);
    oh += __shfl_xor_sync(0xffffffffu, oh, 1);
    oh += __shfl_xor_sync(0xffffffffu, oh, 2);
    ol += W[RL0_OFF_B3];
    oh += W[RL0_OFF_B3];
    // ---- loss and dL/do of rows g and g + 8 ----
    float dl, dh;
    {
        const long long sl = s0 + r0 + g, sh = sl + 8;
        const bool vl = sl < N, vh = sh < N;
        const float yl = vl ? label[sl] : 0.0f, yh = vh ? label[sh] : 0.0f;
        dl = vl ? (1.0f / (1.0f + expf(-ol)) - yl) / (float)N : 0.0f;
        dh = vh ? (1.0f / (1.0f + expf(-oh)) - yh) / (float)N : 0.0f;
        if (q == 0) {
            const double spl = (ol > 0.0f) ? (double)ol + log1p(exp(-(double)ol)) : log1p(exp((double)ol));
            const double sph = (oh > 0.0f) ? (double)oh + log1p(exp(-(double)oh)) : log1p(exp((double)oh));
            s_loss[r0 + g] = vl ? spl - (double)yl * (double)ol : 0.0;
            s_loss[r0 + g + 8] = vh ? sph - (double)yh * (double)oh : 0.0;
            DO[r0 + g] = dl;
            DO[r0 + g + 8] = dh;
        }
    }
    // ---- backward: D2 in c2's layout, D1 = relu'(z1) (D2 W2^T) ----
    float d2[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float w0 = W[RL0_OFF_W3 + 8 * nt + 2 * q], w1 = W[RL0_OFF_W3 + 8 * nt + 2 * q + 1];
        d2[nt][0] = (c2[nt][0] > 0.0f) ? dl * w0 : 0.0f;
        d2[nt][1] = (c2[nt][1] > 0.0f) ? dl * w1 : 0.0f;
        d2[nt][2] = (c2[nt][2] > 0.0f) ? dh * w0 : 0.0f;
        d2[nt][3] = (c2[nt][3] > 0.0f) ? dh * w1 : 0.0f;
    }
    float d1[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) d1[nt][e] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {                        // K = the 32 units of z2
        float v[8];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            v[e] = d2[2 * kk][e];
            v[4 + e] = d2[2 * kk + 1][e];
        }
        unsigned a2[3][4];
        a_frag_split3(v, a2);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {                    // N = the 32 units of z1; B(k, n) = W2[n][k]
            unsigned bw[3][2];
            b_frag_split3_fn([&](int k, int n) { return W[RL0_OFF_W2 + (8 * nt + n) * RL0_HID + 16 * kk + k]; },
                             bw);
            mma_split3x3(d1[nt], a2, bw);
        }
    }
    // fragments to shared memory (rows r0 + g and r0 + g + 8, columns 8nt + 2q + {0, 1})
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int o = (r0 + g + ((e & 2) ? 8 : 0)) * RL0_MLP_LDH + 8 * nt + 2 * q + (e & 1);
            H1[o] = fmaxf(c1[nt][e], 0.0f);
            D1[o] = (c1[nt][e] > 0.0f) ? d1[nt][e] : 0.0f;
            H2[o] = fmaxf(c2[nt][e], 0.0f);
            D2[o] = d2[nt][e];
        }
    __syncthreads();
    // ---- weight matrices: 4 tiles of dW1 (16 x 32) and 8 of dW2 (32 x 32), K = the block's samples ----
    float *P = part + (long long)blockIdx.x * RL0_MLP_PARAMS;
    for (int tile = wid; tile < 12; tile += RL0_MLP_WARPS) {
        const bool l1 = tile < 4;
        const float *X = l1 ? F : H1;                       // A = X^T
        const float *D = l1 ? D1 : D2;                      // B = D
        const int ldx = l1 ? RL0_MLP_LDF : RL0_MLP_LDH;
        const int m0 = l1 ? 0 : 16 * ((tile - 4) >> 2);
        const int n0 = 8 * (l1 ? tile : ((tile - 4) & 3));
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 2
        for (int ks = 0; ks < RL0_MLP_BLOCK / 16; ++ks) {
            unsigned ax[3][4], bd[3][2];
            a_frag_split3_fn([&](int r, int c) { return X[(16 * ks + c) * ldx + m0 + r]; }, ax);
            b_frag_split3_fn([&](int k, int n) { return D[(16 * ks + k) * RL0_MLP_LDH + n0 + n]; }, bd);
            mma_split3x3(acc, ax, bd);
        }
        const int off = l1 ? RL0_OFF_W1 : RL0_OFF_W2;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            P[off + (m0 + g + ((e & 2) ? 8 : 0)) * RL0_HID + n0 + 2 * q + (e & 1)] = acc[e];
    }
    // ---- vectors: db1, db2, dw3 (sums over samples in index order) and db3 ----
    if (t < 3 * RL0_HID + 1) {
        float acc = 0.0f;
        if (t < RL0_HID) {
            for (int s = 0; s < RL0_MLP_BLOCK; ++s) acc += D1[s * RL0_MLP_LDH + t];
            P[RL0_OFF_B1 + t] = acc;
        } else if (t < 2 * RL0_HID) {
            const int o = t - RL0_HID;
            for (int s = 0; s < RL0_MLP_BLOCK; ++s) acc += D2[s * RL0_MLP_LDH + o];
            P[RL0_OFF_B2 + o] = acc;
        } else if (t < 3 * RL0_HID) {
            const int o = t - 2 * RL0_HID;
            for (int s = 0; s < RL0_MLP_BLOCK; ++s) acc = fmaf(H2[s * RL0_MLP_LDH + o], DO[s], acc);
            P[RL0_OFF_W3 + o] = acc;
        } else {
            for (int s = 0; s < RL0_MLP_BLOCK; ++s) acc += DO[s];
            P[RL0_OFF_B3] = acc;
        }
    }
    if (t == 0) {
        double l = 0.0;
        for (int s = 0; s < RL0_MLP_BLOCK; ++s) l += s_loss[s];
        loss_part[blockIdx.x] = l;
    }
}

// grad[p] = sum over blocks (in block order) of the block partials.
__global__ void k_mlp_grad_reduce(const float *part, int nblocks, float *grad, const double *loss_part, double *loss,
                                  long long N)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < RL0_MLP_PARAMS) {
        float acc = 0.0f;
        for (int b = 0; b < nblocks; ++b) acc += part[(long long)b * RL0_MLP_PARAMS + p];
        grad[p] = acc;
    }
    if (p == 0 && loss) {
        double l = 0.0;
        for (int b = 0; b < nblocks; ++b) l += loss_part[b];
        *loss = l / (double)N;
    }
}

// Adam (Kingma and Ba, 2015) with bias correction, on the gradient
// g = sum over blocks (in block order) of the block partials.
__global__ void k_mlp_reduce_adam(const float *part, int nblocks, float *w, float *m, float *v, int step, float lr,
                                  float b1, float b2, float eps)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= RL0_MLP_PARAMS) return;
    float gp = 0.0f;
    for (int b = 0; b < nblocks; ++b) gp += part[(long long)b * RL0_MLP_PARAMS + p];
    const float mp = b1 * m[p] + (1.0f - b1) * gp;
    const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float mh = mp / (1.0f - powf(b1, (float)step));
    const float vh = vp / (1.0f - powf(b2, (float)step));
    w[p] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_mlp_export(const float *w, __nv_bfloat16 *wb)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < RL0_MLP_PARAMS) wb[p] = __float2bfloat16_rn(w[p]);
}

// Logits of N feature rows with the BF16 parameters: the decoder's arithmetic
// (warp_mlp_logits16 on the tensor cores), one warp per 16 rows.
__global__ void __launch_bounds__(256) k_mlp_forward(const __nv_bfloat16 *wb, const float *feat, long long N,
                                                      float *logit)
{
    const long long r0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32 * 16;
    if (r0 >= N) return;                           // whole warps leave together
    auto f = [&](int r, int i) { return (r0 + r < N) ? feat[(r0 + r) * RL0_NFEAT + i] : 0.0f; };
    float lo, hi;
    warp_mlp_logits16(f, wb, &lo, &hi);
    const int g = (threadIdx.x & 31) >> 2;
    if ((threadIdx.x & 3) == 0) {
        if (r0 + g < N) logit[r0 + g] = lo;
        if (r0 + g + 8 < N) logit[r0 + g + 8] = hi;
    }
}

// ---------------------------------------------------------------------------
// Host
// ---------------------------------------------------------------------------
static size_t grad_smem()
{
    return sizeof(float) * (RL0_MLP_PARAMS + 3 + RL0_MLP_BLOCK * (RL0_MLP_LDF + 4 * RL0_MLP_LDH + 1));
}

static int mlp_grad_launch(const float *w, const float *feat, const float *label, long long N, float *grad,
                           double *loss, float *part, double *loss_part, cudaStream_t s)
{
    const int nb = (int)((N + RL0_MLP_BLOCK - 1) / RL0_MLP_BLOCK);
    const size_t sm = grad_smem();
    CK(cudaFuncSetAttribute((const void *)k_mlp_grad_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_mlp_grad_block<<<nb, RL0_MLP_WARPS * 32, sm, s>>>(w, feat, label, N, part, loss_part);
    k_mlp_grad_reduce<<<(RL0_MLP_PARAMS + 255) / 256, 256, 0, s>>>(part, nb, grad, loss_part, loss, N);
    CK(cudaGetLastError());
    return RL0_OK;
}

extern "C" int rl0_mlp_init(uint64_t seed, float *w_dev, void *cuda_stream)
{
    if (!w_dev) return RL0_ERR_INVALID_ARG;
    k_mlp_init<<<(RL0_MLP_PARAMS + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(seed, w_dev);
    CK(cudaGetLastError());
    return RL0_OK;
}

extern "C" int rl0_mlp_grad(const float *w_dev, const float *feat_dev, const float *label_dev, int64_t N,
                            float *grad_dev, double *loss_host, void *cuda_stream)
{
    if (!w_dev || !feat_dev || !label_dev || !grad_dev || N < 1) return RL0_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nb = (int)((N + RL0_MLP_BLOCK - 1) / RL0_MLP_BLOCK);
    float *part = nullptr;
    double *lp = nullptr, *ld = nullptr;
    CK(cudaMallocAsync(&part, (size_t)nb * RL0_MLP_PARAMS * sizeof(float), s));
    CK(cudaMallocAsync(&lp, (size_t)nb * sizeof(double), s));
    CK(cudaMallocAsync(&ld, sizeof(double), s));
    int rc = mlp_grad_launch(w_dev, feat_dev, label_dev, N, grad_dev, ld, part, lp, s);
    double l = 0.0;
    if (!rc) rc = rl0_cuda_err(cudaMemcpyAsync(&l, ld, sizeof(double), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(part, s);
    cudaFreeAsync(lp, s);
    cudaFreeAsync(ld, s);
    if (!rc) rc = rl0_cuda_err(cudaStreamSynchronize(s));
    if (loss_host) *loss_host = l;
    return rc;
}

extern "C" int rl0_mlp_train(float *w_dev, const float *feat_dev, const float *label_dev, int64_t N, int epochs,
                             int batch, float lr, void *wbf16_dev, double *loss_host, void *cuda_stream)
{
    if (!w_dev || !feat_dev || !label_dev || N < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f))
        return RL0_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nbmax = (batch + RL0_MLP_BLOCK - 1) / RL0_MLP_BLOCK;
    float *part = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    double *lp = nullptr, *ld = nullptr;
    CK(cudaMallocAsync(&part, (size_t)nbmax * RL0_MLP_PARAMS * sizeof(float), s));
    CK(cudaMallocAsync(&lp, (size_t)nbmax * sizeof(double), s));
    CK(cudaMallocAsync(&ld, sizeof(double), s));
    CK(cudaMallocAsync(&grad, RL0_MLP_PARAMS * sizeof(float), s));
    CK(cudaMallocAsync(&m, RL0_MLP_PARAMS * sizeof(float), s));
    CK(cudaMallocAsync(&v, RL0_MLP_PARAMS * sizeof(float), s));
    CK(cudaMemsetAsync(m, 0, RL0_MLP_PARAMS * sizeof(float), s));
    CK(cudaMemsetAsync(v, 0, RL0_MLP_PARAMS * sizeof(float), s));
    int rc = RL0_OK, step = 0;
    const size_t sm = grad_smem();
    CK(cudaFuncSetAttribute((const void *)k_mlp_grad_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    for (int ep = 0; ep < epochs && !rc; ++ep) {
        for (int64_t b0 = 0; b0 < N && !rc; b0 += batch) {
            const long long nb = (N - b0 < batch) ? (N - b0) : batch;
            const int nblk = (int)((nb + RL0_MLP_BLOCK - 1) / RL0_MLP_BLOCK);
            k_mlp_grad_block<<<nblk, RL0_MLP_WARPS * 32, sm, s>>>(w_dev, feat_dev + b0 * RL0_NFEAT, label_dev + b0,
                                                                 nb, part, lp);
            ++step;
            k_mlp_reduce_adam<<<(RL0_MLP_PARAMS + 255) / 256, 256, 0, s>>>(part, nblk, w_dev, m, v, step, lr, 0.9f,
                                                                          0.999f, 1e-8f);
            rc = rl0_cuda_err(cudaGetLastError());
        }
    }
    if (!rc) {
        // loss of the final weights over the whole set
        float *pf = nullptr;
        double *pl = nullptr;
        const int nball = (int)((N + RL0_MLP_BLOCK - 1) / RL0_MLP_BLOCK);
        rc = rl0_cuda_err(cudaMallocAsync(&pf, (size_t)nball * RL0_MLP_PARAMS * sizeof(float), s));
        if (!rc) rc = rl0_cuda_err(cudaMallocAsync(&pl, (size_t)nball * sizeof(double), s));
        if (!rc) rc = mlp_grad_launch(w_dev, feat_dev, label_dev, N, grad, ld, pf, pl, s);
        double l = 0.0;
        if (!rc) rc = rl0_cuda_err(cudaMemcpyAsync(&l, ld, sizeof(double), cudaMemcpyDeviceToHost, s));
        if (pf) cudaFreeAsync(pf, s);
        if (pl) cudaFreeAsync(pl, s);
        if (!rc && wbf16_dev)
            k_mlp_export<<<(RL0_MLP_PARAMS + 255) / 256, 256, 0, s>>>(w_dev, (__nv_bfloat16 *)wbf16_dev);
        if (!rc) rc = rl0_cuda_err(cudaStreamSynchronize(s));
        if (loss_host) *loss_host = l;
    }
    cudaFreeAsync(part, s);
    cudaFreeAsync(lp, s);
    cudaFreeAsync(ld, s);
    cudaFreeAsync(grad, s);
    cudaFreeAsync(m, s);
    cudaFreeAsync(v, s);
    cudaStreamSynchronize(s);
    return rc;
}

extern "C" int rl0_mlp_export(const float *w_dev, void *wbf16_dev, void *cuda_stream)
{
    if (!w_dev || !wbf16_dev) return RL0_ERR_INVALID_ARG;
    k_mlp_export<<<(RL0_MLP_PARAMS + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(w_dev,
                                                                                     (__nv_bfloat16 *)wbf16_dev);
    CK(cudaGetLastError());
    return RL0_OK;
}

extern "C" int rl0_mlp_forward(const void *wbf16_dev, const float *feat_dev, int64_t N, float *logit_dev,
                               void *cuda_stream)
{
    if (!wbf16_dev || !feat_dev || !logit_dev || N < 0) return RL0_ERR_INVALID_ARG;
    if (N == 0) return RL0_OK;
    // 16 rows per warp, 8 warps per block
    k_mlp_forward<<<(unsigned)((N + 127) / 128), 256, 0, (cudaStream_t)cuda_stream>>>(
        (const __nv_bfloat16 *)wbf16_dev, feat_dev, N, logit_dev);
    CK(cudaGetLastError());
    return RL0_OK;
}

// ---------------------------------------------------------------------------
// Training data: the candidates met along an analytic decode, labelled
// ---------------------------------------------------------------------------

// sum |v_i| in FP64, one block, fixed order
__global__ void k_l1_f64(const float *v, int n, double *out)
{
    __shared__ double sh[1024];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += fabs((double)v[i]);
    const double r = group_sum_f64(acc, sh, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) *out = r;
}

// label of candidate e: the update x_hat_j + w lands within tol of x_true_j != 0
__global__ void k_label(const int32_t *meta, const float *omega, const float *xhat, const float *xtrue, int c,
                        float tol, float *label)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c) return;
    const int j = meta[4 * e];
    const float xt = xtrue[j];
    const float prop = xhat[j] + omega[e];
    label[e] = (fabsf(prop - xt) <= tol && xt != 0.0f) ? 1.0f : 0.0f;
}

extern "C" int rl0_scorer_log(const rl0_expander *A, const float *y_dev, int64_t k, const rl0_params *params,
                              const float *xtrue_dev, float tol_sigma, int max_rounds, float *feat_dev,
                              float *label_dev, int64_t cap, int64_t *count_out, int *rounds_out,
                              void *cuda_stream)
{
    if (!A || !y_dev || !params || !xtrue_dev || !count_out || cap < 0 || (cap > 0 && (!feat_dev || !label_dev)) ||
        !(tol_sigma > 0.0f) || max_rounds < 2 || max_rounds > RL0_MAX_ROUNDS)
        return RL0_ERR_INVALID_ARG;
    if (params->scorer != 0 || params->adaptive_k) return RL0_ERR_UNSUPPORTED;
    if (!(params->sigma_n > 0.0)) return RL0_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t n = A->n, m = A->m;
    // candidates of one round: at most one per (column, anchor slot)
    const int64_t per_round = std::min<int64_t>(n * A->d, (int64_t)0x7fffffff);
    float *xh = nullptr, *rh = nullptr, *xp = nullptr, *rp = nullptr, *om = nullptr, *ftmp = nullptr;
    int32_t *meta = nullptr;
    double *dl1 = nullptr;
    int rc = RL0_OK;
    auto alloc = [&](void **p, size_t bytes) {
        if (!rc) rc = rl0_cuda_err(cudaMallocAsync(p, bytes, s));
    };
    alloc((void **)&xh, n * sizeof(float));
    alloc((void **)&xp, n * sizeof(float));
    alloc((void **)&rh, m * sizeof(float));
    alloc((void **)&rp, m * sizeof(float));
    alloc((void **)&meta, per_round * 4 * sizeof(int32_t));
    alloc((void **)&om, per_round * sizeof(float));
    alloc((void **)&ftmp, per_round * RL0_NFEAT * sizeof(float));
    alloc((void **)&dl1, sizeof(double));
    if (!rc) rc = rl0_cuda_err(cudaMemsetAsync(xh, 0, n * sizeof(float), s));
    if (!rc) rc = rl0_cuda_err(cudaMemcpyAsync(rh, y_dev, m * sizeof(float), cudaMemcpyDeviceToDevice, s));
    double l1h = 0.0;
    if (!rc) {
        k_l1_f64<<<1, 1024, 0, s>>>(y_dev, (int)m, dl1);
        rc = rl0_cuda_err(cudaMemcpyAsync(&l1h, dl1, sizeof(double), cudaMemcpyDeviceToHost, s));
        if (!rc) rc = rl0_cuda_err(cudaStreamSynchronize(s));
    }
    // the noise floor E||eta||_1 = m sigma_n sqrt(2 / pi): the decode's stop level
    const double stop = (double)m * params->sigma_n * sqrt(2.0 / M_PI);
    const float tol = (float)(tol_sigma * params->sigma_n);
    int64_t total = 0;
    int rounds = 0;
    for (int r = 1; r < max_rounds && !rc; ++r) {
        int c = 0;
        rc = rl0_candidate_features(A, y_dev, k, params, r, xh, rh, ftmp, meta, om, (int)per_round, &c, cuda_stream);
        if (rc) break;
        const int64_t take = std::min<int64_t>(c, cap - std::min(cap, total));
        if (take > 0) {
            rc = rl0_cuda_err(cudaMemcpyAsync(feat_dev + total * RL0_NFEAT, ftmp, take * RL0_NFEAT * sizeof(float),
                                              cudaMemcpyDeviceToDevice, s));
            if (rc) break;
            k_label<<<(unsigned)((take + 255) / 256), 256, 0, s>>>(meta, om, xh, xtrue_dev, (int)take, tol,
                                                                  label_dev + total);
            rc = rl0_cuda_err(cudaGetLastError());
            if (rc) break;
        }
        total += c;
        double l1 = 0.0;
        rc = rl0_round_step(A, y_dev, k, params, r, xh, rh, xp, rp, nullptr, &l1, cuda_stream);
        if (rc) break;
        ++rounds;
        if (l1 < l1h) {                            // accept: ||r||_1 < ||r_hat||_1
            std::swap(xh, xp);
            std::swap(rh, rp);
            l1h = l1;
        }
        if (l1h <= stop) break;
    }
    for (void *p : {(void *)xh, (void *)rh, (void *)xp, (void *)rp, (void *)om, (void *)ftmp, (void *)meta,
                    (void *)dl1})
        if (p) cudaFreeAsync(p, s);
    const int rs = rl0_cuda_err(cudaStreamSynchronize(s));
    if (!rc) rc = rs;
    *count_out = total;
    if (rounds_out) *rounds_out = rounds;
    return rc;
}

extern "C" int rl0_mlp_params(void) { return RL0_MLP_PARAMS; }
