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
//   L = (1/N) sum_s softplus(o_s) - y_s o_s,   dL/do_s = (sigmoid(o_s) - y_s) / N.
__global__ void __launch_bounds__(RL0_MLP_BLOCK) k_mlp_grad_block(const float *__restrict__ w,
                                                                   const float *__restrict__ feat,
                                                                   const float *__restrict__ label, long long N,
                                                                   float *__restrict__ part, double *loss_part)
{
    extern __shared__ float sm[];
    float *W = sm;                                          // RL0_MLP_PARAMS
    float *F = W + RL0_MLP_PARAMS;                          // [B][16]
    float *H1 = F + RL0_MLP_BLOCK * RL0_NFEAT;              // [B][32]
    float *D1 = H1 + RL0_MLP_BLOCK * RL0_HID;               // [B][32] dL/dz1
    float *H2 = D1 + RL0_MLP_BLOCK * RL0_HID;               // [B][32]
    float *D2 = H2 + RL0_MLP_BLOCK * RL0_HID;               // [B][32] dL/dz2
    float *DO = D2 + RL0_MLP_BLOCK * RL0_HID;               // [B]
    __shared__ double s_loss[RL0_MLP_BLOCK];
    const int t = threadIdx.x;
    for (int p = t; p < RL0_MLP_PARAMS; p += RL0_MLP_BLOCK) W[p] = w[p];
    const long long sidx = (long long)blockIdx.x * RL0_MLP_BLOCK + t;
    const bool valid = sidx < N;
    for (int i = 0; i < RL0_NFEAT; ++i) F[t * RL0_NFEAT + i] = valid ? feat[sidx * RL0_NFEAT + i] : 0.0f;
    __syncthreads();
    // forward, one sample per thread
    float z1[RL0_HID], z2[RL0_HID];
#pragma unroll
    for (int o = 0; o < RL0_HID; ++o) {
        float acc = W[RL0_OFF_B1 + o];
#pragma unroll
        for (int i = 0; i < RL0_NFEAT; ++i) acc = fmaf(F[t * RL0_NFEAT + i], W[RL0_OFF_W1 + i * RL0_HID + o], acc);
        z1[o] = acc;
        H1[t * RL0_HID + o] = fmaxf(acc, 0.0f);
    }
    float out = W[RL0_OFF_B3];
#pragma unroll 4
    for (int o = 0; o < RL0_HID; ++o) {
        float acc = W[RL0_OFF_B2 + o];
#pragma unroll
        for (int i = 0; i < RL0_HID; ++i) acc = fmaf(H1[t * RL0_HID + i], W[RL0_OFF_W2 + i * RL0_HID + o], acc);
        z2[o] = acc;
        H2[t * RL0_HID + o] = fmaxf(acc, 0.0f);
        out = fmaf(fmaxf(acc, 0.0f), W[RL0_OFF_W3 + o], out);
    }
    // loss and backward
    const float y = valid ? label[sidx] : 0.0f;
    const float sig = 1.0f / (1.0f + expf(-out));
    const float dout = valid ? (sig - y) / (float)N : 0.0f;
    const double sp = (out > 0.0f) ? (double)out + log1p(exp(-(double)out)) : log1p(exp((double)out));
    s_loss[t] = valid ? (sp - (double)y * (double)out) : 0.0;
    DO[t] = dout;
#pragma unroll
    for (int o = 0; o < RL0_HID; ++o) D2[t * RL0_HID + o] = (z2[o] > 0.0f) ? dout * W[RL0_OFF_W3 + o] : 0.0f;
#pragma unroll 4
    for (int i = 0; i < RL0_HID; ++i) {
        float acc = 0.0f;
#pragma unroll
        for (int o = 0; o < RL0_HID; ++o) acc = fmaf(W[RL0_OFF_W2 + i * RL0_HID + o], D2[t * RL0_HID + o], acc);
        D1[t * RL0_HID + i] = (z1[i] > 0.0f) ? acc : 0.0f;
    }
    __syncthreads();
    // block sums over samples in index order: dW1 = F^T D1, db1 = sum D1, dW2 = H1^T D2, ...
    float *P = part + (long long)blockIdx.x * RL0_MLP_PARAMS;
    for (int p = t; p < RL0_MLP_PARAMS; p += RL0_MLP_BLOCK) {
        float acc = 0.0f;
        if (p < RL0_OFF_B1) {
            const int i = p / RL0_HID, o = p % RL0_HID;
            for (int s = 0; s < RL0_MLP_BLOCK; ++s) acc = fmaf(F[s * RL0_NFEAT + i], D1[s * RL0_HID + o], acc);
        } else if (p < RL0_OFF_W2) {
            const int o = p - RL0_OFF_B1;
            for (int s = 0; s < RL0_MLP_BLOCK; ++s) acc += D1[s * RL0_HID + o];
        } else if (p < RL0_OFF_B2) {
            const int q = p - RL0_OFF_W2, i = q / RL0_HID, o = q % RL0_HID;
            for (int s = 0; s < RL0_MLP_BLOCK; ++s) acc = fmaf(H1[s * RL0_HID + i], D2[s * RL0_HID + o], acc);
        } else if (p < RL0_OFF_W3) {
            const int o = p - RL0_OFF_B2;
            for (int s = 0; s < RL0_MLP_BLOCK; ++s) acc += D2[s * RL0_HID + o];
        } else if (p < RL0_OFF_B3) {
            const int o = p - RL0_OFF_W3;
            for (int s = 0; s < RL0_MLP_BLOCK; ++s) acc = fmaf(H2[s * RL0_HID + o], DO[s], acc);
        } else {
            for (int s = 0; s < RL0_MLP_BLOCK; ++s) acc += DO[s];
        }
        P[p] = acc;
    }
    const double l = group_sum_f64(s_loss[t], s_loss, t, RL0_MLP_BLOCK);
    if (t == 0) loss_part[blockIdx.x] = l;
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

// Adam (Kingma and Ba, 2015) with bias correction.
__global__ void k_mlp_adam(float *w, float *m, float *v, const float *g, int step, float lr, float b1, float b2,
                           float eps)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= RL0_MLP_PARAMS) return;
    const float gp = g[p];
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
    return sizeof(float) * (RL0_MLP_PARAMS + RL0_MLP_BLOCK * (RL0_NFEAT + 4 * RL0_HID + 1));
}

static int mlp_grad_launch(const float *w, const float *feat, const float *label, long long N, float *grad,
                           double *loss, float *part, double *loss_part, cudaStream_t s)
{
    const int nb = (int)((N + RL0_MLP_BLOCK - 1) / RL0_MLP_BLOCK);
    const size_t sm = grad_smem();
    CK(cudaFuncSetAttribute((const void *)k_mlp_grad_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_mlp_grad_block<<<nb, RL0_MLP_BLOCK, sm, s>>>(w, feat, label, N, part, loss_part);
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
    for (int ep = 0; ep < epochs && !rc; ++ep) {
        for (int64_t b0 = 0; b0 < N && !rc; b0 += batch) {
            const long long nb = (N - b0 < batch) ? (N - b0) : batch;
            rc = mlp_grad_launch(w_dev, feat_dev + b0 * RL0_NFEAT, label_dev + b0, nb, grad, ld, part, lp, s);
            ++step;
            k_mlp_adam<<<(RL0_MLP_PARAMS + 255) / 256, 256, 0, s>>>(w_dev, m, v, grad, step, lr, 0.9f, 0.999f,
                                                                   1e-8f);
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

extern "C" int rl0_mlp_params(void) { return RL0_MLP_PARAMS; }
