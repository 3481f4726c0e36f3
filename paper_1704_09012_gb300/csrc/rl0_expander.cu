// rl0_expander.cu -- the expander matrix A of Def. 1.1 and the generating model
// GM(n,m,k,d,mu,nu) (Def. "Generating model", Fig. 1) on the GPU: drawing A,
// validating caller rows, the slot-major and CSR(A^T) copies, and the sketch
// y_hat = A x + eta.
#include <cstdio>
#include <cstring>
#include <new>

#include "rl0_common.cuh"

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 multiplies
// with the key advanced by the golden-ratio Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct PhiloxOut {
    uint32_t v[4];
};

__device__ __forceinline__ PhiloxOut philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                   uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t o0 = hi1 ^ c1 ^ k0, o2 = hi0 ^ c3 ^ k1;
        c0 = o0; c1 = lo1; c2 = o2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    PhiloxOut r;
    r.v[0] = c0; r.v[1] = c1; r.v[2] = c2; r.v[3] = c3;
    return r;
}

// Word stream for one id: counter = (block, id_lo, id_hi, tag), key = seed.
struct WordStream {
    uint32_t k0, k1, id_lo, id_hi, tag, block;
    uint32_t buf[4];
    int pos;
    __device__ uint32_t next()
    {
        if (pos == 4) {
            PhiloxOut o = philox4x32_10(block, id_lo, id_hi, tag, k0, k1);
            buf[0] = o.v[0]; buf[1] = o.v[1]; buf[2] = o.v[2]; buf[3] = o.v[3];
            ++block;
            pos = 0;
        }
        return buf[pos++];
    }
};

#define TAG_EXPANDER 0x41u
#define TAG_NOISE 0x4Eu

// Column j: draw words, map each to [0, m) by Lemire's multiply-shift with
// rejection (exactly uniform), keep the first d distinct values, sort.
__global__ void k_make_expander(int n, int m, int d, uint32_t k0, uint32_t k1, int32_t *rows, int *err)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    WordStream ws{k0, k1, (uint32_t)j, 0u, TAG_EXPANDER, 0u, {0, 0, 0, 0}, 4};
    int32_t col[RL0_MAX_D];
    const uint32_t um = (uint32_t)m;
    const uint32_t thresh = (0u - um) % um;
    int got = 0;
    const int budget = 64 * d + 256;
    for (int draw = 0; draw < budget && got < d; ++draw) {
        uint64_t prod = (uint64_t)ws.next() * um;
        if ((uint32_t)prod < thresh) continue;      // rejected word
        const int32_t cand = (int32_t)(prod >> 32);
        bool dup = false;
        for (int q = 0; q < got; ++q) dup |= (col[q] == cand);
        if (!dup) col[got++] = cand;
    }
    if (got < d) {
        atomicExch(err, 1);
        for (int q = got; q < d; ++q) col[q] = 0;
    }
    for (int a = 1; a < d; ++a) {                   // insertion sort, d <= 32
        const int32_t v = col[a];
        int b = a - 1;
        while (b >= 0 && col[b] > v) { col[b + 1] = col[b]; --b; }
        col[b + 1] = v;
    }
    for (int q = 0; q < d; ++q) rows[(int64_t)j * d + q] = col[q];
}

// Caller rows must be strictly ascending within a column and inside [0, m).
__global__ void k_validate_rows(int n, int m, int d, const int32_t *rows, int *bad)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int32_t prev = -1;
    for (int q = 0; q < d; ++q) {
        const int32_t v = rows[(int64_t)j * d + q];
        if (v <= prev || v >= m) { atomicExch(bad, 1); return; }
        prev = v;
    }
}

__global__ void k_slot_major(int n, int d, const int32_t *rows_cm, int32_t *rows_sm)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * d) return;
    const int j = (int)(e / d), s = (int)(e % d);
    rows_sm[(int64_t)s * n + j] = rows_cm[e];
}

__global__ void k_row_count(int64_t nnz, const int32_t *rows_cm, int32_t *cnt1)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) atomicAdd(&cnt1[rows_cm[e] + 1], 1);
}

// Exclusive-scan building blocks over int32 (m+1 entries): per-block inclusive
// scan of 1024 values, a scan of the block totals, then the offsets.
__global__ void k_scan_blocks(int len, int32_t *a, int32_t *block_tot)
{
    __shared__ int32_t sh[1024];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    sh[threadIdx.x] = (i < len) ? a[i] : 0;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int32_t v = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    if (i < len) a[i] = sh[threadIdx.x];
    if (threadIdx.x == 1023) block_tot[blockIdx.x] = sh[1023];
}

__global__ void k_scan_totals(int nb, int32_t *tot)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int32_t run = 0;
        for (int b = 0; b < nb; ++b) { const int32_t v = tot[b]; tot[b] = run; run += v; }
    }
}

__global__ void k_scan_add(int len, int32_t *a, const int32_t *tot)
{
    const int i = blockIdx.x * 1024 + threadIdx.x;
    if (i < len) a[i] += tot[blockIdx.x];
}

__global__ void k_csr_fill(int n, int d, const int32_t *rows_cm, const int32_t *rowptr, int32_t *fill,
                           int32_t *colidx)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * d) return;
    const int32_t row = rows_cm[e];
    const int32_t pos = rowptr[row] + atomicAdd(&fill[row], 1);
    colidx[pos] = (int32_t)(e / d);
}

// Sort the columns of every row ascending (insertion sort; rows are short).
__global__ void k_csr_sort(int m, const int32_t *rowptr, int32_t *colidx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int32_t b = rowptr[i], e = rowptr[i + 1];
    for (int32_t a = b + 1; a < e; ++a) {
        const int32_t v = colidx[a];
        int32_t q = a - 1;
        while (q >= b && colidx[q] > v) { colidx[q + 1] = colidx[q]; --q; }
        colidx[q + 1] = v;
    }
}

// Def. GM items 4 and 6.  Row i: sum of x over its columns (ascending) in FP64,
// plus sigma_n times a Box-Muller deviate of Philox block (0, i, 0, 'N'),
// rounded to FP32 once.
__global__ void k_sketch(int m, const int32_t *rowptr, const int32_t *colidx, const float *x, double sigma_n,
                         uint32_t k0, uint32_t k1, float *y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double acc = 0.0;
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) acc += (double)x[colidx[p]];
    if (sigma_n > 0.0) {
        PhiloxOut o = philox4x32_10(0u, (uint32_t)i, 0u, TAG_NOISE, k0, k1);
        const double u1 = ((double)o.v[0] + 1.0) / 4294967296.0;
        const double u2 = (double)o.v[1] / 4294967296.0;
        const double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
        acc += sigma_n * z;
    }
    y[i] = (float)acc;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int rl0_cuda_err(cudaError_t e)
{
    if (e == cudaSuccess) return RL0_OK;
    if (e == cudaErrorMemoryAllocation) return RL0_ERR_ALLOC;
    return RL0_ERR_CUDA;
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return rl0_cuda_err(e_);   \
    } while (0)

int rl0_set_device_of(const rl0_expander *A)
{
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != A->device) CK(cudaSetDevice(A->device));
    return RL0_OK;
}

void rl0_expander_release(rl0_expander *A)
{
    if (!A) return;
    rl0_workspace_free(A);
    cudaFree(A->rows_cm);
    cudaFree(A->rows_sm);
    cudaFree(A->rowptr);
    cudaFree(A->colidx);
    cudaFree(A->dev_flag);
    if (A->host_pinned) cudaFreeHost(A->host_pinned);
    delete A;
}

static int check_shape(int64_t n, int64_t m, int d)
{
    if (n < 1 || m < 1 || d < 1 || d > RL0_MAX_D || d > m) return RL0_ERR_INVALID_ARG;
    if (m >= (1LL << 31) || n >= (1LL << 31) || n * (int64_t)d >= (1LL << 31)) return RL0_ERR_INVALID_ARG;
    return RL0_OK;
}

static int alloc_expander(int64_t n, int64_t m, int d, rl0_expander **out)
{
    rl0_expander *A = new (std::nothrow) rl0_expander;
    if (!A) return RL0_ERR_ALLOC;
    std::memset((void *)A, 0, sizeof(*A));
    A->n = n; A->m = m; A->d = d;
    cudaError_t e = cudaGetDevice(&A->device);
    if (e != cudaSuccess) { delete A; return rl0_cuda_err(e); }
    const size_t nnz = (size_t)n * d;
    if (cudaMalloc(&A->rows_cm, nnz * 4) != cudaSuccess || cudaMalloc(&A->rows_sm, nnz * 4) != cudaSuccess ||
        cudaMalloc(&A->rowptr, (size_t)(m + 1) * 4) != cudaSuccess ||
        cudaMalloc(&A->colidx, nnz * 4) != cudaSuccess || cudaMalloc(&A->dev_flag, 64) != cudaSuccess) {
        cudaGetLastError();
        rl0_expander_release(A);
        return RL0_ERR_ALLOC;
    }
    *out = A;
    return RL0_OK;
}

// Builds the slot-major copy and CSR(A^T) from rows_cm, then the workspace.
int rl0_expander_finish(rl0_expander *A, cudaStream_t s)
{
    const int64_t n = A->n, m = A->m;
    const int d = A->d;
    const int64_t nnz = n * d;
    k_slot_major<<<rl0_div_up(nnz, 256), 256, 0, s>>>((int)n, d, A->rows_cm, A->rows_sm);
    CK(cudaMemsetAsync(A->rowptr, 0, (size_t)(m + 1) * 4, s));
    k_row_count<<<rl0_div_up(nnz, 256), 256, 0, s>>>(nnz, A->rows_cm, A->rowptr);
    const int len = (int)(m + 1);
    const int nb = (int)rl0_div_up(len, 1024);
    int32_t *tot = nullptr, *fill = nullptr;
    CK(cudaMallocAsync(&tot, (size_t)nb * 4, s));
    CK(cudaMallocAsync(&fill, (size_t)m * 4, s));
    k_scan_blocks<<<nb, 1024, 0, s>>>(len, A->rowptr, tot);
    k_scan_totals<<<1, 32, 0, s>>>(nb, tot);
    k_scan_add<<<nb, 1024, 0, s>>>(len, A->rowptr, tot);
    CK(cudaMemsetAsync(fill, 0, (size_t)m * 4, s));
    k_csr_fill<<<rl0_div_up(nnz, 256), 256, 0, s>>>((int)n, d, A->rows_cm, A->rowptr, fill, A->colidx);
    k_csr_sort<<<rl0_div_up(m, 128), 128, 0, s>>>((int)m, A->rowptr, A->colidx);
    CK(cudaFreeAsync(tot, s));
    CK(cudaFreeAsync(fill, s));
    CK(cudaGetLastError());
    return rl0_workspace_alloc(A);
}

extern "C" int rl0_make_expander(int64_t n, int64_t m, int d, uint64_t seed, void *cuda_stream,
                                 rl0_expander **out)
{
    if (!out) return RL0_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = check_shape(n, m, d);
    if (rc) return rc;
    rl0_expander *A = nullptr;
    rc = alloc_expander(n, m, d, &A);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int err = 0;
    do {
        if (cudaMemsetAsync(A->dev_flag, 0, 4, s) != cudaSuccess) { err = RL0_ERR_CUDA; break; }
        k_make_expander<<<rl0_div_up(n, 128), 128, 0, s>>>((int)n, (int)m, d, (uint32_t)seed,
                                                           (uint32_t)(seed >> 32), A->rows_cm, A->dev_flag);
        int flag = 0;
        if (cudaMemcpyAsync(&flag, A->dev_flag, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { err = RL0_ERR_CUDA; break; }
        if (flag) { err = RL0_ERR_INVALID_ARG; break; }
        err = rl0_expander_finish(A, s);
        if (!err) err = rl0_cuda_err(cudaStreamSynchronize(s));
    } while (0);
    if (err) { cudaGetLastError(); rl0_expander_release(A); return err; }
    *out = A;
    return RL0_OK;
}

extern "C" int rl0_expander_from_rows(int64_t n, int64_t m, int d, const int32_t *rows_dev, void *cuda_stream,
                                      rl0_expander **out)
{
    if (!out || !rows_dev) return RL0_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = check_shape(n, m, d);
    if (rc) return rc;
    rl0_expander *A = nullptr;
    rc = alloc_expander(n, m, d, &A);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int err = 0;
    do {
        if (cudaMemcpyAsync(A->rows_cm, rows_dev, (size_t)n * d * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(A->dev_flag, 0, 4, s) != cudaSuccess) { err = RL0_ERR_CUDA; break; }
        k_validate_rows<<<rl0_div_up(n, 256), 256, 0, s>>>((int)n, (int)m, d, A->rows_cm, A->dev_flag);
        int flag = 0;
        if (cudaMemcpyAsync(&flag, A->dev_flag, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { err = RL0_ERR_CUDA; break; }
        if (flag) { err = RL0_ERR_INVALID_A; break; }
        err = rl0_expander_finish(A, s);
        if (!err) err = rl0_cuda_err(cudaStreamSynchronize(s));
    } while (0);
    if (err) { cudaGetLastError(); rl0_expander_release(A); return err; }
    *out = A;
    return RL0_OK;
}

extern "C" int rl0_expander_rows(const rl0_expander *A, int32_t *rows_dev, void *cuda_stream)
{
    if (!A || !rows_dev) return RL0_ERR_INVALID_ARG;
    int rc = rl0_set_device_of(A);
    if (rc) return rc;
    CK(cudaMemcpyAsync(rows_dev, A->rows_cm, (size_t)A->n * A->d * 4, cudaMemcpyDeviceToDevice,
                       (cudaStream_t)cuda_stream));
    return RL0_OK;
}

extern "C" int rl0_expander_shape(const rl0_expander *A, int64_t *n, int64_t *m, int *d)
{
    if (!A) return RL0_ERR_INVALID_ARG;
    if (n) *n = A->n;
    if (m) *m = A->m;
    if (d) *d = A->d;
    return RL0_OK;
}

extern "C" void rl0_free_expander(rl0_expander *A)
{
    if (!A) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(A->device);
    cudaDeviceSynchronize();
    rl0_expander_release(A);
    if (prev >= 0) cudaSetDevice(prev);
}

extern "C" int rl0_sketch(const rl0_expander *A, const float *x_dev, double sigma_n, uint64_t noise_seed,
                          float *y_dev, void *cuda_stream)
{
    if (!A || !x_dev || !y_dev || !(sigma_n >= 0.0)) return RL0_ERR_INVALID_ARG;
    int rc = rl0_set_device_of(A);
    if (rc) return rc;
    k_sketch<<<rl0_div_up(A->m, 256), 256, 0, (cudaStream_t)cuda_stream>>>(
        (int)A->m, A->rowptr, A->colidx, x_dev, sigma_n, (uint32_t)noise_seed, (uint32_t)(noise_seed >> 32), y_dev);
    CK(cudaGetLastError());
    return RL0_OK;
}

extern "C" const char *rl0_strerror(int code)
{
    switch (code) {
    case RL0_OK: return "success";
    case RL0_ERR_INVALID_ARG: return "invalid argument";
    case RL0_ERR_CUDA: return "CUDA runtime error";
    case RL0_ERR_ALLOC: return "allocation failed";
    case RL0_ERR_TIMEOUT: return "a bounded device wait gave up";
    case RL0_ERR_UNSUPPORTED: return "unsupported request";
    case RL0_ERR_INVALID_A: return "invalid expander rows (range, order or duplicates)";
    case RL0_ERR_INVALID_Y: return "y_hat holds NaN or Inf";
    case RL0_ERR_TOO_LARGE: return "instance larger than the static workspace (n <= 65536, m <= 32768)";
    default: return "unknown error";
    }
}
