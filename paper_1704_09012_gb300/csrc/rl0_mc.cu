// rl0_mc.cu -- Monte-Carlo check of the posteriors p_z and p_e (arXiv
// 1704.09012, Section "Comparison with empirical probabilities", Fig. 3) with
// the library's own FP32 posterior series: binned counts of the events
// "y_i = 0" over the rows and "y_i = y_l" over the row pairs of each column,
// beside the sum of the posterior the decoder assigns to each sample.
//
// Integer histograms only (per-CTA shared-memory bins, merged with integer
// atomics), so the counts do not depend on scheduling.
#include <algorithm>
#include <cmath>

#include "rl0_common.cuh"
#include "rl0_device.cuh"

#define RL0_MC_MAX_BINS 1024
#define RL0_MC_NT 256

namespace {

__device__ __forceinline__ unsigned long long fixed32(float p)
{
    return __double2ull_rn((double)p * 4294967296.0);     // p in [0, 1], 2^-32 units
}

__device__ __forceinline__ void mc_add(unsigned long long *h, float w, float inv_w, int nbins, bool event, float p)
{
    const float a = fabsf(w) * inv_w;
    if (!(a < (float)nbins)) return;
    const int b = (int)a;
    atomicAdd(&h[3 * b], 1ull);
    if (event) atomicAdd(&h[3 * b + 1], 1ull);
    atomicAdd(&h[3 * b + 2], fixed32(p));
}

__device__ __forceinline__ void mc_flush(unsigned long long *sh, unsigned long long *out, int nbins)
{
    __syncthreads();
    for (int b = threadIdx.x; b < 3 * nbins; b += blockDim.x)
        if (sh[b]) atomicAdd(&out[b], sh[b]);
}

// Rows: bin |yhat_i|; event y0_i == 0; posterior p_breve_z(yhat_i).
__global__ void __launch_bounds__(RL0_MC_NT) k_mc_rows(int m, const float *__restrict__ y0,
                                                       const float *__restrict__ yh, Series pz, int nbins,
                                                       float inv_w, unsigned long long *hz)
{
    __shared__ unsigned long long sh[3 * RL0_MC_MAX_BINS];
    for (int b = threadIdx.x; b < 3 * nbins; b += blockDim.x) sh[b] = 0ull;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const float w = yh[i];
        mc_add(sh, w, inv_w, nbins, y0[i] == 0.0f, series_eval(pz, w));
    }
    mc_flush(sh, hz, nbins);
}

// Row pairs of every column (rows ascending, s < l): bin |yhat_s - yhat_l|;
// event y0_s == y0_l; posterior p_breve_e(yhat_s - yhat_l).
__global__ void __launch_bounds__(RL0_MC_NT) k_mc_pairs(int n, int d, const int32_t *__restrict__ rows_cm,
                                                        const float *__restrict__ y0, const float *__restrict__ yh,
                                                        Series pe, int nbins, float inv_w, unsigned long long *he)
{
    __shared__ unsigned long long sh[3 * RL0_MC_MAX_BINS];
    for (int b = threadIdx.x; b < 3 * nbins; b += blockDim.x) sh[b] = 0ull;
    __syncthreads();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int32_t *N = rows_cm + (size_t)j * d;
        for (int s = 0; s < d; ++s) {
            const int is = N[s];
            for (int l = s + 1; l < d; ++l) {
                const int il = N[l];
                const float D = yh[is] - yh[il];
                mc_add(sh, D, inv_w, nbins, y0[is] == y0[il], series_eval(pe, D));
            }
        }
    }
    mc_flush(sh, he, nbins);
}

}  // namespace

extern "C" int rl0_posterior_mc(const rl0_expander *A, const float *y0_dev, const float *yhat_dev, int64_t k,
                                double sigma_s, double sigma_n, int nbins, double wz_max, double we_max,
                                uint64_t *hz_dev, uint64_t *he_dev, void *cuda_stream)
{
    if (!A || !y0_dev || !yhat_dev || !hz_dev || !he_dev) return RL0_ERR_INVALID_ARG;
    if (k < 1 || k > A->m || !(sigma_s > 0.0) || !(sigma_n > 0.0) || nbins < 1 || nbins > RL0_MC_MAX_BINS ||
        !(wz_max > 0.0) || !(we_max > 0.0))
        return RL0_ERR_INVALID_ARG;
    int rc = rl0_set_device_of(A);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the decoder's posterior series for this sparsity (Eqs. (pz_approx), (pe_approx), ell = 4)
    const double rho = (double)k / (double)A->m;
    const double s2 = sigma_s * sigma_s, n2 = sigma_n * sigma_n;
    const Series pz = rl0::to_device_series(rl0::make_series(A->d * rho, s2, n2, 4));
    const Series pe = rl0::to_device_series(rl0::make_series(2.0 * A->d * rho, s2, 2.0 * n2, 4));
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, A->device);
    nsm = std::max(nsm, 1);
    const int gr = (int)std::min<long long>(rl0_div_up(A->m, RL0_MC_NT), 4LL * nsm);
    const int gp = (int)std::min<long long>(rl0_div_up(A->n, RL0_MC_NT), 4LL * nsm);
    k_mc_rows<<<gr, RL0_MC_NT, 0, s>>>((int)A->m, y0_dev, yhat_dev, pz, nbins, (float)(nbins / wz_max),
                                        (unsigned long long *)hz_dev);
    k_mc_pairs<<<gp, RL0_MC_NT, 0, s>>>((int)A->n, A->d, A->rows_cm, y0_dev, yhat_dev, pe, nbins,
                                         (float)(nbins / we_max), (unsigned long long *)he_dev);
    return rl0_cuda_err(cudaGetLastError());
}
