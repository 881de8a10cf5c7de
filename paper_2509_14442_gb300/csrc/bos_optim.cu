// Device pieces of a BOS reconstruction iteration (Sec. 2.4, Sec. 3.2, without the PINN
// terms): a minibatch of random pixels, L_BOS over that minibatch, and the AdaBelief
// update of the voxel temperatures.
//
//   sample_pixels_kernel -- k-th index = splitmix64 output (draw * npix + k + 1) for the seed,
//                           reduced to [0, n_pixels) by 128-bit multiply-high (uniform)
//   loss_pixels_kernel   -- loss = s sum_k (target[pix_k] - I_k)^2, dL/dI_k = -2 s (target[pix_k] - I_k)
//   adabelief_kernel     -- AdaBelief (Zhuang et al., NeurIPS 2020):
//                             m = b1 m + (1 - b1) g,  s = b2 s + (1 - b2) (g - m)^2 + eps,
//                             theta -= lr (m / (1 - b1^t)) / (sqrt(s / (1 - b2^t)) + eps)
#include <math.h>

#include "../../include/bos.h"
#include "bos_device.cuh"
#include "bos_internal.h"

namespace bos {

__global__ void sample_pixels_kernel(int32_t* __restrict__ pix, long long npix, unsigned long long n_pixels,
                                     unsigned long long seed, unsigned long long draw) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < npix;
         k += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = splitmix64_output(seed, draw * (unsigned long long)npix + (unsigned long long)k + 1ULL);
        pix[k] = (int32_t)__umul64hi(z, n_pixels);
    }
}

__global__ void loss_pixels_kernel(const float* __restrict__ I, const float* __restrict__ target,
                                   const int32_t* __restrict__ pix, long long npix, float scale, double* loss,
                                   float* __restrict__ dLdI) {
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < npix;
         k += (long long)gridDim.x * blockDim.x) {
        const float t = __ldg(target + pix[k]);
        const double r = (double)t - (double)I[k];
        acc += r * r;
        if (dLdI) dLdI[k] = (-2.0f * scale) * (t - I[k]);
    }
    for (int m = 16; m >= 1; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += part[i];
        atomicAdd(loss, (double)scale * s);
    }
}

__global__ void adabelief_kernel(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                                 float* __restrict__ s, long long n, float lr, float b1, float b2, float eps,
                                 float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float d = g - mi;
        const float si = b2 * s[i] + (1.0f - b2) * d * d + eps;
        m[i] = mi;
        s[i] = si;
        theta[i] -= lr * (mi * c1) / (sqrtf(si * c2) + eps);
    }
}

}  // namespace bos

namespace {
int sms_of_current() {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}
}  // namespace

extern "C" {

bos_status_t bos_sample_pixels(int32_t* pix_dev, int64_t npix, int64_t n_pixels, uint64_t seed, uint64_t draw,
                               void* stream) {
    if (!pix_dev || npix <= 0 || n_pixels <= 0 || n_pixels > INT32_MAX) {
        bos::set_last_error("bos_sample_pixels: need npix > 0 and 0 < n_pixels <= 2^31 - 1");
        return BOS_ERR_INVALID_ARG;
    }
    bos::sample_pixels_kernel<<<sms_of_current() * 4, 256, 0, (cudaStream_t)stream>>>(
        pix_dev, npix, (unsigned long long)n_pixels, seed, draw);
    return cudaGetLastError() == cudaSuccess ? BOS_OK : BOS_ERR_CUDA;
}

bos_status_t bos_loss_l2_pixels(const float* I_dev, const float* target_dev, const int32_t* pix_dev, int64_t npix,
                                float scale, double* loss_dev, float* dLdI_dev, void* stream) {
    if (!I_dev || !target_dev || !pix_dev || !loss_dev || npix <= 0 || !(scale > 0.0f) || !isfinite(scale)) {
        bos::set_last_error("bos_loss_l2_pixels: bad argument");
        return BOS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(loss_dev, 0, sizeof(double), st) != cudaSuccess) return BOS_ERR_CUDA;
    bos::loss_pixels_kernel<<<sms_of_current() * 4, 256, 0, st>>>(I_dev, target_dev, pix_dev, npix, scale,
                                                                   loss_dev, dLdI_dev);
    return cudaGetLastError() == cudaSuccess ? BOS_OK : BOS_ERR_CUDA;
}

bos_status_t bos_adabelief_step(float* theta_dev, const float* grad_dev, float* m_dev, float* s_dev, int64_t n,
                                float lr, float beta1, float beta2, float eps, int64_t step, void* stream) {
    if (!theta_dev || !grad_dev || !m_dev || !s_dev || n <= 0 || step < 1 || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f)) {
        bos::set_last_error("bos_adabelief_step: bad argument");
        return BOS_ERR_INVALID_ARG;
    }
    const float c1 = (float)(1.0 / (1.0 - pow((double)beta1, (double)step)));
    const float c2 = (float)(1.0 / (1.0 - pow((double)beta2, (double)step)));
    bos::adabelief_kernel<<<sms_of_current() * 4, 256, 0, (cudaStream_t)stream>>>(theta_dev, grad_dev, m_dev, s_dev, n,
                                                                                   lr, beta1, beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? BOS_OK : BOS_ERR_CUDA;
}

}  // extern "C"
