// Device pieces of a BOS reconstruction iteration (Sec. 2.4, Sec. 3.2, without the PINN
// terms): a minibatch of random pixels, L_BOS over that minibatch, and the AdaBelief
// update of the voxel temperatures.
//
//   sample_pixels_kernel -- k-th index = splitmix64 output (draw * npix + k + 1) for the seed,
//                           reduced to [0, n_pixels) by 128-bit multiply-high (uniform)
//   loss_pixels_kernel   -- loss = s sum_k (target[pix_k] - I_k)^2, dL/dI_k = -2 s (target[pix_k] - I_k)
//   counter_add_kernel   -- an on-device iteration counter (draw and step numbers of a
//                           captured CUDA graph)
//   sort_pixels_kernel   -- orders a minibatch by the Morton key of its pixels, so that each
//                           warp of the tracers gets neighbouring pixels (coherent rays)
//   adabelief_kernel     -- AdaBelief (Zhuang et al., NeurIPS 2020):
//                             m = b1 m + (1 - b1) g,  s = b2 s + (1 - b2) (g - m)^2 + eps,
//                             theta -= lr (m / (1 - b1^t)) / (sqrt(s / (1 - b2^t)) + eps)
#include <math.h>

#include "../../include/bos.h"
#include "bos_device.cuh"
#include "bos_internal.h"

namespace bos {

__global__ void sample_pixels_kernel(int32_t* __restrict__ pix, long long npix, unsigned long long n_pixels,
                                     unsigned long long seed, unsigned long long draw0,
                                     const unsigned long long* __restrict__ draw_dev) {
    const unsigned long long draw = draw0 + (draw_dev ? *draw_dev : 0ULL);
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
                                 long long step0, const unsigned long long* __restrict__ step_dev) {
    // bias corrections 1 / (1 - b^t) for step t (t >= 1)
    const float t = (float)(step0 + (long long)(step_dev ? *step_dev : 0ULL));
    const float c1 = 1.0f / (1.0f - powf(b1, t));
    const float c2 = 1.0f / (1.0f - powf(b2, t));
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

__global__ void counter_add_kernel(unsigned long long* c, unsigned long long inc) { *c += inc; }

// Interleave the bits of x (even positions) and y (odd positions), 16 bits each.
__device__ __forceinline__ uint32_t morton2(uint32_t x, uint32_t y) {
    auto spread = [](uint32_t v) {
        v &= 0xffffu;
        v = (v | (v << 8)) & 0x00ff00ffu;
        v = (v | (v << 4)) & 0x0f0f0f0fu;
        v = (v | (v << 2)) & 0x33333333u;
        v = (v | (v << 1)) & 0x55555555u;
        return v;
    };
    return spread(x) | (spread(y) << 1);
}

// One block sorts a pixel list (n <= kSortMax) by the Morton key of (px, py), bitonic
// sort in shared memory; entries past n are padded with the largest key.
constexpr int kSortMax = 16384;
constexpr int kSortThreads = 1024;

__global__ void __launch_bounds__(kSortThreads) sort_pixels_kernel(int32_t* __restrict__ pix, int n, int width,
                                                                   int m) {
    extern __shared__ uint32_t sh[];
    uint32_t* key = sh;
    uint32_t* val = sh + m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        if (i < n) {
            const uint32_t p = (uint32_t)pix[i];
            key[i] = morton2(p % (uint32_t)width, p / (uint32_t)width);
            val[i] = p;
        } else {
            key[i] = 0xffffffffu;
            val[i] = 0xffffffffu;
        }
    }
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const uint32_t a = key[i], b = key[l];
                    if ((a > b) == up) {
                        key[i] = b;
                        key[l] = a;
                        const uint32_t t = val[i];
                        val[i] = val[l];
                        val[l] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) pix[i] = (int32_t)val[i];
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
                               const uint64_t* draw_dev, void* stream) {
    if (!pix_dev || npix <= 0 || n_pixels <= 0 || n_pixels > INT32_MAX) {
        bos::set_last_error("bos_sample_pixels: need npix > 0 and 0 < n_pixels <= 2^31 - 1");
        return BOS_ERR_INVALID_ARG;
    }
    bos::sample_pixels_kernel<<<sms_of_current() * 4, 256, 0, (cudaStream_t)stream>>>(
        pix_dev, npix, (unsigned long long)n_pixels, seed, draw, (const unsigned long long*)draw_dev);
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
                                float lr, float beta1, float beta2, float eps, int64_t step, const uint64_t* step_dev,
                                void* stream) {
    if (!theta_dev || !grad_dev || !m_dev || !s_dev || n <= 0 || (step < 1 && !step_dev) || step < 0 ||
        !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f)) {
        bos::set_last_error("bos_adabelief_step: bad argument");
        return BOS_ERR_INVALID_ARG;
    }
    bos::adabelief_kernel<<<sms_of_current() * 4, 256, 0, (cudaStream_t)stream>>>(
        theta_dev, grad_dev, m_dev, s_dev, n, lr, beta1, beta2, eps, (long long)step,
        (const unsigned long long*)step_dev);
    return cudaGetLastError() == cudaSuccess ? BOS_OK : BOS_ERR_CUDA;
}

bos_status_t bos_sort_pixels(int32_t* pix_dev, int64_t npix, int width, int height, void* stream) {
    if (!pix_dev || npix <= 0 || npix > bos::kSortMax || width <= 0 || height <= 0 || width > 65535 ||
        height > 65535) {
        bos::set_last_error("bos_sort_pixels: need 1 <= npix <= 16384 and an image of at most 65535 x 65535");
        return BOS_ERR_INVALID_ARG;
    }
    int m = 1;
    while (m < npix) m <<= 1;
    const size_t smem = 2 * (size_t)m * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(bos::sort_pixels_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * bos::kSortMax * sizeof(uint32_t)));
    if (e != cudaSuccess) return BOS_ERR_CUDA;
    bos::sort_pixels_kernel<<<1, bos::kSortThreads, smem, (cudaStream_t)stream>>>(pix_dev, (int)npix, width, m);
    return cudaGetLastError() == cudaSuccess ? BOS_OK : BOS_ERR_CUDA;
}

bos_status_t bos_counter_add(uint64_t* counter_dev, uint64_t inc, void* stream) {
    if (!counter_dev) {
        bos::set_last_error("bos_counter_add: NULL counter");
        return BOS_ERR_INVALID_ARG;
    }
    bos::counter_add_kernel<<<1, 1, 0, (cudaStream_t)stream>>>((unsigned long long*)counter_dev, inc);
    return cudaGetLastError() == cudaSuccess ? BOS_OK : BOS_ERR_CUDA;
}

}  // extern "C"
