// Arithmetic-throughput probe (no counterpart in the paper): the FP32 and FP64 fused
// multiply-add rates of this GPU, measured in the same run as the tracer so that its
// arithmetic roofline is stated against this device and clock.
//
// Every thread runs eight independent recurrences x <- x * a + b for `repeats` x 16
// rounds; a and b are kernel arguments, so nothing folds at compile time, and the sum of
// the recurrences is written only under a condition the compiler cannot decide, which
// keeps the chains alive.  With 32 warps per SM and eight chains per thread the FMA
// latency is hidden, so the launch time is set by the FMA pipes alone.
#include "bos_device.cuh"
#include "bos_internal.h"

namespace bos {

constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 16;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;

// KIND 0: scalar float32 fma; 1: packed float32 pairs (fma.rn.f32x2, two FMAs per
// instruction); 2: float64 fma.
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) probe_fma_kernel(int repeats, float a, float b, float* sink) {
    const float seed = (float)threadIdx.x * 1e-3f;
    if constexpr (KIND == 0) {
        float x[kProbeChains];
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) x[i] = seed + (float)i;
        for (int r = 0; r < repeats; ++r) {
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
                for (int i = 0; i < kProbeChains; ++i) x[i] = fmaf(x[i], a, b);
        }
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) s += x[i];
        if (s == 1234.5678f) sink[0] = s;
    } else if constexpr (KIND == 1) {
        const f32x2 aa = pack2(a, a), bb = pack2(b, b);
        f32x2 x[kProbeChains];
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) x[i] = pack2(seed + (float)i, seed - (float)i);
        for (int r = 0; r < repeats; ++r) {
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
                for (int i = 0; i < kProbeChains; ++i) x[i] = fma2(x[i], aa, bb);
        }
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) {
            float lo, hi;
            unpack2(x[i], lo, hi);
            s += lo + hi;
        }
        if (s == 1234.5678f) sink[0] = s;
    } else {
        const double ad = (double)a, bd = (double)b;
        double x[kProbeChains];
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) x[i] = (double)seed + (double)i;
        for (int r = 0; r < repeats; ++r) {
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
                for (int i = 0; i < kProbeChains; ++i) x[i] = fma(x[i], ad, bd);
        }
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) s += x[i];
        if (s == 1234.5678) sink[0] = (float)s;
    }
}

cudaError_t launch_probe_fma(int kind, int repeats, float* sink, int num_sms, double* flops, cudaStream_t st) {
    const unsigned blocks = (unsigned)num_sms * kProbeBlocksPerSm;
    // 0.9999999 keeps every recurrence bounded (it converges to b / (1 - a))
    const float a = 0.9999999f, b = 1e-7f;
    if (kind == 0)
        probe_fma_kernel<0><<<blocks, kProbeThreads, 0, st>>>(repeats, a, b, sink);
    else if (kind == 1)
        probe_fma_kernel<1><<<blocks, kProbeThreads, 0, st>>>(repeats, a, b, sink);
    else
        probe_fma_kernel<2><<<blocks, kProbeThreads, 0, st>>>(repeats, a, b, sink);
    if (flops)
        *flops = 2.0 * (kind == 1 ? 2.0 : 1.0) * (double)blocks * kProbeThreads * (double)repeats * kProbeUnroll *
                 kProbeChains;
    return cudaGetLastError();
}

}  // namespace bos
