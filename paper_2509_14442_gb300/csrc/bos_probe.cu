// Throughput probes (no counterpart in the paper), measured in the same run as the tracer
// so that its rooflines are stated against this device and clock: the FP32 and FP64 fused
// multiply-add rates, and the L1 read bandwidth of the 256-bit loads the gathers use.
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

// L1 read bandwidth: every block streams the same small buffer (it stays resident in each
// SM's L1) `repeats` times with the 256-bit non-coherent loads the tracer's gathers use,
// eight per thread in flight, and folds the values into a register.
__global__ void __launch_bounds__(kProbeThreads) probe_read_l1_kernel(const float* __restrict__ buf, int n8,
                                                                      int repeats, float* sink) {
    float acc = 0.0f;
    for (int r = 0; r < repeats; ++r) {
        for (int i = threadIdx.x; i < n8; i += 8 * kProbeThreads) {
            float v[8][8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = i + u * kProbeThreads;
                const float* p = buf + 8 * (size_t)(j < n8 ? j : i);
                asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                             : "=f"(v[u][0]), "=f"(v[u][1]), "=f"(v[u][2]), "=f"(v[u][3]), "=f"(v[u][4]),
                               "=f"(v[u][5]), "=f"(v[u][6]), "=f"(v[u][7])
                             : "l"(p));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                acc += ((v[u][0] + v[u][1]) + (v[u][2] + v[u][3])) + ((v[u][4] + v[u][5]) + (v[u][6] + v[u][7]));
        }
    }
    if (acc == 1234.5678f) sink[0] = acc;
}

cudaError_t launch_probe_read_l1(const void* buf, long long bytes, int repeats, float* sink, int num_sms,
                                 double* bytes_read, cudaStream_t st) {
    const unsigned blocks = (unsigned)num_sms * kProbeBlocksPerSm;
    const int n8 = (int)(bytes / 32);
    probe_read_l1_kernel<<<blocks, kProbeThreads, 0, st>>>((const float*)buf, n8, repeats, sink);
    // each block issues 8 x 256 loads per round (lanes past the end re-read their first
    // element), ceil(n8 / 2048) rounds per pass
    const long long rounds = (n8 + 8 * kProbeThreads - 1) / (8 * kProbeThreads);
    if (bytes_read) *bytes_read = (double)blocks * (double)repeats * (double)rounds * (8.0 * kProbeThreads) * 32.0;
    return cudaGetLastError();
}

}  // namespace bos
