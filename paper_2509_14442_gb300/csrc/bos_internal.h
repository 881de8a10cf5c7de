// Host/device interface between the C-ABI layer and the kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bos_device.cuh"

namespace bos {

constexpr size_t kAlign = 256;

// Limits every entry point enforces: warp tiles per launch (the tile index and the tile
// queue are 32-bit; 2^30 leaves room for the warps that overshoot the last tile) and the
// fixed step count per ray.
constexpr long long kMaxTiles = 1LL << 30;
constexpr int kMaxFixedSteps = 1 << 24;
inline size_t align_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

// Resident blocks per SM of `kernel` (threads, dynamic shared memory smem), after setting
// its shared-memory carveout to what those blocks need: the tracers' gathers are served
// from L1, which gets the rest of the SM's 256 KB (a larger L1 measured ~1 % faster for
// the adjoint, and the largest shared carveout 7.5 % slower).  The preference is dropped
// again if the driver's choice for it would lower the occupancy.
template <class Kernel>
inline cudaError_t occupancy_prefer_l1(Kernel kernel, int threads, size_t smem, int& per_sm) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess || per_sm < 1) return e;
    int dev = 0, max_sm = 0, reserved = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return e;
    const long long need = (long long)per_sm * ((long long)smem + (long long)fa.sharedSizeBytes + reserved);
    int pct = max_sm > 0 ? (int)((100 * need + max_sm - 1) / max_sm) : 100;
    pct = pct < 0 ? 0 : pct > 100 ? 100 : pct;
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct)) != cudaSuccess) return e;
    int after = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&after, kernel, threads, smem)) != cudaSuccess) return e;
    if (after < per_sm)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, -1);
    return cudaSuccess;
}

struct RenderOut {
    float* I;
    float* disp;
    double* hit;
};

struct WorkDev {
    int* tile_counter;              // warp tile queue (zeroed per launch)
    unsigned long long* steps;      // sum of N over traced rays
    int* err;                       // sticky device error word
};

// Ray state every K steps (float4 x3 per checkpoint: dr + cr.x, dv + cr.y, cv + cr.z),
// index ((c * 3 + q) * nrays + slot), plus the path-length excess of every ray.  A ray's
// slot is (tile * 32 + lane) * samples_per_lane + sample, so a warp's loads coalesce.
struct CkptDev {
    float4* state;                  // nullptr: do not save
    float* excess;
    long long nrays;                // number of slots (tiles * 32 * samples_per_lane)
    int every;
    int max_ckpt;
    // refracted projector connection (light mode 2), kept when state != nullptr:
    float4* pstate;                 // checkpoints of each slot's projector ray (same layout as state)
    float4* conn;                   // 2 per slot: (x_w - x_ref, cos/len), (x_w - a_1, 0)
    int* err;                       // the context's error word (the checked build's reports)
};

// Grid adjoint accumulators: per node (d L/d deta, d L/d grad eta) in float32.
struct AdjDev {
    float4* acc;                    // float64 precision: four doubles per node
    const float* dLdI;              // bos_backward_f64: points at doubles
    int* err;
    float* seg;          // per-warp segment states of the Sharma adjoint (adjoint_segment_bytes)
};

// The Sharma adjoint keeps each recomputed segment's K steps (state and stage terms
// (dr, dv, A, B): 12 floats per lane and step) in a per-warp slice of global memory (L1/L2-resident while the segment is reversed)
// rather than in shared memory, which would cap the kernel at fewer resident warps.  Its
// grid is capped at kAdjMaxBlocks blocks of kAdjWarpsPerBlock warps.
constexpr int kAdjMaxBlocks = 1024;
constexpr int kAdjWarpsPerBlock = 2;
inline size_t adjoint_segment_bytes(int K) {
    return (size_t)kAdjMaxBlocks * kAdjWarpsPerBlock * (size_t)K * 12 * 32 * sizeof(float);
}

// One request's share of a batched launch (the request server): its scene, buffers and the
// range of its warp tiles in the launch.  Work item g of the launch is tile
// tile0 + (g - first) of the job j with first(j) <= g < first(j + 1).
struct BatchJob {
    SceneDev S;
    RenderOut out;
    WorkDev wk;
    CkptDev ck;
    AdjDev adj;
    int tile0;
    int first;
};

__host__ __device__ __forceinline__ int batch_job_of(const BatchJob* jobs, int njobs, int g) {
    int lo = 0, hi = njobs - 1;            // the last job whose first item is <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].first <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Message returned by bos_last_error() on the calling thread.
void set_last_error(const char* msg);

// Ray-independent float64 set-up terms of a scene (S.g, S.cam, S.w, S.L and S.it filled in).
RayConst ray_const_of(const SceneDev& S);

cudaError_t launch_build_store(const GridDev& g, const float* T, void* store, cudaStream_t st);
cudaError_t launch_render(int mode, const SceneDev& S, const RenderOut& o, const WorkDev& w, const CkptDev& ck,
                          int num_sms, cudaStream_t st);
// Batched launches over several jobs' warp tiles (modes 1, 2 = FP32_COMP, BF16_COMP;
// integrator 0 = Sharma RKN, 2 = quasi-linear; light modes 0 and 1).  `counter` is zeroed
// by the caller; seg_base holds kAdjMaxBlocks x kAdjWarpsPerBlock segment slices of K_max
// steps for the Sharma adjoint.
cudaError_t launch_render_batch(int mode, int integ, const BatchJob* jobs, int njobs, int total, int* counter,
                                int num_sms, cudaStream_t st);
cudaError_t launch_adjoint_batch(int mode, int integ, const BatchJob* jobs, int njobs, int total, int* counter,
                                 float* seg_base, int k_max, int num_sms, cudaStream_t st);
cudaError_t launch_gradient(const GridDev& g, const float4* acc, const float* T, float* dLdT, int num_sms,
                            cudaStream_t st);
cudaError_t launch_ray_steps(const SceneDev& S, int32_t* nsteps, int num_sms, cudaStream_t st);
cudaError_t launch_export_nodes(const GridDev& g, void* out, int num_sms, cudaStream_t st);
cudaError_t launch_loss_l2(const float* I, const float* target, long long n, double* loss, float* dLdI, int num_sms,
                           cudaStream_t st);
cudaError_t launch_probe_read(const void* buf, long long bytes, int repeats, float* sink, int num_sms,
                              cudaStream_t st);
cudaError_t launch_probe_fma(int kind, int repeats, float* sink, int num_sms, double* flops, cudaStream_t st);
cudaError_t launch_probe_read_l1(const void* buf, long long bytes, int repeats, float* sink, int num_sms,
                                 double* bytes_read, cudaStream_t st);
cudaError_t launch_backward_fp64(const SceneDev& S, const CkptDev& ck, const AdjDev& adj, const WorkDev& w,
                                 const float* T, void* dLdT, bool f64, int num_sms, cudaStream_t st);
cudaError_t launch_backward(int mode, const SceneDev& S, const CkptDev& ck, const AdjDev& adj, const WorkDev& w,
                            const float* T, float* dLdT, int num_sms, cudaStream_t st);

}  // namespace bos
