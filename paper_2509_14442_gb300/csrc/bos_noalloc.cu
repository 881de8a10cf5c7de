// bos_render_noalloc: the forward render for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code running inside a latency-critical
// loop (cudaMalloc and cudaFree can synchronise the whole device), or a host application
// whose device memory is already handed out by another allocator (a framework's caching
// allocator or a fixed partition per process).  For them this entry point builds the
// field store and renders with scratch memory that lives in a file-scope device array
// of fixed size, reserved when the library is loaded on a GPU and held until the
// process exits.  The caller passes only its inputs and outputs.
//
// The array is shared by every call: calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it and must be serialised by the caller.
// The array keeps the previous call's contents; every call clears what has to start at
// zero and rebuilds the whole store before rendering.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "../../include/bos.h"
#include "bos_ctx_internal.h"
#include "bos_internal.h"

namespace {

// Scratch: 256 bytes of work counters, then the field store.
constexpr size_t kScratchBytes = (size_t)128 << 20;    // 128 MiB
constexpr size_t kCounterBytes = 256;
constexpr size_t kErrOffset = 4;                          // int error word after the tile counter
constexpr int kMaxDevices = 64;

__device__ __align__(256) static unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};                   // device address of g_scratch, per device

bos_status_t refuse(bos_status_t s, const char* fmt, ...) {
    char buf[512];
    int k = snprintf(buf, sizeof buf, "bos_render_noalloc: ");
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf + k, sizeof buf - k, fmt, ap);
    va_end(ap);
    bos::set_last_error(buf);        // reported by bos_last_error()
    return s;
}

bool finite3(const double* v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

// Device address of the scratch array on the current device, looked up once per device.
bos_status_t scratch_on(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return refuse(BOS_ERR_INVALID_ARG, "device %d out of range", device);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return refuse(BOS_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
        }
        g_scratch_dev[device] = p;
    }
    *out = (unsigned char*)g_scratch_dev[device];
    return BOS_OK;
}

bos::CamDev cam_dev(const bos_camera_desc& c) {
    bos::CamDev d;
    for (int a = 0; a < 3; ++a) {
        d.pos[a] = c.pos[a];
        d.fwd[a] = c.fwd[a];
        d.up[a] = c.up[a];
    }
    d.fx = c.fx;
    d.fy = c.fy;
    d.cx = c.cx;
    d.cy = c.cy;
    d.width = c.width;
    d.height = c.height;
    d.spp = c.spp;
    d.seed = c.seed;
    return d;
}

}  // namespace

extern "C" bos_status_t bos_render_noalloc(const bos_grid_desc* grid, const float* T_dev, const bos_camera_desc* cam,
                                           const bos_wall_desc* wall, const bos_light_desc* light,
                                           const float* pattern_dev, const bos_integrator_desc* integ, float* I_dev,
                                           float* disp_dev, void* stream) {
    using namespace bos;
    if (!grid || !T_dev || !cam || !wall || !light || !pattern_dev || !integ || !I_dev)
        return refuse(BOS_ERR_INVALID_ARG, "NULL argument");
    // the same descriptor checks as bos_set_grid and bos_set_geometry
    bos_status_t s0 = check_grid_desc(grid, "bos_render_noalloc");
    if (s0 != BOS_OK) return s0;
    s0 = check_geometry_desc(cam, wall, light, pattern_dev, integ, "bos_render_noalloc");
    if (s0 != BOS_OK) return s0;
    if (light->mode == 2 && grid->prec != BOS_PREC_FP32_COMP && grid->prec != BOS_PREC_BF16_COMP)
        return refuse(BOS_ERR_UNIMPLEMENTED, "the refracted projector connection needs a compensated precision");

    GridDev g{};
    const int n[3] = {grid->nx, grid->ny, grid->nz};
    for (int a = 0; a < 3; ++a) {
        g.n[a] = n[a];
        g.nb[a] = (n[a] - 1 + kBrick - 1) / kBrick;
        g.origin[a] = grid->origin[a];
        g.extent[a] = grid->extent[a];
        g.h[a] = grid->extent[a] / (double)n[a];
        g.inv_h[a] = 1.0 / g.h[a];
        g.inv_hf[a] = (float)(1.0 / g.h[a]);
        g.hf[a] = (float)g.h[a];
    }
    g.K = grid->rho0 * grid->G * grid->T0;
    g.prec = grid->prec;
    const size_t elem = grid->prec == BOS_PREC_BF16_COMP ? 16 : 32;   // store element (x pairs, or FP64 records)
    const size_t slots = (size_t)morton3(g.nb[0] - 1, g.nb[1] - 1, g.nb[2] - 1) + 1;
    const size_t store_bytes = slots * kBrickCells * elem;
    g.store_elems = (uint32_t)(slots * kBrickCells);
    if (store_bytes > kScratchBytes - kCounterBytes)
        return refuse(BOS_ERR_INVALID_ARG,
                      "the field store of this grid needs %zu bytes; the fixed scratch holds at most %zu bytes",
                      store_bytes, kScratchBytes - kCounterBytes);

    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return refuse(BOS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    unsigned char* scratch = nullptr;
    bos_status_t s = scratch_on(device, &scratch);
    if (s != BOS_OK) return s;
    int num_sms = 1;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);

    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemsetAsync(scratch, 0, kCounterBytes, st);      // tile counter, step counter, error word
    if (e != cudaSuccess) return refuse(BOS_ERR_CUDA, "clearing the counters: %s", cudaGetErrorString(e));
    g.store = scratch + kCounterBytes;
    e = launch_build_store(g, T_dev, scratch + kCounterBytes, st);
    if (e != cudaSuccess) return refuse(BOS_ERR_CUDA, "field build: %s", cudaGetErrorString(e));

    SceneDev S;
    S.pix = nullptr;
    S.npix = 0;
    S.g = g;
    S.cam = cam_dev(*cam);
    for (int a = 0; a < 3; ++a) {
        S.w.origin[a] = wall->origin[a];
        S.w.eu[a] = wall->eu[a];
        S.w.ev[a] = wall->ev[a];
        S.w.normal[a] = wall->normal[a];
    }
    S.w.size_u = wall->size_u;
    S.w.size_v = wall->size_v;
    S.L.mode = light->mode;
    S.L.proj = cam_dev(light->proj);
    S.L.tw = light->tw;
    S.L.th = light->th;
    S.L.connect_iters = light->mode == 2 ? light->connect_iters : 0;
    S.L.pattern = pattern_dev;
    S.it.fixed_steps = integ->fixed_steps;
    S.it.max_step_vox = integ->max_step_vox;
    S.it.integrator = integ->integrator;
    S.it.ckpt_every = integ->ckpt_every;
    if (integ->fixed_steps > 0) {
        S.it.max_steps = integ->fixed_steps;
    } else {
        double hmin = fmin(g.h[0], fmin(g.h[1], g.h[2]));
        double diag = sqrt(g.extent[0] * g.extent[0] + g.extent[1] * g.extent[1] + g.extent[2] * g.extent[2]);
        double b = ceil(diag / (integ->max_step_vox * hmin)) + 2.0;
        S.it.max_steps = b > 2e9 ? 2000000000 : (int)b;
    }
    S.rc = ray_const_of(S);
    const int mode = grid->prec == BOS_PREC_FP32_COMP ? 1 : grid->prec == BOS_PREC_BF16_COMP ? 2
                     : grid->prec == BOS_PREC_FP32     ? 3
                                                       : 4;
    WorkDev w{(int*)scratch, (unsigned long long*)(scratch + 64), (int*)(scratch + kErrOffset)};
    S.g.err = w.err;
    CkptDev ck{};
    ck.every = integ->ckpt_every;
    RenderOut o{I_dev, disp_dev, nullptr};
    e = launch_render(mode, S, o, w, ck, num_sms, st);
    if (e != cudaSuccess) return refuse(BOS_ERR_CUDA, "render: %s", cudaGetErrorString(e));
    return BOS_OK;
}

// Device-detected errors of the allocation-free render live in the shared array's error
// word (written by the kernels, cleared by the next bos_render_noalloc).  Read it on the
// current device after synchronising the stream of the call in question; it races with any
// bos_render_noalloc still running on the device, like the array itself.
extern "C" bos_status_t bos_noalloc_status(void) {
    using namespace bos;
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return refuse(BOS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    unsigned char* scratch = nullptr;
    bos_status_t s = scratch_on(device, &scratch);
    if (s != BOS_OK) return s;
    int err = 0;
    e = cudaMemcpy(&err, scratch + kErrOffset, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return refuse(BOS_ERR_CUDA, "reading the error word: %s", cudaGetErrorString(e));
    switch (err) {
        case DEV_OK: return BOS_OK;
        case DEV_STEP_BUDGET: return refuse(BOS_ERR_DEVICE_CHECK, "a ray needed more steps than the step bound");
        case DEV_BAD_PIXEL: return refuse(BOS_ERR_DEVICE_CHECK, "a pixel index is outside the image");
        case DEV_BOUNDS: return refuse(BOS_ERR_DEVICE_CHECK, "an index fell outside its buffer (checked build)");
        default: return refuse(BOS_ERR_DEVICE_CHECK, "device error %d", err);
    }
}
