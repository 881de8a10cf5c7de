// C ABI of the BOS library: argument validation, context-owned device memory and
// kernel launches.  Declarations and contracts: include/bos.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>

#include "../../include/bos.h"
#include "bos_ctx_internal.h"
#include "bos_internal.h"

using namespace bos;

namespace {

thread_local std::string g_last_error;

bos_status_t fail(bos_status_t s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
bos_status_t fail(bos_status_t s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

bos_status_t cuda_fail(cudaError_t e, const char* what) {
    return fail(BOS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool finite3(const double* v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }
double norm3(const double* v) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }
bool unit3(const double* v) { return finite3(v) && fabs(norm3(v) - 1.0) < 1e-9; }

bos_status_t check_camera(const bos_camera_desc* c, const char* who) {
    if (!c) return fail(BOS_ERR_INVALID_ARG, "%s: NULL camera", who);
    if (!finite3(c->pos) || !unit3(c->fwd) || !unit3(c->up))
        return fail(BOS_ERR_INVALID_ARG, "%s: pos must be finite, fwd and up unit vectors", who);
    double dot = c->fwd[0] * c->up[0] + c->fwd[1] * c->up[1] + c->fwd[2] * c->up[2];
    if (fabs(dot) > 1e-9) return fail(BOS_ERR_INVALID_ARG, "%s: fwd and up must be orthogonal", who);
    if (!(c->fx > 0) || !(c->fy > 0) || !isfinite(c->fx) || !isfinite(c->fy) || !isfinite(c->cx) ||
        !isfinite(c->cy))
        return fail(BOS_ERR_INVALID_ARG, "%s: focal lengths must be > 0 and finite", who);
    if (c->width <= 0 || c->height <= 0 || c->spp <= 0)
        return fail(BOS_ERR_INVALID_ARG, "%s: width, height and spp must be > 0", who);
    if ((long long)c->width * c->height * c->spp > (1LL << 40))
        return fail(BOS_ERR_INVALID_ARG, "%s: too many rays", who);
    // the warp-tile index and the tile queue are 32-bit: keep the tile count (plus the
    // warps of a grid that overshoot it) far below INT_MAX
    const TileShape ts = tile_shape(c->width, c->height, c->spp);
    if ((long long)ts.tiles_x * ts.tiles_y > kMaxTiles)
        return fail(BOS_ERR_INVALID_ARG, "%s: %lld warp tiles of %d x %d pixels, at most %lld", who,
                    (long long)ts.tiles_x * ts.tiles_y, ts.TW, ts.TH, kMaxTiles);
    return BOS_OK;
}

template <class T>
void copy3(T* dst, const double* src) {
    for (int a = 0; a < 3; ++a) dst[a] = src[a];
}

CamDev to_dev(const bos_camera_desc& c) {
    CamDev d;
    copy3(d.pos, c.pos);
    copy3(d.fwd, c.fwd);
    copy3(d.up, c.up);
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

// Bytes per store element: float32 and bfloat16 records are stored as x pairs (F4P, B4P).
size_t elem_bytes(int prec) { return prec == BOS_PREC_FP64 ? 32 : prec == BOS_PREC_BF16_COMP ? 16 : 32; }

// Tracer variant of a precision (see the MODE switch of the render kernel).
int mode_of(int prec) {
    switch (prec) {
        case BOS_PREC_FP32_COMP: return 1;
        case BOS_PREC_BF16_COMP: return 2;
        case BOS_PREC_FP32: return 3;
        default: return 4;
    }
}

}  // namespace

struct bos_ctx {
    int device = 0;
    int num_sms = 1;
    uint64_t mem_limit = 0;
    uint64_t bytes = 0;

    bool has_grid = false, has_geom = false;
    bos_grid_desc grid{};
    GridDev g{};
    void* store = nullptr;
    size_t store_bytes = 0;
    const float* T = nullptr;

    CamDev cam{};
    WallDev wall{};
    LightDev light{};
    IntegDev integ{};

    void* small = nullptr;          // tile counter, step counter, error word
    int* tile_counter = nullptr;
    unsigned long long* steps = nullptr;
    int* err = nullptr;

    float4* ckpt = nullptr;
    size_t ckpt_bytes = 0;
    float* excess = nullptr;
    size_t excess_bytes = 0;
    float4* pckpt = nullptr;        // projector-ray checkpoints (light mode 2)
    size_t pckpt_bytes = 0;
    float4* conn = nullptr;         // per-slot connection records (light mode 2)
    size_t conn_bytes = 0;
    bool saved = false;
    CkptDev saved_ck{};
    int saved_mode = 0;
    const int32_t* saved_pix = nullptr;   // pixel list of the saved render (nullptr: whole image)
    long long saved_npix = 0;

    float4* acc = nullptr;
    float* seg = nullptr;           // adjoint segment states
    size_t seg_bytes = 0;
    size_t acc_bytes = 0;

    // Optional caller-provided device arena: when set, buffers are carved from it and
    // nothing is allocated or freed (used by the request server).
    char* arena = nullptr;
    size_t arena_size = 0, arena_used = 0;
};

namespace {

bos_status_t dev_alloc(bos_ctx* c, void** p, size_t* have, size_t want, const char* what) {
    if (*have >= want && *p) return BOS_OK;
    if (c->arena) {
        size_t need = bos::align_up(want);
        if (c->arena_used + need > c->arena_size)
            return fail(BOS_ERR_OOM, "%s: %zu bytes do not fit the request's arena (%zu of %zu used)", what, want,
                        c->arena_used, c->arena_size);
        *p = c->arena + c->arena_used;
        c->arena_used += need;
        *have = want;
        return BOS_OK;
    }
    if (c->mem_limit && c->bytes - *have + want > c->mem_limit)
        return fail(BOS_ERR_OOM, "%s: %zu bytes would exceed the context limit of %llu bytes", what, want,
                    (unsigned long long)c->mem_limit);
    if (*p) {
        cudaError_t e = cudaFree(*p);
        if (e != cudaSuccess) return cuda_fail(e, what);
        c->bytes -= *have;
        *p = nullptr;
        *have = 0;
    }
    cudaError_t e = cudaMalloc(p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(BOS_ERR_OOM, "%s: cudaMalloc(%zu) failed: %s", what, want, cudaGetErrorString(e));
    }
    *have = want;
    c->bytes += want;
    return BOS_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

SceneDev scene_of(const bos_ctx* c) {
    SceneDev S;
    S.g = c->g;
    S.cam = c->cam;
    S.w = c->wall;
    S.L = c->light;
    S.it = c->integ;
    S.rc = bos::ray_const_of(S);
    S.pix = nullptr;
    S.npix = 0;
    return S;
}

// Upper bound of N over all rays: fixed, or the box diagonal over the step length.
int step_bound(const bos_ctx* c) {
    if (c->integ.fixed_steps > 0) return c->integ.fixed_steps;
    double hmin = fmin(c->g.h[0], fmin(c->g.h[1], c->g.h[2]));
    double diag = norm3(c->g.extent);
    double b = ceil(diag / (c->integ.max_step_vox * hmin)) + 2.0;
    return b > 2e9 ? 2000000000 : (int)b;
}

}  // namespace

namespace bos {

void set_last_error(const char* msg) { g_last_error = msg; }

bos_status_t check_grid_desc(const bos_grid_desc* d, const char* who) {
    if (!d) return fail(BOS_ERR_INVALID_ARG, "%s: NULL grid", who);
    if (d->nx < 2 || d->ny < 2 || d->nz < 2 || d->nx > 8192 || d->ny > 8192 || d->nz > 8192)
        return fail(BOS_ERR_INVALID_ARG, "%s: need 2 <= n <= 8192 cells per axis, got %d x %d x %d", who, d->nx,
                    d->ny, d->nz);
    if ((long long)d->nx * d->ny * d->nz >= (1LL << 31))
        return fail(BOS_ERR_INVALID_ARG, "%s: at most 2^31 - 1 cells", who);
    if (!finite3(d->origin) || !finite3(d->extent) || !(d->extent[0] > 0) || !(d->extent[1] > 0) ||
        !(d->extent[2] > 0))
        return fail(BOS_ERR_INVALID_ARG, "%s: origin must be finite and extent > 0", who);
    if (!(d->T0 > 0) || !(d->rho0 > 0) || !(d->G > 0) || !isfinite(d->T0 * d->rho0 * d->G))
        return fail(BOS_ERR_INVALID_ARG, "%s: T0, rho0 and G must be > 0", who);
    if (d->prec < BOS_PREC_FP64 || d->prec > BOS_PREC_BF16_COMP)
        return fail(BOS_ERR_INVALID_ARG, "%s: unknown precision %d", who, d->prec);
    return BOS_OK;
}

bos_status_t check_geometry_desc(const bos_camera_desc* cam, const bos_wall_desc* wall, const bos_light_desc* light,
                                 const float* pattern_dev, const bos_integrator_desc* it, const char* who) {
    char w[96];
    if (!wall || !light || !it) return fail(BOS_ERR_INVALID_ARG, "%s: NULL argument", who);
    snprintf(w, sizeof w, "%s: camera", who);
    bos_status_t s = check_camera(cam, w);
    if (s != BOS_OK) return s;
    if (!finite3(wall->origin) || !unit3(wall->eu) || !unit3(wall->ev) || !unit3(wall->normal) ||
        !(wall->size_u > 0) || !(wall->size_v > 0) || !isfinite(wall->size_u) || !isfinite(wall->size_v))
        return fail(BOS_ERR_INVALID_ARG, "%s: wall needs a finite origin, unit axes and finite sizes > 0", who);
    if (light->mode < 0 || light->mode > 2) return fail(BOS_ERR_INVALID_ARG, "%s: light mode %d", who, light->mode);
    if (light->tw <= 0 || light->th <= 0 || !pattern_dev)
        return fail(BOS_ERR_INVALID_ARG, "%s: pattern size must be > 0 and pattern non-NULL", who);
    if ((long long)light->tw * light->th >= (1LL << 31))
        return fail(BOS_ERR_INVALID_ARG, "%s: pattern of more than 2^31 - 1 texels", who);
    if (light->mode == 2 && (light->connect_iters < 1 || light->connect_iters > 16))
        return fail(BOS_ERR_INVALID_ARG, "%s: connect_iters must be in [1, 16]", who);
    if (light->mode >= 1) {
        snprintf(w, sizeof w, "%s: projector", who);
        s = check_camera(&light->proj, w);
        if (s != BOS_OK) return s;
    }
    if (it->fixed_steps < 0 || it->fixed_steps > kMaxFixedSteps)
        return fail(BOS_ERR_INVALID_ARG, "%s: fixed_steps must be in [0, %d]", who, kMaxFixedSteps);
    if (it->fixed_steps == 0 && !(it->max_step_vox > 1e-3 && it->max_step_vox < 1e6))
        return fail(BOS_ERR_INVALID_ARG, "%s: max_step_vox must be in (1e-3, 1e6)", who);
    if (it->integrator < 0 || it->integrator > 2)
        return fail(BOS_ERR_INVALID_ARG, "%s: integrator %d", who, it->integrator);
    if (it->ckpt_every < 1 || it->ckpt_every > 4096)
        return fail(BOS_ERR_INVALID_ARG, "%s: ckpt_every must be in [1, 4096]", who);
    return BOS_OK;
}

// Host IEEE double (this file is built without FMA contraction), in the order the
// per-ray device code used for the same terms.
RayConst ray_const_of(const SceneDev& S) {
    RayConst rc;
    const double* f = S.cam.fwd;
    const double* u = S.cam.up;
    const double* p = S.cam.pos;
    rc.right[0] = f[1] * u[2] - f[2] * u[1];
    rc.right[1] = f[2] * u[0] - f[0] * u[2];
    rc.right[2] = f[0] * u[1] - f[1] * u[0];
    for (int a = 0; a < 3; ++a) {
        rc.lo_m[a] = S.g.origin[a] - p[a];
        rc.hi_m[a] = (S.g.origin[a] + S.g.extent[a]) - p[a];
    }
    const double q[3] = {S.w.origin[0] - p[0], S.w.origin[1] - p[1], S.w.origin[2] - p[2]};
    rc.qn = (q[0] * S.w.normal[0] + q[1] * S.w.normal[1]) + q[2] * S.w.normal[2];
    double hmin = S.g.h[0] < S.g.h[1] ? S.g.h[0] : S.g.h[1];
    hmin = S.g.h[2] < hmin ? S.g.h[2] : hmin;
    rc.step = S.it.max_step_vox * hmin;
    const double* pp = S.L.proj.pos;
    for (int a = 0; a < 3; ++a) {
        rc.plo_m[a] = S.g.origin[a] - pp[a];
        rc.phi_m[a] = (S.g.origin[a] + S.g.extent[a]) - pp[a];
    }
    const double pq[3] = {S.w.origin[0] - pp[0], S.w.origin[1] - pp[1], S.w.origin[2] - pp[2]};
    rc.pqn = (pq[0] * S.w.normal[0] + pq[1] * S.w.normal[1]) + pq[2] * S.w.normal[2];
    return rc;
}

// Bind a context to a device arena (nullptr: back to its own allocations).  Drops the
// context's grid, geometry and saved render.
void ctx_bind_arena(bos_ctx* c, void* base, size_t bytes, cudaStream_t stream) {
    if (!c->arena) {
        void* bufs[] = {c->store, c->ckpt, c->excess, c->acc, c->pckpt, c->conn, c->seg};
        for (void* p : bufs)
            if (p) cudaFree(p);
        c->bytes = 256;
    }
    c->seg = nullptr;
    c->seg_bytes = 0;
    c->store = nullptr;
    c->ckpt = nullptr;
    c->excess = nullptr;
    c->acc = nullptr;
    c->pckpt = nullptr;
    c->conn = nullptr;
    c->store_bytes = c->ckpt_bytes = c->excess_bytes = c->acc_bytes = c->pckpt_bytes = c->conn_bytes = 0;
    c->arena = (char*)base;
    c->arena_size = bytes;
    c->arena_used = 0;
    c->has_grid = c->has_geom = c->saved = false;
    if (c->small) cudaMemsetAsync(c->small, 0, 256, stream);
}

// Device bytes a render (and, with adjoint != 0, its backward) needs, as carved from an
// arena: the same sizes render_impl / bos_set_grid / bos_backward allocate.
size_t request_bytes(const bos_grid_desc& g, const bos_camera_desc& cam, const bos_light_desc& light,
                     const bos_integrator_desc& it, int adjoint) {
    uint32_t nb[3] = {(uint32_t)(g.nx - 1 + kBrick - 1) / kBrick, (uint32_t)(g.ny - 1 + kBrick - 1) / kBrick,
                      (uint32_t)(g.nz - 1 + kBrick - 1) / kBrick};
    size_t slots = (size_t)morton3(nb[0] - 1, nb[1] - 1, nb[2] - 1) + 1;
    size_t bytes = align_up(slots * kBrickCells * elem_bytes(g.prec));
    if (adjoint) {
        TileShape ts = tile_shape(cam.width, cam.height, cam.spp);
        size_t nslots = (size_t)ts.tiles_x * ts.tiles_y * 32 * ts.samples_per_lane;
        int bound;
        if (it.fixed_steps > 0) {
            bound = it.fixed_steps;
        } else {
            double h[3] = {g.extent[0] / g.nx, g.extent[1] / g.ny, g.extent[2] / g.nz};
            double hmin = fmin(h[0], fmin(h[1], h[2]));
            double b = ceil(norm3(g.extent) / (it.max_step_vox * hmin)) + 2.0;
            bound = b > 2e9 ? 2000000000 : (int)b;
        }
        size_t max_ckpt = it.integrator == 2 ? 1 : (size_t)((bound + it.ckpt_every - 1) / it.ckpt_every);
        bytes += align_up(max_ckpt * 3 * nslots * sizeof(float4));
        bytes += align_up(nslots * (g.prec == BOS_PREC_FP64 ? 8 : 4));
        if (light.mode == 2) {   // the projector rays' checkpoints and the connection records
            bytes += align_up(max_ckpt * 3 * nslots * sizeof(float4));
            bytes += align_up(2 * nslots * sizeof(float4));
        }
        bytes += align_up((size_t)g.nx * g.ny * g.nz * (g.prec == BOS_PREC_FP64 ? 32 : 16));
        if (it.integrator != 2) bytes += align_up(adjoint_segment_bytes(it.ckpt_every));
    }
    return bytes;
}

}  // namespace bos

extern "C" {

const char* bos_error_string(bos_status_t s) {
    switch (s) {
        case BOS_OK: return "ok";
        case BOS_ERR_INVALID_ARG: return "invalid argument";
        case BOS_ERR_NOT_READY: return "not ready";
        case BOS_ERR_OOM: return "out of device memory";
        case BOS_ERR_ADMISSION: return "request exceeds the admission limit";
        case BOS_ERR_CUDA: return "CUDA error";
        case BOS_ERR_TIMEOUT: return "timed out";
        case BOS_ERR_DEVICE_CHECK: return "device-side check failed";
        case BOS_ERR_UNIMPLEMENTED: return "unimplemented";
    }
    return "unknown status";
}

const char* bos_last_error(void) { return g_last_error.c_str(); }

bos_status_t bos_create(bos_ctx** out, int device, uint64_t mem_limit_bytes) {
    if (!out) return fail(BOS_ERR_INVALID_ARG, "bos_create: NULL out");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "bos_create: cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(BOS_ERR_INVALID_ARG, "bos_create: no CUDA device %d", device);
    DeviceGuard dg(device);
    bos_ctx* c = new bos_ctx();
    c->device = device;
    c->mem_limit = mem_limit_bytes;
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "bos_create: SM count");
    }
    size_t have = 0;
    bos_status_t s = dev_alloc(c, &c->small, &have, 256, "bos_create");
    if (s != BOS_OK) {
        delete c;
        return s;
    }
    e = cudaMemset(c->small, 0, 256);
    if (e != cudaSuccess) {
        cudaFree(c->small);
        delete c;
        return cuda_fail(e, "bos_create: memset");
    }
    c->tile_counter = (int*)c->small;
    c->err = (int*)c->small + 1;
    c->steps = (unsigned long long*)((char*)c->small + 64);
    *out = c;
    return BOS_OK;
}

bos_status_t bos_destroy(bos_ctx* c) {
    if (!c) return BOS_OK;
    DeviceGuard dg(c->device);
    if (c->small) cudaFree(c->small);
    if (!c->arena) {
        void* bufs[] = {c->store, c->ckpt, c->excess, c->acc, c->pckpt, c->conn, c->seg};
        for (void* p : bufs)
            if (p) cudaFree(p);
    }
    delete c;
    return BOS_OK;
}

uint64_t bos_device_bytes(bos_ctx* c) { return c ? c->bytes : 0; }

bos_status_t bos_set_grid(bos_ctx* c, const bos_grid_desc* d, const float* T_dev, void* stream) {
    if (!c || !d || !T_dev) return fail(BOS_ERR_INVALID_ARG, "bos_set_grid: NULL argument");
    bos_status_t s0 = check_grid_desc(d, "bos_set_grid");
    if (s0 != BOS_OK) return s0;
    DeviceGuard dg(c->device);
    GridDev g{};
    int n[3] = {d->nx, d->ny, d->nz};
    for (int a = 0; a < 3; ++a) {
        g.n[a] = n[a];
        g.nb[a] = (n[a] - 1 + kBrick - 1) / kBrick;
        g.origin[a] = d->origin[a];
        g.extent[a] = d->extent[a];
        g.h[a] = d->extent[a] / (double)n[a];
        g.inv_h[a] = 1.0 / g.h[a];
        g.inv_hf[a] = (float)(1.0 / g.h[a]);
        g.hf[a] = (float)g.h[a];
    }
    g.K = d->rho0 * d->G * d->T0;
    g.prec = d->prec;
    size_t slots = (size_t)morton3(g.nb[0] - 1, g.nb[1] - 1, g.nb[2] - 1) + 1;
    size_t want = slots * kBrickCells * elem_bytes(d->prec);
    g.store_elems = (uint32_t)(slots * kBrickCells);
    g.err = c->err;
    bos_status_t s = dev_alloc(c, &c->store, &c->store_bytes, want, "bos_set_grid: brick store");
    if (s != BOS_OK) return s;
    g.store = c->store;
    cudaError_t e = launch_build_store(g, T_dev, c->store, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "bos_set_grid: launch");
    c->grid = *d;
    c->g = g;
    c->T = T_dev;
    c->has_grid = true;
    c->saved = false;
    return BOS_OK;
}

bos_status_t bos_set_geometry(bos_ctx* c, const bos_camera_desc* cam, const bos_wall_desc* wall,
                              const bos_light_desc* light, const float* pattern_dev, const bos_integrator_desc* it) {
    if (!c || !wall || !light || !it) return fail(BOS_ERR_INVALID_ARG, "bos_set_geometry: NULL argument");
    bos_status_t s = check_geometry_desc(cam, wall, light, pattern_dev, it, "bos_set_geometry");
    if (s != BOS_OK) return s;
    c->cam = to_dev(*cam);
    copy3(c->wall.origin, wall->origin);
    copy3(c->wall.eu, wall->eu);
    copy3(c->wall.ev, wall->ev);
    copy3(c->wall.normal, wall->normal);
    c->wall.size_u = wall->size_u;
    c->wall.size_v = wall->size_v;
    c->light.mode = light->mode;
    c->light.proj = to_dev(light->proj);
    c->light.tw = light->tw;
    c->light.th = light->th;
    c->light.pattern = pattern_dev;
    c->light.connect_iters = light->mode == 2 ? light->connect_iters : 0;
    c->integ.fixed_steps = it->fixed_steps;
    c->integ.max_step_vox = it->max_step_vox;
    c->integ.integrator = it->integrator;
    c->integ.ckpt_every = it->ckpt_every;
    c->has_geom = true;
    c->saved = false;
    return BOS_OK;
}

// Checks, checkpoint buffers and counters of a render (everything but the launch).
static bos_status_t render_prepare(bos_ctx* c, int mode, int save, cudaStream_t st, const int32_t* pix, long long npix,
                                   SceneDev& S, CkptDev& ck) {
    if (!c->has_grid || !c->has_geom) return fail(BOS_ERR_NOT_READY, "bos_render: set_grid and set_geometry first");
    if (c->light.mode == 2 && (mode == 3 || mode == 4))
        return fail(BOS_ERR_UNIMPLEMENTED, "bos_render: the refracted projector connection needs FP32_COMP or BF16_COMP");
    c->integ.max_steps = step_bound(c);
    S = scene_of(c);
    S.pix = pix;
    S.npix = npix;
    ck = CkptDev{};
    ck.every = c->integ.ckpt_every;
    ck.err = c->err;
    {
        TileShape ts = tile_shape(c->cam.width, c->cam.height, c->cam.spp);
        long long tiles = pix ? (npix + (32 / ts.G) - 1) / (32 / ts.G) : (long long)ts.tiles_x * ts.tiles_y;
        ck.nrays = tiles * 32 * ts.samples_per_lane;
    }
    if (save) {
        if (mode != 1 && mode != 2 && mode != 4)
            return fail(BOS_ERR_UNIMPLEMENTED, "bos_render: save_for_backward needs FP32_COMP, BF16_COMP or FP64");
        if (c->integ.integrator == 1)
            return fail(BOS_ERR_UNIMPLEMENTED, "bos_render: no adjoint for the RK4 integrator");
        if (mode == 4 && c->integ.integrator != 0)
            return fail(BOS_ERR_UNIMPLEMENTED, "bos_render: the FP64 adjoint needs Sharma RKN");
        // quasi-linear tracing keeps only the final state (one-sweep adjoint)
        ck.max_ckpt = c->integ.integrator == 2 ? 1 : (c->integ.max_steps + ck.every - 1) / ck.every;
        size_t want = (size_t)ck.max_ckpt * 3 * (size_t)ck.nrays * sizeof(float4);
        bos_status_t s = dev_alloc(c, (void**)&c->ckpt, &c->ckpt_bytes, want, "bos_render: checkpoints");
        if (s != BOS_OK) return s;
        // path-length record per ray: the float32 excess over ell, or (FP64) the float64 length
        s = dev_alloc(c, (void**)&c->excess, &c->excess_bytes, (size_t)ck.nrays * (mode == 4 ? 8 : 4),
                      "bos_render: excess");
        if (s != BOS_OK) return s;
        ck.state = c->ckpt;
        ck.excess = c->excess;
        if (c->light.mode == 2) {
            if (c->integ.integrator != 0 || c->light.connect_iters != 1)
                return fail(BOS_ERR_UNIMPLEMENTED,
                            "bos_render: the refracted connection's adjoint needs Sharma RKN and connect_iters = 1");
            s = dev_alloc(c, (void**)&c->pckpt, &c->pckpt_bytes, want, "bos_render: projector checkpoints");
            if (s != BOS_OK) return s;
            s = dev_alloc(c, (void**)&c->conn, &c->conn_bytes, 2 * (size_t)ck.nrays * sizeof(float4),
                          "bos_render: connection records");
            if (s != BOS_OK) return s;
            ck.pstate = c->pckpt;
            ck.conn = c->conn;
        }
    }
    cudaError_t e = cudaMemsetAsync(c->small, 0, 4, st);               // tile counter
    if (e == cudaSuccess && mode != 0) e = cudaMemsetAsync(c->steps, 0, 8, st);   // the reference traces nothing
    if (e != cudaSuccess) return cuda_fail(e, "bos_render: memset");
    return BOS_OK;
}

static bos_status_t render_impl(bos_ctx* c, int mode, float* I, float* disp, double* hit, int save, void* stream,
                                const int32_t* pix = nullptr, long long npix = 0) {
    if (!c || !I) return fail(BOS_ERR_INVALID_ARG, "bos_render: NULL context or I");
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    SceneDev S;
    CkptDev ck;
    bos_status_t s = render_prepare(c, mode, save, st, pix, npix, S, ck);
    if (s != BOS_OK) return s;
    WorkDev w{c->tile_counter, c->steps, c->err};
    RenderOut o{I, disp, hit};
    cudaError_t e = launch_render(mode, S, o, w, ck, c->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(e, "bos_render: launch");
    c->saved = save != 0;
    c->saved_ck = ck;
    c->saved_mode = mode;
    c->saved_pix = pix;
    c->saved_npix = npix;
    return BOS_OK;
}

bos_status_t bos_render(bos_ctx* c, float* I, float* disp, double* hit, int save_for_backward, void* stream) {
    if (!c) return fail(BOS_ERR_INVALID_ARG, "bos_render: NULL context");
    return render_impl(c, mode_of(c->grid.prec), I, disp, hit, save_for_backward, stream);
}

bos_status_t bos_render_pixels(bos_ctx* c, const int32_t* pix, int64_t npix, float* I, float* disp,
                               int save_for_backward, void* stream) {
    if (!c) return fail(BOS_ERR_INVALID_ARG, "bos_render_pixels: NULL context");
    if (!pix || npix <= 0 || npix > kMaxTiles)
        return fail(BOS_ERR_INVALID_ARG, "bos_render_pixels: need a pixel list of 1 .. 2^30 entries");
    return render_impl(c, mode_of(c->grid.prec), I, disp, nullptr, save_for_backward, stream, pix, npix);
}

bos_status_t bos_render_reference(bos_ctx* c, float* I, float* disp, double* hit, void* stream) {
    return render_impl(c, 0, I, disp, hit, 0, stream);
}

bos_status_t bos_ray_steps(bos_ctx* c, int32_t* nsteps, void* stream) {
    if (!c || !nsteps) return fail(BOS_ERR_INVALID_ARG, "bos_ray_steps: NULL argument");
    if (!c->has_grid || !c->has_geom) return fail(BOS_ERR_NOT_READY, "bos_ray_steps: set_grid and set_geometry first");
    DeviceGuard dg(c->device);
    c->integ.max_steps = step_bound(c);
    cudaError_t e = launch_ray_steps(scene_of(c), nsteps, c->num_sms, (cudaStream_t)stream);
    return e == cudaSuccess ? BOS_OK : cuda_fail(e, "bos_ray_steps");
}

bos_status_t bos_last_ray_steps(bos_ctx* c, uint64_t* out) {
    if (!c || !out) return fail(BOS_ERR_INVALID_ARG, "bos_last_ray_steps: NULL argument");
    DeviceGuard dg(c->device);
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpy(&v, c->steps, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "bos_last_ray_steps");
    *out = v;
    return BOS_OK;
}

bos_status_t bos_loss_l2(const float* I, const float* target, int64_t n, double* loss, float* dLdI, void* stream) {
    if (!I || !target || !loss || n < 0) return fail(BOS_ERR_INVALID_ARG, "bos_loss_l2: bad argument");
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = launch_loss_l2(I, target, n, loss, dLdI, sms, (cudaStream_t)stream);
    return e == cudaSuccess ? BOS_OK : cuda_fail(e, "bos_loss_l2");
}

static bos_status_t backward_impl(bos_ctx* c, const void* dLdI, void* dLdT, bool f64, void* stream) {
    if (!c || !dLdI || !dLdT) return fail(BOS_ERR_INVALID_ARG, "bos_backward: NULL argument");
    if (!c->saved) return fail(BOS_ERR_NOT_READY, "bos_backward: needs a bos_render with save_for_backward=1");
    if (f64 && c->saved_mode != 4)
        return fail(BOS_ERR_UNIMPLEMENTED, "bos_backward_f64: needs a render of the FP64 precision");
    DeviceGuard dg(c->device);
    size_t cells = (size_t)c->g.n[0] * c->g.n[1] * c->g.n[2];
    const size_t acc_bytes = cells * (c->saved_mode == 4 ? 32 : 16);   // float4, or four doubles (FP64) per node
    bos_status_t s = dev_alloc(c, (void**)&c->acc, &c->acc_bytes, acc_bytes, "bos_backward: accumulators");
    if (s != BOS_OK) return s;
    if (c->integ.integrator != 2) {   // the quasi-linear adjoint keeps no segment states
        s = dev_alloc(c, (void**)&c->seg, &c->seg_bytes, adjoint_segment_bytes(c->saved_ck.every),
                      "bos_backward: segment states");
        if (s != BOS_OK) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(c->acc, 0, acc_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->small, 0, 4, st);
    if (e != cudaSuccess) return cuda_fail(e, "bos_backward: memset");
    AdjDev adj{c->acc, static_cast<const float*>(dLdI), c->err, c->seg};
    WorkDev w{c->tile_counter, c->steps, c->err};
    SceneDev S = scene_of(c);
    S.pix = c->saved_pix;
    S.npix = c->saved_npix;
    e = f64 ? launch_backward_fp64(S, c->saved_ck, adj, w, c->T, dLdT, true, c->num_sms, st)
            : launch_backward(c->saved_mode, S, c->saved_ck, adj, w, c->T, static_cast<float*>(dLdT), c->num_sms, st);
    if (e == cudaErrorNotSupported) return fail(BOS_ERR_UNIMPLEMENTED, "bos_backward: not available for this mode");
    return e == cudaSuccess ? BOS_OK : cuda_fail(e, "bos_backward: launch");
}

bos_status_t bos_backward(bos_ctx* c, const float* dLdI, float* dLdT, void* stream) {
    return backward_impl(c, dLdI, dLdT, false, stream);
}

bos_status_t bos_backward_f64(bos_ctx* c, const double* dLdI, double* dLdT, void* stream) {
    return backward_impl(c, dLdI, dLdT, true, stream);
}

bos_status_t bos_export_nodes(bos_ctx* c, void* out, void* stream) {
    if (!c || !out) return fail(BOS_ERR_INVALID_ARG, "bos_export_nodes: NULL argument");
    if (!c->has_grid) return fail(BOS_ERR_NOT_READY, "bos_export_nodes: set_grid first");
    DeviceGuard dg(c->device);
    cudaError_t e = launch_export_nodes(c->g, out, c->num_sms, (cudaStream_t)stream);
    return e == cudaSuccess ? BOS_OK : cuda_fail(e, "bos_export_nodes");
}

bos_status_t bos_probe_read(const void* buf, uint64_t bytes, int repeats, float* sink, void* stream) {
    if (!buf || !sink || bytes < 16 || (bytes & 15) || repeats < 1 || ((uintptr_t)buf & 15))
        return fail(BOS_ERR_INVALID_ARG, "bos_probe_read: need a 16-byte aligned buffer of a multiple of 16 bytes");
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = launch_probe_read(buf, (long long)bytes, repeats, sink, sms, (cudaStream_t)stream);
    return e == cudaSuccess ? BOS_OK : cuda_fail(e, "bos_probe_read");
}

bos_status_t bos_probe_fma(int kind, int repeats, float* sink, double* flops, void* stream) {
    if (!sink || kind < 0 || kind > 2 || repeats < 1)
        return fail(BOS_ERR_INVALID_ARG, "bos_probe_fma: need kind 0, 1 or 2, repeats >= 1 and a sink");
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = launch_probe_fma(kind, repeats, sink, sms, flops, (cudaStream_t)stream);
    return e == cudaSuccess ? BOS_OK : cuda_fail(e, "bos_probe_fma");
}

bos_status_t bos_probe_read_l1(const void* buf, uint64_t bytes, int repeats, float* sink, double* bytes_read,
                               void* stream) {
    if (!buf || !sink || bytes < 32 || bytes > (64u << 10) || (bytes & 31) || repeats < 1 || ((uintptr_t)buf & 31))
        return fail(BOS_ERR_INVALID_ARG,
                    "bos_probe_read_l1: need a 32-byte aligned buffer of 32 B .. 64 KiB in multiples of 32 bytes");
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = launch_probe_read_l1(buf, (long long)bytes, repeats, sink, sms, bytes_read, (cudaStream_t)stream);
    return e == cudaSuccess ? BOS_OK : cuda_fail(e, "bos_probe_read_l1");
}

bos_status_t bos_debug_store_bound(bos_ctx* c, uint32_t elems) {
#if BOS_CHECKED
    if (!c || !c->has_grid) return fail(BOS_ERR_NOT_READY, "bos_debug_store_bound: set_grid first");
    if (elems < c->g.store_elems) c->g.store_elems = elems;
    return BOS_OK;
#else
    (void)c;
    (void)elems;
    return fail(BOS_ERR_UNIMPLEMENTED, "bos_debug_store_bound: bounds checks exist only in the checked build");
#endif
}

int bos_checked_build(void) { return BOS_CHECKED; }

bos_status_t bos_status(bos_ctx* c) {
    if (!c) return fail(BOS_ERR_INVALID_ARG, "bos_status: NULL context");
    DeviceGuard dg(c->device);
    int err = 0;
    cudaError_t e = cudaMemcpy(&err, c->err, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "bos_status");
    switch (err) {
        case DEV_OK: return BOS_OK;
        case DEV_STEP_BUDGET: return fail(BOS_ERR_DEVICE_CHECK, "a ray needed more steps than the step bound");
        case DEV_CKPT_OVERFLOW: return fail(BOS_ERR_DEVICE_CHECK, "a ray needed more checkpoints than allocated");
        case DEV_BAD_PIXEL: return fail(BOS_ERR_DEVICE_CHECK, "a pixel index of the list is outside the image");
        case DEV_BOUNDS: return fail(BOS_ERR_DEVICE_CHECK, "an index fell outside its buffer (checked build)");
        default: return fail(BOS_ERR_DEVICE_CHECK, "device error %d", err);
    }
}

}  // extern "C"

namespace bos {

// ---- hooks of the request server's batched launches

bool ctx_batchable(const bos_ctx* c) {
    const int mode = mode_of(c->grid.prec);
    return (mode == 1 || mode == 2) && (c->integ.integrator == 0 || c->integ.integrator == 2) && c->light.mode != 2 &&
           c->integ.ckpt_every <= 64;
}

bos_status_t ctx_batch_render(bos_ctx* c, float* I, float* disp, int save, cudaStream_t st, BatchJob* J, int* ntiles,
                              double* steps_per_tile) {
    DeviceGuard dg(c->device);
    const int mode = mode_of(c->grid.prec);
    SceneDev S;
    CkptDev ck;
    bos_status_t s = render_prepare(c, mode, save, st, nullptr, 0, S, ck);
    if (s != BOS_OK) return s;
    *J = BatchJob{};
    J->S = S;
    J->out = RenderOut{I, disp, nullptr};
    J->wk = WorkDev{c->tile_counter, c->steps, c->err};
    J->ck = ck;
    const TileShape ts = tile_shape(c->cam.width, c->cam.height, c->cam.spp);
    *ntiles = tile_count(S, ts);
    *steps_per_tile = 32.0 * ts.samples_per_lane * (double)c->integ.max_steps;
    c->saved = save != 0;
    c->saved_ck = ck;
    c->saved_mode = mode;
    c->saved_pix = nullptr;
    c->saved_npix = 0;
    return BOS_OK;
}

bos_status_t ctx_batch_backward(bos_ctx* c, const float* dLdI, cudaStream_t st, BatchJob* J) {
    if (!c->saved) return fail(BOS_ERR_NOT_READY, "bos_backward: needs a bos_render with save_for_backward=1");
    DeviceGuard dg(c->device);
    const size_t cells = (size_t)c->g.n[0] * c->g.n[1] * c->g.n[2];
    bos_status_t s = dev_alloc(c, (void**)&c->acc, &c->acc_bytes, cells * sizeof(float4), "bos_backward: accumulators");
    if (s != BOS_OK) return s;
    cudaError_t e = cudaMemsetAsync(c->acc, 0, cells * sizeof(float4), st);
    if (e != cudaSuccess) return cuda_fail(e, "bos_backward: memset");
    J->adj = AdjDev{c->acc, dLdI, c->err, nullptr};
    J->ck = c->saved_ck;
    return BOS_OK;
}

bos_status_t ctx_gradient(bos_ctx* c, float* dLdT, cudaStream_t st) {
    DeviceGuard dg(c->device);
    cudaError_t e = launch_gradient(c->g, c->acc, c->T, dLdT, c->num_sms, st);
    return e == cudaSuccess ? BOS_OK : cuda_fail(e, "bos_backward: gradient");
}

int ctx_num_sms(const bos_ctx* c) { return c->num_sms; }

}  // namespace bos
