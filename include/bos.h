/*
 * bos.h -- C ABI of the GB300 (sm_103a) BOS forward model and its adjoint.
 *
 * The library renders what a camera sees of a patterned back wall through a
 * heated, refracting air volume, and differentiates an image loss with respect
 * to the temperature field (single-view background-oriented schlieren,
 * arxiv 2509.14442):
 *
 *   a1  eta(T) = 1 + rho0 G T0 / T on the cell grid, grad eta by central
 *       differences (Sec. 2.1), stored in bricks              -> bos_set_grid
 *   a2  pinhole rays, tent-filter Monte Carlo over each pixel (Sec. 2.3)
 *   a3  nonlinear ray tracing dr/dt = v, dv/dt = eta grad eta (Sec. 2.2, Eq. 1)
 *       with Sharma's Runge-Kutta-Nystrom steps
 *   a4  straight extrapolation to the back wall
 *   a5  radiance L_wall <n_w, v_w> / |path| per ray, averaged over the pixel
 *       (Sec. 2.3, Eq. 2)                                      -> bos_render
 *   a6  gradient of L_BOS = sum_j (I_flow_j - I_j)^2 (Sec. 2.4) with respect
 *       to T by a discrete adjoint                            -> bos_backward
 *
 * Conventions (every call):
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *    library never frees them.  The library owns its own device buffers (the
 *    brick store, checkpoints, accumulators) and frees them in bos_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Every call that launches work is asynchronous on that stream and
 *    returns as soon as the work is enqueued.
 *  - Every call returns a bos_status_t; no exception or abort crosses the ABI.
 *    bos_last_error() gives a message for the most recent failure on the
 *    calling thread.  Errors found by a kernel (bounded waits that timed out,
 *    step budgets exceeded) are sticky in the context and read by bos_status()
 *    after the caller has synchronised the stream.
 *  - A context is not thread-safe: use one context per host thread / stream.
 *  - Layouts: T is (nz, ny, nx) float32, x fastest.  Images are (height, width)
 *    row-major, row 0 at the top.  Wall coordinates are metres along (eu, ev).
 */
#ifndef BOS_H
#define BOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bos_ctx bos_ctx;

typedef enum {
    BOS_OK = 0,
    BOS_ERR_INVALID_ARG = 1,   /* a descriptor or pointer failed validation */
    BOS_ERR_NOT_READY = 2,     /* a call needs set_grid / set_geometry / a saved render first */
    BOS_ERR_OOM = 3,           /* a device allocation failed or would exceed the context limit */
    BOS_ERR_ADMISSION = 4,     /* the request does not fit the server's memory limit */
    BOS_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    BOS_ERR_TIMEOUT = 6,       /* a bounded wait ran out */
    BOS_ERR_DEVICE_CHECK = 7,  /* a kernel flagged an error (see bos_last_error) */
    BOS_ERR_UNIMPLEMENTED = 8  /* the combination of options is not supported */
} bos_status_t;

/* Arithmetic of the field store and of the integrator.
 *  FP64:       float64 store (32 B per cell), float64 ray state.
 *  FP32:       float32 store (32 B per cell: the cell's record and its difference to
 *              the next cell along x), plain float32 absolute ray state.
 *  FP32_COMP:  float32 store; each ray keeps its straight line in 32.32 fixed
 *              point (grid units) derived from its float64 origin and integrates
 *              only its small deviation from that line in float32 with
 *              compensated (Kahan) sums; float64 only at the ray origin and the
 *              wall intersection.
 *  BF16_COMP:  as FP32_COMP with a bfloat16 store (16 B per cell: the cell's record
 *              and the next one along x). */
typedef enum {
    BOS_PREC_FP64 = 0,
    BOS_PREC_FP32 = 1,
    BOS_PREC_FP32_COMP = 2,
    BOS_PREC_BF16_COMP = 3
} bos_precision_t;

/* Voxel grid: nx*ny*nz cells over the box [origin, origin + extent]; the
 * sample of cell (i, j, k) sits at its centre origin + (i + 1/2, j + 1/2, k + 1/2) h,
 * h = extent / n.  T0 (K), rho0 (kg/m^3) and G (m^3/kg) enter eta(T) = 1 + rho0 G T0 / T
 * (Sec. 2.1).  Requires 2 <= n <= 8192 along every axis and fewer than 2^31 cells,
 * extent > 0, T0 rho0 G > 0. */
typedef struct {
    int nx, ny, nz;
    double origin[3];
    double extent[3];
    double T0, rho0, G;
    int prec;                   /* bos_precision_t */
} bos_grid_desc;

/* Pinhole camera (and projector): position, unit viewing direction `fwd`, unit
 * `up` orthogonal to it; right = fwd x up.  Image point (x, y) in pixels (y down)
 * looks along normalise(((x - cx)/fx) right - ((y - cy)/fy) up + fwd).  At most 2^40
 * rays (width*height*spp) and 2^30 warp tiles of 32 rays (8x4 pixels at spp = 1).
 * spp rays per pixel: one ray through the pixel centre if spp == 1, otherwise
 * tent-filter (radius 1 px) offsets drawn from splitmix64 output k = 1 + (pixel*spp + s)
 * for `seed` (Sec. 2.3: triangular filter, Monte Carlo over the pixel). */
typedef struct {
    double pos[3], fwd[3], up[3];
    double fx, fy, cx, cy;
    int width, height, spp;
    uint64_t seed;
} bos_camera_desc;

/* Back-wall plane through `origin` spanned by unit eu, ev; unit `normal` points
 * away from the camera (so <normal, v> > 0 for rays that reach it). */
typedef struct {
    double origin[3], eu[3], ev[3], normal[3];
    double size_u, size_v;
} bos_wall_desc;

/* Wall luminance (Sec. 2.3): mode 0 -- a tw x th texture covering the wall
 * rectangle [0, size_u] x [0, size_v]; mode 1 -- a pinhole projector `proj`
 * casting a tw x th pattern, connected to the wall point by a straight line;
 * mode 2 -- the same projector with a refracted connection: the pattern point that
 * lights wall point x_w is the one whose own ray, traced through the field like a
 * camera ray, lands on x_w, found by connect_iters (1..16) rounds of aiming
 * a <- a + (x_w - y(a)) from a = x_w, y(a) the wall hit of the projector ray aimed at a.
 * Mode 2 renders with the compensated tracers (BOS_PREC_FP32_COMP, BOS_PREC_BF16_COMP);
 * its backward needs Sharma RKN and connect_iters = 1.  All patterns are bilinear on
 * texel centres and zero outside.  connect_iters is ignored in modes 0 and 1. */
typedef struct {
    int mode;
    bos_camera_desc proj;
    int tw, th;
    int connect_iters;
} bos_light_desc;

/* Integrator: fixed_steps in [1, 2^24] gives every ray that many steps; fixed_steps = 0
 * gives N = ceil(ell / (max_step_vox * min h)) for the straight in-box segment of
 * length ell, max_step_vox in (1e-3, 1e6).  integrator 0 = Sharma's Runge-Kutta-Nystrom,
 * 1 = classic RK4 (forward only), 2 = quasi-linear (the index field sampled on the
 * straight line, Sec. 2.2).  ckpt_every = K in [1, 4096]: the adjoint keeps the ray state
 * every K steps. */
typedef struct {
    int fixed_steps;
    double max_step_vox;
    int integrator;
    int ckpt_every;
} bos_integrator_desc;

/* Create a context on CUDA `device`.  mem_limit_bytes caps the library's own
 * device allocations (0 = no cap); exceeding it gives BOS_ERR_OOM. */
bos_status_t bos_create(bos_ctx** out, int device, uint64_t mem_limit_bytes);

/* Free every buffer the context owns.  The caller must have synchronised the
 * streams the context used.  NULL is accepted. */
bos_status_t bos_destroy(bos_ctx* ctx);

/* Step a1 (Sec. 2.1): build the field store from T_dev (nz*ny*nx float32 kelvin,
 * all > 0).  Per cell, in float64: deta = rho0 G T0 / T; grad eta by central
 * differences (deta[i+1] - deta[i-1]) / (2h), one-sided (deta[1]-deta[0])/h at the
 * faces; then rounded to the store type of desc->prec.  The store is a Morton-ordered
 * array of 8x8x8-cell bricks with a one-cell apron, so every trilinear corner sits at a
 * fixed offset; float32 and bf16 stores keep x pairs, so a cell's 8 corners are four
 * 32-byte (bf16: 16-byte) loads, and a float64 store eight 32-byte loads.
 * T_dev must stay allocated and unchanged until the last bos_backward that uses
 * this grid (the adjoint's chain rule d eta / dT = -rho0 G T0 / T^2 reads it). */
bos_status_t bos_set_grid(bos_ctx* ctx, const bos_grid_desc* desc, const float* T_dev, void* stream);

/* Camera, wall, light and integrator (Sec. 2.3).  Descriptors are copied;
 * pattern_dev (th*tw float32, row 0 = v 0 for a texture, = top row for a
 * projector) is caller-owned and must stay valid until the last render/backward. */
bos_status_t bos_set_geometry(bos_ctx* ctx, const bos_camera_desc* cam, const bos_wall_desc* wall,
                              const bos_light_desc* light, const float* pattern_dev,
                              const bos_integrator_desc* integ);

/* Steps a2-a5 (Eq. 1, Eq. 2): trace every ray of every pixel through the field
 * and write per pixel
 *   I_dev    (height*width float32): mean over the pixel's rays of L_wall <n_w, v_w>/(|v_w| len),
 *   disp_dev (height*width*2 float32, nullable): mean wall-plane displacement of the
 *            hit from the straight (no-flow) hit of the same ray, metres along (eu, ev),
 *   hit_dev  (height*width*2 float64, nullable): mean wall coordinates of the hits.
 * Rays that never reach the wall plane contribute zero.  save_for_backward != 0
 * stores the ray state every ckpt_every steps for bos_backward: FP32_COMP or BF16_COMP with
 * Sharma RKN or quasi-linear tracing, or FP64 with Sharma RKN (the absolute (r, v) as six
 * doubles); otherwise BOS_ERR_UNIMPLEMENTED. */
bos_status_t bos_render(bos_ctx* ctx, float* I_dev, float* disp_dev, double* hit_dev, int save_for_backward,
                        void* stream);

/* Steps a2-a5 for a subset of the pixels (the paper's reconstruction draws 5000 random
 * pixels of the BOS image per iteration, Sec. 3.2): pix_dev holds npix (1 .. 2^30) flat pixel indices
 * y*width + x (any order, repeats allowed; indices outside the image are skipped and
 * flagged in bos_status).  I_dev receives npix float32 values and disp_dev (nullable)
 * npix*2, entry k belonging to pix_dev[k].  With save_for_backward, the next
 * bos_backward takes dL/dI as npix values in the same order; pix_dev must stay valid
 * until then. */
bos_status_t bos_render_pixels(bos_ctx* ctx, const int32_t* pix_dev, int64_t npix, float* I_dev, float* disp_dev,
                               int save_for_backward, void* stream);

/* The reference image I_ref (Sec. 2.1: no flow): the same rays, straight, with
 * the ambient index.  Same outputs as bos_render. */
bos_status_t bos_render_reference(bos_ctx* ctx, float* I_dev, float* disp_dev, double* hit_dev, void* stream);

/* Step count of every ray (height*width*spp int32, ray = pixel*spp + s): the
 * integer decision of step a2, for checks. */
bos_status_t bos_ray_steps(bos_ctx* ctx, int32_t* nsteps_dev, void* stream);

/* Total ray-steps of the most recent bos_render (sum over rays of N), read after
 * the render's stream has been synchronised. */
bos_status_t bos_last_ray_steps(bos_ctx* ctx, uint64_t* out);

/* L_BOS (Sec. 2.4) for n pixels: loss_dev (1 float64) = sum_j (target_j - I_j)^2 and
 * dLdI_dev (n float32, nullable) = -2 (target_j - I_j). */
bos_status_t bos_loss_l2(const float* I_dev, const float* target_dev, int64_t n, double* loss_dev,
                         float* dLdI_dev, void* stream);

/* L_BOS over a pixel minibatch (Sec. 2.4, Sec. 3.2), times a constant scale s > 0:
 * loss_dev (1 float64) = s sum_k (target[pix_k] - I_k)^2 and dLdI_dev (npix float32,
 * nullable) = -2 s (target[pix_k] - I_k), with I_dev from bos_render_pixels over pix_dev
 * and target_dev a whole image.  The scale brings image-loss gradients (often 1e-10 per
 * voxel, since I carries the 1/path-length weight) above an optimiser's epsilon. */
bos_status_t bos_loss_l2_pixels(const float* I_dev, const float* target_dev, const int32_t* pix_dev, int64_t npix,
                                float scale, double* loss_dev, float* dLdI_dev, void* stream);

/* A minibatch of npix uniformly random pixel indices in [0, n_pixels) (with repeats):
 * entry k is the splitmix64 output number d*npix + k + 1 for `seed`, scaled to the range
 * by a 64x64-bit multiply-high, with draw number d = draw + *draw_dev (draw_dev nullable,
 * read on the device, so a captured CUDA graph can replay successive draws).  Used for the
 * random BOS-pixel minibatches of Sec. 3.2. */
bos_status_t bos_sample_pixels(int32_t* pix_dev, int64_t npix, int64_t n_pixels, uint64_t seed, uint64_t draw,
                               const uint64_t* draw_dev, void* stream);

/* One AdaBelief step (the optimiser of Sec. 3.2; Zhuang et al., NeurIPS 2020) on n float32
 * parameters: m = b1 m + (1-b1) g; s = b2 s + (1-b2) (g-m)^2 + eps;
 * theta -= lr (m / (1 - b1^t)) / (sqrt(s / (1 - b2^t)) + eps), with step number
 * t = step + *step_dev (step_dev nullable, read on the device); t >= 1; m and s start at 0. */
bos_status_t bos_adabelief_step(float* theta_dev, const float* grad_dev, float* m_dev, float* s_dev, int64_t n,
                                float lr, float beta1, float beta2, float eps, int64_t step, const uint64_t* step_dev,
                                void* stream);

/* Reorder a pixel list in place (npix <= 16384, width and height <= 65535) by the Morton
 * (Z-order) key of (px, py), so that the 32 rays of a warp come from neighbouring pixels.
 * The list keeps its entries (with repeats), so every sum over it is unchanged up to
 * summation order; random minibatches (Sec. 3.2) otherwise give each warp rays from all over
 * the image.  One block; asynchronous on `stream`. */
bos_status_t bos_sort_pixels(int32_t* pix_dev, int64_t npix, int width, int height, void* stream);

/* *counter_dev += inc on the device (an iteration counter for bos_sample_pixels and
 * bos_adabelief_step inside a captured CUDA graph). */
bos_status_t bos_counter_add(uint64_t* counter_dev, uint64_t inc, void* stream);

/* Step a6 (Sec. 2.4): given dL/dI (height*width float32, or npix values after
 * bos_render_pixels) for the most recent render with save_for_backward=1, write dL/dT
 * (nz*ny*nx float32).  Needs the FP32_COMP or BF16_COMP precision with Sharma RKN
 * (ckpt_every <= 64) or quasi-linear tracing (integrator 2), or the FP64 precision with
 * Sharma RKN (ckpt_every <= 64), which runs the whole adjoint in float64 (else
 * BOS_ERR_UNIMPLEMENTED).
 * dLdI_dev must not alias the accumulators.  Sharma RKN: reverses the steps of every ray
 * from its checkpoints; quasi-linear: one forward-order sweep per ray from its final
 * state (its field samples lie on the straight line, Sec. 2.2).  Both scatter
 * d L / d(deta, grad eta) into the grid with warp-aggregated atomics, then apply the
 * transpose of the difference stencil and d deta/dT = -rho0 G T0 / T^2. */
bos_status_t bos_backward(bos_ctx* ctx, const float* dLdI_dev, float* dLdT_dev, void* stream);

/* Step a6 for the FP64 precision with a float64 seed and result (Sec. 2.4): as
 * bos_backward, for the most recent FP64 render with save_for_backward=1 (Sharma RKN,
 * ckpt_every <= 64), with dL/dI given as float64 (height*width, or npix after
 * bos_render_pixels) and dL/dT written as float64 (nz*ny*nx), so that the float64 adjoint's
 * result is not rounded to float32 at the boundary.  BOS_ERR_UNIMPLEMENTED for a render of
 * another precision. */
bos_status_t bos_backward_f64(bos_ctx* ctx, const double* dLdI_dev, double* dLdT_dev, void* stream);

/* Copy the stored node values back in grid order: out_dev receives nz*ny*nx*4
 * values (deta, d eta/dx, d eta/dy, d eta/dz) of the store type (float32, bf16 as
 * uint16 bit patterns, or float64), read through the brick addressing. */
bos_status_t bos_export_nodes(bos_ctx* ctx, void* out_dev, void* stream);

/* Measurement probe, no counterpart in the paper: read `bytes` (a multiple of 16, 16-byte
 * aligned) of buf_dev `repeats` times with coalesced 16-byte loads that bypass L1, so that
 * with a buffer smaller than L2 the caller can time the L2 read bandwidth that bounds
 * the tracer's gathers.  sink_dev (1 float) is written only to keep the loads alive. */
bos_status_t bos_probe_read(const void* buf_dev, uint64_t bytes, int repeats, float* sink_dev, void* stream);

/* Measurement probe, no counterpart in the paper: the fused multiply-add throughput of
 * this GPU.  kind 0 = float32 fma, 1 = packed float32 pairs (fma.rn.f32x2), 2 = float64
 * fma.  Launches 4 blocks of 256 threads per SM; each thread runs eight independent
 * recurrences x <- x*a + b for repeats x 16 rounds.  The caller times the launch on
 * `stream`; *flops_out (host, may be NULL) receives the launch's flop count (2 per FMA,
 * 4 per packed FMA).  sink_dev (1 float) is written only to keep the chains alive.
 * Errors: BOS_ERR_INVALID_ARG for another kind, repeats < 1 or a NULL sink. */
bos_status_t bos_probe_fma(int kind, int repeats, float* sink_dev, double* flops_out, void* stream);

/* Measurement probe, no counterpart in the paper: the L1 read bandwidth of the 256-bit
 * non-coherent loads (ld.global.nc.v8.f32) the tracer's gathers use.  Launches 4 blocks of
 * 256 threads per SM; every block reads all of buf_dev (32 B .. 64 KiB, a multiple of 32,
 * 32-byte aligned, so it stays resident in each SM's L1) `repeats` times.  The caller
 * times the launch on `stream`; *bytes_out (host, may be NULL) receives the bytes read.
 * sink_dev (1 float) is written only to keep the loads alive.
 * Errors: BOS_ERR_INVALID_ARG for another size or alignment, repeats < 1 or a NULL pointer. */
bos_status_t bos_probe_read_l1(const void* buf_dev, uint64_t bytes, int repeats, float* sink_dev, double* bytes_out,
                               void* stream);

/* Forward render that allocates nothing, for callers that must not call cudaMalloc
 * (a latency-critical loop, where allocation and freeing can synchronise the device, or
 * a host whose device memory is already handed out by another allocator).  No
 * counterpart in the paper: it runs the same field build and render as bos_set_grid +
 * bos_set_geometry + bos_render (any precision, light mode and integrator those accept;
 * no checkpoints), with the field store and the work counters in one file-scope device
 * array of 128 MiB that the library reserves on every GPU it is loaded on, until the
 * process exits.  The caller passes the inputs (T_dev, pattern_dev) and outputs (I_dev,
 * disp_dev nullable) as in bos_render.  The descriptors are checked exactly as
 * bos_set_grid and bos_set_geometry check them (BOS_ERR_INVALID_ARG).
 * Grids whose field store exceeds the array (128 MiB - 256 B; e.g. 128x128x96 cells
 * fit in float32, 256x256x192 do not) are rejected with BOS_ERR_INVALID_ARG and a
 * message in bos_last_error().  The first call on a device looks up the array's
 * address with that device current; make that first call before any stream capture.
 * Every call shares the array: calls whose work overlaps on the GPU race and must be
 * serialised by the caller.  Each call clears the counters and the error word and
 * rebuilds the store, so leftovers of the previous call do not matter.  Errors the
 * kernels detect are read with bos_noalloc_status.  Asynchronous on `stream`. */
bos_status_t bos_render_noalloc(const bos_grid_desc* grid, const float* T_dev, const bos_camera_desc* cam,
                                const bos_wall_desc* wall, const bos_light_desc* light, const float* pattern_dev,
                                const bos_integrator_desc* integ, float* I_dev, float* disp_dev, void* stream);

/* Device-detected errors of the most recent bos_render_noalloc on the current device
 * (the kernels' sticky error word inside the shared array): BOS_OK, or
 * BOS_ERR_DEVICE_CHECK with a message in bos_last_error().  Call it after synchronising
 * that render's stream; like the array, it races with a bos_render_noalloc still running.
 * Allocates nothing (one 4-byte device-to-host copy). */
bos_status_t bos_noalloc_status(void);

/* The checked build (library built with BOS_CHECKED=1, libbos_checked.so), a stand-in for a
 * memory checker: every gather from the field store, every node-accumulator atomic and
 * every checkpoint access is checked against the extent of its buffer; an index outside it
 * is recorded in the context's error word (bos_status then returns BOS_ERR_DEVICE_CHECK)
 * and replaced by index 0, so the access stays inside the buffer.  No counterpart in the
 * paper.  bos_checked_build returns 1 in that build and 0 otherwise. */
int bos_checked_build(void);

/* Checked build only, for testing the checks: lower the field-store bound the checks use to
 * `elems` elements (never above the real extent), so that gathers beyond it are reported
 * while every access still lands inside the real store.  BOS_ERR_UNIMPLEMENTED in the
 * ordinary build; BOS_ERR_NOT_READY before bos_set_grid; bos_set_grid restores the bound. */
bos_status_t bos_debug_store_bound(bos_ctx* ctx, uint32_t elems);

/* Sticky device-side status of the context (call after synchronising). */
bos_status_t bos_status(bos_ctx* ctx);

/* Static description of a status code. */
const char* bos_error_string(bos_status_t s);

/* Message of the last failing call on this thread ("" if none). */
const char* bos_last_error(void);

/* Bytes of device memory the context currently owns. */
uint64_t bos_device_bytes(bos_ctx* ctx);

/* ------------------------------------------------------------------ request server
 *
 * Continuous batching of renders on one GPU.  A request is one frame: a temperature field
 * on the device plus geometry; it is a forward render, or with target_dev set a forward +
 * adjoint render (L_BOS against target_dev, then dL/dT).  Requests queue in arrival order;
 * the server admits the head when fewer than `slots` requests are in flight and the
 * request's exact device footprint (bos_request_footprint) fits in the unused part of the
 * server's arena, one allocation of mem_limit_bytes made at creation.  Admitted requests
 * share batched launches: each launch pulls warp tiles of every admitted request in the
 * same phase (render, or adjoint) from one device work list, oldest request first, with a
 * few milliseconds of work per launch, so a request that arrives while others run joins
 * the next launch and the work of all admitted requests overlaps on the device.  Requests
 * with FP32_COMP or BF16_COMP stores, Sharma RKN or quasi-linear tracing, light mode 0 or 1
 * and ckpt_every <= 64 are batched; others run their own launches in the same order.  All
 * device buffers named in a request are caller-owned and must stay valid until the request
 * is done.  The server never blocks without a bound: bos_wait and bos_server_destroy take
 * timeouts and return BOS_ERR_TIMEOUT; no kernel waits on the host. */

typedef struct bos_server bos_server;

typedef struct {
    bos_grid_desc grid;
    const float* T_dev;            /* nz*ny*nx float32 */
    bos_camera_desc cam;
    bos_wall_desc wall;
    bos_light_desc light;
    const float* pattern_dev;      /* th*tw float32 */
    bos_integrator_desc integ;
    float* I_dev;                  /* out: height*width float32 */
    float* disp_dev;               /* out, nullable: height*width*2 float32 */
    const float* target_dev;       /* nullable: height*width float32; set -> forward + adjoint */
    double* loss_dev;              /* out with target: 1 float64 */
    float* dLdT_dev;               /* out with target: nz*ny*nx float32 */
} bos_request;

typedef struct {
    uint64_t submit_ns, admit_ns, done_ns;   /* host steady-clock times (0 = not yet) */
    uint64_t footprint_bytes;
    int status;                              /* the request's bos_status_t once done */
    int done;
    int slot;
} bos_ticket_info;

/* Run the scheduler without touching a GPU: admitted requests "run" for a time
 * proportional to their footprint.  For tests of admission and queueing. */
#define BOS_SERVER_FAKE_EXECUTOR 1

/* Device bytes the server reserves for this request while it runs. */
bos_status_t bos_request_footprint(const bos_request* req, uint64_t* bytes);

/* Create a server on `device` with an arena of mem_limit_bytes and `slots` concurrent
 * requests (1..64).  BOS_ERR_OOM if the arena cannot be allocated.  With an arena of at
 * least 804 MiB, 201 MiB of it hold the batched Sharma adjoint's per-warp segment states;
 * below that, forward + adjoint Sharma requests run their own launches. */
bos_status_t bos_server_create(bos_server** out, int device, uint64_t mem_limit_bytes, int slots, int flags);

/* Queue a request (descriptors are copied).  BOS_ERR_ADMISSION if its footprint exceeds
 * the arena, BOS_ERR_INVALID_ARG for a malformed request. */
bos_status_t bos_submit(bos_server* s, const bos_request* req, uint64_t* ticket);

/* Wait up to timeout_ns for a request; returns its status, or BOS_ERR_TIMEOUT. */
bos_status_t bos_wait(bos_server* s, uint64_t ticket, uint64_t timeout_ns);

/* Times, footprint and status of a request. */
bos_status_t bos_ticket(bos_server* s, uint64_t ticket, bos_ticket_info* info);

/* Arena size, peak arena use, queued and running requests. */
bos_status_t bos_server_stats(bos_server* s, uint64_t* arena_bytes, uint64_t* peak_used_bytes, int* queued,
                              int* running);

/* Batched launches so far: their number, the warp tiles they ran, the sum over launches of
 * the requests each one served, and the most requests one launch served. */
bos_status_t bos_server_batches(bos_server* s, uint64_t* launches, uint64_t* tiles, uint64_t* job_shares,
                                int* max_jobs);

/* Stop accepting requests, wait up to timeout_ns for queued and running ones, then free
 * everything.  BOS_ERR_TIMEOUT leaves the server running (call again). */
bos_status_t bos_server_destroy(bos_server* s, uint64_t timeout_ns);

#ifdef __cplusplus
}
#endif

#endif /* BOS_H */
