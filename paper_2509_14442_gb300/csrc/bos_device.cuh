// Device-side building blocks of the BOS library (sm_103a).
//
// Internal to the CUDA library: the brick store layout, the float64 ray set-up
// (bit-exact integer decisions), trilinear field evaluation for each store type and
// the float64 wall/luminance epilogue.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef BOS_CHECKED
#define BOS_CHECKED 0   // 1: the checked build (bounds checks on every indexed device buffer)
#endif

namespace bos {

// Device-side error word: first error code wins.
enum DeviceError : int { DEV_OK = 0, DEV_STEP_BUDGET = 1, DEV_CKPT_OVERFLOW = 2, DEV_BAD_PIXEL = 3, DEV_BOUNDS = 4 };

__device__ __forceinline__ void flag_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// Index i into a buffer of n elements.  The checked build records an index outside the
// buffer in the error word and returns 0 instead, so the access stays inside the buffer;
// the ordinary build returns i as it is.
__device__ __forceinline__ uint32_t bounded(uint32_t i, uint32_t n, int* err) {
#if BOS_CHECKED
    if (i >= n) {
        flag_error(err, DEV_BOUNDS);
        return 0;
    }
#endif
    return i;
}
__device__ __forceinline__ size_t bounded(size_t i, size_t n, int* err) {
#if BOS_CHECKED
    if (i >= n) {
        flag_error(err, DEV_BOUNDS);
        return 0;
    }
#endif
    return i;
}

// ------------------------------------------------------------------ descriptors

struct GridDev {
    int n[3];          // cells per axis
    int nb[3];         // bricks per axis (covering base cells 0 .. n-2)
    double origin[3];
    double extent[3];
    double h[3];       // extent / n
    double inv_h[3];   // 1 / h
    double K;          // rho0 * G * T0
    float inv_hf[3];   // 1 / h (float)
    float hf[3];
    int prec;
    const void* store; // bricks: slot * 729 + (lz * 9 + ly) * 9 + lx
    uint32_t store_elems;   // elements of the store (the checked build's bound)
    int* err;               // the context's error word (the checked build's reports)
};

struct CamDev {
    double pos[3], fwd[3], up[3];
    double fx, fy, cx, cy;
    int width, height, spp;
    unsigned long long seed;
};

struct WallDev {
    double origin[3], eu[3], ev[3], normal[3];
    double size_u, size_v;
};

struct LightDev {
    int mode;            // 0 texture, 1 projector (straight connection), 2 projector (refracted)
    CamDev proj;
    int tw, th;
    const float* pattern;
    int connect_iters;   // mode 2: aiming rounds per wall point
};

struct IntegDev {
    int fixed_steps;
    double max_step_vox;
    int integrator;
    int ckpt_every;
    int max_steps;     // bound on N for any ray of this grid/camera (sizes checkpoints)
};

// Ray-independent float64 terms of the ray set-up, formed on the host with the same IEEE
// operations (and order) the per-ray code would apply, so every ray sees the same bits.
struct RayConst {
    double right[3];       // fwd x up
    double lo_m[3];        // grid origin - camera position
    double hi_m[3];        // (grid origin + extent) - camera position
    double qn;             // (wall origin - camera position) . wall normal
    double step;           // max_step_vox * min(h)
    double plo_m[3];       // the same three terms for the projector pinhole (light modes 1, 2)
    double phi_m[3];
    double pqn;
};

struct SceneDev {
    GridDev g;
    CamDev cam;
    WallDev w;
    LightDev L;
    IntegDev it;
    RayConst rc;
    const int32_t* pix;   // nullptr: the whole image; else a list of flat pixel indices
    long long npix;
};

struct D4 {            // float64 store element
    double x, y, z, w;
};

constexpr int kBrick = 8;
constexpr int kBrickSide = 9;                     // 8 cells + 1 apron cell
constexpr int kBrickCells = kBrickSide * kBrickSide * kBrickSide;

// ------------------------------------------------------------------ float64, no contraction
// The ray set-up must round exactly like a plain IEEE double program evaluated in
// source order, so every operation is an explicit round-to-nearest intrinsic.

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dsqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ double ddot(const double a[3], const double b[3]) {
    return dadd(dadd(dmul(a[0], b[0]), dmul(a[1], b[1])), dmul(a[2], b[2]));
}

// ------------------------------------------------------------------ brick addressing

__host__ __device__ __forceinline__ uint32_t spread3(uint32_t x) {   // 10 bits -> every third bit
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__host__ __device__ __forceinline__ uint32_t morton3(uint32_t bx, uint32_t by, uint32_t bz) {
    return spread3(bx) | (spread3(by) << 1) | (spread3(bz) << 2);
}

// Offset (in elements) of base corner (i, j, k), 0 <= i <= n-2: its brick's Morton slot
// and its place inside the brick; the 7 other corners follow at +1, +9, +10, +81, +82,
// +90, +91.
__host__ __device__ __forceinline__ uint32_t brick_offset(int i, int j, int k) {
    uint32_t slot = morton3((uint32_t)i >> 3, (uint32_t)j >> 3, (uint32_t)k >> 3);
    return slot * (uint32_t)kBrickCells + (uint32_t)(((k & 7) * kBrickSide + (j & 7)) * kBrickSide + (i & 7));
}

// Per-ray cache of the current brick's slot base.
struct BrickCache {
    uint32_t key;
    uint32_t base;
};

__device__ __forceinline__ uint32_t cached_offset(BrickCache& bc, int i, int j, int k) {
    uint32_t key = ((uint32_t)i >> 3) | (((uint32_t)j >> 3) << 10) | (((uint32_t)k >> 3) << 20);
    if (key != bc.key) {
        bc.key = key;
        bc.base = morton3((uint32_t)i >> 3, (uint32_t)j >> 3, (uint32_t)k >> 3) * (uint32_t)kBrickCells;
    }
    return bc.base + (uint32_t)(((k & 7) * kBrickSide + (j & 7)) * kBrickSide + (i & 7));
}

// ------------------------------------------------------------------ store loads

__device__ __forceinline__ float4 load_cell(const float4* s, uint32_t o) { return __ldg(s + o); }

__device__ __forceinline__ float4 load_cell(const uint2* s, uint32_t o) {
    uint2 u = __ldg(s + o);
    float4 r;
    r.x = __uint_as_float(u.x << 16);
    r.y = __uint_as_float(u.x & 0xffff0000u);
    r.z = __uint_as_float(u.y << 16);
    r.w = __uint_as_float(u.y & 0xffff0000u);
    return r;
}

// Packed pairs of float32 (sm_100+ f32x2 arithmetic: each lane rounds like the scalar op).
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// a + t (b - a), per lane exactly fmaf(t, b - a, a)
__device__ __forceinline__ f32x2 lerp2(f32x2 a, f32x2 b, f32x2 t) { return fma2(t, sub2(b, a), a); }

struct Cell2 {           // one (deta, gx, gy, gz) record as two packed pairs
    f32x2 lo, hi;
};

__device__ __forceinline__ Cell2 load_cell2(const float4* s, uint32_t o) {
    float4 v = __ldg(s + o);
    return Cell2{pack2(v.x, v.y), pack2(v.z, v.w)};
}
__device__ __forceinline__ Cell2 load_cell2(const uint2* s, uint32_t o) {
    uint2 u = __ldg(s + o);
    return Cell2{pack2(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u)),
                 pack2(__uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u))};
}
__device__ __forceinline__ Cell2 lerpc(Cell2 a, Cell2 b, f32x2 t) { return Cell2{lerp2(a.lo, b.lo, t), lerp2(a.hi, b.hi, t)}; }

// ---- paired store elements
//
// The compensated and plain float32 tracers read their store as pairs along x: element o
// holds record o and what the first interpolation level needs of record o + 1, so the 8
// corners of a cell are 4 loads.  Float32: (record, record[o+1] - record[o]) -- the
// difference is the float32 subtraction the interpolation would make, so one fma gives
// the x-interpolated value, bit-identical to lerp(record[o], record[o+1]).  32 bytes,
// read with one 256-bit load.  Bfloat16: the two raw records (16 bytes).
struct __align__(32) F4P {
    float4 v, d;
};
struct __align__(16) B4P {
    uint2 a, b;
};

__device__ __forceinline__ void load_pair(const F4P* s, uint32_t o, Cell2& v, Cell2& d) {
    float v0, v1, v2, v3, d0, d1, d2, d3;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v0), "=f"(v1), "=f"(v2), "=f"(v3), "=f"(d0), "=f"(d1), "=f"(d2), "=f"(d3)
        : "l"(s + o));
    v = Cell2{pack2(v0, v1), pack2(v2, v3)};
    d = Cell2{pack2(d0, d1), pack2(d2, d3)};
}

__device__ __forceinline__ Cell2 bf16_cell(uint2 u) {
    return Cell2{pack2(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u)),
                 pack2(__uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u))};
}

// x-interpolated corner pair at element o (t0 = the x fraction, packed) and the x
// difference record[o+1] - record[o].
__device__ __forceinline__ void xlerp(const F4P* s, uint32_t o, f32x2 t0, Cell2& lerped, Cell2& diff) {
    Cell2 v;
    load_pair(s, o, v, diff);
    lerped = Cell2{fma2(t0, diff.lo, v.lo), fma2(t0, diff.hi, v.hi)};
}
__device__ __forceinline__ void xlerp(const B4P* s, uint32_t o, f32x2 t0, Cell2& lerped, Cell2& diff) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(s + o));
    const Cell2 a = bf16_cell(make_uint2(u.x, u.y)), b = bf16_cell(make_uint2(u.z, u.w));
    diff = Cell2{sub2(b.lo, a.lo), sub2(b.hi, a.hi)};
    lerped = Cell2{fma2(t0, diff.lo, a.lo), fma2(t0, diff.hi, a.hi)};
}

// The record at element o (for reading nodes back).
__device__ __forceinline__ float4 pair_record(const F4P* s, uint32_t o) { return s[o].v; }

// Trilinear (deta, grad eta) in packed arithmetic from a paired store; bit-identical to
// `trilinear` on the records.
template <class E>
__device__ __forceinline__ float4 trilinear2(const E* s, uint32_t o, float f0, float f1, float f2) {
    const f32x2 t0 = pack2(f0, f0), t1 = pack2(f1, f1), t2 = pack2(f2, f2);
    Cell2 a0, a1, a2, a3, d;
    xlerp(s, o, t0, a0, d);
    xlerp(s, o + 9, t0, a1, d);
    xlerp(s, o + 81, t0, a2, d);
    xlerp(s, o + 90, t0, a3, d);
    Cell2 r = lerpc(lerpc(a0, a1, t1), lerpc(a2, a3, t1), t2);
    float4 v;
    unpack2(r.lo, v.x, v.y);
    unpack2(r.hi, v.z, v.w);
    return v;
}

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float t) {
    return make_float4(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y), fmaf(t, b.z - a.z, a.z),
                       fmaf(t, b.w - a.w, a.w));
}

// Trilinear (deta, grad eta) from the 4 pairs at base offset o, fractions f (scalar
// float32: fma(t, d, v) along x is lerp(record[o], record[o+1]) exactly).
__device__ __forceinline__ float4 xlerp4(const F4P* s, uint32_t o, float t) {
    const F4P p = s[o];
    return make_float4(fmaf(t, p.d.x, p.v.x), fmaf(t, p.d.y, p.v.y), fmaf(t, p.d.z, p.v.z), fmaf(t, p.d.w, p.v.w));
}

__device__ __forceinline__ float4 trilinear(const F4P* s, uint32_t o, float f0, float f1, float f2) {
    float4 a0 = xlerp4(s, o, f0), a1 = xlerp4(s, o + 9, f0);
    float4 a2 = xlerp4(s, o + 81, f0), a3 = xlerp4(s, o + 90, f0);
    float4 b0 = lerp4(a0, a1, f1), b1 = lerp4(a2, a3, f1);
    return lerp4(b0, b1, f2);
}

__device__ __forceinline__ D4 dlerp(D4 a, D4 b, double t) {
    D4 r;
    r.x = a.x + t * (b.x - a.x);
    r.y = a.y + t * (b.y - a.y);
    r.z = a.z + t * (b.z - a.z);
    r.w = a.w + t * (b.w - a.w);
    return r;
}

__device__ __forceinline__ D4 load_d4(const D4* s, uint32_t o) {
    const double2* p = reinterpret_cast<const double2*>(s + o);
    double2 a = __ldg(p), b = __ldg(p + 1);
    D4 r;
    r.x = a.x;
    r.y = a.y;
    r.z = b.x;
    r.w = b.y;
    return r;
}

__device__ __forceinline__ D4 trilinear_d(const D4* s, uint32_t o, double f0, double f1, double f2) {
    D4 a0 = dlerp(load_d4(s, o), load_d4(s, o + 1), f0);
    D4 a1 = dlerp(load_d4(s, o + 9), load_d4(s, o + 10), f0);
    D4 a2 = dlerp(load_d4(s, o + 81), load_d4(s, o + 82), f0);
    D4 a3 = dlerp(load_d4(s, o + 90), load_d4(s, o + 91), f0);
    return dlerp(dlerp(a0, a1, f1), dlerp(a2, a3, f1), f2);
}

// Cell coordinates of a point given in grid units u = (x - o)/h - 1/2 (any type):
// base i = clamp(floor(u), 0, n - 2), fraction f = u - i (linear extrapolation of the
// edge cells beyond the outer centres).
template <class T>
__device__ __forceinline__ void split_coord(T u, int n, int& i, T& f) {
    T fl = floor(u);
    fl = fl < T(0) ? T(0) : fl;
    fl = fl > T(n - 2) ? T(n - 2) : fl;
    i = (int)fl;
    f = u - fl;
}

// Field at an absolute position, in T arithmetic (the FP64 and plain-FP32 paths).
__device__ __forceinline__ void field_at(const GridDev& g, const double x[3], double& eta, double grad[3]) {
    int i[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double u = (x[a] - g.origin[a]) / g.h[a] - 0.5;
        split_coord(u, g.n[a], i[a], f[a]);
    }
    uint32_t o = bounded(brick_offset(i[0], i[1], i[2]) + 91u, g.store_elems, g.err);
    o = o ? o - 91u : 0u;
    D4 v = trilinear_d(static_cast<const D4*>(g.store), o, f[0], f[1], f[2]);
    eta = 1.0 + v.x;
    grad[0] = v.y;
    grad[1] = v.z;
    grad[2] = v.w;
}

// ------------------------------------------------------------------ sampling (Sec. 2.3)

__device__ __forceinline__ unsigned long long splitmix64_output(unsigned long long seed, unsigned long long k) {
    unsigned long long z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double tent_offset(double xi) {
    if (xi < 0.5) return dsub(dsqrt(dmul(2.0, xi)), 1.0);
    return dsub(1.0, dsqrt(dsub(2.0, dmul(2.0, xi))));
}

__device__ __forceinline__ void image_point(const CamDev& c, int px, int py, int s, double& x, double& y) {
    double t1 = 0.0, t2 = 0.0;
    if (c.spp > 1) {
        unsigned long long counter =
            ((unsigned long long)py * (unsigned long long)c.width + (unsigned long long)px) * (unsigned long long)c.spp +
            (unsigned long long)s;
        unsigned long long z = splitmix64_output(c.seed, counter + 1ULL);
        double xi1 = (double)(z >> 40) * (1.0 / 16777216.0);
        double xi2 = (double)((z >> 16) & 0xFFFFFFULL) * (1.0 / 16777216.0);
        t1 = tent_offset(xi1);
        t2 = tent_offset(xi2);
    }
    x = dadd(dadd((double)px, 0.5), t1);
    y = dadd(dadd((double)py, 0.5), t2);
}

__device__ __forceinline__ void pinhole_direction(const CamDev& c, const double right[3], double x, double y,
                                                  double d[3]) {
    double a = ddiv(dsub(x, c.cx), c.fx);
    double b = ddiv(dsub(y, c.cy), c.fy);
    for (int i = 0; i < 3; ++i) d[i] = dadd(dsub(dmul(a, right[i]), dmul(b, c.up[i])), c.fwd[i]);
    double n = dsqrt(ddot(d, d));
    for (int i = 0; i < 3; ++i) d[i] = ddiv(d[i], n);
}

struct Ray {
    double d[3];
    double tw;      // straight distance to the wall plane
    double t_in;    // box entry (>= 0)
    double ell;     // traced segment length
    int N;          // steps (0: straight to the wall)
    bool wall;      // reaches the wall plane
    signed char in_axis;    // slab axis that sets t_in (-1: t_in = 0)
    signed char out_axis;   // slab axis that sets the segment end (3: the wall plane)
};

// Slab test and step count of the straight ray rs + t d (unit d) whose direction is
// already in R.d: wall-plane distance, traced segment [t_in, min(t_out, t_w)] and N, bit-exact
// with a plain IEEE double evaluation of the same formulas.  lo_m / hi_m are the box faces
// minus rs and qn = (wall origin - rs) . normal.
__device__ __forceinline__ void ray_segment(const SceneDev& S, const double rs[3], const double lo_m[3],
                                            const double hi_m[3], double qn, Ray& R) {
    R.N = 0;
    R.t_in = 0.0;
    R.ell = 0.0;
    R.tw = 0.0;
    R.in_axis = -1;
    R.out_axis = 3;
    double den = ddot(R.d, S.w.normal);
    R.wall = den > 0.0;
    if (!R.wall) return;
    R.tw = ddiv(qn, den);
    double t_in = 0.0, t_out = __longlong_as_double(0x7ff0000000000000LL);
    int ia = -1, oa = -1;
    bool inside = true;
    for (int a = 0; a < 3; ++a) {
        if (R.d[a] == 0.0) {
            if (rs[a] < S.g.origin[a] || rs[a] > dadd(S.g.origin[a], S.g.extent[a])) inside = false;
            continue;
        }
        double t0 = ddiv(lo_m[a], R.d[a]);
        double t1 = ddiv(hi_m[a], R.d[a]);
        if (t0 > t1) {
            double t = t0;
            t0 = t1;
            t1 = t;
        }
        if (t0 > t_in) {
            t_in = t0;
            ia = a;
        }
        if (t1 < t_out) {
            t_out = t1;
            oa = a;
        }
    }
    double t_end = R.tw;
    int ea = 3;
    if (t_out < R.tw) {
        t_end = t_out;
        ea = oa;
    }
    if (!inside || !(t_in < t_end)) return;
    R.t_in = t_in;
    R.in_axis = (signed char)ia;
    R.out_axis = (signed char)ea;
    R.ell = dsub(t_end, t_in);
    if (S.it.fixed_steps > 0) {
        R.N = S.it.fixed_steps;
    } else {
        double nn = ceil(ddiv(R.ell, S.rc.step));
        R.N = nn > (double)S.it.max_steps ? -1 : (int)nn;   // -1: over the step budget
    }
}

// Straight-line set-up of a camera ray: wall plane, slab test, traced segment and N
// (bit-exact with a plain IEEE double evaluation of the same formulas).  SLAB = false: the
// direction and the wall plane only (a straight ray needs no segment or step count).
template <bool SLAB = true>
__device__ __forceinline__ Ray ray_setup(const SceneDev& S, int px, int py, int s) {
    Ray R;
    double x, y;
    image_point(S.cam, px, py, s, x, y);
    pinhole_direction(S.cam, S.rc.right, x, y, R.d);
    if constexpr (SLAB) {
        ray_segment(S, S.cam.pos, S.rc.lo_m, S.rc.hi_m, S.rc.qn, R);
    } else {
        R.N = 0;
        R.t_in = R.ell = 0.0;
        R.in_axis = -1;
        R.out_axis = 3;
        const double den = ddot(R.d, S.w.normal);
        R.wall = den > 0.0;
        R.tw = R.wall ? ddiv(S.rc.qn, den) : 0.0;
    }
    return R;
}

// The projector ray aimed at wall point base + e (base float64, e a small float offset):
// unit direction q / |q| from the projector pinhole, q = aim - P, and its segment.
__device__ __forceinline__ Ray projector_setup(const SceneDev& S, const double base[3], const float e[3]) {
    Ray R;
    const double* P = S.L.proj.pos;
    double q[3];
    for (int a = 0; a < 3; ++a) q[a] = dadd(dsub(base[a], P[a]), (double)e[a]);
    double nq = dsqrt(ddot(q, q));
    for (int a = 0; a < 3; ++a) R.d[a] = ddiv(q[a], nq);
    ray_segment(S, P, S.rc.plo_m, S.rc.phi_m, S.rc.pqn, R);
    return R;
}

// ------------------------------------------------------------------ wall (Sec. 2.3)

__device__ __forceinline__ double texel(const LightDev& L, int i, int j) {
    if (i < 0 || j < 0 || i >= L.tw || j >= L.th) return 0.0;
    return (double)__ldg(L.pattern + (size_t)j * L.tw + i);
}

__device__ __forceinline__ double bilinear(const LightDev& L, double s, double t, double* ds = nullptr,
                                           double* dt = nullptr) {
    s -= 0.5;
    t -= 0.5;
    double fi = floor(s), fj = floor(t);
    int i = (int)fmax(fmin(fi, 2.0e9), -2.0e9), j = (int)fmax(fmin(fj, 2.0e9), -2.0e9);
    double fs = s - fi, ft = t - fj;
    double p00 = texel(L, i, j), p10 = texel(L, i + 1, j), p01 = texel(L, i, j + 1), p11 = texel(L, i + 1, j + 1);
    if (ds) {
        *ds = (1.0 - ft) * (p10 - p00) + ft * (p11 - p01);
        *dt = (1.0 - fs) * (p01 - p00) + fs * (p11 - p10);
    }
    return (1.0 - fs) * ((1.0 - ft) * p00 + ft * p01) + fs * ((1.0 - ft) * p10 + ft * p11);
}

// Wall luminance at x (Eq. 2's L_wall) and, if g != nullptr, its gradient in x.
__device__ __forceinline__ double wall_luminance(const LightDev& L, const WallDev& w, const double x[3],
                                                 double* g = nullptr) {
    if (L.mode == 0) {
        double q[3] = {x[0] - w.origin[0], x[1] - w.origin[1], x[2] - w.origin[2]};
        double su = w.size_u / L.tw, sv = w.size_v / L.th;
        double wu = q[0] * w.eu[0] + q[1] * w.eu[1] + q[2] * w.eu[2];
        double wv = q[0] * w.ev[0] + q[1] * w.ev[1] + q[2] * w.ev[2];
        double ds, dt;
        double v = bilinear(L, wu / su, wv / sv, &ds, &dt);
        if (g)
            for (int a = 0; a < 3; ++a) g[a] = ds * w.eu[a] / su + dt * w.ev[a] / sv;
        return v;
    }
    const CamDev& P = L.proj;
    double right[3] = {P.fwd[1] * P.up[2] - P.fwd[2] * P.up[1], P.fwd[2] * P.up[0] - P.fwd[0] * P.up[2],
                       P.fwd[0] * P.up[1] - P.fwd[1] * P.up[0]};
    double q[3] = {x[0] - P.pos[0], x[1] - P.pos[1], x[2] - P.pos[2]};
    double z = q[0] * P.fwd[0] + q[1] * P.fwd[1] + q[2] * P.fwd[2];
    if (!(z > 0.0)) {
        if (g) g[0] = g[1] = g[2] = 0.0;
        return 0.0;
    }
    double xx = q[0] * right[0] + q[1] * right[1] + q[2] * right[2];
    double yy = q[0] * P.up[0] + q[1] * P.up[1] + q[2] * P.up[2];
    double ds, dt;
    double v = bilinear(L, P.cx + P.fx * xx / z, P.cy - P.fy * yy / z, &ds, &dt);
    if (g)
        for (int a = 0; a < 3; ++a) {
            double dpx = P.fx * (right[a] / z - xx * P.fwd[a] / (z * z));
            double dpy = -P.fy * (P.up[a] / z - yy * P.fwd[a] / (z * z));
            g[a] = ds * dpx + dt * dpy;
        }
    return v;
}

struct RayResult {
    double I;        // L cos / len
    double hit[2];   // wall coordinates
    double disp[2];  // hit minus straight hit
};

// From the end state (r_N, v_N) and the path length before r_N: straight to the wall,
// luminance, cosine over length.
__device__ __forceinline__ RayResult wall_epilogue(const SceneDev& S, const double rs[3], const Ray& R,
                                                   const double rN[3], const double vN[3], double len_before) {
    RayResult o;
    o.I = 0.0;
    o.hit[0] = o.hit[1] = o.disp[0] = o.disp[1] = 0.0;
    const WallDev& w = S.w;
    double vn = vN[0] * w.normal[0] + vN[1] * w.normal[1] + vN[2] * w.normal[2];
    if (!(vn > 0.0)) return o;
    double q[3] = {w.origin[0] - rN[0], w.origin[1] - rN[1], w.origin[2] - rN[2]};
    double ts = (q[0] * w.normal[0] + q[1] * w.normal[1] + q[2] * w.normal[2]) / vn;
    double xw[3], dx[3];
    for (int a = 0; a < 3; ++a) xw[a] = rN[a] + ts * vN[a];
    double vl = sqrt(vN[0] * vN[0] + vN[1] * vN[1] + vN[2] * vN[2]);
    double len = len_before + ts * vl;   // signed: t* < 0 when r_N lies behind the wall
    double cw = vn / vl;
    o.I = wall_luminance(S.L, w, xw) * cw / len;
    for (int a = 0; a < 3; ++a) {
        double xr = rs[a] + R.tw * R.d[a];
        dx[a] = xw[a] - xr;
        q[a] = xw[a] - w.origin[a];
    }
    o.hit[0] = q[0] * w.eu[0] + q[1] * w.eu[1] + q[2] * w.eu[2];
    o.hit[1] = q[0] * w.ev[0] + q[1] * w.ev[1] + q[2] * w.ev[2];
    o.disp[0] = dx[0] * w.eu[0] + dx[1] * w.eu[1] + dx[2] * w.eu[2];
    o.disp[1] = dx[0] * w.ev[0] + dx[1] * w.ev[1] + dx[2] * w.ev[2];
    return o;
}

// ------------------------------------------------------------------ warp tiles

// A warp renders a tile of 32 rays: G lanes per pixel (G = spp if spp is a power of
// two <= 32, else 1 lane per pixel that loops over the samples), TW x TH pixels.
struct TileShape {
    int G, TW, TH, tiles_x, tiles_y, samples_per_lane;
};

__host__ __device__ __forceinline__ TileShape tile_shape(int width, int height, int spp) {
    TileShape t;
    bool pow2 = spp >= 1 && spp <= 32 && (spp & (spp - 1)) == 0;
    t.G = pow2 ? spp : 1;
    t.samples_per_lane = pow2 ? 1 : spp;
    int P = 32 / t.G;
    t.TW = P >= 32 ? 8 : P >= 16 ? 4 : P >= 8 ? 4 : P >= 4 ? 2 : P >= 2 ? 2 : 1;
    t.TH = P / t.TW;
    t.tiles_x = (width + t.TW - 1) / t.TW;
    t.tiles_y = (height + t.TH - 1) / t.TH;
    return t;
}

// Pixel of a lane of warp tile t.  Whole image: TW x TH pixel tiles in row-major order,
// outputs indexed by pixel.  Pixel list: P = 32/G consecutive list entries per tile,
// outputs (and dL/dI seeds) indexed by list entry; out-of-range indices are skipped.
struct TilePix {
    int px, py;
    long long out;
    bool valid, bad;
};

__host__ __device__ __forceinline__ int tile_count(const SceneDev& S, const TileShape& ts) {
    if (S.pix) return (int)((S.npix + (32 / ts.G) - 1) / (32 / ts.G));
    return ts.tiles_x * ts.tiles_y;
}

__device__ __forceinline__ TilePix tile_pixel(const SceneDev& S, const TileShape& ts, int t, int lane) {
    TilePix r;
    const int lp = lane / ts.G;
    r.bad = false;
    if (S.pix) {
        const long long e = (long long)t * (32 / ts.G) + lp;
        const long long npx = (long long)S.cam.width * S.cam.height;
        long long p = e < S.npix ? (long long)__ldg(S.pix + e) : -1;
        r.bad = e < S.npix && (p < 0 || p >= npx);
        r.valid = e < S.npix && !r.bad;
        if (!r.valid) p = 0;
        r.px = (int)(p % S.cam.width);
        r.py = (int)(p / S.cam.width);
        r.out = e;
    } else {
        const int tx = t % ts.tiles_x, ty = t / ts.tiles_x;
        r.px = tx * ts.TW + lp % ts.TW;
        r.py = ty * ts.TH + lp / ts.TW;
        r.valid = r.px < S.cam.width && r.py < S.cam.height;
        r.out = (long long)r.py * S.cam.width + r.px;
    }
    return r;
}


}  // namespace bos
