// Plain FP64 CPU oracle of the BOS forward model and of its gradient.
//
// TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg of
// the benchmark load this library; the product (the CUDA library) never calls it and
// shares no code, header, table or helper with it.
//
// It is written for a reader to check against the paper by eye: textbook formulas,
// one ray at a time, no blocking, no fusion, no reordering.  Built with
// -ffp-contract=off and without fast-math, so every double operation is one IEEE
// round-to-nearest operation in the written order.
//
// What it computes (paper section / equation in brackets):
//   eta(T) = 1 + rho0 * G * T0 / T                              [Sec. 2.1]
//   grad eta on the cell centres by central differences, one-sided at the faces
//   trilinear eta and grad eta; D = eta * grad eta               [Eq. 1, right-hand side]
//   Sharma's Runge-Kutta-Nystrom step for dr/dt = v, dv/dt = D   [Sec. 2.2, Eq. 1]
//   classic RK4 on (r, v) as a cross-check integrator            [Eq. 1]
//   quasi-linear tracing: the index field sampled on the straight line r_in + t v0
//   drives the velocity equation, which drives the position equation  [Sec. 2.2]
//   pinhole camera, tent (triangular) pixel filter sampled by its inverse CDF,
//   Monte Carlo over the pixel, wall hit by straight extrapolation, textured or
//   pinhole-projector wall luminance, weight <n_w, v_w> / path length  [Sec. 2.3, Eq. 2]
//   refracted projector connection: the projector point that lights wall point x_w is the
//   one whose own ray, traced through the same field, lands on x_w; found by M rounds of
//   aiming a_{k+1} = a_k + (x_w - y(a_k)) from a_0 = x_w                    [Sec. 2.3]
//   L_BOS = sum_j (I_flow_j - I_j)^2 and its gradient with respect to T by a
//   discrete adjoint over a full tape of ray states              [Sec. 2.4]
//   complex-step directional derivatives (the same code run on std::complex<double>)
//
// Parity status: every function here is pinned by the CPU tests (closed forms,
// invariants, brute force, complex step); none is "parity unpinned".
//
// Sample jitter uses the splitmix64 generator (Steele, Lea and Flood, OOPSLA 2014):
// the k-th output for seed s is mix(s + k * 0x9E3779B97F4A7C15).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

typedef std::complex<double> cplx;

static inline double re(double x) { return x; }
static inline double re(const cplx& x) { return x.real(); }

extern "C" {

// The oracle's own plain-C descriptors (mirrored by oracle.py with ctypes).
typedef struct {
    int n[3];              // cells along x, y, z
    double origin[3];      // box corner (m)
    double extent[3];      // box size (m)
    double T0, rho0, G;    // ambient temperature (K), ambient density, Gladstone-Dale coefficient
} orc_grid;

typedef struct {
    double pos[3], fwd[3], up[3];   // pinhole, unit viewing direction, unit up direction
    double fx, fy, cx, cy;          // focal lengths and principal point in pixels
    int width, height, spp;         // image size, rays per pixel
    uint64_t seed;                  // jitter seed
} orc_camera;

typedef struct {
    double origin[3], eu[3], ev[3], normal[3];   // wall plane frame; normal points away from the camera
    double size_u, size_v;                       // extent along eu, ev (m)
} orc_wall;

typedef struct {
    int mode;              // 0: luminance is a texture on the wall, 1: pinhole projector with a
                           // straight projector-to-wall connection, 2: the projector's own rays
                           // traced through the field too (refracted connection)
    orc_camera proj;       // projector pinhole (modes 1, 2); width/height = pattern size
    int tw, th;            // texture / pattern size (texels)
    const float* pattern;  // th rows of tw values
    int connect_iters;     // mode 2: projector rays traced per wall point (M >= 1)
} orc_light;

typedef struct {
    int fixed_steps;       // > 0: steps per ray; 0: ceil(ell / (max_step_vox * min h))
    double max_step_vox;
    int integrator;        // 0: Sharma RKN, 1: classic RK4, 2: quasi-linear (RKN weights, stages on the line)
} orc_integ;

// Field description.  kind 0: trilinear on node arrays deta (eta - 1) and grad (3 per
// node), both FP64, node index (k*ny + j)*nx + i.  Analytic kinds (no grid):
//   1: eta^2 = p0 + p1 x + p2 y + p3 z
//   2: eta   = p0 + p1 x + p2 y + p3 z
//   3: eta   = 1 + p0 + p1 exp(-|x - (p2,p3,p4)|^2 / (2 p5^2))
typedef struct {
    int kind;
    const double* deta;
    const double* grad;
    double p[8];
} orc_field;

}  // extern "C"

namespace {

// ---------------------------------------------------------------- field [Sec. 2.1]

template <class S>
struct Field {
    const orc_grid* g;
    int kind;
    const S* deta;
    const S* grad;
    double p[8];
    double h[3];
};

inline size_t node_index(const orc_grid& g, long i, long j, long k) {
    return ((size_t)k * (size_t)g.n[1] + (size_t)j) * (size_t)g.n[0] + (size_t)i;
}

inline double spacing(const orc_grid& g, int a) { return g.extent[a] / (double)g.n[a]; }

// eta - 1 = rho0 * G * T0 / T  (ideal gas at constant pressure + Gladstone-Dale).
template <class S>
void deta_from_T(const orc_grid& g, const S* T, S* deta) {
    const double K = g.rho0 * g.G * g.T0;
    const size_t n = (size_t)g.n[0] * g.n[1] * g.n[2];
    for (size_t c = 0; c < n; ++c) deta[c] = K / T[c];
}

// grad eta at every cell centre: central difference inside, one-sided at the two faces.
template <class S>
void grad_from_deta(const orc_grid& g, const S* deta, S* grad) {
    const long nx = g.n[0], ny = g.n[1], nz = g.n[2];
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long idx[3] = {i, j, k};
                for (int a = 0; a < 3; ++a) {
                    long lo = idx[a] - 1, hi = idx[a] + 1;
                    double den = 2.0 * spacing(g, a);
                    if (lo < 0) { lo = idx[a]; den = spacing(g, a); }
                    if (hi > g.n[a] - 1) { hi = idx[a]; den = spacing(g, a); }
                    long ilo[3] = {i, j, k}, ihi[3] = {i, j, k};
                    ilo[a] = lo;
                    ihi[a] = hi;
                    S d = deta[node_index(g, ihi[0], ihi[1], ihi[2])] -
                          deta[node_index(g, ilo[0], ilo[1], ilo[2])];
                    grad[3 * node_index(g, i, j, k) + a] = d / den;
                }
            }
}

// Trilinear interpolation point: for each axis u = (x - o)/h - 1/2 (cell-centre units),
// base node i = clamp(floor(u), 0, n - 2), fraction f = u - i (so beyond the outer cell
// centres the edge cells are extrapolated linearly; the interpolant stays continuous).
template <class S>
void cell_coords(const orc_grid& g, const S x[3], long i0[3], S f[3]) {
    for (int a = 0; a < 3; ++a) {
        S u = (x[a] - g.origin[a]) / spacing(g, a) - 0.5;
        double fl = std::floor(re(u));
        if (fl < 0.0) fl = 0.0;
        if (fl > (double)(g.n[a] - 2)) fl = (double)(g.n[a] - 2);
        i0[a] = (long)fl;
        f[a] = u - fl;
    }
}

struct Corner {
    size_t node;
    double w;         // trilinear weight
    double dw[3];     // d w / d x_a
};

// eta and grad eta at x.
template <class S>
void field_eval(const Field<S>& F, const S x[3], S& eta, S grad[3]) {
    if (F.kind == 0) {
        const orc_grid& g = *F.g;
        long i0[3];
        S f[3];
        cell_coords(g, x, i0, f);
        S acc[4] = {S(0), S(0), S(0), S(0)};
        for (int c = 0; c < 8; ++c) {
            int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
            S w = (di ? f[0] : S(1.0) - f[0]) * (dj ? f[1] : S(1.0) - f[1]) *
                  (dk ? f[2] : S(1.0) - f[2]);
            size_t nd = node_index(g, i0[0] + di, i0[1] + dj, i0[2] + dk);
            acc[0] += w * F.deta[nd];
            for (int a = 0; a < 3; ++a) acc[1 + a] += w * F.grad[3 * nd + a];
        }
        eta = S(1.0) + acc[0];
        for (int a = 0; a < 3; ++a) grad[a] = acc[1 + a];
    } else if (F.kind == 1) {
        S e2 = F.p[0] + F.p[1] * x[0] + F.p[2] * x[1] + F.p[3] * x[2];
        eta = std::sqrt(e2);
        for (int a = 0; a < 3; ++a) grad[a] = F.p[1 + a] / (2.0 * eta);
    } else if (F.kind == 2) {
        eta = F.p[0] + F.p[1] * x[0] + F.p[2] * x[1] + F.p[3] * x[2];
        for (int a = 0; a < 3; ++a) grad[a] = S(F.p[1 + a]);
    } else {
        S d[3] = {x[0] - F.p[2], x[1] - F.p[3], x[2] - F.p[4]};
        S r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        S e = F.p[1] * std::exp(-r2 / (2.0 * F.p[5] * F.p[5]));
        eta = 1.0 + F.p[0] + e;
        for (int a = 0; a < 3; ++a) grad[a] = -d[a] / (F.p[5] * F.p[5]) * e;
    }
}

// Right-hand side of the velocity equation of Eq. 1: D = eta * grad eta.
template <class S>
void rhs(const Field<S>& F, const S x[3], S D[3]) {
    S eta, g[3];
    field_eval(F, x, eta, g);
    for (int a = 0; a < 3; ++a) D[a] = eta * g[a];
}

// ---------------------------------------------------------------- integrators [Eq. 1]

// One step of Sharma's Runge-Kutta-Nystrom scheme for r'' = D(r), with v = r':
//   A = dt D(r),  B = dt D(r + dt/2 v + dt/8 A),  C = dt D(r + dt v + dt/2 B)
//   r <- r + dt (v + (A + 2B)/6),  v <- v + (A + 4B + C)/6
template <class S>
void step_rkn(const Field<S>& F, S r[3], S v[3], S dt) {
    S A[3], B[3], C[3], p[3], D[3];
    rhs(F, r, D);
    for (int a = 0; a < 3; ++a) A[a] = dt * D[a];
    for (int a = 0; a < 3; ++a) p[a] = r[a] + (dt * 0.5) * v[a] + (dt * 0.125) * A[a];
    rhs(F, p, D);
    for (int a = 0; a < 3; ++a) B[a] = dt * D[a];
    for (int a = 0; a < 3; ++a) p[a] = r[a] + dt * v[a] + (dt * 0.5) * B[a];
    rhs(F, p, D);
    for (int a = 0; a < 3; ++a) C[a] = dt * D[a];
    for (int a = 0; a < 3; ++a) {
        r[a] = r[a] + dt * (v[a] + (A[a] + 2.0 * B[a]) / 6.0);
        v[a] = v[a] + (A[a] + 4.0 * B[a] + C[a]) / 6.0;
    }
}

// One classic fourth-order Runge-Kutta step on the first-order system (r, v).
template <class S>
void step_rk4(const Field<S>& F, S r[3], S v[3], S dt) {
    S k1r[3], k1v[3], k2r[3], k2v[3], k3r[3], k3v[3], k4r[3], k4v[3], p[3];
    for (int a = 0; a < 3; ++a) k1r[a] = v[a];
    rhs(F, r, k1v);
    for (int a = 0; a < 3; ++a) { k2r[a] = v[a] + (dt * 0.5) * k1v[a]; p[a] = r[a] + (dt * 0.5) * k1r[a]; }
    rhs(F, p, k2v);
    for (int a = 0; a < 3; ++a) { k3r[a] = v[a] + (dt * 0.5) * k2v[a]; p[a] = r[a] + (dt * 0.5) * k2r[a]; }
    rhs(F, p, k3v);
    for (int a = 0; a < 3; ++a) { k4r[a] = v[a] + dt * k3v[a]; p[a] = r[a] + dt * k3r[a]; }
    rhs(F, p, k4v);
    for (int a = 0; a < 3; ++a) {
        r[a] = r[a] + dt / 6.0 * (k1r[a] + 2.0 * k2r[a] + 2.0 * k3r[a] + k4r[a]);
        v[a] = v[a] + dt / 6.0 * (k1v[a] + 2.0 * k2v[a] + 2.0 * k3v[a] + k4v[a]);
    }
}

// One step of quasi-linear tracing (Sec. 2.2): the right-hand side of the velocity
// equation is taken on the straight line r_lin(t) = r_in + t v0 instead of on the ray, so
// the velocity no longer feeds back into where the field is sampled.  Step n covers
// [n dt, (n+1) dt]; the stages sit at the start, middle and end of it on the line, with
// Sharma's weights:
//   A = dt D(r_lin(n dt)), B = dt D(r_lin((n+1/2) dt)), C = dt D(r_lin((n+1) dt))
//   r <- r + dt (v + (A + 2B)/6),  v <- v + (A + 4B + C)/6
template <class S>
void step_quasi(const Field<S>& F, const S rin[3], const S v0[3], long n, S r[3], S v[3], S dt) {
    S A[3], B[3], C[3], p[3], D[3];
    for (int a = 0; a < 3; ++a) p[a] = rin[a] + ((double)n * dt) * v0[a];
    rhs(F, p, D);
    for (int a = 0; a < 3; ++a) A[a] = dt * D[a];
    for (int a = 0; a < 3; ++a) p[a] = rin[a] + (((double)n + 0.5) * dt) * v0[a];
    rhs(F, p, D);
    for (int a = 0; a < 3; ++a) B[a] = dt * D[a];
    for (int a = 0; a < 3; ++a) p[a] = rin[a] + (((double)n + 1.0) * dt) * v0[a];
    rhs(F, p, D);
    for (int a = 0; a < 3; ++a) C[a] = dt * D[a];
    for (int a = 0; a < 3; ++a) {
        r[a] = r[a] + dt * (v[a] + (A[a] + 2.0 * B[a]) / 6.0);
        v[a] = v[a] + (A[a] + 4.0 * B[a] + C[a]) / 6.0;
    }
}

template <class S>
S norm3(const S a[3]) { return std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

// ---------------------------------------------------------------- camera rays [Sec. 2.3]

inline uint64_t splitmix64_output(uint64_t seed, uint64_t k) {
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Inverse CDF of the triangular density on [-1, 1]: F(t) = (1+t)^2/2 for t < 0,
// 1 - (1-t)^2/2 for t >= 0.
inline double tent_inverse(double xi) {
    if (xi < 0.5) return std::sqrt(2.0 * xi) - 1.0;
    return 1.0 - std::sqrt(2.0 - 2.0 * xi);
}

// Image-plane point of sample s of pixel (px, py): pixel centre plus a tent-filter
// offset; with one sample per pixel the pixel centre.
void sample_point(const orc_camera& cam, long px, long py, int s, double& x, double& y) {
    double t1 = 0.0, t2 = 0.0;
    if (cam.spp > 1) {
        uint64_t counter = ((uint64_t)py * (uint64_t)cam.width + (uint64_t)px) * (uint64_t)cam.spp + (uint64_t)s;
        uint64_t z = splitmix64_output(cam.seed, counter + 1);
        double xi1 = (double)(z >> 40) * (1.0 / 16777216.0);
        double xi2 = (double)((z >> 16) & 0xFFFFFFULL) * (1.0 / 16777216.0);
        t1 = tent_inverse(xi1);
        t2 = tent_inverse(xi2);
    }
    x = ((double)px + 0.5) + t1;
    y = ((double)py + 0.5) + t2;
}

// Unit direction of the pinhole ray through image point (x, y); image y grows downward.
void pinhole_dir(const orc_camera& cam, double x, double y, double d[3]) {
    double right[3] = {cam.fwd[1] * cam.up[2] - cam.fwd[2] * cam.up[1],
                       cam.fwd[2] * cam.up[0] - cam.fwd[0] * cam.up[2],
                       cam.fwd[0] * cam.up[1] - cam.fwd[1] * cam.up[0]};
    double a = (x - cam.cx) / cam.fx;
    double b = (y - cam.cy) / cam.fy;
    for (int i = 0; i < 3; ++i) d[i] = a * right[i] - b * cam.up[i] + cam.fwd[i];
    double n = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; ++i) d[i] = d[i] / n;
}

struct RayGeom {
    double rs[3];    // pinhole (start of the ray)
    double d[3];     // unit direction
    bool wall;       // the straight ray reaches the wall plane (d . n > 0)
    double tw;       // straight distance to the wall plane
    bool traced;     // a segment inside the box lies before the wall
    double t_in;     // entry distance into the box (>= 0)
    double ell;      // length of the traced segment
    long N;          // integrator steps
};

// Straight-line set-up of one ray: slab test against the box, wall plane distance,
// traced segment [t_in, min(t_out, t_w)] and its step count.
RayGeom ray_geometry(const orc_grid& g, const orc_wall& w, const orc_integ& it,
                     const double rs[3], const double d[3]) {
    RayGeom R;
    for (int a = 0; a < 3; ++a) { R.rs[a] = rs[a]; R.d[a] = d[a]; }
    double den = d[0] * w.normal[0] + d[1] * w.normal[1] + d[2] * w.normal[2];
    R.wall = den > 0.0;
    R.tw = 0.0;
    R.traced = false;
    R.t_in = 0.0;
    R.ell = 0.0;
    R.N = 0;
    if (!R.wall) return R;
    double q[3] = {w.origin[0] - rs[0], w.origin[1] - rs[1], w.origin[2] - rs[2]};
    R.tw = (q[0] * w.normal[0] + q[1] * w.normal[1] + q[2] * w.normal[2]) / den;
    double t_in = 0.0, t_out = INFINITY;
    bool inside = true;
    for (int a = 0; a < 3; ++a) {
        double lo = g.origin[a], hi = g.origin[a] + g.extent[a];
        if (d[a] == 0.0) {
            if (rs[a] < lo || rs[a] > hi) inside = false;
            continue;
        }
        double t0 = (lo - rs[a]) / d[a];
        double t1 = (hi - rs[a]) / d[a];
        if (t0 > t1) std::swap(t0, t1);
        if (t0 > t_in) t_in = t0;
        if (t1 < t_out) t_out = t1;
    }
    double t_end = std::min(t_out, R.tw);
    if (!inside || !(t_in < t_end)) return R;
    R.traced = true;
    R.t_in = t_in;
    R.ell = t_end - t_in;
    if (it.fixed_steps > 0) {
        R.N = it.fixed_steps;
    } else {
        double hmin = std::min(spacing(g, 0), std::min(spacing(g, 1), spacing(g, 2)));
        double step = it.max_step_vox * hmin;
        R.N = (long)std::ceil(R.ell / step);
    }
    return R;
}

// ---------------------------------------------------------------- wall luminance [Sec. 2.3]

template <class S>
S texel(const orc_light& L, long i, long j) {
    if (i < 0 || j < 0 || i >= L.tw || j >= L.th) return S(0.0);
    return S((double)L.pattern[(size_t)j * L.tw + i]);
}

// Bilinear lookup with texel centres at integer + 1/2 and zero outside the pattern.
template <class S>
S bilinear(const orc_light& L, S s, S t) {
    s = s - 0.5;
    t = t - 0.5;
    double fi = std::floor(re(s)), fj = std::floor(re(t));
    long i = (long)fi, j = (long)fj;
    S fs = s - fi, ft = t - fj;
    return (S(1.0) - fs) * (S(1.0) - ft) * texel<S>(L, i, j) + fs * (S(1.0) - ft) * texel<S>(L, i + 1, j) +
           (S(1.0) - fs) * ft * texel<S>(L, i, j + 1) + fs * ft * texel<S>(L, i + 1, j + 1);
}

// Luminance arriving from wall point x: the wall texture there, or the projector
// pattern at the pinhole projection of x (the projector-to-wall connection is straight).
template <class S>
S luminance(const orc_light& L, const orc_wall& w, const S x[3]) {
    if (L.mode == 0) {
        S q[3] = {x[0] - w.origin[0], x[1] - w.origin[1], x[2] - w.origin[2]};
        S wu = q[0] * w.eu[0] + q[1] * w.eu[1] + q[2] * w.eu[2];
        S wv = q[0] * w.ev[0] + q[1] * w.ev[1] + q[2] * w.ev[2];
        return bilinear<S>(L, wu / (w.size_u / L.tw), wv / (w.size_v / L.th));
    }
    const orc_camera& P = L.proj;
    double right[3] = {P.fwd[1] * P.up[2] - P.fwd[2] * P.up[1], P.fwd[2] * P.up[0] - P.fwd[0] * P.up[2],
                       P.fwd[0] * P.up[1] - P.fwd[1] * P.up[0]};
    S q[3] = {x[0] - P.pos[0], x[1] - P.pos[1], x[2] - P.pos[2]};
    S z = q[0] * P.fwd[0] + q[1] * P.fwd[1] + q[2] * P.fwd[2];
    if (re(z) <= 0.0) return S(0.0);
    S xx = q[0] * right[0] + q[1] * right[1] + q[2] * right[2];
    S yy = q[0] * P.up[0] + q[1] * P.up[1] + q[2] * P.up[2];
    S px = P.cx + P.fx * xx / z;
    S py = P.cy - P.fy * yy / z;
    return bilinear<S>(L, px, py);
}

// ---------------------------------------------------------------- one ray [Eq. 1, Eq. 2]

template <class S>
struct RayOut {
    S I;            // L * <n_w, v_w>/|v_w| / len
    S hit[2];       // wall coordinates of the hit (m)
    S disp[2];      // hit minus the straight (reference) hit, in wall coordinates (m)
    long N;
    bool valid;
};

struct Scene {
    const orc_grid* g;
    const orc_camera* cam;
    const orc_wall* w;
    const orc_light* L;
    const orc_integ* it;
};

template <class S>
void wall_coords(const orc_wall& w, const S x[3], S out[2]) {
    S q[3] = {x[0] - w.origin[0], x[1] - w.origin[1], x[2] - w.origin[2]};
    out[0] = q[0] * w.eu[0] + q[1] * w.eu[1] + q[2] * w.eu[2];
    out[1] = q[0] * w.ev[0] + q[1] * w.ev[1] + q[2] * w.ev[2];
}

// ---------------------------------------------------------------- projector rays [Sec. 2.3]

// Geometry of the projector ray aimed at wall point `aim`: unit direction from the
// projector pinhole, the box segment [t_in, t_end] (t_end = min(box exit, wall plane)) and
// its step count.  The same slab test as a camera ray, written for real or complex
// arithmetic; branch decisions and N use the real parts.  in_axis / out_axis name the
// slab face that fixes t_in / t_end (-1: t_in = 0 inside the box; out_axis = 3: the wall).
template <class S>
struct ProjGeom {
    S q[3], nq, d[3];
    bool wall, traced;
    S tw, t_in, t_end, ell;
    int in_axis, out_axis;
    long N;
};

template <class S>
ProjGeom<S> projector_geometry(const Scene& sc, const S aim[3]) {
    const orc_grid& g = *sc.g;
    const orc_wall& w = *sc.w;
    const double* P = sc.L->proj.pos;
    ProjGeom<S> G;
    for (int a = 0; a < 3; ++a) G.q[a] = aim[a] - P[a];
    G.nq = norm3(G.q);
    for (int a = 0; a < 3; ++a) G.d[a] = G.q[a] / G.nq;
    S den = G.d[0] * w.normal[0] + G.d[1] * w.normal[1] + G.d[2] * w.normal[2];
    G.wall = re(den) > 0.0;
    G.traced = false;
    G.N = 0;
    G.in_axis = -1;
    G.out_axis = 3;
    G.tw = G.t_in = G.t_end = G.ell = S(0.0);
    if (!G.wall) return G;
    double qw[3] = {w.origin[0] - P[0], w.origin[1] - P[1], w.origin[2] - P[2]};
    G.tw = (qw[0] * w.normal[0] + qw[1] * w.normal[1] + qw[2] * w.normal[2]) / den;
    S t_in = S(0.0), t_out = S(INFINITY);
    int ia = -1, oa = -1;
    bool inside = true;
    for (int a = 0; a < 3; ++a) {
        double lo = g.origin[a], hi = g.origin[a] + g.extent[a];
        if (re(G.d[a]) == 0.0) {
            if (P[a] < lo || P[a] > hi) inside = false;
            continue;
        }
        S t0 = (lo - P[a]) / G.d[a], t1 = (hi - P[a]) / G.d[a];
        if (re(t0) > re(t1)) std::swap(t0, t1);
        if (re(t0) > re(t_in)) { t_in = t0; ia = a; }
        if (re(t1) < re(t_out)) { t_out = t1; oa = a; }
    }
    S t_end = G.tw;
    int ea = 3;
    if (re(t_out) < re(G.tw)) { t_end = t_out; ea = oa; }
    if (!inside || !(re(t_in) < re(t_end))) return G;
    G.traced = true;
    G.t_in = t_in;
    G.t_end = t_end;
    G.in_axis = ia;
    G.out_axis = ea;
    G.ell = t_end - t_in;
    if (sc.it->fixed_steps > 0) {
        G.N = sc.it->fixed_steps;
    } else {
        double hmin = std::min(spacing(g, 0), std::min(spacing(g, 1), spacing(g, 2)));
        G.N = (long)std::ceil(re(G.ell) / (sc.it->max_step_vox * hmin));
    }
    return G;
}

// Wall hit y of the projector ray aimed at `aim`: straight to the box, N integrator steps
// of Eq. 1 inside it (v0 = eta(r_in) d, dt = ell / (N eta(r_in)), as for camera rays), then
// straight from (r_N, v_N) to the wall plane.  Without a box segment y is the straight hit.
// Returns the steps taken.
template <class S>
long trace_projector(const Scene& sc, const Field<S>& F, const S aim[3], S y[3]) {
    const orc_wall& w = *sc.w;
    const double* P = sc.L->proj.pos;
    ProjGeom<S> G = projector_geometry(sc, aim);
    if (!G.wall) {
        for (int a = 0; a < 3; ++a) y[a] = aim[a];
        return 0;
    }
    if (!G.traced) {
        for (int a = 0; a < 3; ++a) y[a] = P[a] + G.tw * G.d[a];
        return 0;
    }
    S rin[3], r[3], v[3], eta_in, gd[3];
    for (int a = 0; a < 3; ++a) rin[a] = P[a] + G.t_in * G.d[a];
    field_eval(F, rin, eta_in, gd);
    for (int a = 0; a < 3; ++a) { r[a] = rin[a]; v[a] = eta_in * G.d[a]; }
    S dt = G.ell / ((double)G.N * eta_in);
    const S v0[3] = {v[0], v[1], v[2]};
    for (long n = 0; n < G.N; ++n) {
        if (sc.it->integrator == 1) step_rk4(F, r, v, dt);
        else if (sc.it->integrator == 2) step_quasi(F, rin, v0, n, r, v, dt);
        else step_rkn(F, r, v, dt);
    }
    S vn = v[0] * w.normal[0] + v[1] * w.normal[1] + v[2] * w.normal[2];
    S qq[3] = {w.origin[0] - r[0], w.origin[1] - r[1], w.origin[2] - r[2]};
    S ts = (qq[0] * w.normal[0] + qq[1] * w.normal[1] + qq[2] * w.normal[2]) / vn;
    for (int a = 0; a < 3; ++a) y[a] = r[a] + ts * v[a];
    return G.N;
}

// The wall point whose projector pattern value lights x_w: M rounds of
// a_{k+1} = a_k + (x_w - y(a_k)) from a_0 = x_w (mode 2; modes 0, 1 return x_w).
// Returns the projector-ray steps taken.
template <class S>
long connect_projector(const Scene& sc, const Field<S>& F, const S xw[3], S a[3]) {
    for (int c = 0; c < 3; ++c) a[c] = xw[c];
    if (sc.L->mode != 2) return 0;
    long steps = 0;
    for (int k = 0; k < sc.L->connect_iters; ++k) {
        S y[3];
        steps += trace_projector(sc, F, a, y);
        for (int c = 0; c < 3; ++c) a[c] = a[c] + (xw[c] - y[c]);
    }
    return steps;
}

// Trace one ray: straight to the box, N integrator steps of Eq. 1 inside it with
// v0 = eta(r_in) d and dt = ell / (N eta(r_in)) (so |v| = eta, dt = ds / eta), then straight
// from (r_N, v_N) to the wall.  `straight` forces the reference (no-flow) ray.
template <class S>
RayOut<S> trace_ray(const Scene& sc, const Field<S>& F, const RayGeom& R, bool straight) {
    RayOut<S> o;
    o.I = S(0.0);
    o.hit[0] = o.hit[1] = o.disp[0] = o.disp[1] = S(0.0);
    o.N = 0;
    o.valid = R.wall;
    if (!R.wall) return o;
    const orc_wall& w = *sc.w;
    double xref[3];
    for (int a = 0; a < 3; ++a) xref[a] = R.rs[a] + R.tw * R.d[a];
    S xw[3], vN[3], len;
    if (straight || !R.traced) {
        for (int a = 0; a < 3; ++a) { xw[a] = S(xref[a]); vN[a] = S(R.d[a]); }
        len = S(R.tw);
    } else {
        S rin[3];
        for (int a = 0; a < 3; ++a) rin[a] = S(R.rs[a] + R.t_in * R.d[a]);
        S eta_in, gdummy[3];
        field_eval(F, rin, eta_in, gdummy);
        S r[3], v[3];
        for (int a = 0; a < 3; ++a) { r[a] = rin[a]; v[a] = eta_in * R.d[a]; }
        S dt = R.ell / ((double)R.N * eta_in);
        S lensum = S(0.0);
        const S v0[3] = {v[0], v[1], v[2]};
        for (long n = 0; n < R.N; ++n) {
            S r0[3] = {r[0], r[1], r[2]};
            if (sc.it->integrator == 1) step_rk4(F, r, v, dt);
            else if (sc.it->integrator == 2) step_quasi(F, rin, v0, n, r, v, dt);
            else step_rkn(F, r, v, dt);
            S dr[3] = {r[0] - r0[0], r[1] - r0[1], r[2] - r0[2]};
            lensum += norm3(dr);
        }
        S vn = v[0] * w.normal[0] + v[1] * w.normal[1] + v[2] * w.normal[2];
        if (!(re(vn) > 0.0)) { o.valid = false; return o; }
        S q[3] = {w.origin[0] - r[0], w.origin[1] - r[1], w.origin[2] - r[2]};
        S tstar = (q[0] * w.normal[0] + q[1] * w.normal[1] + q[2] * w.normal[2]) / vn;
        for (int a = 0; a < 3; ++a) { xw[a] = r[a] + tstar * v[a]; vN[a] = v[a]; }
        // path length to the wall: entry distance, traced polyline, and the straight
        // continuation from r_N, signed (t* < 0 when the traced segment ends behind the wall)
        S seg_in[3] = {rin[0] - R.rs[0], rin[1] - R.rs[1], rin[2] - R.rs[2]};
        len = norm3(seg_in) + lensum + tstar * norm3(v);
        o.N = R.N;
    }
    S cosw = (vN[0] * w.normal[0] + vN[1] * w.normal[1] + vN[2] * w.normal[2]) / norm3(vN);
    S xl[3];   // where the luminance is read: x_w, or its refracted projector connection
    if (straight) {
        for (int a = 0; a < 3; ++a) xl[a] = xw[a];
    } else {
        o.N += connect_projector(sc, F, xw, xl);   // steps count the projector rays too
    }
    o.I = luminance<S>(*sc.L, w, xl) * cosw / len;
    wall_coords(w, xw, o.hit);
    S dx[3] = {xw[0] - xref[0], xw[1] - xref[1], xw[2] - xref[2]};
    o.disp[0] = dx[0] * w.eu[0] + dx[1] * w.eu[1] + dx[2] * w.eu[2];
    o.disp[1] = dx[0] * w.ev[0] + dx[1] * w.ev[1] + dx[2] * w.ev[2];
    return o;
}

RayGeom pixel_ray(const Scene& sc, long pix, int s) {
    const orc_camera& cam = *sc.cam;
    long px = pix % cam.width, py = pix / cam.width;
    double x, y, d[3];
    sample_point(cam, px, py, s, x, y);
    pinhole_dir(cam, x, y, d);
    return ray_geometry(*sc.g, *sc.w, *sc.it, cam.pos, d);
}

template <class Fn>
void parallel_for(long n, int threads, Fn fn) {
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    if (threads > n) threads = (int)std::max(1L, n);
    std::atomic<long> next(0);
    auto work = [&]() {
        const long chunk = 16;
        for (;;) {
            long b = next.fetch_add(chunk);
            if (b >= n) break;
            long e = std::min(n, b + chunk);
            for (long i = b; i < e; ++i) fn(i);
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(work);
    work();
    for (auto& th : pool) th.join();
}

Field<double> make_field(const orc_grid* g, const orc_field* f) {
    Field<double> F;
    F.g = g;
    F.kind = f->kind;
    F.deta = f->deta;
    F.grad = f->grad;
    for (int i = 0; i < 8; ++i) F.p[i] = f->p[i];
    for (int a = 0; a < 3; ++a) F.h[a] = spacing(*g, a);
    return F;
}

// ---------------------------------------------------------------- adjoint [Sec. 2.4]

// Corners and weights of the trilinear interpolant at x, with the weight derivatives.
void corners_at(const orc_grid& g, const double x[3], Corner C[8]) {
    long i0[3];
    double f[3];
    cell_coords(g, x, i0, f);
    for (int c = 0; c < 8; ++c) {
        int dd[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        double fac[3], dfac[3];
        for (int a = 0; a < 3; ++a) {
            fac[a] = dd[a] ? f[a] : 1.0 - f[a];
            dfac[a] = (dd[a] ? 1.0 : -1.0) / spacing(g, a);
        }
        C[c].node = node_index(g, i0[0] + dd[0], i0[1] + dd[1], i0[2] + dd[2]);
        C[c].w = fac[0] * fac[1] * fac[2];
        C[c].dw[0] = dfac[0] * fac[1] * fac[2];
        C[c].dw[1] = fac[0] * dfac[1] * fac[2];
        C[c].dw[2] = fac[0] * fac[1] * dfac[2];
    }
}

struct NodeAdj {
    double* deta;   // dL/d(deta) per node
    double* grad;   // dL/d(grad) per node, 3 per node
};

// D = (1 + deta(x)) grad(x) at x; given Dbar, return xbar = (dD/dx)^T Dbar and add the
// node adjoints: deta_c += w_c (Dbar . grad(x)),  grad_c += w_c (1 + deta(x)) Dbar.
void rhs_adjoint(const Field<double>& F, const double x[3], const double Dbar[3], double xbar[3], NodeAdj& acc) {
    Corner C[8];
    corners_at(*F.g, x, C);
    double de = 0.0, g[3] = {0, 0, 0}, dde[3] = {0, 0, 0}, dg[3][3] = {{0}};
    for (int c = 0; c < 8; ++c) {
        double vde = F.deta[C[c].node];
        de += C[c].w * vde;
        for (int k = 0; k < 3; ++k) dde[k] += C[c].dw[k] * vde;
        for (int a = 0; a < 3; ++a) {
            double vg = F.grad[3 * C[c].node + a];
            g[a] += C[c].w * vg;
            for (int k = 0; k < 3; ++k) dg[a][k] += C[c].dw[k] * vg;
        }
    }
    double eta = 1.0 + de;
    double Dg = Dbar[0] * g[0] + Dbar[1] * g[1] + Dbar[2] * g[2];
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += Dbar[a] * dg[a][k];
        xbar[k] = dde[k] * Dg + eta * s;
    }
    for (int c = 0; c < 8; ++c) {
        acc.deta[C[c].node] += C[c].w * Dg;
        for (int a = 0; a < 3; ++a) acc.grad[3 * C[c].node + a] += C[c].w * eta * Dbar[a];
    }
}

// Gradient of the bilinear lookup with respect to its pixel coordinates (s, t).
void bilinear_grad(const orc_light& L, double s, double t, double& ds, double& dt) {
    s -= 0.5;
    t -= 0.5;
    double fi = std::floor(s), fj = std::floor(t);
    long i = (long)fi, j = (long)fj;
    double fs = s - fi, ft = t - fj;
    double p00 = texel<double>(L, i, j), p10 = texel<double>(L, i + 1, j);
    double p01 = texel<double>(L, i, j + 1), p11 = texel<double>(L, i + 1, j + 1);
    ds = (1.0 - ft) * (p10 - p00) + ft * (p11 - p01);
    dt = (1.0 - fs) * (p01 - p00) + fs * (p11 - p10);
}

// d luminance / d x at wall point x.
void luminance_grad(const orc_light& L, const orc_wall& w, const double x[3], double gx[3]) {
    if (L.mode == 0) {
        double q[3] = {x[0] - w.origin[0], x[1] - w.origin[1], x[2] - w.origin[2]};
        double su = w.size_u / L.tw, sv = w.size_v / L.th;
        double wu = q[0] * w.eu[0] + q[1] * w.eu[1] + q[2] * w.eu[2];
        double wv = q[0] * w.ev[0] + q[1] * w.ev[1] + q[2] * w.ev[2];
        double ds, dt;
        bilinear_grad(L, wu / su, wv / sv, ds, dt);
        for (int a = 0; a < 3; ++a) gx[a] = ds * w.eu[a] / su + dt * w.ev[a] / sv;
        return;
    }
    const orc_camera& P = L.proj;
    double right[3] = {P.fwd[1] * P.up[2] - P.fwd[2] * P.up[1], P.fwd[2] * P.up[0] - P.fwd[0] * P.up[2],
                       P.fwd[0] * P.up[1] - P.fwd[1] * P.up[0]};
    double q[3] = {x[0] - P.pos[0], x[1] - P.pos[1], x[2] - P.pos[2]};
    double z = q[0] * P.fwd[0] + q[1] * P.fwd[1] + q[2] * P.fwd[2];
    if (z <= 0.0) { gx[0] = gx[1] = gx[2] = 0.0; return; }
    double xx = q[0] * right[0] + q[1] * right[1] + q[2] * right[2];
    double yy = q[0] * P.up[0] + q[1] * P.up[1] + q[2] * P.up[2];
    double ds, dt;
    bilinear_grad(L, P.cx + P.fx * xx / z, P.cy - P.fy * yy / z, ds, dt);
    for (int a = 0; a < 3; ++a) {
        double dpx = P.fx * (right[a] / z - xx * P.fwd[a] / (z * z));
        double dpy = -P.fy * (P.up[a] / z - yy * P.fwd[a] / (z * z));
        gx[a] = ds * dpx + dt * dpy;
    }
}

// Reverse one Sharma step (r_n, v_n) -> (r_{n+1}, v_{n+1}).  On entry rb, vb hold the
// adjoints of r_{n+1}, v_{n+1}; on exit those of r_n, v_n.  dtb accumulates dL/d dt.
void step_rkn_adjoint(const Field<double>& F, const double r[3], const double v[3], double dt,
                      double rb[3], double vb[3], double& dtb, NodeAdj& acc) {
    double A[3], B[3], p1[3], p2[3], p3[3], D1[3], D2[3], D3[3];
    for (int a = 0; a < 3; ++a) p1[a] = r[a];
    rhs(F, p1, D1);
    for (int a = 0; a < 3; ++a) A[a] = dt * D1[a];
    for (int a = 0; a < 3; ++a) p2[a] = r[a] + (dt * 0.5) * v[a] + (dt * 0.125) * A[a];
    rhs(F, p2, D2);
    for (int a = 0; a < 3; ++a) B[a] = dt * D2[a];
    for (int a = 0; a < 3; ++a) p3[a] = r[a] + dt * v[a] + (dt * 0.5) * B[a];
    rhs(F, p3, D3);

    double Ab[3], Bb[3], Cb[3], rn[3], vn[3];
    for (int a = 0; a < 3; ++a) {
        // r' = r + dt (v + (A + 2B)/6),  v' = v + (A + 4B + C)/6
        Ab[a] = dt / 6.0 * rb[a] + vb[a] / 6.0;
        Bb[a] = dt / 3.0 * rb[a] + 4.0 * vb[a] / 6.0;
        Cb[a] = vb[a] / 6.0;
        rn[a] = rb[a];
        vn[a] = vb[a] + dt * rb[a];
        dtb += rb[a] * (v[a] + (A[a] + 2.0 * B[a]) / 6.0);
    }
    double Db[3], pb[3];
    // C = dt D(p3)
    for (int a = 0; a < 3; ++a) { dtb += Cb[a] * D3[a]; Db[a] = dt * Cb[a]; }
    rhs_adjoint(F, p3, Db, pb, acc);
    // p3 = r + dt v + dt/2 B
    for (int a = 0; a < 3; ++a) {
        rn[a] += pb[a];
        vn[a] += dt * pb[a];
        Bb[a] += dt * 0.5 * pb[a];
        dtb += pb[a] * (v[a] + 0.5 * B[a]);
    }
    // B = dt D(p2)
    for (int a = 0; a < 3; ++a) { dtb += Bb[a] * D2[a]; Db[a] = dt * Bb[a]; }
    rhs_adjoint(F, p2, Db, pb, acc);
    // p2 = r + dt/2 v + dt/8 A
    for (int a = 0; a < 3; ++a) {
        rn[a] += pb[a];
        vn[a] += dt * 0.5 * pb[a];
        Ab[a] += dt * 0.125 * pb[a];
        dtb += pb[a] * (0.5 * v[a] + 0.125 * A[a]);
    }
    // A = dt D(p1), p1 = r
    for (int a = 0; a < 3; ++a) { dtb += Ab[a] * D1[a]; Db[a] = dt * Ab[a]; }
    rhs_adjoint(F, p1, Db, pb, acc);
    for (int a = 0; a < 3; ++a) {
        rn[a] += pb[a];
        rb[a] = rn[a];
        vb[a] = vn[a];
    }
}

// Reverse one quasi-linear step.  The stage points lie on the straight line
// r_in + t v0 with t v0 = (n + c) ell/N d, which does not depend on the field, so no
// position adjoint flows back through the field samples (their dt and v0 dependences
// cancel exactly, and both are left out).
void step_quasi_adjoint(const Field<double>& F, const double rin[3], const double v0[3], long n, const double v[3],
                        double dt, double rb[3], double vb[3], double& dtb, NodeAdj& acc) {
    double p1[3], p2[3], p3[3], D1[3], D2[3], D3[3], A[3], B[3];
    for (int a = 0; a < 3; ++a) {
        p1[a] = rin[a] + ((double)n * dt) * v0[a];
        p2[a] = rin[a] + (((double)n + 0.5) * dt) * v0[a];
        p3[a] = rin[a] + (((double)n + 1.0) * dt) * v0[a];
    }
    rhs(F, p1, D1);
    rhs(F, p2, D2);
    rhs(F, p3, D3);
    for (int a = 0; a < 3; ++a) {
        A[a] = dt * D1[a];
        B[a] = dt * D2[a];
    }
    double Ab[3], Bb[3], Cb[3], Db[3], pb[3];
    for (int a = 0; a < 3; ++a) {
        Ab[a] = dt / 6.0 * rb[a] + vb[a] / 6.0;
        Bb[a] = dt / 3.0 * rb[a] + 4.0 * vb[a] / 6.0;
        Cb[a] = vb[a] / 6.0;
        dtb += rb[a] * (v[a] + (A[a] + 2.0 * B[a]) / 6.0);
    }
    for (int a = 0; a < 3; ++a) { dtb += Cb[a] * D3[a]; Db[a] = dt * Cb[a]; }
    rhs_adjoint(F, p3, Db, pb, acc);
    for (int a = 0; a < 3; ++a) { dtb += Bb[a] * D2[a]; Db[a] = dt * Bb[a]; }
    rhs_adjoint(F, p2, Db, pb, acc);
    for (int a = 0; a < 3; ++a) { dtb += Ab[a] * D1[a]; Db[a] = dt * Ab[a]; }
    rhs_adjoint(F, p1, Db, pb, acc);
    for (int a = 0; a < 3; ++a) vb[a] = vb[a] + dt * rb[a];
}

inline double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Adjoint of y = trace_projector(aim) (Sharma RKN, full tape): for the seed yb = dL/dy,
// adds the node adjoints of the projector ray's samples and returns ab = dL/d aim, which
// flows through the ray's direction d = q / |q| (q = aim - P), its box segment (t_in and
// t_end on the slab faces or the wall plane) and its entry state v0 = eta(r_in) d,
// dt = ell / (N eta(r_in)).  N is an integer and has no derivative.
void projector_adjoint(const Scene& sc, const Field<double>& F, const double aim[3], const double yb[3],
                       NodeAdj& acc, double ab[3]) {
    const orc_wall& w = *sc.w;
    const double* P = sc.L->proj.pos;
    ProjGeom<double> G = projector_geometry(sc, aim);
    if (!G.wall) {   // y = aim
        for (int a = 0; a < 3; ++a) ab[a] = yb[a];
        return;
    }
    const double den = dot3(G.d, w.normal);
    double db[3] = {0, 0, 0};
    if (!G.traced) {
        // y = P + t_w d,  t_w = ((o - P) . n) / (d . n)
        double twb = dot3(yb, G.d);
        for (int a = 0; a < 3; ++a) db[a] = G.tw * yb[a] - twb * G.tw * w.normal[a] / den;
    } else {
        const long N = G.N;
        double rin[3], eta_in, gdum[3];
        for (int a = 0; a < 3; ++a) rin[a] = P[a] + G.t_in * G.d[a];
        field_eval(F, rin, eta_in, gdum);
        const double dt = G.ell / ((double)N * eta_in);
        std::vector<double> tape((size_t)(N + 1) * 6);
        double r[3], v[3];
        for (int a = 0; a < 3; ++a) { r[a] = rin[a]; v[a] = eta_in * G.d[a]; }
        for (int a = 0; a < 3; ++a) { tape[a] = r[a]; tape[3 + a] = v[a]; }
        for (long n = 0; n < N; ++n) {
            step_rkn(F, r, v, dt);
            for (int a = 0; a < 3; ++a) { tape[6 * (n + 1) + a] = r[a]; tape[6 * (n + 1) + 3 + a] = v[a]; }
        }
        // y = r_N + t* v_N,  t* = ((o - r_N) . n) / (v_N . n)
        const double vn = dot3(v, w.normal);
        double qq[3] = {w.origin[0] - r[0], w.origin[1] - r[1], w.origin[2] - r[2]};
        const double ts = dot3(qq, w.normal) / vn;
        double rb[3], vb[3], dtb = 0.0;
        const double tb = dot3(yb, v);
        for (int a = 0; a < 3; ++a) {
            rb[a] = yb[a] - tb * w.normal[a] / vn;
            vb[a] = ts * yb[a] - tb * ts * w.normal[a] / vn;
        }
        for (long n = N - 1; n >= 0; --n) step_rkn_adjoint(F, &tape[6 * n], &tape[6 * n + 3], dt, rb, vb, dtb, acc);
        // eta_in = 1 + deta(r_in): node adjoints, and its slope moves r_in's adjoint
        const double etab = dot3(vb, G.d) - dtb * dt / eta_in;
        Corner C[8];
        corners_at(*F.g, rin, C);
        for (int c = 0; c < 8; ++c) {
            acc.deta[C[c].node] += C[c].w * etab;
            for (int k = 0; k < 3; ++k) rb[k] += etab * C[c].dw[k] * F.deta[C[c].node];
        }
        // r_in = P + t_in d,  v0 = eta_in d,  ell = t_end - t_in
        for (int a = 0; a < 3; ++a) db[a] = eta_in * vb[a] + G.t_in * rb[a];
        const double ellb = dtb / ((double)N * eta_in);
        const double tinb = dot3(rb, G.d) - ellb, tendb = ellb;
        if (G.in_axis >= 0) db[G.in_axis] += tinb * (-G.t_in / G.d[G.in_axis]);   // t_in = (face - P) / d
        if (G.out_axis == 3) {
            for (int a = 0; a < 3; ++a) db[a] += tendb * (-G.tw * w.normal[a] / den);   // t_end = t_w
        } else {
            db[G.out_axis] += tendb * (-G.t_end / G.d[G.out_axis]);
        }
    }
    // d = q / |q|
    const double dd = dot3(db, G.d);
    for (int a = 0; a < 3; ++a) ab[a] = (db[a] - dd * G.d[a]) / G.nq;
}

// Adjoint of the luminance read at the projector connection of x_w (Lb = dL/dL_wall):
// reverses a_{k+1} = a_k + (x_w - y(a_k)), a_0 = x_w, and returns dL/dx_w (modes 0 and 1:
// Lb times the luminance gradient at x_w).
void connection_adjoint(const Scene& sc, const Field<double>& F, const double xw[3], double Lb, NodeAdj& acc,
                        double xwb[3]) {
    const int M = sc.L->mode == 2 ? sc.L->connect_iters : 0;
    std::vector<double> a((size_t)(M + 1) * 3);
    for (int c = 0; c < 3; ++c) a[c] = xw[c];
    for (int k = 0; k < M; ++k) {
        double y[3];
        trace_projector(sc, F, &a[3 * k], y);
        for (int c = 0; c < 3; ++c) a[3 * (k + 1) + c] = a[3 * k + c] + (xw[c] - y[c]);
    }
    double gL[3], abar[3];
    luminance_grad(*sc.L, *sc.w, &a[3 * M], gL);
    for (int c = 0; c < 3; ++c) {
        abar[c] = Lb * gL[c];
        xwb[c] = 0.0;
    }
    for (int k = M - 1; k >= 0; --k) {
        double yb[3], ak[3];
        for (int c = 0; c < 3; ++c) {
            xwb[c] += abar[c];
            yb[c] = -abar[c];
        }
        projector_adjoint(sc, F, &a[3 * k], yb, acc, ak);
        for (int c = 0; c < 3; ++c) abar[c] += ak[c];
    }
    for (int c = 0; c < 3; ++c) xwb[c] += abar[c];
}

// Adjoint of one traced ray with seed Ib = dL/dI_ray, accumulating node adjoints.
void ray_adjoint(const Scene& sc, const Field<double>& F, const RayGeom& R, double Ib, NodeAdj& acc,
                 std::vector<double>& tape) {
    if (!R.wall || Ib == 0.0) return;
    const orc_wall& w = *sc.w;
    if (!R.traced) {
        // the straight camera ray does not depend on the field; a refracted projector
        // connection of its wall point still does
        if (sc.L->mode == 2) {
            double xw[3], xwb[3];
            for (int a = 0; a < 3; ++a) xw[a] = R.rs[a] + R.tw * R.d[a];
            double cosw = dot3(R.d, w.normal);
            connection_adjoint(sc, F, xw, Ib * cosw / R.tw, acc, xwb);
        }
        return;
    }
    const long N = R.N;
    double rin[3];
    for (int a = 0; a < 3; ++a) rin[a] = R.rs[a] + R.t_in * R.d[a];
    double eta_in, gd[3];
    field_eval(F, rin, eta_in, gd);
    double dt = R.ell / ((double)N * eta_in);
    tape.resize((size_t)(N + 1) * 6);
    double r[3], v[3];
    for (int a = 0; a < 3; ++a) { r[a] = rin[a]; v[a] = eta_in * R.d[a]; }
    for (int a = 0; a < 3; ++a) { tape[a] = r[a]; tape[3 + a] = v[a]; }
    double lensum = 0.0;
    const double v0[3] = {v[0], v[1], v[2]};
    for (long n = 0; n < N; ++n) {
        double r0[3] = {r[0], r[1], r[2]};
        if (sc.it->integrator == 2) step_quasi(F, rin, v0, n, r, v, dt);
        else step_rkn(F, r, v, dt);
        double dr[3] = {r[0] - r0[0], r[1] - r0[1], r[2] - r0[2]};
        lensum += norm3(dr);
        for (int a = 0; a < 3; ++a) { tape[6 * (n + 1) + a] = r[a]; tape[6 * (n + 1) + 3 + a] = v[a]; }
    }
    double vn = v[0] * w.normal[0] + v[1] * w.normal[1] + v[2] * w.normal[2];
    if (!(vn > 0.0)) return;
    double q[3] = {w.origin[0] - r[0], w.origin[1] - r[1], w.origin[2] - r[2]};
    double tstar = (q[0] * w.normal[0] + q[1] * w.normal[1] + q[2] * w.normal[2]) / vn;
    double xw[3];
    for (int a = 0; a < 3; ++a) xw[a] = r[a] + tstar * v[a];
    double si[3] = {rin[0] - R.rs[0], rin[1] - R.rs[1], rin[2] - R.rs[2]};
    double vlen = norm3(v);
    double len = norm3(si) + lensum + tstar * vlen;   // signed continuation, as in trace_ray
    double cosw = vn / vlen;
    double xl[3];
    connect_projector(sc, F, xw, xl);
    double Lw = luminance<double>(*sc.L, w, xl);

    // I = Lw * cosw / len
    double Lb = Ib * cosw / len, cb = Ib * Lw / len, lenb = -Ib * Lw * cosw / (len * len);
    double gL[3];   // dL/dx_w through the luminance (and the projector connection)
    connection_adjoint(sc, F, xw, Lb, acc, gL);
    // x_w - r_N = t* v, so the length of the continuation t* |v| has the adjoint
    // lenb v / |v| on x_w and its negative on r_N (t* passed through x_w below).
    double xwb[3], rb[3], vb[3];
    for (int a = 0; a < 3; ++a) {
        double uo = v[a] / vlen;
        xwb[a] = gL[a] + lenb * uo;   // luminance and t* |v|
        rb[a] = -lenb * uo;
        vb[a] = cb * (w.normal[a] / vlen - vn * v[a] / (vlen * vlen * vlen));   // cosine
    }
    // x_w = r + t* v,  t* = ((o - r) . n) / (v . n)
    double tb = xwb[0] * v[0] + xwb[1] * v[1] + xwb[2] * v[2];
    for (int a = 0; a < 3; ++a) {
        rb[a] += xwb[a] - tb * w.normal[a] / vn;
        vb[a] += tstar * xwb[a] - tb * tstar * w.normal[a] / vn;
    }
    double dtb = 0.0;
    for (long n = N - 1; n >= 0; --n) {
        const double* rn = &tape[6 * n];
        const double* vn_ = &tape[6 * n + 3];
        const double* r1 = &tape[6 * (n + 1)];
        double dr[3] = {r1[0] - rn[0], r1[1] - rn[1], r1[2] - rn[2]};
        double l = norm3(dr);
        for (int a = 0; a < 3; ++a) rb[a] += lenb * dr[a] / l;            // |r_{n+1} - r_n| term
        if (sc.it->integrator == 2) step_quasi_adjoint(F, rin, v0, n, vn_, dt, rb, vb, dtb, acc);
        else step_rkn_adjoint(F, rn, vn_, dt, rb, vb, dtb, acc);
        for (int a = 0; a < 3; ++a) rb[a] -= lenb * dr[a] / l;
    }
    // v0 = eta_in d, dt = ell / (N eta_in), eta_in = 1 + deta(r_in)
    double etab = vb[0] * R.d[0] + vb[1] * R.d[1] + vb[2] * R.d[2] - dtb * dt / eta_in;
    Corner C[8];
    corners_at(*F.g, rin, C);
    for (int c = 0; c < 8; ++c) acc.deta[C[c].node] += C[c].w * etab;
}

}  // namespace

// =============================================================== C ABI of the oracle
extern "C" {

int orc_abi_version(void) { return 4; }

void orc_deta_from_T(const orc_grid* g, const double* T, double* deta) { deta_from_T<double>(*g, T, deta); }

void orc_grad_from_deta(const orc_grid* g, const double* deta, double* grad) {
    grad_from_deta<double>(*g, deta, grad);
}

// eta and grad eta at npts points (for interpolation tests).
void orc_field_eval(const orc_grid* g, const orc_field* f, long npts, const double* x, double* eta, double* grad) {
    Field<double> F = make_field(g, f);
    for (long i = 0; i < npts; ++i) field_eval(F, x + 3 * i, eta[i], grad + 3 * i);
}

// Integrate one ray segment: N steps from r_in along unit d with v0 = eta(r_in) d and
// dt = ell / (N eta(r_in)).  Outputs r_N, v_N, the polyline length and, if tape is not
// NULL, all (N + 1) states (r, v) as 6 doubles each.
void orc_trace_segment(const orc_grid* g, const orc_field* f, const double* r_in, const double* d, double ell,
                       long N, int integrator, double* r_out, double* v_out, double* lensum, double* tape) {
    Field<double> F = make_field(g, f);
    double eta_in, gd[3];
    field_eval(F, r_in, eta_in, gd);
    double r[3], v[3];
    for (int a = 0; a < 3; ++a) { r[a] = r_in[a]; v[a] = eta_in * d[a]; }
    double dt = ell / ((double)N * eta_in);
    double ls = 0.0;
    if (tape) for (int a = 0; a < 3; ++a) { tape[a] = r[a]; tape[3 + a] = v[a]; }
    const double rin[3] = {r[0], r[1], r[2]}, v0[3] = {v[0], v[1], v[2]};
    for (long n = 0; n < N; ++n) {
        double r0[3] = {r[0], r[1], r[2]};
        if (integrator == 1) step_rk4(F, r, v, dt);
        else if (integrator == 2) step_quasi(F, rin, v0, n, r, v, dt);
        else step_rkn(F, r, v, dt);
        double dr[3] = {r[0] - r0[0], r[1] - r0[1], r[2] - r0[2]};
        ls += norm3(dr);
        if (tape) for (int a = 0; a < 3; ++a) { tape[6 * (n + 1) + a] = r[a]; tape[6 * (n + 1) + 3 + a] = v[a]; }
    }
    for (int a = 0; a < 3; ++a) { r_out[a] = r[a]; v_out[a] = v[a]; }
    *lensum = ls;
}

// Camera ray set-up for sample s of pixel pix: image point, direction, entry, segment, N.
void orc_ray_setup(const orc_grid* g, const orc_camera* cam, const orc_wall* w, const orc_integ* it, long pix,
                   int s, double* xy, double* d, double* t_in, double* ell, double* tw, long* N, int* flags) {
    Scene sc = {g, cam, w, nullptr, it};
    long px = pix % cam->width, py = pix / cam->width;
    sample_point(*cam, px, py, s, xy[0], xy[1]);
    RayGeom R = pixel_ray(sc, pix, s);
    for (int a = 0; a < 3; ++a) d[a] = R.d[a];
    *t_in = R.t_in;
    *ell = R.ell;
    *tw = R.tw;
    *N = R.N;
    *flags = (R.wall ? 1 : 0) | (R.traced ? 2 : 0);
}

uint64_t orc_splitmix64_output(uint64_t seed, uint64_t k) { return splitmix64_output(seed, k); }
double orc_tent_inverse(double xi) { return tent_inverse(xi); }

// Projector connection (mode 2) of npts wall points x: the aim a after the light's
// connect_iters rounds (or `iters` >= 0 rounds when given) and the wall hit y(a) of the
// projector ray aimed at it.  The camera is not used.
void orc_connect(const orc_grid* g, const orc_field* f, const orc_wall* w, const orc_light* L, const orc_integ* it,
                 long npts, const double* x, int iters, double* a_out, double* y_out) {
    Field<double> F = make_field(g, f);
    orc_light L2 = *L;
    L2.mode = 2;
    if (iters >= 0) L2.connect_iters = iters;
    Scene sc = {g, nullptr, w, &L2, it};
    for (long i = 0; i < npts; ++i) {
        connect_projector(sc, F, x + 3 * i, a_out + 3 * i);
        trace_projector(sc, F, a_out + 3 * i, y_out + 3 * i);
    }
}

// Luminance at npts wall points.
void orc_luminance(const orc_light* L, const orc_wall* w, long npts, const double* x, double* out) {
    for (long i = 0; i < npts; ++i) out[i] = luminance<double>(*L, *w, x + 3 * i);
}

// Render npix pixels (pix = NULL: all, in order).  Per pixel: I (mean over samples of
// L cos / len), disp (mean over samples, 2), hit (mean wall coordinates, 2).  nsteps
// (NULL or npix * spp) receives N of every sample.  straight != 0 renders the
// reference image (no flow).
void orc_render(const orc_grid* g, const orc_field* f, const orc_camera* cam, const orc_wall* w,
                const orc_light* L, const orc_integ* it, long npix, const long* pix, int straight, int threads,
                double* I, double* disp, double* hit, long* nsteps) {
    Field<double> F = make_field(g, f);
    Scene sc = {g, cam, w, L, it};
    const int spp = cam->spp;
    parallel_for(npix, threads, [&](long q) {
        long p = pix ? pix[q] : q;
        double Is = 0.0, d0 = 0.0, d1 = 0.0, h0 = 0.0, h1 = 0.0;
        for (int s = 0; s < spp; ++s) {
            RayGeom R = pixel_ray(sc, p, s);
            RayOut<double> o = trace_ray<double>(sc, F, R, straight != 0);
            Is += o.I;
            d0 += o.disp[0];
            d1 += o.disp[1];
            h0 += o.hit[0];
            h1 += o.hit[1];
            if (nsteps) nsteps[q * spp + s] = o.N;
        }
        I[q] = Is / spp;
        if (disp) { disp[2 * q] = d0 / spp; disp[2 * q + 1] = d1 / spp; }
        if (hit) { hit[2 * q] = h0 / spp; hit[2 * q + 1] = h1 / spp; }
    });
}

// Complex-step directional derivative of I with respect to T along dT:
// dI = Im(I(T + i h dT)) / h, computed through eta(T), the central differences and the
// whole forward model in complex arithmetic.
void orc_render_cs(const orc_grid* g, const double* T, const double* dT, double h, const orc_camera* cam,
                   const orc_wall* w, const orc_light* L, const orc_integ* it, long npix, const long* pix,
                   int threads, double* dI, double* ddisp) {
    const size_t n = (size_t)g->n[0] * g->n[1] * g->n[2];
    std::vector<cplx> Tc(n), de(n), gr(3 * n);
    for (size_t c = 0; c < n; ++c) Tc[c] = cplx(T[c], h * dT[c]);
    deta_from_T<cplx>(*g, Tc.data(), de.data());
    grad_from_deta<cplx>(*g, de.data(), gr.data());
    Field<cplx> F;
    F.g = g;
    F.kind = 0;
    F.deta = de.data();
    F.grad = gr.data();
    for (int a = 0; a < 3; ++a) F.h[a] = spacing(*g, a);
    Scene sc = {g, cam, w, L, it};
    const int spp = cam->spp;
    parallel_for(npix, threads, [&](long q) {
        long p = pix ? pix[q] : q;
        cplx Is = 0.0, d0 = 0.0, d1 = 0.0;
        for (int s = 0; s < spp; ++s) {
            RayGeom R = pixel_ray(sc, p, s);
            RayOut<cplx> o = trace_ray<cplx>(sc, F, R, false);
            Is += o.I;
            d0 += o.disp[0];
            d1 += o.disp[1];
        }
        dI[q] = Is.imag() / h / spp;
        if (ddisp) { ddisp[2 * q] = d0.imag() / h / spp; ddisp[2 * q + 1] = d1.imag() / h / spp; }
    });
}

// Gradient of sum_j w_j I_j with respect to the node fields (deta, grad) and to T, by a
// discrete adjoint over a full tape of ray states (Sharma RKN or quasi-linear).  w = dL/dI per pixel
// (all pixels).  Node adjoints (may be NULL) receive the direct node sensitivities;
// dLdT receives the total derivative with respect to T through the central differences
// and d eta / d T = -rho0 G T0 / T^2.
void orc_grad(const orc_grid* g, const double* T, const orc_camera* cam, const orc_wall* w, const orc_light* L,
              const orc_integ* it, const double* dLdI, int threads, double* dLdT, double* node_deta,
              double* node_grad) {
    const size_t n = (size_t)g->n[0] * g->n[1] * g->n[2];
    if (L->mode == 2 && it->integrator != 0) {   // the projector-ray adjoint is written for Sharma RKN
        for (size_t c = 0; c < n; ++c) dLdT[c] = NAN;
        return;
    }
    std::vector<double> de(n), gr(3 * n);
    deta_from_T<double>(*g, T, de.data());
    grad_from_deta<double>(*g, de.data(), gr.data());
    orc_field f;
    f.kind = 0;
    f.deta = de.data();
    f.grad = gr.data();
    Field<double> F = make_field(g, &f);
    Scene sc = {g, cam, w, L, it};
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    const long npix = (long)cam->width * cam->height;
    const int spp = cam->spp;
    std::vector<std::vector<double>> acc_de(threads, std::vector<double>(n, 0.0));
    std::vector<std::vector<double>> acc_g(threads, std::vector<double>(3 * n, 0.0));
    std::atomic<long> next(0);
    auto work = [&](int t) {
        NodeAdj acc = {acc_de[t].data(), acc_g[t].data()};
        std::vector<double> tape;
        for (;;) {
            long p = next.fetch_add(1);
            if (p >= npix) break;
            if (dLdI[p] == 0.0) continue;   // no sensitivity: nothing to propagate
            for (int s = 0; s < spp; ++s) {
                RayGeom R = pixel_ray(sc, p, s);
                ray_adjoint(sc, F, R, dLdI[p] / spp, acc, tape);
            }
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
    std::vector<double> bde(n, 0.0), bg(3 * n, 0.0);
    for (int t = 0; t < threads; ++t) {
        for (size_t c = 0; c < n; ++c) bde[c] += acc_de[t][c];
        for (size_t c = 0; c < 3 * n; ++c) bg[c] += acc_g[t][c];
    }
    if (node_deta) std::memcpy(node_deta, bde.data(), n * sizeof(double));
    if (node_grad) std::memcpy(node_grad, bg.data(), 3 * n * sizeof(double));
    // transpose of the difference stencil: grad_m[a] = (deta[hi] - deta[lo]) / den
    std::vector<double> tot(bde);
    const long nx = g->n[0], ny = g->n[1], nz = g->n[2];
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long idx[3] = {i, j, k};
                size_t m = node_index(*g, i, j, k);
                for (int a = 0; a < 3; ++a) {
                    long lo = idx[a] - 1, hi = idx[a] + 1;
                    double den = 2.0 * spacing(*g, a);
                    if (lo < 0) { lo = idx[a]; den = spacing(*g, a); }
                    if (hi > g->n[a] - 1) { hi = idx[a]; den = spacing(*g, a); }
                    long ilo[3] = {i, j, k}, ihi[3] = {i, j, k};
                    ilo[a] = lo;
                    ihi[a] = hi;
                    tot[node_index(*g, ihi[0], ihi[1], ihi[2])] += bg[3 * m + a] / den;
                    tot[node_index(*g, ilo[0], ilo[1], ilo[2])] -= bg[3 * m + a] / den;
                }
            }
    const double K = g->rho0 * g->G * g->T0;
    for (size_t c = 0; c < n; ++c) dLdT[c] = tot[c] * (-K / (T[c] * T[c]));
}

}  // extern "C"
