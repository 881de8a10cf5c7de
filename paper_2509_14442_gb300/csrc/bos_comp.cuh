// Float32 deviation integrator (FP32_COMP / BF16_COMP), shared by the forward and the
// adjoint kernels so that the adjoint recomputes exactly the forward's arithmetic.
#pragma once

#include "bos_device.cuh"

namespace bos {

// ---- float32 deviation from a fixed-point straight line (FP32_COMP / BF16_COMP) -----
//
// A ray's straight line S(m) = r_in + m (ell/N) d is kept in 32.32 fixed point grid
// units (hi word = cell, lo word = fraction), exact under repeated addition; the ray
// state is r = S(n) + dr, v = eta_in d + dv with dr, dv small and carried in float32
// with Kahan compensation.  Sharma's step in these variables:
//   A = dt D(S(n) + dr)
//   B = dt D(S(n+1/2) + dr + dt/2 dv + dt/8 A)
//   C = dt D(S(n+1) + dr + dt dv + dt/2 B)
//   dr += dt (dv + (A + 2B)/6),  dv += (A + 4B + C)/6

template <class E>
struct CompField {
    const E* store;
    int n[3];
    float inv_h[3];
    uint32_t nelem;   // store elements (the checked build's bound)
    int* err;
};

template <class E>
__device__ __forceinline__ CompField<E> comp_field(const GridDev& g) {
    return CompField<E>{static_cast<const E*>(g.store), {g.n[0], g.n[1], g.n[2]}, {g.inv_hf[0], g.inv_hf[1], g.inv_hf[2]},
                        g.store_elems, g.err};
}

// Store offset of the base corner of a cell: the x-paired elements of its 8 corners span
// o .. o + 90 (the checked build bounds that range).
template <class E>
__device__ __forceinline__ uint32_t comp_offset(const CompField<E>& F, BrickCache& bc, const int ci[3]) {
    const uint32_t o = cached_offset(bc, ci[0], ci[1], ci[2]);
#if BOS_CHECKED
    const uint32_t b = bounded(o + 90u, F.nelem, F.err);
    return b ? b - 90u : 0u;
#else
    return o;
#endif
}

// Cell and fraction of fixed-point straight position U plus deviation q (metres).  The
// 32-bit fraction word becomes a float through its top 23 bits (U carries a +2^-24 bias
// from the set-up, so this truncation rounds to nearest); fractions outside [0, 1) and
// cells outside [0, n-2] (near the box faces, where the edge cells extrapolate) take a
// rarely used exact path.
template <class E>
__device__ __forceinline__ void comp_cell(const CompField<E>& F, const long long U[3], const float q[3], int ci[3],
                                          float cf[3]) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const uint32_t lo = (uint32_t)U[a];
        ci[a] = (int)(U[a] >> 32);
        const float fr = __uint_as_float((lo >> 9) | 0x3f800000u) - 1.0f;
        cf[a] = fmaf(q[a], F.inv_h[a], fr);
        // 0 <= f < 1 exactly when the bit pattern is below that of 1.0f (negatives have the
        // sign bit set); 0 <= i <= n - 2 as one unsigned compare
        ok = ok && __float_as_uint(cf[a]) < 0x3f800000u && (uint32_t)ci[a] <= (uint32_t)(F.n[a] - 2);
    }
    if (!ok) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float fl = floorf(cf[a]);
            int I = ci[a] + (int)fl;
            float f = cf[a] - fl;
            int Ic = min(max(I, 0), F.n[a] - 2);
            ci[a] = Ic;
            cf[a] = f + (float)(I - Ic);
        }
    }
}

// Field at fixed-point straight position U plus deviation q (metres).
template <class E>
__device__ __forceinline__ float4 comp_eval(const CompField<E>& F, const long long U[3], const float q[3],
                                            BrickCache& bc, int ci[3], float cf[3]) {
    comp_cell(F, U, q, ci, cf);
    const uint32_t o = comp_offset(F, bc, ci);
    return trilinear2(F.store, o, cf[0], cf[1], cf[2]);
}

// The four paired records of the last cell a ray gathered, as the first interpolation level
// uses them: each record and its x difference.  A ray's consecutive stage points are a
// quarter of a voxel apart or less, and the next step's first stage is within rounding of
// this step's third, so most evaluations find their cell here and load (and, for the
// bfloat16 store, widen) nothing; the interpolation is the same operations on the same
// values as `trilinear2`, so the results are bit-identical.
struct CellRecs {
    uint32_t o;            // element offset of the cached cell's base corner (0xffffffff: none)
    Cell2 v[4], d[4];      // pairs at o, o + 9, o + 81, o + 90: records and x differences
};

__device__ __forceinline__ void load_rec(const F4P* s, uint32_t o, Cell2& v, Cell2& d) { load_pair(s, o, v, d); }
__device__ __forceinline__ void load_rec(const B4P* s, uint32_t o, Cell2& v, Cell2& d) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(s + o));
    const Cell2 b = bf16_cell(make_uint2(u.z, u.w));
    v = bf16_cell(make_uint2(u.x, u.y));
    d = Cell2{sub2(b.lo, v.lo), sub2(b.hi, v.hi)};
}

template <class E>
__device__ __forceinline__ float4 trilinear_cached(const E* s, uint32_t o, float f0, float f1, float f2, CellRecs& c) {
    if (o != c.o) {   // per lane: lanes whose cell is cached issue no load
        load_rec(s, o, c.v[0], c.d[0]);
        load_rec(s, o + 9, c.v[1], c.d[1]);
        load_rec(s, o + 81, c.v[2], c.d[2]);
        load_rec(s, o + 90, c.v[3], c.d[3]);
        c.o = o;
    }
    const f32x2 t0 = pack2(f0, f0), t1 = pack2(f1, f1), t2 = pack2(f2, f2);
    Cell2 a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = Cell2{fma2(t0, c.d[i].lo, c.v[i].lo), fma2(t0, c.d[i].hi, c.v[i].hi)};
    const Cell2 r = lerpc(lerpc(a[0], a[1], t1), lerpc(a[2], a[3], t1), t2);
    float4 v;
    unpack2(r.lo, v.x, v.y);
    unpack2(r.hi, v.z, v.w);
    return v;
}

// comp_eval through the cell cache (the paired float32 and bfloat16 stores).
template <class E>
__device__ __forceinline__ float4 comp_eval_c(const CompField<E>& F, const long long U[3], const float q[3],
                                              BrickCache& bc, CellRecs& cr, int ci[3], float cf[3]) {
    comp_cell(F, U, q, ci, cf);
    const uint32_t o = comp_offset(F, bc, ci);
    return trilinear_cached(F.store, o, cf[0], cf[1], cf[2], cr);
}

__device__ __forceinline__ void rhs_of(float4 v, float D[3]) {
    float eta = 1.0f + v.x;
    D[0] = eta * v.y;
    D[1] = eta * v.z;
    D[2] = eta * v.w;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

struct CompState {
    long long U[3];     // straight position at step start (32.32 grid units)
    float dr[3], cr[3]; // deviation and its Kahan compensation (true = dr - cr)
    float dv[3], cv[3];
    float excess;       // sum over steps of |step| - ell/N
};

struct CompConst {
    long long dU[3], dUh[3];   // straight step and half step (32.32 grid units)
    float dS[3];               // straight step (m)
    float dhat[3];
    float step_len;            // ell / N
    float dt;
};

// One step; with AB != nullptr (Sharma RKN) the step's A and B are also written to AB[0..5]
// (the adjoint's recompute keeps them, so its reverse step knows all three stage points).
template <class E, int INTEG>
__device__ __forceinline__ void comp_step(const CompField<E>& F, CompState& st, const CompConst& k, BrickCache& bc,
                                          float* AB = nullptr) {
    int ci[3];
    float cf[3], D[3];
    float inc_r[3], inc_v[3];
    const float dt = k.dt;
    if constexpr (INTEG != 1) {
        float A[3], B[3], C[3], q[3];
        long long U2[3], U3[3];
        rhs_of(comp_eval(F, st.U, st.dr, bc, ci, cf), D);
        for (int a = 0; a < 3; ++a) A[a] = dt * D[a];
        for (int a = 0; a < 3; ++a) {
            q[a] = st.dr[a] + (0.5f * dt) * st.dv[a] + (0.125f * dt) * A[a];
            U2[a] = st.U[a] + k.dUh[a];
        }
        rhs_of(comp_eval(F, U2, q, bc, ci, cf), D);
        for (int a = 0; a < 3; ++a) B[a] = dt * D[a];
        for (int a = 0; a < 3; ++a) {
            q[a] = st.dr[a] + dt * st.dv[a] + (0.5f * dt) * B[a];
            U3[a] = st.U[a] + k.dU[a];
        }
        rhs_of(comp_eval(F, U3, q, bc, ci, cf), D);
        for (int a = 0; a < 3; ++a) C[a] = dt * D[a];
        for (int a = 0; a < 3; ++a) {
            inc_r[a] = dt * (st.dv[a] + (A[a] + 2.0f * B[a]) * (1.0f / 6.0f));
            inc_v[a] = (A[a] + 4.0f * B[a] + C[a]) * (1.0f / 6.0f);
        }
        if (AB != nullptr)
            for (int a = 0; a < 3; ++a) {
                AB[a] = A[a];
                AB[3 + a] = B[a];
            }
    } else {
        // classic RK4 on (r, v): k1v..k4v are D at the four stage positions
        float k1[3], k2[3], k3[3], k4[3], q[3];
        long long U2[3], U3[3];
        rhs_of(comp_eval(F, st.U, st.dr, bc, ci, cf), k1);
        for (int a = 0; a < 3; ++a) {
            q[a] = st.dr[a] + (0.5f * dt) * st.dv[a];
            U2[a] = st.U[a] + k.dUh[a];
        }
        rhs_of(comp_eval(F, U2, q, bc, ci, cf), k2);
        for (int a = 0; a < 3; ++a) q[a] = st.dr[a] + (0.5f * dt) * (st.dv[a] + (0.5f * dt) * k1[a]);
        rhs_of(comp_eval(F, U2, q, bc, ci, cf), k3);
        for (int a = 0; a < 3; ++a) {
            q[a] = st.dr[a] + dt * (st.dv[a] + (0.5f * dt) * k2[a]);
            U3[a] = st.U[a] + k.dU[a];
        }
        rhs_of(comp_eval(F, U3, q, bc, ci, cf), k4);
        for (int a = 0; a < 3; ++a) {
            inc_r[a] = dt * st.dv[a] + (dt * dt * (1.0f / 6.0f)) * (k1[a] + k2[a] + k3[a]);
            inc_v[a] = (dt * (1.0f / 6.0f)) * (k1[a] + 2.0f * k2[a] + 2.0f * k3[a] + k4[a]);
        }
    }
    // |dS + inc| - |dS| = (2 dS.inc + |inc|^2) / (|dS + inc| + |dS|)
    float si = k.dS[0] * inc_r[0] + k.dS[1] * inc_r[1] + k.dS[2] * inc_r[2];
    float ii = inc_r[0] * inc_r[0] + inc_r[1] * inc_r[1] + inc_r[2] * inc_r[2];
    float di = k.dhat[0] * inc_r[0] + k.dhat[1] * inc_r[1] + k.dhat[2] * inc_r[2];
    st.excess += __fdividef(2.0f * si + ii, 2.0f * k.step_len + di);
    for (int a = 0; a < 3; ++a) {
        kahan_add(st.dr[a], st.cr[a], inc_r[a]);
        kahan_add(st.dv[a], st.cv[a], inc_v[a]);
        st.U[a] += k.dU[a];
    }
}

__device__ __forceinline__ long long to_fixed(double u, double scale) { return __double2ll_rn(u * scale); }

// Set-up shared by the forward and the adjoint: fixed-point line, eta at entry, dt.
// Set-up of the compensated state of the ray rs + t d (camera or projector pinhole rs).
template <class E>
__device__ __forceinline__ void comp_setup(const SceneDev& S, const CompField<E>& F, const double rs[3], const Ray& R,
                                           CompState& st, CompConst& k, double& eta_in, double rin[3]) {
    const GridDev& g = S.g;
    double sl = R.ell / (double)R.N;
    for (int a = 0; a < 3; ++a) {
        rin[a] = rs[a] + R.t_in * R.d[a];
        double u = (rin[a] - g.origin[a]) * g.inv_h[a] - 0.5;
        double du = sl * R.d[a] * g.inv_h[a];
        st.U[a] = to_fixed(u, 4294967296.0) + 256;   // +2^-24: see comp_cell
        k.dU[a] = to_fixed(du, 4294967296.0);
        k.dUh[a] = k.dU[a] >> 1;
        k.dS[a] = (float)(sl * R.d[a]);
        k.dhat[a] = (float)R.d[a];
        st.dr[a] = st.cr[a] = st.dv[a] = st.cv[a] = 0.0f;
    }
    st.excess = 0.0f;
    BrickCache bc = {0xffffffffu, 0u};
    int ci[3];
    float cf[3];
    float zero[3] = {0.0f, 0.0f, 0.0f};
    float4 v = comp_eval(F, st.U, zero, bc, ci, cf);
    eta_in = 1.0 + (double)v.x;
    k.dt = (float)sl / (float)eta_in;   // dt = (ell / N) / eta_in; float precision is all it carries
    k.step_len = (float)sl;
}


// ------------------------------------------------------------------ wall (Eq. 2) in float32
//
// With r_N = r_s + (t_in + ell) d + dr and v_N = eta_in d + dv, the wall hit relative to
// the straight hit x_ref = r_s + t_w d only involves small quantities:
//   t* = (L c - n.dr) / (eta_in c + n.dv),          c = n.d,  L = t_w - t_in - ell
//   x_w - x_ref = dr + t* dv - ((eta_in n.dr + L n.dv) / (eta_in c + n.dv)) d
// so float32 keeps ~1e-7 of the displacement; float64 is used only for x_ref.

__device__ __forceinline__ float texel_f(const LightDev& L, int i, int j) {
    if (i < 0 || j < 0 || i >= L.tw || j >= L.th) return 0.0f;
    return __ldg(L.pattern + (size_t)j * L.tw + i);
}

__device__ __forceinline__ float bilinear_f(const LightDev& L, float s, float t) {
    s -= 0.5f;
    t -= 0.5f;
    float fi = floorf(fminf(fmaxf(s, -4.0f), (float)L.tw + 4.0f));
    float fj = floorf(fminf(fmaxf(t, -4.0f), (float)L.th + 4.0f));
    int i = (int)fi, j = (int)fj;
    float fs = s - fi, ft = t - fj;
    float p00 = texel_f(L, i, j), p10 = texel_f(L, i + 1, j), p01 = texel_f(L, i, j + 1), p11 = texel_f(L, i + 1, j + 1);
    return (1.0f - fs) * ((1.0f - ft) * p00 + ft * p01) + fs * ((1.0f - ft) * p10 + ft * p11);
}

// Luminance at x_ref + dx.
__device__ __forceinline__ float luminance_rel(const SceneDev& S, const double xref[3], const float dx[3]) {
    const LightDev& L = S.L;
    const WallDev& w = S.w;
    if (L.mode == 0) {
        double q[3] = {xref[0] - w.origin[0], xref[1] - w.origin[1], xref[2] - w.origin[2]};
        float hu = (float)(q[0] * w.eu[0] + q[1] * w.eu[1] + q[2] * w.eu[2]) +
                   (dx[0] * (float)w.eu[0] + dx[1] * (float)w.eu[1] + dx[2] * (float)w.eu[2]);
        float hv = (float)(q[0] * w.ev[0] + q[1] * w.ev[1] + q[2] * w.ev[2]) +
                   (dx[0] * (float)w.ev[0] + dx[1] * (float)w.ev[1] + dx[2] * (float)w.ev[2]);
        return bilinear_f(L, hu * (float)(L.tw / w.size_u), hv * (float)(L.th / w.size_v));
    }
    const CamDev& P = L.proj;
    float q[3];
    for (int a = 0; a < 3; ++a) q[a] = (float)(xref[a] - P.pos[a]) + dx[a];
    float fw[3] = {(float)P.fwd[0], (float)P.fwd[1], (float)P.fwd[2]};
    float up[3] = {(float)P.up[0], (float)P.up[1], (float)P.up[2]};
    float rt[3] = {fw[1] * up[2] - fw[2] * up[1], fw[2] * up[0] - fw[0] * up[2], fw[0] * up[1] - fw[1] * up[0]};
    float z = q[0] * fw[0] + q[1] * fw[1] + q[2] * fw[2];
    if (!(z > 0.0f)) return 0.0f;
    float iz = 1.0f / z;
    float px = (float)P.cx + (float)P.fx * ((q[0] * rt[0] + q[1] * rt[1] + q[2] * rt[2]) * iz);
    float py = (float)P.cy - (float)P.fy * ((q[0] * up[0] + q[1] * up[1] + q[2] * up[2]) * iz);
    return bilinear_f(L, px, py);
}

// Wall hit of a traced ray relative to its straight hit rs + t_w d, from the end
// deviation (dr, dv): dx = x_w - x_ref, the cosine factor <n, v_N> / |v_N| and the path
// length (signed straight continuation t* |v_N|).  valid = the ray reaches the wall.
struct WallRel {
    float dx[3];
    float cosw, len;
    bool valid;
};

__device__ __forceinline__ WallRel comp_wall(const SceneDev& S, const Ray& R, double eta_in, const float dr[3],
                                             const float dv[3], float excess) {
    WallRel h;
    const WallDev& w = S.w;
    float nf[3] = {(float)w.normal[0], (float)w.normal[1], (float)w.normal[2]};
    float df[3] = {(float)R.d[0], (float)R.d[1], (float)R.d[2]};
    const float cd = df[0] * nf[0] + df[1] * nf[1] + df[2] * nf[2];
    const float Lrem = (float)(R.tw - R.t_in - R.ell);
    const float e = (float)eta_in;
    const float ndr = nf[0] * dr[0] + nf[1] * dr[1] + nf[2] * dr[2];
    const float ndv = nf[0] * dv[0] + nf[1] * dv[1] + nf[2] * dv[2];
    const float den = e * cd + ndv;                       // <n, v_N>
    h.valid = den > 0.0f;
    if (!h.valid) {
        h.dx[0] = h.dx[1] = h.dx[2] = 0.0f;
        h.cosw = h.len = 0.0f;
        return h;
    }
    const float iden = 1.0f / den;
    const float ts = (Lrem * cd - ndr) * iden;
    const float kk = -(e * ndr + Lrem * ndv) * iden;
    for (int a = 0; a < 3; ++a) h.dx[a] = dr[a] + ts * dv[a] + kk * df[a];
    const float ddv = df[0] * dv[0] + df[1] * dv[1] + df[2] * dv[2];
    const float vl = sqrtf(e * e + 2.0f * e * ddv + (dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]));
    h.len = (float)(R.t_in + R.ell) + (excess + ts * vl);   // signed continuation t* |v|
    h.cosw = den / vl;
    return h;
}

// Finish a camera ray whose wall point is x_ref + dx, reading the luminance at x_ref + e
// (e = dx, or the refracted projector connection of the wall point).
__device__ __forceinline__ RayResult comp_finish(const SceneDev& S, const Ray& R, const WallRel& h, const float e[3],
                                                 bool want_hit) {
    RayResult o;
    o.I = 0.0;
    o.hit[0] = o.hit[1] = o.disp[0] = o.disp[1] = 0.0;
    if (!h.valid) return o;
    const WallDev& w = S.w;
    const float* dx = h.dx;
    double xref[3];
    for (int a = 0; a < 3; ++a) xref[a] = S.cam.pos[a] + R.tw * R.d[a];
    const float Lw = luminance_rel(S, xref, e);
    o.I = (double)(Lw * h.cosw / h.len);
    o.disp[0] = (double)(dx[0] * (float)w.eu[0] + dx[1] * (float)w.eu[1] + dx[2] * (float)w.eu[2]);
    o.disp[1] = (double)(dx[0] * (float)w.ev[0] + dx[1] * (float)w.ev[1] + dx[2] * (float)w.ev[2]);
    if (want_hit) {
        double q[3] = {xref[0] - w.origin[0], xref[1] - w.origin[1], xref[2] - w.origin[2]};
        o.hit[0] = q[0] * w.eu[0] + q[1] * w.eu[1] + q[2] * w.eu[2] + o.disp[0];
        o.hit[1] = q[0] * w.ev[0] + q[1] * w.ev[1] + q[2] * w.ev[2] + o.disp[1];
    }
    return o;
}

// The straight (no-flow) ray: hit x_ref, cosine <n, d>, length t_w.
__device__ __forceinline__ RayResult straight_epilogue(const SceneDev& S, const Ray& R, bool want_hit) {
    const float zero[3] = {0.0f, 0.0f, 0.0f};
    RayResult o;
    o.I = 0.0;
    o.hit[0] = o.hit[1] = o.disp[0] = o.disp[1] = 0.0;
    const WallDev& w = S.w;
    const float cd = (float)(R.d[0] * w.normal[0] + R.d[1] * w.normal[1] + R.d[2] * w.normal[2]);
    if (!(cd > 0.0f)) return o;
    double xref[3];
    for (int a = 0; a < 3; ++a) xref[a] = S.cam.pos[a] + R.tw * R.d[a];
    o.I = (double)(luminance_rel(S, xref, zero) * cd / (float)R.tw);
    if (want_hit) {
        double q[3] = {xref[0] - w.origin[0], xref[1] - w.origin[1], xref[2] - w.origin[2]};
        o.hit[0] = q[0] * w.eu[0] + q[1] * w.eu[1] + q[2] * w.eu[2];
        o.hit[1] = q[0] * w.ev[0] + q[1] * w.ev[1] + q[2] * w.ev[2];
    }
    return o;
}

}  // namespace bos
