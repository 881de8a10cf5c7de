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
};

// Field at fixed-point straight position U plus deviation q (metres).
template <class E>
__device__ __forceinline__ float4 comp_eval(const CompField<E>& F, const long long U[3], const float q[3],
                                            BrickCache& bc, int ci[3], float cf[3]) {
    for (int a = 0; a < 3; ++a) {
        int I = (int)(U[a] >> 32);
        float f = fmaf(q[a], F.inv_h[a], __uint2float_rn((uint32_t)U[a]) * 2.3283064365386963e-10f);
        float fl = floorf(f);
        I += (int)fl;
        f -= fl;
        int Ic = min(max(I, 0), F.n[a] - 2);
        f += (float)(I - Ic);
        ci[a] = Ic;
        cf[a] = f;
    }
    uint32_t o = cached_offset(bc, ci[0], ci[1], ci[2]);
    return trilinear(F.store, o, cf[0], cf[1], cf[2]);
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

template <class E, int INTEG>
__device__ __forceinline__ void comp_step(const CompField<E>& F, CompState& st, const CompConst& k, BrickCache& bc) {
    int ci[3];
    float cf[3], D[3];
    float inc_r[3], inc_v[3];
    const float dt = k.dt;
    if (INTEG == 0) {
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
    st.excess += (2.0f * si + ii) / (2.0f * k.step_len + di);
    for (int a = 0; a < 3; ++a) {
        kahan_add(st.dr[a], st.cr[a], inc_r[a]);
        kahan_add(st.dv[a], st.cv[a], inc_v[a]);
        st.U[a] += k.dU[a];
    }
}

__device__ __forceinline__ long long to_fixed(double u, double scale) { return __double2ll_rn(u * scale); }

// Set-up shared by the forward and the adjoint: fixed-point line, eta at entry, dt.
template <class E>
__device__ __forceinline__ void comp_setup(const SceneDev& S, const CompField<E>& F, const Ray& R, CompState& st,
                                           CompConst& k, double& eta_in, double rin[3]) {
    const GridDev& g = S.g;
    double sl = R.ell / (double)R.N;
    for (int a = 0; a < 3; ++a) {
        rin[a] = S.cam.pos[a] + R.t_in * R.d[a];
        double u = (rin[a] - g.origin[a]) / g.h[a] - 0.5;
        double du = sl * R.d[a] / g.h[a];
        st.U[a] = to_fixed(u, 4294967296.0);
        k.dU[a] = to_fixed(du, 4294967296.0);
        k.dUh[a] = to_fixed(du, 2147483648.0);
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
    double dt = R.ell / ((double)R.N * eta_in);
    k.dt = (float)dt;
    k.step_len = (float)sl;
}


}  // namespace bos
