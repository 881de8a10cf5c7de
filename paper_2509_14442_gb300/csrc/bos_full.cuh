// Full-state integration in absolute coordinates, T = float (plain FP32 tracer) or
// double (FP64 tracer and its adjoint): the field at a point and one Sharma RKN or classic
// RK4 step of dr/dt = v, dv/dt = eta grad eta (Sec. 2.2, Eq. 1).  Shared by the forward
// and the adjoint so that the adjoint recomputes exactly the forward's arithmetic.
#pragma once

#include "bos_comp.cuh"
#include "bos_device.cuh"

namespace bos {

template <class T>
struct FullField;

template <>
struct FullField<double> {
    GridDev g;
    __device__ __forceinline__ void rhs(const double x[3], double D[3]) const {
        double eta, gr[3];
        field_at(g, x, eta, gr);
        for (int a = 0; a < 3; ++a) D[a] = eta * gr[a];
    }
    __device__ __forceinline__ double eta(const double x[3]) const {
        double e, gr[3];
        field_at(g, x, e, gr);
        return e;
    }
};

template <>
struct FullField<float> {
    GridDev g;
    __device__ __forceinline__ float4 at(const float x[3]) const {
        int i[3];
        float f[3];
        for (int a = 0; a < 3; ++a) {
            float u = (x[a] - (float)g.origin[a]) * g.inv_hf[a] - 0.5f;
            split_coord(u, g.n[a], i[a], f[a]);
        }
        uint32_t o = bounded(brick_offset(i[0], i[1], i[2]) + 90u, g.store_elems, g.err);
        o = o ? o - 90u : 0u;
        return trilinear(static_cast<const F4P*>(g.store), o, f[0], f[1], f[2]);
    }
    __device__ __forceinline__ void rhs(const float x[3], float D[3]) const { rhs_of(at(x), D); }
    __device__ __forceinline__ float eta(const float x[3]) const { return 1.0f + at(x).x; }
};

template <class T, int INTEG>
__device__ __forceinline__ void full_step(const FullField<T>& F, T r[3], T v[3], T dt) {
    if (INTEG == 0) {
        T A[3], B[3], C[3], p[3], D[3];
        F.rhs(r, D);
        for (int a = 0; a < 3; ++a) A[a] = dt * D[a];
        for (int a = 0; a < 3; ++a) p[a] = r[a] + (dt * T(0.5)) * v[a] + (dt * T(0.125)) * A[a];
        F.rhs(p, D);
        for (int a = 0; a < 3; ++a) B[a] = dt * D[a];
        for (int a = 0; a < 3; ++a) p[a] = r[a] + dt * v[a] + (dt * T(0.5)) * B[a];
        F.rhs(p, D);
        for (int a = 0; a < 3; ++a) C[a] = dt * D[a];
        for (int a = 0; a < 3; ++a) {
            r[a] = r[a] + dt * (v[a] + (A[a] + T(2) * B[a]) / T(6));
            v[a] = v[a] + (A[a] + T(4) * B[a] + C[a]) / T(6);
        }
    } else {
        T k1v[3], k2v[3], k3v[3], k4v[3], k2r[3], k3r[3], k4r[3], p[3];
        F.rhs(r, k1v);
        for (int a = 0; a < 3; ++a) {
            k2r[a] = v[a] + (dt * T(0.5)) * k1v[a];
            p[a] = r[a] + (dt * T(0.5)) * v[a];
        }
        F.rhs(p, k2v);
        for (int a = 0; a < 3; ++a) {
            k3r[a] = v[a] + (dt * T(0.5)) * k2v[a];
            p[a] = r[a] + (dt * T(0.5)) * k2r[a];
        }
        F.rhs(p, k3v);
        for (int a = 0; a < 3; ++a) {
            k4r[a] = v[a] + dt * k3v[a];
            p[a] = r[a] + dt * k3r[a];
        }
        F.rhs(p, k4v);
        for (int a = 0; a < 3; ++a) {
            r[a] = r[a] + dt / T(6) * (v[a] + T(2) * k2r[a] + T(2) * k3r[a] + k4r[a]);
            v[a] = v[a] + dt / T(6) * (k1v[a] + T(2) * k2v[a] + T(2) * k3v[a] + k4v[a]);
        }
    }
}

}  // namespace bos
