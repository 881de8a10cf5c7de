// Forward kernels of the BOS library for sm_103a:
//   build_store   -- step a1: T -> (eta - 1, grad eta) bricks                 (Sec. 2.1)
//   render        -- steps a2-a5: rays, Sharma RKN tracing, wall, radiance    (Eq. 1, Eq. 2)
//   ray_steps     -- the integer step count of every ray (step a2)
//   export_nodes  -- read the store back through the brick addressing
//   loss_l2       -- L_BOS and its seed dL/dI                                 (Sec. 2.4)
#include "bos_comp.cuh"
#include "bos_device.cuh"
#include "bos_full.cuh"
#include "bos_internal.h"

namespace bos {

// ===================================================================== a1: field store

template <class E>
__device__ __forceinline__ void store_cell(E* dst, double de, double gx, double gy, double gz);

template <>
__device__ __forceinline__ void store_cell<float4>(float4* dst, double de, double gx, double gy, double gz) {
    *dst = make_float4(__double2float_rn(de), __double2float_rn(gx), __double2float_rn(gy), __double2float_rn(gz));
}

template <>
__device__ __forceinline__ void store_cell<uint2>(uint2* dst, double de, double gx, double gy, double gz) {
    uint32_t a = __bfloat16_as_ushort(__double2bfloat16(de)), b = __bfloat16_as_ushort(__double2bfloat16(gx));
    uint32_t c = __bfloat16_as_ushort(__double2bfloat16(gy)), d = __bfloat16_as_ushort(__double2bfloat16(gz));
    *dst = make_uint2(a | (b << 16), c | (d << 16));
}

template <>
__device__ __forceinline__ void store_cell<D4>(D4* dst, double de, double gx, double gy, double gz) {
    double2* p = reinterpret_cast<double2*>(dst);
    p[0] = make_double2(de, gx);
    p[1] = make_double2(gy, gz);
}

__device__ __forceinline__ double deta_at(const GridDev& g, const float* T, int i, int j, int k) {
    double t = (double)__ldg(T + ((size_t)k * g.n[1] + j) * g.n[0] + i);
    return ddiv(g.K, t);
}

// One block per brick: deta = K / T is computed once for every cell of the brick's 9^3
// records plus a one-cell halo (11^3 values in shared memory), then each record takes
// its central or one-sided differences from there.  Bricks cover base cells 0..n-2;
// coordinates beyond the grid are clamped (those records are never read).
constexpr int kHalo = kBrickSide + 2;   // 11

// Store element of each record type: float32 and bfloat16 records are stored as x pairs
// (F4P, B4P), float64 records as they are.
template <class R>
struct StoreElem {
    using type = R;
};
template <>
struct StoreElem<float4> {
    using type = F4P;
};
template <>
struct StoreElem<uint2> {
    using type = B4P;
};

__device__ __forceinline__ void write_elem(F4P* dst, const float4* rec, int l, bool next) {
    const float4 a = rec[l], b = next ? rec[l + 1] : a;
    F4P p;
    p.v = a;
    p.d = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, b.w - a.w);   // float32 subtractions
    *dst = p;
}
__device__ __forceinline__ void write_elem(B4P* dst, const uint2* rec, int l, bool next) {
    B4P p;
    p.a = rec[l];
    p.b = next ? rec[l + 1] : make_uint2(0u, 0u);
    *dst = p;
}
__device__ __forceinline__ void write_elem(D4* dst, const D4* rec, int l, bool) { store_cell<D4>(dst, rec[l].x, rec[l].y, rec[l].z, rec[l].w); }

template <class R>
__global__ void __launch_bounds__(256) build_store_kernel(GridDev g, const float* __restrict__ T,
                                                          typename StoreElem<R>::type* __restrict__ store) {
    __shared__ double de[kHalo * kHalo * kHalo];
    __shared__ __align__(32) R rec[kBrickCells];   // records are written with 16-byte stores
    const int b = blockIdx.x;
    const int bx = b % g.nb[0], by = (b / g.nb[0]) % g.nb[1], bz = b / (g.nb[0] * g.nb[1]);
    const int ox = bx * kBrick - 1, oy = by * kBrick - 1, oz = bz * kBrick - 1;
    for (int t = threadIdx.x; t < kHalo * kHalo * kHalo; t += blockDim.x) {
        const int hx = t % kHalo, hy = (t / kHalo) % kHalo, hz = t / (kHalo * kHalo);
        const int i = min(max(ox + hx, 0), g.n[0] - 1), j = min(max(oy + hy, 0), g.n[1] - 1),
                  k = min(max(oz + hz, 0), g.n[2] - 1);
        de[t] = deta_at(g, T, i, j, k);
    }
    __syncthreads();
    for (int local = threadIdx.x; local < kBrickCells; local += blockDim.x) {
        const int lx = local % kBrickSide, ly = (local / kBrickSide) % kBrickSide, lz = local / (kBrickSide * kBrickSide);
        const int c[3] = {min(bx * kBrick + lx, g.n[0] - 1), min(by * kBrick + ly, g.n[1] - 1),
                          min(bz * kBrick + lz, g.n[2] - 1)};
        // halo index of a (clamped) grid cell
        auto at = [&](int i, int j, int k) { return de[((k - oz) * kHalo + (j - oy)) * kHalo + (i - ox)]; };
        double gr[3];
        for (int a = 0; a < 3; ++a) {
            int lo[3] = {c[0], c[1], c[2]}, hi[3] = {c[0], c[1], c[2]};
            double den = dmul(2.0, g.h[a]);
            lo[a] = c[a] - 1;
            hi[a] = c[a] + 1;
            if (lo[a] < 0) {
                lo[a] = c[a];
                den = g.h[a];
            }
            if (hi[a] > g.n[a] - 1) {
                hi[a] = c[a];
                den = g.h[a];
            }
            gr[a] = ddiv(dsub(at(hi[0], hi[1], hi[2]), at(lo[0], lo[1], lo[2])), den);
        }
        store_cell<R>(rec + local, at(c[0], c[1], c[2]), gr[0], gr[1], gr[2]);
    }
    __syncthreads();
    const uint32_t slot = morton3((uint32_t)bx, (uint32_t)by, (uint32_t)bz);
    for (int local = threadIdx.x; local < kBrickCells; local += blockDim.x)
        write_elem(store + (size_t)slot * kBrickCells + local, rec, local, local % kBrickSide < kBrickSide - 1);
}

// ===================================================================== a3: integrators

// ===================================================================== a2-a5: render

struct Sums {
    double I, du, dv, hu, hv;
};

// Integrate one ray of the comp path (N > 0) from the pinhole rs; optionally store its
// checkpoints every K steps in `state` (slot `ray`).  Leaves the end state in st.  CACHE:
// the Sharma stages go through the ray's cell cache (the refracted connection's kernels,
// which hold a second ray's state, go without: at 96 registers they spill).
template <class E, int INTEG, bool CACHE = true>
__device__ __forceinline__ void comp_run(const SceneDev& S, const CompField<E>& F, const double rs[3], const Ray& R,
                                         const CkptDev& ck, float4* state, long long ray, CompState& st,
                                         double& eta_in) {
    CompConst k;
    double rin[3];
    comp_setup(S, F, rs, R, st, k, eta_in, rin);
    BrickCache bc = {0xffffffffu, 0u};
    CellRecs cr;
    cr.o = 0xffffffffu;
    auto eval = [&](const long long U[3], const float q[3], BrickCache& b, int ci[3], float cf[3]) {
        if constexpr (CACHE) return comp_eval_c(F, U, q, b, cr, ci, cf);
        else return comp_eval(F, U, q, b, ci, cf);
    };
    const int K = ck.every;
#ifndef BOS_FWD_PIPELINE
#define BOS_FWD_PIPELINE 1
#endif
    if constexpr (INTEG == 2) {
        // Quasi-linear tracing (Sec. 2.2): the field is sampled on the straight line at the
        // start, middle and end of every step (Sharma's weights); the end sample is the next
        // step's start sample, so each step gathers twice, with no dependence on the ray.
        const float zero[3] = {0.0f, 0.0f, 0.0f};
        int ci[3];
        float cf[3], A[3], B[3], C[3], D[3];
        float usum[3] = {0.0f, 0.0f, 0.0f};
        const float dt = k.dt;
        rhs_of(comp_eval(F, st.U, zero, bc, ci, cf), D);
        for (int a = 0; a < 3; ++a) A[a] = dt * D[a];
        // two steps per iteration: their four line samples do not depend on one another,
        // so their gathers overlap (the quasi-linear kernel gets a larger register budget for this)
#pragma unroll 2
        for (int n = 0; n < R.N; ++n) {
            long long U2[3], U3[3];
            for (int a = 0; a < 3; ++a) {
                U2[a] = st.U[a] + k.dUh[a];
                U3[a] = st.U[a] + k.dU[a];
            }
            rhs_of(comp_eval(F, U2, zero, bc, ci, cf), D);
            for (int a = 0; a < 3; ++a) B[a] = dt * D[a];
            rhs_of(comp_eval(F, U3, zero, bc, ci, cf), D);
            float inc_r[3], inc_v[3];
            for (int a = 0; a < 3; ++a) {
                C[a] = dt * D[a];
                inc_r[a] = dt * (st.dv[a] + (A[a] + 2.0f * B[a]) * (1.0f / 6.0f));
                inc_v[a] = (A[a] + 4.0f * B[a] + C[a]) * (1.0f / 6.0f);
            }
            float si = k.dS[0] * inc_r[0] + k.dS[1] * inc_r[1] + k.dS[2] * inc_r[2];
            float ii = inc_r[0] * inc_r[0] + inc_r[1] * inc_r[1] + inc_r[2] * inc_r[2];
            float di = k.dhat[0] * inc_r[0] + k.dhat[1] * inc_r[1] + k.dhat[2] * inc_r[2];
            st.excess += __fdividef(2.0f * si + ii, 2.0f * k.step_len + di);
            if (state != nullptr) {          // sum of the unit step directions, for the adjoint
                float w[3] = {k.dS[0] + inc_r[0], k.dS[1] + inc_r[1], k.dS[2] + inc_r[2]};
                float rn = rsqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
                for (int a = 0; a < 3; ++a) usum[a] += w[a] * rn;
            }
            for (int a = 0; a < 3; ++a) {
                kahan_add(st.dr[a], st.cr[a], inc_r[a]);
                kahan_add(st.dv[a], st.cv[a], inc_v[a]);
                st.U[a] = U3[a];
                A[a] = C[a];
            }
        }
        if (state != nullptr) {   // the final state, for the one-sweep adjoint
            state[0 * ck.nrays + ray] = make_float4(st.dr[0] - st.cr[0], st.dr[1] - st.cr[1], st.dr[2] - st.cr[2],
                                                       st.excess);
            state[1 * ck.nrays + ray] = make_float4(st.dv[0] - st.cv[0], st.dv[1] - st.cv[1], st.dv[2] - st.cv[2],
                                                       usum[0]);
            state[2 * ck.nrays + ray] = make_float4(usum[1], usum[2], 0.0f, 0.0f);
        }
    } else if constexpr (INTEG == 0 && BOS_FWD_PIPELINE) {
        // Sharma steps, software-pipelined: the next step's first stage needs only the new
        // position r' = r + dt (v + (A + 2B)/6), not C, so it is evaluated together with this
        // step's third stage.  Same operations as comp_step, in a different order in time.
        BrickCache bc1 = {0xffffffffu, 0u};
        int ci[3];
        float cf[3], A[3], D[3];
        rhs_of(eval(st.U, st.dr, bc1, ci, cf), D);
        const float dt = k.dt;
        for (int a = 0; a < 3; ++a) A[a] = dt * D[a];
        for (int n = 0; n < R.N; ++n) {
            if (state != nullptr && n % K == 0) {
                const size_t c = bounded((size_t)(n / K), (size_t)ck.max_ckpt, ck.err);
                state[(c * 3 + 0) * ck.nrays + ray] = make_float4(st.dr[0], st.dr[1], st.dr[2], st.cr[0]);
                state[(c * 3 + 1) * ck.nrays + ray] = make_float4(st.dv[0], st.dv[1], st.dv[2], st.cr[1]);
                state[(c * 3 + 2) * ck.nrays + ray] = make_float4(st.cv[0], st.cv[1], st.cv[2], st.cr[2]);
            }
            float B[3], C[3], q[3], inc_r[3], inc_v[3];
            long long U2[3], U3[3];
            for (int a = 0; a < 3; ++a) {
                q[a] = st.dr[a] + (0.5f * dt) * st.dv[a] + (0.125f * dt) * A[a];
                U2[a] = st.U[a] + k.dUh[a];
                U3[a] = st.U[a] + k.dU[a];
            }
            rhs_of(eval(U2, q, bc, ci, cf), D);
            for (int a = 0; a < 3; ++a) B[a] = dt * D[a];
            for (int a = 0; a < 3; ++a) {
                q[a] = st.dr[a] + dt * st.dv[a] + (0.5f * dt) * B[a];
                inc_r[a] = dt * (st.dv[a] + (A[a] + 2.0f * B[a]) * (1.0f / 6.0f));
            }
            float dr1[3], cr1[3];
            for (int a = 0; a < 3; ++a) {
                dr1[a] = st.dr[a];
                cr1[a] = st.cr[a];
                kahan_add(dr1[a], cr1[a], inc_r[a]);
            }
            // independent: stage 3 of this step and stage 1 of the next
            float D1[3] = {0.0f, 0.0f, 0.0f};
            rhs_of(eval(U3, q, bc, ci, cf), D);
            if (n + 1 < R.N) {
                int ci1[3];
                float cf1[3];
                rhs_of(eval(U3, dr1, bc1, ci1, cf1), D1);
            }
            for (int a = 0; a < 3; ++a) {
                C[a] = dt * D[a];
                inc_v[a] = (A[a] + 4.0f * B[a] + C[a]) * (1.0f / 6.0f);
            }
            float si = k.dS[0] * inc_r[0] + k.dS[1] * inc_r[1] + k.dS[2] * inc_r[2];
            float ii = inc_r[0] * inc_r[0] + inc_r[1] * inc_r[1] + inc_r[2] * inc_r[2];
            float di = k.dhat[0] * inc_r[0] + k.dhat[1] * inc_r[1] + k.dhat[2] * inc_r[2];
            st.excess += __fdividef(2.0f * si + ii, 2.0f * k.step_len + di);
            for (int a = 0; a < 3; ++a) {
                st.dr[a] = dr1[a];
                st.cr[a] = cr1[a];
                kahan_add(st.dv[a], st.cv[a], inc_v[a]);
                st.U[a] = U3[a];
                A[a] = dt * D1[a];
            }
        }
    } else {
        for (int n = 0; n < R.N; ++n) {
            if (state != nullptr && n % K == 0) {
                const size_t c = bounded((size_t)(n / K), (size_t)ck.max_ckpt, ck.err);
                state[(c * 3 + 0) * ck.nrays + ray] = make_float4(st.dr[0], st.dr[1], st.dr[2], st.cr[0]);
                state[(c * 3 + 1) * ck.nrays + ray] = make_float4(st.dv[0], st.dv[1], st.dv[2], st.cr[1]);
                state[(c * 3 + 2) * ck.nrays + ray] = make_float4(st.cv[0], st.cv[1], st.cv[2], st.cr[2]);
            }
            comp_step<E, INTEG>(F, st, k, bc);
        }
    }
}

__device__ __forceinline__ void comp_end(const CompState& st, float dr[3], float dv[3]) {
    for (int a = 0; a < 3; ++a) {
        dr[a] = st.dr[a] - st.cr[a];
        dv[a] = st.dv[a] - st.cv[a];
    }
}

// Trace one camera ray of the comp path (checkpoints every K steps when ck.state is set).
// With CONN (light mode 2) the luminance is read at the refracted projector connection of
// the wall point x_w = x_ref + dx: M rounds of a <- a + (x_w - y(a)) from a = x_w, y(a) the
// wall hit of the projector ray aimed at a (traced like a camera ray), so that
// a = x_ref + e with e <- dx - (y(a) - (P + t_w d_p)) - ((P + t_w d_p) - a).
template <class E, int INTEG, bool CONN>
__device__ RayResult trace_comp(const SceneDev& S, const CompField<E>& F, const Ray& R, const CkptDev& ck,
                                long long ray, bool want_hit, unsigned long long& steps) {
    WallRel h;
    if (R.N > 0) {
        CompState st;
        double eta_in;
        comp_run<E, INTEG, !CONN>(S, F, S.cam.pos, R, ck, ck.state, ray, st, eta_in);
        if (ck.state != nullptr) ck.excess[ray] = st.excess;
        steps += (unsigned long long)R.N;
        float dr[3], dv[3];
        comp_end(st, dr, dv);
        h = comp_wall(S, R, eta_in, dr, dv, st.excess);
    } else {   // straight camera ray (only with CONN: the projector rays may still bend)
        h.dx[0] = h.dx[1] = h.dx[2] = 0.0f;
        h.cosw = (float)(R.d[0] * S.w.normal[0] + R.d[1] * S.w.normal[1] + R.d[2] * S.w.normal[2]);
        h.len = (float)R.tw;
        h.valid = h.cosw > 0.0f;
        if (ck.state != nullptr) ck.excess[ray] = 0.0f;
    }
    float e[3] = {h.dx[0], h.dx[1], h.dx[2]};
    if constexpr (CONN) {
        if (h.valid) {
            double xref[3];
            for (int a = 0; a < 3; ++a) xref[a] = S.cam.pos[a] + R.tw * R.d[a];
            const double* P = S.L.proj.pos;
            for (int m = 0; m < S.L.connect_iters; ++m) {
                const Ray Rp = projector_setup(S, xref, e);
                float yrel[3] = {0.0f, 0.0f, 0.0f};
                if (Rp.wall && Rp.N > 0) {
                    CompState sp;
                    double eta_p;
                    comp_run<E, INTEG, !CONN>(S, F, P, Rp, ck, m == 0 ? ck.pstate : nullptr, ray, sp, eta_p);
                    steps += (unsigned long long)Rp.N;
                    float pr[3], pv[3];
                    comp_end(sp, pr, pv);
                    const WallRel hp = comp_wall(S, Rp, eta_p, pr, pv, 0.0f);
                    if (hp.valid)
                        for (int a = 0; a < 3; ++a) yrel[a] = hp.dx[a];
                }
                for (int a = 0; a < 3; ++a) {
                    const double eps = (xref[a] + (double)e[a]) - (P[a] + Rp.tw * Rp.d[a]);
                    e[a] = (h.dx[a] - yrel[a]) + (float)eps;
                }
            }
        }
        if (ck.conn != nullptr) {   // (a zero cosine factor marks a ray that misses the wall)
            ck.conn[2 * ray] = make_float4(h.dx[0], h.dx[1], h.dx[2], h.valid ? h.cosw / h.len : 0.0f);
            ck.conn[2 * ray + 1] = make_float4(h.dx[0] - e[0], h.dx[1] - e[1], h.dx[2] - e[2], 0.0f);
        }
    }
    return comp_finish(S, R, h, e, want_hit);
}

// Plain FP32 / FP64 tracer.  For the float64 adjoint (T = double, Sharma RKN) the state
// (r, v) is kept every K steps as six doubles, plane q of checkpoint c at
// ((c * 6 + q) * nrays + ray) of ck.state, and the path length of the traced steps per ray
// in ck.excess (as a double).
template <class T, int INTEG>
__device__ RayResult trace_full(const SceneDev& S, const FullField<T>& F, const Ray& R, const CkptDev& ck,
                                long long ray) {
    T r[3], v[3];
    double rin[3];
    double* const save = (sizeof(T) == 8 && INTEG == 0) ? reinterpret_cast<double*>(ck.state) : nullptr;
    for (int a = 0; a < 3; ++a) {
        rin[a] = S.cam.pos[a] + R.t_in * R.d[a];
        r[a] = (T)rin[a];
    }
    T eta_in = F.eta(r);
    for (int a = 0; a < 3; ++a) v[a] = eta_in * (T)R.d[a];
    T dt = (T)R.ell / ((T)R.N * eta_in);
    T lensum = 0;
    const T rl[3] = {r[0], r[1], r[2]}, v0[3] = {v[0], v[1], v[2]};
    for (int n = 0; n < R.N; ++n) {
        if (save != nullptr && n % ck.every == 0) {
            const size_t c = bounded((size_t)(n / ck.every), (size_t)ck.max_ckpt, ck.err);
            for (int q = 0; q < 3; ++q) {
                save[(c * 6 + q) * ck.nrays + ray] = (double)r[q];
                save[(c * 6 + 3 + q) * ck.nrays + ray] = (double)v[q];
            }
        }
        T r0[3] = {r[0], r[1], r[2]};
        if constexpr (INTEG == 2) {
            // quasi-linear: the field on the straight line at the start, middle and end of the step
            T A[3], B[3], C[3], p[3], D[3];
            for (int a = 0; a < 3; ++a) p[a] = rl[a] + ((T)n * dt) * v0[a];
            F.rhs(p, D);
            for (int a = 0; a < 3; ++a) A[a] = dt * D[a];
            for (int a = 0; a < 3; ++a) p[a] = rl[a] + (((T)n + T(0.5)) * dt) * v0[a];
            F.rhs(p, D);
            for (int a = 0; a < 3; ++a) B[a] = dt * D[a];
            for (int a = 0; a < 3; ++a) p[a] = rl[a] + (((T)n + T(1)) * dt) * v0[a];
            F.rhs(p, D);
            for (int a = 0; a < 3; ++a) C[a] = dt * D[a];
            for (int a = 0; a < 3; ++a) {
                r[a] = r[a] + dt * (v[a] + (A[a] + T(2) * B[a]) / T(6));
                v[a] = v[a] + (A[a] + T(4) * B[a] + C[a]) / T(6);
            }
        } else {
            full_step<T, INTEG>(F, r, v, dt);
        }
        T d0 = r[0] - r0[0], d1 = r[1] - r0[1], d2 = r[2] - r0[2];
        lensum += sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
    if (save != nullptr) reinterpret_cast<double*>(ck.excess)[ray] = (double)lensum;
    double rN[3] = {(double)r[0], (double)r[1], (double)r[2]};
    double vN[3] = {(double)v[0], (double)v[1], (double)v[2]};
    return wall_epilogue(S, S.cam.pos, R, rN, vN, R.t_in + (double)lensum);
}

template <int MODE>   // 0 straight, 1 comp fp32, 2 comp bf16, 3 full fp32, 4 full fp64
struct Tracer;

template <int MODE, int INTEG, bool CONN>
__device__ __forceinline__ RayResult trace_ray(const SceneDev& S, const Ray& R, const CkptDev& ck, long long ray,
                                               bool want_hit, unsigned long long& steps) {
    if constexpr (MODE == 0) {
        return straight_epilogue(S, R, want_hit);
    } else if constexpr (MODE == 1) {
        const CompField<F4P> F = comp_field<F4P>(S.g);
        return trace_comp<F4P, INTEG, CONN>(S, F, R, ck, ray, want_hit, steps);
    } else if constexpr (MODE == 2) {
        const CompField<B4P> F = comp_field<B4P>(S.g);
        return trace_comp<B4P, INTEG, CONN>(S, F, R, ck, ray, want_hit, steps);
    } else if constexpr (MODE == 3) {
        FullField<float> F = {S.g};
        steps += (unsigned long long)R.N;
        return trace_full<float, INTEG>(S, F, R, ck, ray);
    } else {
        FullField<double> F = {S.g};
        steps += (unsigned long long)R.N;
        return trace_full<double, INTEG>(S, F, R, ck, ray);
    }
}

#ifndef BOS_FWD_MIN_BLOCKS
#define BOS_FWD_MIN_BLOCKS 6              // resident 128-thread blocks per SM the register budget is cut for
#endif
#ifndef BOS_FWD_CACHED_MIN_BLOCKS
#define BOS_FWD_CACHED_MIN_BLOCKS 5       // the same for the Sharma tracer on the paired stores, whose cell
#endif                                    // cache holds 32 more values per ray (96 registers)
#ifndef BOS_FWD_QUASI_MIN_BLOCKS
#define BOS_FWD_QUASI_MIN_BLOCKS 3        // the same for quasi-linear tracing (more registers, more overlap)
#endif
constexpr int render_min_blocks(int mode, int integ, bool conn) {
    return integ == 2 ? BOS_FWD_QUASI_MIN_BLOCKS
                      : ((mode == 1 || mode == 2) && integ == 0 && !conn && BOS_FWD_PIPELINE) ? BOS_FWD_CACHED_MIN_BLOCKS
                                                                                             : BOS_FWD_MIN_BLOCKS;
}
// One warp tile of a render: the rays of its (up to) 32 lanes, averaged per pixel, written
// to the outputs; adds the traced ray-steps to my_steps.
template <int MODE, int INTEG, bool CONN>
__device__ __forceinline__ void render_tile(const SceneDev& S, const RenderOut& out, const WorkDev& wk,
                                            const CkptDev& ck, const TileShape& ts, int t, int lane,
                                            unsigned long long& my_steps) {
    const int spp = S.cam.spp;
    const int sl = lane % ts.G;
    const TilePix tp = tile_pixel(S, ts, t, lane);
    if (tp.bad) flag_error(wk.err, DEV_BAD_PIXEL);
    const int px = tp.px, py = tp.py;
    const bool valid = tp.valid;
    Sums acc = {0, 0, 0, 0, 0};
    if (valid) {
        for (int q = 0; q < ts.samples_per_lane; ++q) {
            const int s = ts.samples_per_lane == 1 ? sl : q;
            const long long ray = ((long long)t * 32 + lane) * ts.samples_per_lane + q;   // checkpoint slot
            Ray R = ray_setup<MODE != 0>(S, px, py, s);
            if (!R.wall) continue;
            if (R.N < 0) {
                flag_error(wk.err, DEV_STEP_BUDGET);
                continue;
            }
            RayResult r;
            if (MODE == 0 || (R.N == 0 && !CONN)) {
                r = straight_epilogue(S, R, out.hit != nullptr);
                if (MODE != 0 && R.N == 0 && ck.state != nullptr) {
                    if (MODE == 4) reinterpret_cast<double*>(ck.excess)[ray] = 0.0;
                    else ck.excess[ray] = 0.0f;
                }
            } else {
                r = trace_ray<MODE, INTEG, CONN>(S, R, ck, ray, out.hit != nullptr, my_steps);
            }
            acc.I += r.I;
            acc.du += r.disp[0];
            acc.dv += r.disp[1];
            acc.hu += r.hit[0];
            acc.hv += r.hit[1];
        }
    }
    for (int m = 1; m < ts.G; m <<= 1) {
        acc.I += __shfl_xor_sync(0xffffffffu, acc.I, m);
        acc.du += __shfl_xor_sync(0xffffffffu, acc.du, m);
        acc.dv += __shfl_xor_sync(0xffffffffu, acc.dv, m);
        acc.hu += __shfl_xor_sync(0xffffffffu, acc.hu, m);
        acc.hv += __shfl_xor_sync(0xffffffffu, acc.hv, m);
    }
    if (valid && sl == 0) {
        const size_t p = (size_t)tp.out;
        const double inv = 1.0 / spp;
        out.I[p] = (float)(acc.I * inv);
        if (out.disp) {
            out.disp[2 * p] = (float)(acc.du * inv);
            out.disp[2 * p + 1] = (float)(acc.dv * inv);
        }
        if (out.hit) {
            out.hit[2 * p] = acc.hu * inv;
            out.hit[2 * p + 1] = acc.hv * inv;
        }
    }
}

__device__ __forceinline__ void add_steps(unsigned long long* steps, unsigned long long my_steps, int lane) {
    for (int m = 16; m >= 1; m >>= 1) my_steps += __shfl_xor_sync(0xffffffffu, my_steps, m);
    if (lane == 0 && my_steps) atomicAdd(steps, my_steps);
}

// FEW: the form for launches with few warp tiles (a pixel minibatch), without a register
// cap: the GPU is not full either way, and each ray finishes sooner without spills.
template <int MODE, int INTEG, bool CONN, bool FEW = false>
__global__ void __launch_bounds__(128, FEW ? 1 : render_min_blocks(MODE, INTEG, CONN))
    render_kernel(SceneDev S, RenderOut out, WorkDev wk, CkptDev ck) {
    const TileShape ts = tile_shape(S.cam.width, S.cam.height, S.cam.spp);
    const int ntiles = tile_count(S, ts);
    const int lane = threadIdx.x & 31;
    unsigned long long my_steps = 0;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(wk.tile_counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        render_tile<MODE, INTEG, CONN>(S, out, wk, ck, ts, t, lane, my_steps);
    }
    add_steps(wk.steps, my_steps, lane);
}

// Batched render: one launch covers warp tiles of several requests' renders (the request
// server's continuous batching).  Work item g belongs to job j with jobs[j].first <= g <
// jobs[j + 1].first and is that job's tile jobs[j].tile0 + (g - jobs[j].first).  Warps
// pull items in order, so the jobs' tiles are interleaved as they are listed.
template <int MODE, int INTEG>
__global__ void __launch_bounds__(128, render_min_blocks(MODE, INTEG, false))
    render_batch_kernel(const BatchJob* __restrict__ jobs, int njobs, int total, int* counter) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(counter, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= total) break;
        const int j = batch_job_of(jobs, njobs, g);
        const BatchJob& J = jobs[j];
        const TileShape ts = tile_shape(J.S.cam.width, J.S.cam.height, J.S.cam.spp);
        unsigned long long my_steps = 0;
        render_tile<MODE, INTEG, false>(J.S, J.out, J.wk, J.ck, ts, J.tile0 + (g - J.first), lane, my_steps);
        add_steps(J.wk.steps, my_steps, lane);
    }
}

// ===================================================================== small kernels

__global__ void ray_steps_kernel(SceneDev S, int32_t* __restrict__ nsteps) {
    const long long nrays = (long long)S.cam.width * S.cam.height * S.cam.spp;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrays;
         r += (long long)gridDim.x * blockDim.x) {
        long long pix = r / S.cam.spp;
        int s = (int)(r % S.cam.spp);
        Ray R = ray_setup(S, (int)(pix % S.cam.width), (int)(pix / S.cam.width), s);
        nsteps[r] = R.wall ? R.N : 0;
    }
}

__device__ __forceinline__ float4 node_record(const F4P& p) { return p.v; }
__device__ __forceinline__ uint2 node_record(const B4P& p) { return p.a; }
__device__ __forceinline__ D4 node_record(const D4& p) { return p; }

template <class R>
__global__ void export_nodes_kernel(GridDev g, R* __restrict__ out) {
    using E = typename StoreElem<R>::type;
    const long long n = (long long)g.n[0] * g.n[1] * g.n[2];
    const E* st = static_cast<const E*>(g.store);
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]), k = (int)(c / ((long long)g.n[0] * g.n[1]));
        // read node (i, j, k) as a corner of the cell whose base is clamped to n-2
        int bi = min(i, g.n[0] - 2), bj = min(j, g.n[1] - 2), bk = min(k, g.n[2] - 2);
        uint32_t o = brick_offset(bi, bj, bk) + (uint32_t)((k - bk) * 81 + (j - bj) * 9 + (i - bi));
        out[c] = node_record(st[o]);
    }
}

__global__ void loss_l2_kernel(const float* __restrict__ I, const float* __restrict__ target, long long n,
                               double* loss, float* __restrict__ dLdI) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double r = (double)target[i] - (double)I[i];     // exact for two floats
        acc += r * r;
        if (dLdI) dLdI[i] = -2.0f * (target[i] - I[i]);
    }
    for (int m = 16; m >= 1; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
    __shared__ double part[32];
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) part[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += part[i];
        atomicAdd(loss, s);
    }
}

// ===================================================================== measurement probe

// Streams `n4` float4 of an L2-resident buffer `repeats` times (grid-stride, L1 bypassed)
// and folds them into a register; measures the L2 read bandwidth.
__global__ void probe_read_kernel(const float4* __restrict__ buf, long long n4, int repeats, float* sink) {
    float acc = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < repeats; ++r)
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            float4 v = __ldcg(buf + i);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    if (acc == 1234.5678f) sink[0] = acc;
}

cudaError_t launch_probe_read(const void* buf, long long bytes, int repeats, float* sink, int num_sms,
                              cudaStream_t st) {
    probe_read_kernel<<<num_sms * 8, 256, 0, st>>>((const float4*)buf, bytes / 16, repeats, sink);
    return cudaGetLastError();
}

// ===================================================================== launchers

cudaError_t launch_build_store(const GridDev& g, const float* T, void* store, cudaStream_t st) {
    const unsigned blocks = (unsigned)g.nb[0] * g.nb[1] * g.nb[2];
    switch (g.prec) {
        case 0: build_store_kernel<D4><<<blocks, 256, 0, st>>>(g, T, (D4*)store); break;
        case 3: build_store_kernel<uint2><<<blocks, 256, 0, st>>>(g, T, (B4P*)store); break;
        default: build_store_kernel<float4><<<blocks, 256, 0, st>>>(g, T, (F4P*)store); break;
    }
    return cudaGetLastError();
}

template <int MODE, int INTEG, bool CONN, bool FEW = false>
static cudaError_t launch_render_c(const SceneDev& S, const RenderOut& o, const WorkDev& w, const CkptDev& ck,
                                   int num_sms, cudaStream_t st) {
    int per_sm = 0;
    cudaError_t e = occupancy_prefer_l1(render_kernel<MODE, INTEG, CONN, FEW>, 128, 0, per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    render_kernel<MODE, INTEG, CONN, FEW><<<num_sms * per_sm, 128, 0, st>>>(S, o, w, ck);
    return cudaGetLastError();
}

// The refracted projector connection (light mode 2) has its own instantiation for the
// compensated tracers; the straight reference render and the plain tracers do not use it.
template <int MODE, int INTEG>
static cudaError_t launch_render_t(const SceneDev& S, const RenderOut& o, const WorkDev& w, const CkptDev& ck,
                                   int num_sms, cudaStream_t st) {
    if constexpr (MODE == 1 || MODE == 2) {
        if (S.L.mode == 2) return launch_render_c<MODE, INTEG, true>(S, o, w, ck, num_sms, st);
        // quasi-linear tracing of a few tiles (up to 8 warps per SM): the uncapped form
        if constexpr (INTEG == 2) {
            if (tile_count(S, tile_shape(S.cam.width, S.cam.height, S.cam.spp)) <= num_sms * 8)
                return launch_render_c<MODE, INTEG, false, true>(S, o, w, ck, num_sms, st);
        }
    }
    return launch_render_c<MODE, INTEG, false>(S, o, w, ck, num_sms, st);
}

cudaError_t launch_render(int mode, const SceneDev& S, const RenderOut& o, const WorkDev& w, const CkptDev& ck,
                          int num_sms, cudaStream_t st) {
    const int integ = S.it.integrator;
#define BOS_CASE(M)                                                                        \
    case M:                                                                                \
        return integ == 1   ? launch_render_t<M, 1>(S, o, w, ck, num_sms, st)              \
               : integ == 2 ? launch_render_t<M, 2>(S, o, w, ck, num_sms, st)              \
                            : launch_render_t<M, 0>(S, o, w, ck, num_sms, st);
    switch (mode) {
        BOS_CASE(0)
        BOS_CASE(1)
        BOS_CASE(2)
        BOS_CASE(3)
        BOS_CASE(4)
        default: return cudaErrorInvalidValue;
    }
#undef BOS_CASE
}

template <int MODE, int INTEG>
static cudaError_t launch_render_batch_c(const BatchJob* jobs, int njobs, int total, int* counter, int num_sms,
                                         cudaStream_t st) {
    int per_sm = 0;
    cudaError_t e = occupancy_prefer_l1(render_batch_kernel<MODE, INTEG>, 128, 0, per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    render_batch_kernel<MODE, INTEG><<<num_sms * per_sm, 128, 0, st>>>(jobs, njobs, total, counter);
    return cudaGetLastError();
}

cudaError_t launch_render_batch(int mode, int integ, const BatchJob* jobs, int njobs, int total, int* counter,
                                int num_sms, cudaStream_t st) {
    if (mode == 1) return integ == 2 ? launch_render_batch_c<1, 2>(jobs, njobs, total, counter, num_sms, st)
                                     : launch_render_batch_c<1, 0>(jobs, njobs, total, counter, num_sms, st);
    if (mode == 2) return integ == 2 ? launch_render_batch_c<2, 2>(jobs, njobs, total, counter, num_sms, st)
                                     : launch_render_batch_c<2, 0>(jobs, njobs, total, counter, num_sms, st);
    return cudaErrorNotSupported;
}

cudaError_t launch_ray_steps(const SceneDev& S, int32_t* nsteps, int num_sms, cudaStream_t st) {
    ray_steps_kernel<<<num_sms * 8, 256, 0, st>>>(S, nsteps);
    return cudaGetLastError();
}

cudaError_t launch_export_nodes(const GridDev& g, void* out, int num_sms, cudaStream_t st) {
    switch (g.prec) {
        case 0: export_nodes_kernel<D4><<<num_sms * 8, 256, 0, st>>>(g, (D4*)out); break;
        case 3: export_nodes_kernel<uint2><<<num_sms * 8, 256, 0, st>>>(g, (uint2*)out); break;
        default: export_nodes_kernel<float4><<<num_sms * 8, 256, 0, st>>>(g, (float4*)out); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_loss_l2(const float* I, const float* target, long long n, double* loss, float* dLdI, int num_sms,
                           cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    loss_l2_kernel<<<num_sms * 4, 256, 0, st>>>(I, target, n, loss, dLdI);
    return cudaGetLastError();
}

}  // namespace bos
