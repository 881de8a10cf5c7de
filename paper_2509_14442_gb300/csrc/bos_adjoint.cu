// Adjoint of the BOS forward model (step a6, Sec. 2.4): dL/dT for a given dL/dI.
//
//   adjoint_kernel  -- per ray, reverse Sharma's steps segment by segment from the
//                      checkpoints the forward kept every K steps (each segment is
//                      recomputed forward into shared memory, then reversed), starting
//                      from the adjoint of the wall epilogue (luminance, cosine, path
//                      length of Eq. 2).  Each stage's field value and gradient come
//                      from one packed trilinear evaluation.  The sensitivities of the
//                      8 trilinear corners are summed per lane while the ray stays in a
//                      cell, and flushed into per-node accumulators (d L/d deta,
//                      d L/d grad eta) with warp-aggregated atomics: lanes whose rows
//                      belong to the same cell are summed in shared memory, so each
//                      (corner, channel) gets one atomic per cell visit per warp.
//   gradient_kernel -- per node: the transpose of the central-difference stencil applied
//                      to the grad-eta sensitivities, plus the deta sensitivity, times
//                      d deta/dT = -rho0 G T0 / T^2.  A gather, so it is deterministic.
#include "bos_comp.cuh"
#include "bos_device.cuh"
#include "bos_full.cuh"
#include "bos_internal.h"

namespace bos {

constexpr int kAdjWarps = kAdjWarpsPerBlock;   // warps per block
#ifndef BOS_ADJ_MIN_BLOCKS
#define BOS_ADJ_MIN_BLOCKS 5              // resident blocks per SM the register budget is cut for
#endif
#ifndef BOS_ADJ_QUASI_MIN_BLOCKS
#define BOS_ADJ_QUASI_MIN_BLOCKS 7        // the same for the quasi-linear adjoint (128 registers, 16 warps/SM),
#endif                                    // used when there are more than 12 warp tiles per SM
#ifndef BOS_ADJ_QUASI_SMALL_MIN_BLOCKS
#define BOS_ADJ_QUASI_SMALL_MIN_BLOCKS 1  // the quasi-linear adjoint for few tiles (no register cap)
#endif
constexpr int kRow = 36;              // floats per lane row of the cell accumulators (16-byte aligned rows)
constexpr int kConnDoubles = 20;      // per-lane shared doubles of the refracted connection's adjoint
constexpr uint32_t kNoKey = 0xffffffffu;

struct InterpGrad {
    float4 v, d0, d1, d2;   // value and derivatives with respect to the three fractions
};

__device__ __forceinline__ Cell2 subc(Cell2 a, Cell2 b) { return Cell2{sub2(a.lo, b.lo), sub2(a.hi, b.hi)}; }
__device__ __forceinline__ float4 to4(Cell2 c) {
    float4 v;
    unpack2(c.lo, v.x, v.y);
    unpack2(c.hi, v.z, v.w);
    return v;
}

// Value (same operations as `trilinear2`, so bit-identical) and its derivatives with respect
// to the three fractions, in packed f32x2 arithmetic.
template <class E>
__device__ __forceinline__ InterpGrad trilinear_grad2(const E* s, uint32_t o, float f0, float f1, float f2) {
    const f32x2 t0 = pack2(f0, f0), t1 = pack2(f1, f1), t2 = pack2(f2, f2);
    Cell2 a0, a1, a2, a3, e0, e1, e2, e3;   // x-interpolated corner pairs and their x differences
    xlerp(s, o, t0, a0, e0);
    xlerp(s, o + 9, t0, a1, e1);
    xlerp(s, o + 81, t0, a2, e2);
    xlerp(s, o + 90, t0, a3, e3);
    const Cell2 b0 = lerpc(a0, a1, t1), b1 = lerpc(a2, a3, t1);
    InterpGrad r;
    r.v = to4(lerpc(b0, b1, t2));
    r.d2 = to4(subc(b1, b0));
    r.d1 = to4(lerpc(subc(a1, a0), subc(a3, a2), t2));
    r.d0 = to4(lerpc(lerpc(e0, e1, t1), lerpc(e2, e3, t1), t2));
    return r;
}

struct Stage {
    uint32_t key;   // node index of the cell's base corner
    float cf[3];
    InterpGrad ig;
};

template <class E>
__device__ __forceinline__ uint32_t cell_key_of(const CompField<E>& F, const int ci[3]) {
    return (uint32_t)ci[0] + (uint32_t)ci[1] * (uint32_t)F.n[0] + (uint32_t)ci[2] * ((uint32_t)F.n[0] * (uint32_t)F.n[1]);
}

__device__ __forceinline__ void rhs_from(const InterpGrad& ig, float D[3]) {
    float eta = 1.0f + ig.v.x;
    D[0] = eta * ig.v.y;
    D[1] = eta * ig.v.z;
    D[2] = eta * ig.v.w;
}

template <class E>
__device__ __forceinline__ void stage_eval(const CompField<E>& F, const long long U[3], const float q[3], BrickCache& bc,
                                           Stage& s) {
    int ci[3];
    comp_cell(F, U, q, ci, s.cf);
    s.key = cell_key_of(F, ci);
    const uint32_t o = comp_offset(F, bc, ci);
    s.ig = trilinear_grad2(F.store, o, s.cf[0], s.cf[1], s.cf[2]);
}

// Adjoint of D = (1 + deta) grad at a stage point: given Db, the position adjoint (metres)
// and the per-corner record Q (corner c receives w_c Q).
template <class E>
__device__ __forceinline__ void rhs_adjoint(const CompField<E>& F, const InterpGrad& ig, const float Db[3], float pb[3],
                                            float4& Q) {
    const float eta = 1.0f + ig.v.x;
    const float Dg = Db[0] * ig.v.y + Db[1] * ig.v.z + Db[2] * ig.v.w;
    const float4 dv[3] = {ig.d0, ig.d1, ig.d2};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        pb[a] = F.inv_h[a] * (dv[a].x * Dg + eta * (Db[0] * dv[a].y + Db[1] * dv[a].z + Db[2] * dv[a].w));
    Q = make_float4(Dg, eta * Db[0], eta * Db[1], eta * Db[2]);
}

// Per-lane accumulation of corner sensitivities for the lane's current cell; the row
// (8 corners x 4 channels) lives in shared memory.  When a lane's stage point leaves the
// cell, the warp flushes: lanes whose rows belong to the same cell are summed column by
// column (lane l owns corner l/4, channel l%4) and each sum is one atomic.
struct CellAcc {
    uint32_t key;      // node index of the accumulated cell's base corner, kNoKey if empty
    uint32_t ncells;   // nodes of the accumulators (the checked build's bound)
    int* err;
};

__device__ __forceinline__ void flush_rows(float* rows, bool flag, CellAcc& ca, float* acc, int nx, int nxy) {
    unsigned pend = __ballot_sync(0xffffffffu, flag);
    if (!pend) return;
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const int corner = lane >> 2;
    const uint32_t off = (uint32_t)(corner & 1) + (uint32_t)((corner >> 1) & 1) * (uint32_t)nx +
                         (uint32_t)(corner >> 2) * (uint32_t)nxy;
    const uint32_t mykey = flag ? ca.key : kNoKey;
    while (pend) {
        const int leader = __ffs(pend) - 1;
        const uint32_t lk = __shfl_sync(0xffffffffu, mykey, leader);
        const unsigned grp = __ballot_sync(0xffffffffu, mykey == lk);
        pend &= ~grp;
        // column sum over the group's rows, sixteen rows at a time with independent loads
        // and a pairwise tree (warp tiles are coherent, so a group is often the whole warp)
        float sum = 0.0f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const unsigned part = (grp >> (16 * q)) & 0xffffu;
            if (part) {
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = (part >> i) & 1u ? rows[(16 * q + i) * kRow + lane] : 0.0f;
#pragma unroll
                for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
                    for (int i = 0; i < w; ++i) v[i] += v[i + w];
                sum += v[0];
            }
        }
        if (sum != 0.0f) atomicAdd(acc + ((size_t)bounded(lk + off, ca.ncells, ca.err) << 2) + (lane & 3), sum);
    }
    __syncwarp();
    if (flag) {
        float4* row = reinterpret_cast<float4*>(rows + lane * kRow);
#pragma unroll
        for (int c = 0; c < 8; ++c) row[c] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        ca.key = kNoKey;
    }
    __syncwarp();
}

// Warp-collective: add w_c(cf) Q to the lane's cell row (flushing first where the cell changes).
__device__ __forceinline__ void accumulate(float* rows, bool act, uint32_t cell, const float cf[3], float4 Q,
                                           CellAcc& ca, float* acc, int nx, int nxy) {
    const int lane = threadIdx.x & 31;
    const uint32_t key = act ? cell : kNoKey;
    flush_rows(rows, act && ca.key != kNoKey && ca.key != key, ca, acc, nx, nxy);
    if (act) {
        ca.key = key;
        float4* row = reinterpret_cast<float4*>(rows + lane * kRow);
        const float g0 = 1.0f - cf[0], g1 = 1.0f - cf[1], g2 = 1.0f - cf[2];
        const f32x2 qlo = pack2(Q.x, Q.y), qhi = pack2(Q.z, Q.w);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float w = ((c & 1) ? cf[0] : g0) * ((c & 2) ? cf[1] : g1) * ((c & 4) ? cf[2] : g2);
            const f32x2 ww = pack2(w, w);
            float4 r = row[c];
            f32x2 lo = fma2(ww, qlo, pack2(r.x, r.y)), hi = fma2(ww, qhi, pack2(r.z, r.w));
            unpack2(lo, r.x, r.y);
            unpack2(hi, r.z, r.w);
            row[c] = r;
        }
    }
}

// Warp-collective: add w_c(cf) Q and, where `dual`, then w_c(cf2) Q2 (a second sample in
// the same cell) to the lane's cell row: the same two FMAs per value, in the same order, as
// two calls of `accumulate`, with one read and one write of the row.
__device__ __forceinline__ void accumulate_dual(float* rows, bool act, uint32_t cell, const float cf[3], float4 Q,
                                                bool dual, const float cf2[3], float4 Q2, CellAcc& ca, float* acc,
                                                int nx, int nxy) {
    const int lane = threadIdx.x & 31;
    const uint32_t key = act ? cell : kNoKey;
    flush_rows(rows, act && ca.key != kNoKey && ca.key != key, ca, acc, nx, nxy);
    if (act) {
        ca.key = key;
        float4* row = reinterpret_cast<float4*>(rows + lane * kRow);
        const float g0 = 1.0f - cf[0], g1 = 1.0f - cf[1], g2 = 1.0f - cf[2];
        const float h0 = 1.0f - cf2[0], h1 = 1.0f - cf2[1], h2 = 1.0f - cf2[2];
        const f32x2 qlo = pack2(Q.x, Q.y), qhi = pack2(Q.z, Q.w);
        const f32x2 q2lo = pack2(Q2.x, Q2.y), q2hi = pack2(Q2.z, Q2.w);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float w = ((c & 1) ? cf[0] : g0) * ((c & 2) ? cf[1] : g1) * ((c & 4) ? cf[2] : g2);
            const f32x2 ww = pack2(w, w);
            float4 r = row[c];
            f32x2 lo = fma2(ww, qlo, pack2(r.x, r.y)), hi = fma2(ww, qhi, pack2(r.z, r.w));
            if (dual) {
                const float v = ((c & 1) ? cf2[0] : h0) * ((c & 2) ? cf2[1] : h1) * ((c & 4) ? cf2[2] : h2);
                const f32x2 vv = pack2(v, v);
                lo = fma2(vv, q2lo, lo);
                hi = fma2(vv, q2hi, hi);
            }
            unpack2(lo, r.x, r.y);
            unpack2(hi, r.z, r.w);
            row[c] = r;
        }
    }
}

// Warp-collective: add w_c(cf) Q and, where with2 / with1, w_c(cf2) Q2 and w_c(cf1) Q1 (other
// samples in the same cell) to the lane's cell row, in one read and one write of the row.
__device__ __forceinline__ void accumulate3(float* rows, bool act, uint32_t cell, const float cf[3], float4 Q,
                                            bool with2, const float cf2[3], float4 Q2, bool with1, const float cf1[3],
                                            float4 Q1, CellAcc& ca, float* acc, int nx, int nxy) {
    const int lane = threadIdx.x & 31;
    const uint32_t key = act ? cell : kNoKey;
    flush_rows(rows, act && ca.key != kNoKey && ca.key != key, ca, acc, nx, nxy);
    if (act) {
        ca.key = key;
        float4* row = reinterpret_cast<float4*>(rows + lane * kRow);
        const f32x2 qlo = pack2(Q.x, Q.y), qhi = pack2(Q.z, Q.w);
        const f32x2 q2lo = pack2(Q2.x, Q2.y), q2hi = pack2(Q2.z, Q2.w);
        const f32x2 q1lo = pack2(Q1.x, Q1.y), q1hi = pack2(Q1.z, Q1.w);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float w = ((c & 1) ? cf[0] : 1.0f - cf[0]) * ((c & 2) ? cf[1] : 1.0f - cf[1]) *
                            ((c & 4) ? cf[2] : 1.0f - cf[2]);
            const float w2 = with2 ? ((c & 1) ? cf2[0] : 1.0f - cf2[0]) * ((c & 2) ? cf2[1] : 1.0f - cf2[1]) *
                                         ((c & 4) ? cf2[2] : 1.0f - cf2[2])
                                   : 0.0f;
            const float w1 = with1 ? ((c & 1) ? cf1[0] : 1.0f - cf1[0]) * ((c & 2) ? cf1[1] : 1.0f - cf1[1]) *
                                         ((c & 4) ? cf1[2] : 1.0f - cf1[2])
                                   : 0.0f;
            float4 r = row[c];
            f32x2 lo = fma2(pack2(w, w), qlo, pack2(r.x, r.y)), hi = fma2(pack2(w, w), qhi, pack2(r.z, r.w));
            lo = fma2(pack2(w2, w2), q2lo, lo);
            hi = fma2(pack2(w2, w2), q2hi, hi);
            lo = fma2(pack2(w1, w1), q1lo, lo);
            hi = fma2(pack2(w1, w1), q1hi, hi);
            unpack2(lo, r.x, r.y);
            unpack2(hi, r.z, r.w);
            row[c] = r;
        }
    }
}

// Adjoint of the wall epilogue for seed Ib = dL/dI of this ray: returns the adjoints of
// (r_N, v_N) and of the path length (which the per-step lengths feed).
// With the refracted projector connection the luminance is read at xl (not at x_w) and
// its sensitivity to x_w arrives as xlb; otherwise xl = xlb = nullptr.
__device__ __forceinline__ void wall_adjoint(const SceneDev& S, const double rN[3], const double vN[3],
                                             double len_before, double Ib, double rb[3], double vb[3],
                                             double& lenb, const double* xl = nullptr, const double* xlb = nullptr) {
    const WallDev& w = S.w;
    rb[0] = rb[1] = rb[2] = vb[0] = vb[1] = vb[2] = 0.0;
    lenb = 0.0;
    double vn = vN[0] * w.normal[0] + vN[1] * w.normal[1] + vN[2] * w.normal[2];
    if (!(vn > 0.0)) return;
    double q[3] = {w.origin[0] - rN[0], w.origin[1] - rN[1], w.origin[2] - rN[2]};
    double ts = (q[0] * w.normal[0] + q[1] * w.normal[1] + q[2] * w.normal[2]) / vn;
    double xw[3];
    for (int a = 0; a < 3; ++a) xw[a] = rN[a] + ts * vN[a];
    double vl = sqrt(vN[0] * vN[0] + vN[1] * vN[1] + vN[2] * vN[2]);
    double len = len_before + ts * vl;              // signed continuation x_w - r_N = t* v
    double cw = vn / vl;
    double gL[3];
    double Lw = xl ? wall_luminance(S.L, w, xl) : wall_luminance(S.L, w, xw, gL);
    double Lb = Ib * cw / len, cb = Ib * Lw / len;
    lenb = -Ib * Lw * cw / (len * len);
    double xwb[3];
    for (int a = 0; a < 3; ++a) {
        double u = vN[a] / vl;                      // d(t* |v|) through x_w = r_N + t* v
        xwb[a] = (xl ? xlb[a] : Lb * gL[a]) + lenb * u;
        rb[a] = -lenb * u;
        vb[a] = cb * (w.normal[a] / vl - vn * vN[a] / (vl * vl * vl));
    }
    double tb = xwb[0] * vN[0] + xwb[1] * vN[1] + xwb[2] * vN[2];
    for (int a = 0; a < 3; ++a) {
        rb[a] += xwb[a] - tb * w.normal[a] / vn;
        vb[a] += ts * xwb[a] - tb * ts * w.normal[a] / vn;
    }
}

// Adjoint of a projector ray's wall hit y = r_N + t* v_N, t* = ((o - r_N) . n) / (v_N . n),
// for the seed yb.
__device__ __forceinline__ void hit_adjoint(const SceneDev& S, const double rN[3], const double vN[3],
                                            const double yb[3], double rb[3], double vb[3]) {
    const WallDev& w = S.w;
    rb[0] = rb[1] = rb[2] = vb[0] = vb[1] = vb[2] = 0.0;
    double vn = vN[0] * w.normal[0] + vN[1] * w.normal[1] + vN[2] * w.normal[2];
    if (!(vn > 0.0)) return;
    double q[3] = {w.origin[0] - rN[0], w.origin[1] - rN[1], w.origin[2] - rN[2]};
    double ts = (q[0] * w.normal[0] + q[1] * w.normal[1] + q[2] * w.normal[2]) / vn;
    double tb = yb[0] * vN[0] + yb[1] * vN[1] + yb[2] * vN[2];
    for (int a = 0; a < 3; ++a) {
        rb[a] = yb[a] - tb * w.normal[a] / vn;
        vb[a] = ts * rb[a];
    }
}

// d/d aim of the straight projector ray's wall hit y = P + t_w d (d = q / |q|,
// t_w = ((o - P) . n) / (d . n)), for the seed yb.
__device__ __forceinline__ void straight_aim_adjoint(const SceneDev& S, const Ray& Rp, double nq, const double yb[3],
                                                     double ab[3]) {
    const WallDev& w = S.w;
    double den = Rp.d[0] * w.normal[0] + Rp.d[1] * w.normal[1] + Rp.d[2] * w.normal[2];
    double twb = yb[0] * Rp.d[0] + yb[1] * Rp.d[1] + yb[2] * Rp.d[2];
    double db[3];
    for (int a = 0; a < 3; ++a) db[a] = Rp.tw * yb[a] - twb * Rp.tw * w.normal[a] / den;
    double dd = db[0] * Rp.d[0] + db[1] * Rp.d[1] + db[2] * Rp.d[2];
    for (int a = 0; a < 3; ++a) ab[a] = (db[a] - dd * Rp.d[a]) / nq;
}

__host__ __device__ constexpr size_t adj_warp_floats(int K) {
    return (size_t)32 * kRow;   // K is carried by the global segment states
}

// Floats per lane and step of the recomputed segment: (dr, dv, A, B) of Sharma's step.
constexpr int kSegFloats = 12;

// One warp tile of the Sharma adjoint: reverse every ray of the tile from its checkpoints
// and scatter its sensitivities into the lane rows (flushed into acc as the cells change).
template <class E, bool CONN>
__device__ __forceinline__ void adjoint_tile(const SceneDev& S, const CkptDev& ck, const AdjDev& adj,
                                             const CompField<E>& F, const TileShape& ts, int t, int lane,
                                             float* rows, float* st_buf, float* acc, CellAcc& ca, double* xlum) {
    const int nx = S.g.n[0], nxy = S.g.n[0] * S.g.n[1];
    const int spp = S.cam.spp;
    const int K = ck.every;
    double* const xlb = xlum + 3;
    double* const ybar = xlum + 6;
    double* const drbw = xlum + 9;
    double* const dvbw = xlum + 12;
    double* const tpb = xlum + 15;
    double* const nqp = xlum + 18;
    const int sl = lane % ts.G;
    const TilePix tp = tile_pixel(S, ts, t, lane);
    const int px = tp.px, py = tp.py;
    const bool valid = tp.valid;
    for (int qs = 0; qs < ts.samples_per_lane; ++qs) {
        const int s = ts.samples_per_lane == 1 ? sl : qs;
        const long long slot = ((long long)t * 32 + lane) * ts.samples_per_lane + qs;
        bool act = valid;
        Ray R;
        R.N = 0;
        R.wall = false;
        double Ib = 0.0;
        if (act) {
            R = ray_setup(S, px, py, s);
            Ib = (double)adj.dLdI[(size_t)tp.out] / spp;
        }
        const bool act0 = act && R.wall && R.N >= 0 && Ib != 0.0;
        // Refracted projector connection (light mode 2, one aiming round): the luminance is
        // read at a_1 = 2 x_w - y(x_w), y the wall hit of the projector ray aimed at x_w.
        // Pass 0 reverses that projector ray for the seed -dL/da_1 and turns its entry state
        // into dL/d aim; pass 1 reverses the camera ray with dL/dx_w = 2 dL/da_1 + dL/d aim.
        Ray Rp;
        Rp.N = 0;
        Rp.wall = false;
        bool pact = false;
        if constexpr (CONN) {
            for (int a = 0; a < 3; ++a) xlum[a] = xlb[a] = ybar[a] = 0.0;
            nqp[0] = 1.0;
            if (act0) {
                const float4 c0 = ck.conn[2 * slot], c1 = ck.conn[2 * slot + 1];
                const float dxf[3] = {c0.x, c0.y, c0.z};
                double xref[3], gL[3], q[3];
                for (int a = 0; a < 3; ++a) {
                    xref[a] = S.cam.pos[a] + R.tw * R.d[a];
                    xlum[a] = xref[a] + ((double)dxf[a] - (double)(&c1.x)[a]);
                }
                const double Lb = Ib * (double)c0.w;
                wall_luminance(S.L, S.w, xlum, gL);
                for (int a = 0; a < 3; ++a) {
                    ybar[a] = -Lb * gL[a];
                    xlb[a] = 2.0 * Lb * gL[a];
                    q[a] = (xref[a] - S.L.proj.pos[a]) + (double)dxf[a];
                }
                nqp[0] = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
                Rp = projector_setup(S, xref, dxf);
                const bool seeded = ybar[0] != 0.0 || ybar[1] != 0.0 || ybar[2] != 0.0;
                if (!Rp.wall) {                 // y = aim
                    for (int a = 0; a < 3; ++a) xlb[a] += ybar[a];
                } else if (Rp.N <= 0) {         // straight projector ray
                    double ab[3];
                    straight_aim_adjoint(S, Rp, nqp[0], ybar, ab);
                    for (int a = 0; a < 3; ++a) xlb[a] += ab[a];
                } else {
                    pact = seeded;
                }
            }
        }
        for (int pass = CONN ? 0 : 1; pass < 2; ++pass) {
        const bool proj = CONN && pass == 0;
        const Ray& RR = proj ? Rp : R;
        const double* rs = proj ? S.L.proj.pos : S.cam.pos;
        const float4* cstate = proj ? ck.pstate : ck.state;
        act = proj ? pact : (act0 && R.N > 0);
        CompState st0;
        CompConst k;
        double eta_in = 1.0, rin[3] = {0, 0, 0};
        if (act) comp_setup(S, F, rs, RR, st0, k, eta_in, rin);
        const int N = act ? RR.N : 0;
        const int nseg = (N + K - 1) / K;
        const int nseg_max = __reduce_max_sync(0xffffffffu, (unsigned)nseg);
        float rb[3] = {0, 0, 0}, vb[3] = {0, 0, 0}, dtb = 0.0f, lenb = 0.0f;
        double etab = 0.0;
        if constexpr (CONN)
            for (int a = 0; a < 3; ++a) tpb[a] = 0.0;
        const float dt = act ? k.dt : 0.0f;
        BrickCache bc = {kNoKey, 0u};
        for (int c = nseg_max - 1; c >= 0; --c) {
            const int n0 = c * K;
            const int n1 = min(n0 + K, N);
            const bool seg = act && n0 < N;
            // ---- recompute the segment from its checkpoint, keeping each step's state
            if (seg) {
                CompState st;
                const size_t cc = bounded((size_t)c, (size_t)ck.max_ckpt, ck.err);
                const float4 s0 = cstate[(cc * 3 + 0) * ck.nrays + slot];
                const float4 s1 = cstate[(cc * 3 + 1) * ck.nrays + slot];
                const float4 s2 = cstate[(cc * 3 + 2) * ck.nrays + slot];
                st.dr[0] = s0.x; st.dr[1] = s0.y; st.dr[2] = s0.z;
                st.dv[0] = s1.x; st.dv[1] = s1.y; st.dv[2] = s1.z;
                st.cv[0] = s2.x; st.cv[1] = s2.y; st.cv[2] = s2.z;
                st.cr[0] = s0.w; st.cr[1] = s1.w; st.cr[2] = s2.w;
                st.excess = 0.0f;
                for (int a = 0; a < 3; ++a) st.U[a] = st0.U[a] + (long long)n0 * k.dU[a];
                for (int n = n0; n < n1; ++n) {
                    float* p = st_buf + (size_t)(n - n0) * kSegFloats * 32 + lane;
                    p[0] = st.dr[0]; p[32] = st.dr[1]; p[64] = st.dr[2];
                    p[96] = st.dv[0]; p[128] = st.dv[1]; p[160] = st.dv[2];
                    float AB[6];
                    comp_step<E, 0>(F, st, k, bc, AB);
                    for (int q = 0; q < 6; ++q) p[192 + 32 * q] = AB[q];
                }
                if (c == nseg - 1) {
                    // the lane's last segment: start from the adjoint of the wall epilogue
                    double rN[3], vN[3], drb[3], dvb[3], lb = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        rN[a] = rin[a] + RR.ell * RR.d[a] + ((double)st.dr[a] - (double)st.cr[a]);
                        vN[a] = eta_in * RR.d[a] + ((double)st.dv[a] - (double)st.cv[a]);
                    }
                    if (proj) {
                        hit_adjoint(S, rN, vN, ybar, drb, dvb);
                        for (int a = 0; a < 3; ++a) {
                            drbw[a] = drb[a];
                            dvbw[a] = dvb[a];
                        }
                    } else {
                        double len_before = R.t_in + R.ell + (double)ck.excess[slot];
                        wall_adjoint(S, rN, vN, len_before, Ib, drb, dvb, lb, CONN ? xlum : nullptr,
                                     CONN ? xlb : nullptr);
                    }
                    for (int a = 0; a < 3; ++a) {
                        rb[a] = (float)drb[a];
                        vb[a] = (float)dvb[a];
                    }
                    lenb = (float)lb;
                    etab += dvb[0] * RR.d[0] + dvb[1] * RR.d[1] + dvb[2] * RR.d[2];
                }
            }
            __syncwarp();
            const float rseg[3] = {rb[0], rb[1], rb[2]};   // rb before this segment's steps
            // ---- reverse the segment's steps
            const int n_hi = __reduce_max_sync(0xffffffffu, (unsigned)(seg ? n1 : 0));
            float tps[3] = {0.0f, 0.0f, 0.0f};   // sum over the segment's stages of (t / dt_step) pb
            for (int n = n_hi - 1; n >= n0; --n) {
                const bool a_ = seg && n < n1;
                // the step's state and stage terms from the recompute: all three stage
                // points are known, so each stage is evaluated (value and gradient) when
                // its adjoint is formed, in the order 3, 2, 1
                float dr[3] = {0, 0, 0}, dvv[3] = {0, 0, 0}, A[3] = {0, 0, 0}, B[3] = {0, 0, 0};
                if (a_) {
                    const float* p = st_buf + (size_t)(n - n0) * kSegFloats * 32 + lane;
                    dr[0] = p[0]; dr[1] = p[32]; dr[2] = p[64];
                    dvv[0] = p[96]; dvv[1] = p[128]; dvv[2] = p[160];
                    A[0] = p[192]; A[1] = p[224]; A[2] = p[256];
                    B[0] = p[288]; B[1] = p[320]; B[2] = p[352];
                }
                long long U[3];
                for (int a = 0; a < 3; ++a) U[a] = st0.U[a] + (long long)n * k.dU[a];
                float u[3] = {0, 0, 0};
                if (a_) {
                    float inc[3], nn = 0.0f;
                    for (int a = 0; a < 3; ++a) {
                        inc[a] = k.dS[a] + dt * (dvv[a] + (A[a] + 2.0f * B[a]) * (1.0f / 6.0f));
                        nn += inc[a] * inc[a];
                    }
                    const float rn = rsqrtf(nn);
                    for (int a = 0; a < 3; ++a) {
                        u[a] = inc[a] * rn;             // unit step direction: d|r_{n+1} - r_n|
                        rb[a] += lenb * u[a];
                    }
                }
                // r' = r + dt (v + (A + 2B)/6),  v' = v + (A + 4B + C)/6
                float Ab[3], Bb[3], Cb[3], rn_[3], vn_[3];
                for (int a = 0; a < 3; ++a) {
                    Ab[a] = (dt * (1.0f / 6.0f)) * rb[a] + vb[a] * (1.0f / 6.0f);
                    Bb[a] = (dt * (1.0f / 3.0f)) * rb[a] + vb[a] * (4.0f / 6.0f);
                    Cb[a] = vb[a] * (1.0f / 6.0f);
                    rn_[a] = rb[a];
                    vn_[a] = vb[a] + dt * rb[a];
                    dtb += rb[a] * (dvv[a] + (A[a] + 2.0f * B[a]) * (1.0f / 6.0f));
                }
                float Db[3], pb[3] = {0, 0, 0}, D[3] = {0, 0, 0}, q[3];
                long long Us[3];
                Stage s;
                float4 Q3 = make_float4(0, 0, 0, 0), Q2 = Q3, Q1 = Q3;
                uint32_t key3 = kNoKey, key2 = kNoKey, key1 = kNoKey;
                float cf3[3] = {0, 0, 0}, cf2[3] = {0, 0, 0}, cf1[3] = {0, 0, 0};
                // C = dt D(p3),  p3 = S(n+1) + dr + dt dv + dt/2 B
                if (a_) {
                    for (int a = 0; a < 3; ++a) {
                        q[a] = dr[a] + dt * dvv[a] + (0.5f * dt) * B[a];
                        Us[a] = U[a] + k.dU[a];
                    }
                    stage_eval(F, Us, q, bc, s);
                    rhs_from(s.ig, D);
                }
                for (int a = 0; a < 3; ++a) {
                    dtb += Cb[a] * D[a];
                    Db[a] = dt * Cb[a];
                }
                if (a_) {
                    rhs_adjoint(F, s.ig, Db, pb, Q3);
                    key3 = s.key;
                    for (int a = 0; a < 3; ++a) cf3[a] = s.cf[a];
                }
                if constexpr (CONN) {
                    const float tn = (float)(n + 1 - n0);
                    for (int a = 0; a < 3; ++a) tps[a] += tn * pb[a];
                }
                for (int a = 0; a < 3; ++a) {
                    rn_[a] += pb[a];
                    vn_[a] += dt * pb[a];
                    Bb[a] += (0.5f * dt) * pb[a];
                    dtb += pb[a] * (dvv[a] + 0.5f * B[a]);
                }
                // B = dt D(p2),  p2 = S(n+1/2) + dr + dt/2 dv + dt/8 A
                if (a_) {
                    for (int a = 0; a < 3; ++a) {
                        q[a] = dr[a] + (0.5f * dt) * dvv[a] + (0.125f * dt) * A[a];
                        Us[a] = U[a] + k.dUh[a];
                    }
                    stage_eval(F, Us, q, bc, s);
                    rhs_from(s.ig, D);
                }
                for (int a = 0; a < 3; ++a) {
                    dtb += Bb[a] * D[a];
                    Db[a] = dt * Bb[a];
                }
                if (a_) {
                    rhs_adjoint(F, s.ig, Db, pb, Q2);
                    key2 = s.key;
                    for (int a = 0; a < 3; ++a) cf2[a] = s.cf[a];
                }
                if constexpr (CONN) {
                    const float tn = (float)(n - n0) + 0.5f;
                    for (int a = 0; a < 3; ++a) tps[a] += tn * pb[a];
                }
                for (int a = 0; a < 3; ++a) {
                    rn_[a] += pb[a];
                    vn_[a] += (0.5f * dt) * pb[a];
                    Ab[a] += (0.125f * dt) * pb[a];
                    dtb += pb[a] * (0.5f * dvv[a] + 0.125f * A[a]);
                }
                // A = dt D(p1),  p1 = S(n) + dr
                if (a_) {
                    stage_eval(F, U, dr, bc, s);
                    rhs_from(s.ig, D);
                }
                for (int a = 0; a < 3; ++a) {
                    dtb += Ab[a] * D[a];
                    Db[a] = dt * Ab[a];
                }
                if (a_) {
                    rhs_adjoint(F, s.ig, Db, pb, Q1);
                    key1 = s.key;
                    for (int a = 0; a < 3; ++a) cf1[a] = s.cf[a];
                }
                if constexpr (CONN) {
                    const float tn = (float)(n - n0);
                    for (int a = 0; a < 3; ++a) tps[a] += tn * pb[a];
                }
                if (a_) {
                    for (int a = 0; a < 3; ++a) {
                        rb[a] = rn_[a] + pb[a] - lenb * u[a];
                        vb[a] = vn_[a];
                    }
                }
                // scatter the three stages: one pass over the lane's cell row for the
                // stages in stage 3's cell, then the others (a step that crosses a face)
#ifndef BOS_ADJ_ONE_PASS
#define BOS_ADJ_ONE_PASS 1
#endif
                const bool same2 = BOS_ADJ_ONE_PASS && key2 == key3, same1 = BOS_ADJ_ONE_PASS && key1 == key3;
                accumulate3(rows, a_, key3, cf3, Q3, same2, cf2, Q2, same1, cf1, Q1, ca, acc, nx, nxy);
                accumulate(rows, a_ && !same2, key2, cf2, Q2, ca, acc, nx, nxy);
                accumulate(rows, a_ && !same1, key1, cf1, Q1, ca, acc, nx, nxy);
            }
            if constexpr (CONN) {
                if (proj && seg)
                    for (int a = 0; a < 3; ++a) tpb[a] += (double)tps[a] + (double)n0 * (double)(rb[a] - rseg[a]);
            }
            __syncwarp();
        }
        // ---- entry: v0 = eta_in d and dt = ell / (N eta_in), eta_in = 1 + deta(r_in)
        int ci[3] = {0, 0, 0};
        float cf[3] = {0, 0, 0};
        if (act) {
            etab -= (double)dtb * (double)dt / eta_in;
            const float zero[3] = {0, 0, 0};
            comp_cell(F, st0.U, zero, ci, cf);
        }
        accumulate(rows, act, cell_key_of(F, ci), cf, make_float4((float)etab, 0.0f, 0.0f, 0.0f), ca, acc, nx, nxy);
        if constexpr (CONN) {
            if (proj && act) {
                // the projector ray's entry state as a function of its aim: r_in = P + t_in d,
                // v0 = eta_in d (base of v_N), straight step (ell/N) d, dt = ell / (N eta_in),
                // eta_in = 1 + deta(r_in), d = q / |q|, t_in and t_end on slab faces or the wall
                const double Nd = (double)RR.N, ds = RR.ell / Nd;
                Stage se;
                const float zero[3] = {0, 0, 0};
                stage_eval(F, st0.U, zero, bc, se);
                const double ge[3] = {(double)se.ig.d0.x * (double)F.inv_h[0], (double)se.ig.d1.x * (double)F.inv_h[1],
                                      (double)se.ig.d2.x * (double)F.inv_h[2]};
                double dSb[3], rbi[3], db[3];
                for (int a = 0; a < 3; ++a) {
                    dSb[a] = tpb[a] + Nd * drbw[a];
                    rbi[a] = (double)rb[a] + etab * ge[a];
                    db[a] = eta_in * dvbw[a] + ds * dSb[a] + RR.t_in * rbi[a];
                }
                const double ellb = (double)dtb / (Nd * eta_in) +
                                    (RR.d[0] * dSb[0] + RR.d[1] * dSb[1] + RR.d[2] * dSb[2]) / Nd;
                const double tinb = RR.d[0] * rbi[0] + RR.d[1] * rbi[1] + RR.d[2] * rbi[2] - ellb;
                if (RR.in_axis >= 0) db[RR.in_axis] += tinb * (-RR.t_in / RR.d[RR.in_axis]);
                if (RR.out_axis == 3) {
                    const double den = RR.d[0] * S.w.normal[0] + RR.d[1] * S.w.normal[1] + RR.d[2] * S.w.normal[2];
                    for (int a = 0; a < 3; ++a) db[a] += ellb * (-RR.tw * S.w.normal[a] / den);
                } else {
                    const int oa = RR.out_axis;
                    db[oa] += ellb * (-(RR.t_in + RR.ell) / RR.d[oa]);
                }
                const double dd = db[0] * RR.d[0] + db[1] * RR.d[1] + db[2] * RR.d[2];
                for (int a = 0; a < 3; ++a) xlb[a] += (db[a] - dd * RR.d[a]) / nqp[0];
            }
        }
        }   // passes
    }
}

template <class E, bool CONN_T>
__global__ void __launch_bounds__(kAdjWarps * 32, BOS_ADJ_MIN_BLOCKS) adjoint_kernel(SceneDev S, CkptDev ck, AdjDev adj, WorkDev wk) {
    constexpr bool CONN = CONN_T;
    extern __shared__ float4 smem4[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Refracted connection: values that live across a whole ray reversal are parked in
    // shared memory (per lane: a_1, dL/dx_w, the projector seed, the projector's wall-seed
    // adjoints, the straight-step adjoint sum and |q|) rather than held in registers
    // through the hot loop.
    __shared__ double conn_sh[CONN ? kAdjWarps * 32 * kConnDoubles : 1];
    double* const xlum = conn_sh + (CONN ? (warp * 32 + lane) * kConnDoubles : 0);
    const int K = ck.every;
    float* rows = reinterpret_cast<float*>(smem4) + (size_t)warp * adj_warp_floats(K);      // [32][kRow]
    // [K][12][32] step states and stage terms (dr, dv, A, B) of the segment being reversed
    // (this warp's slice)
    float* st_buf = adj.seg + ((size_t)blockIdx.x * kAdjWarps + warp) * ((size_t)K * kSegFloats * 32);
    const CompField<E> F = comp_field<E>(S.g);
    const TileShape ts = tile_shape(S.cam.width, S.cam.height, S.cam.spp);
    const int ntiles = tile_count(S, ts);
    float* acc = reinterpret_cast<float*>(adj.acc);
    {
        float4* row = reinterpret_cast<float4*>(rows + lane * kRow);
        for (int c = 0; c < 8; ++c) row[c] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncwarp();
    CellAcc ca = {kNoKey, (uint32_t)S.g.n[0] * S.g.n[1] * S.g.n[2], S.g.err};
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(wk.tile_counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        adjoint_tile<E, CONN>(S, ck, adj, F, ts, t, lane, rows, st_buf, acc, ca, xlum);
    }
    flush_rows(rows, ca.key != kNoKey, ca, acc, S.g.n[0], S.g.n[0] * S.g.n[1]);
}

// Adjoint of quasi-linear tracing (Sec. 2.2).  The stage points lie on the straight
// line, so the outputs are linear in the sampled D values and no position adjoint flows
// back through them.  Reversing a step leaves the position adjoint unchanged and adds
// dt (r_bar + len_bar u_n) to the velocity adjoint (u_n the unit direction of step n), so
//   v_bar_{n+1} = v_bar_N + dt (N - n - 1) r_bar + dt len_bar sum_{m > n} u_m
// is known from the final state and a running prefix of u: one sweep in forward order
// recomputes the samples and scatters every stage's sensitivity (the end sample of a
// step and the start sample of the next are one point and one scatter).
// A quasi-linear line sample: its cell and the field value only (the samples sit on the
// straight line, so no position adjoint and hence no field gradient is needed).
struct LineSample {
    uint32_t key;
    float cf[3];
    float4 v;   // (deta, grad eta)
};

template <class E>
__device__ __forceinline__ void line_sample(const CompField<E>& F, const long long U[3], BrickCache& bc,
                                            LineSample& p) {
    const float zero[3] = {0.0f, 0.0f, 0.0f};
    int ci[3];
    comp_cell(F, U, zero, ci, p.cf);
    p.key = cell_key_of(F, ci);
    p.v = trilinear2(F.store, comp_offset(F, bc, ci), p.cf[0], p.cf[1], p.cf[2]);
}

// Corner record of D = (1 + deta) grad at a line sample for the adjoint Db of D.
__device__ __forceinline__ float4 line_corner_record(const float4 v, const float Db[3]) {
    const float eta = 1.0f + v.x;
    return make_float4(Db[0] * v.y + Db[1] * v.z + Db[2] * v.w, eta * Db[0], eta * Db[1], eta * Db[2]);
}

// One warp tile of the quasi-linear adjoint (one forward-order sweep per ray).
template <class E>
__device__ __forceinline__ void adjoint_quasi_tile(const SceneDev& S, const CkptDev& ck, const AdjDev& adj,
                                                   const CompField<E>& F, const TileShape& ts, int t, int lane,
                                                   float* rows, float* acc, CellAcc& ca) {
    const int nx = S.g.n[0], nxy = S.g.n[0] * S.g.n[1];
    const int spp = S.cam.spp;
    const float zero[3] = {0.0f, 0.0f, 0.0f};
    const int sl = lane % ts.G;
    const TilePix tp = tile_pixel(S, ts, t, lane);
    const int px = tp.px, py = tp.py;
    const bool valid = tp.valid;
    for (int qs = 0; qs < ts.samples_per_lane; ++qs) {
        const int s = ts.samples_per_lane == 1 ? sl : qs;
        const long long slot = ((long long)t * 32 + lane) * ts.samples_per_lane + qs;
        bool act = valid;
        Ray R;
        R.N = 0;
        R.wall = false;
        double Ib = 0.0;
        if (act) {
            R = ray_setup(S, px, py, s);
            Ib = (double)adj.dLdI[(size_t)tp.out] / spp;
        }
        act = act && R.wall && R.N > 0 && Ib != 0.0;
        CompState st;
        CompConst k;
        double eta_in = 1.0, rin[3] = {0, 0, 0};
        float rb[3] = {0, 0, 0}, vbN[3] = {0, 0, 0}, lenb = 0.0f, usum[3] = {0, 0, 0};
        double etab = 0.0;
        if (act) {
            comp_setup(S, F, S.cam.pos, R, st, k, eta_in, rin);
            const float4 s0 = ck.state[0 * ck.nrays + slot];
            const float4 s1 = ck.state[1 * ck.nrays + slot];
            const float4 s2 = ck.state[2 * ck.nrays + slot];
            usum[0] = s1.w;
            usum[1] = s2.x;
            usum[2] = s2.y;
            double rN[3], vN[3], drb[3], dvb[3], lb;
            const float drN[3] = {s0.x, s0.y, s0.z}, dvN[3] = {s1.x, s1.y, s1.z};
            for (int a = 0; a < 3; ++a) {
                rN[a] = rin[a] + R.ell * R.d[a] + (double)drN[a];
                vN[a] = eta_in * R.d[a] + (double)dvN[a];
            }
            wall_adjoint(S, rN, vN, R.t_in + R.ell + (double)s0.w, Ib, drb, dvb, lb);
            for (int a = 0; a < 3; ++a) {
                rb[a] = (float)drb[a];
                vbN[a] = (float)dvb[a];
            }
            lenb = (float)lb;
            etab = dvb[0] * R.d[0] + dvb[1] * R.d[1] + dvb[2] * R.d[2];
        }
        const int N = act ? R.N : 0;
        const int n_max = __reduce_max_sync(0xffffffffu, (unsigned)N);
        const float dt = act ? k.dt : 0.0f;
        BrickCache bc = {kNoKey, 0u};
        // the start sample of step 0
        LineSample p0 = {};
        float A[3] = {0, 0, 0}, dv[3] = {0, 0, 0}, prefix[3] = {0, 0, 0}, carry[3] = {0, 0, 0}, dtb = 0.0f;
        if (act) {
            line_sample(F, st.U, bc, p0);
            float D[3];
            rhs_of(p0.v, D);
            for (int a = 0; a < 3; ++a) A[a] = dt * D[a];
        }
        for (int n = 0; n < n_max; ++n) {
            const bool a_ = act && n < N;
            LineSample pm = {}, pe = {};
            float B[3] = {0, 0, 0}, C[3] = {0, 0, 0}, u[3] = {0, 0, 0}, Dm[3] = {0, 0, 0}, De[3] = {0, 0, 0};
            float Db0[3] = {0, 0, 0}, Dbm[3] = {0, 0, 0};
            if (a_) {
                long long U2[3], U3[3];
                for (int a = 0; a < 3; ++a) {
                    U2[a] = st.U[a] + (long long)n * k.dU[a] + k.dUh[a];
                    U3[a] = st.U[a] + (long long)(n + 1) * k.dU[a];
                }
                line_sample(F, U2, bc, pm);
                rhs_of(pm.v, Dm);
                line_sample(F, U3, bc, pe);
                rhs_of(pe.v, De);
                float inc[3], nn = 0.0f;
                for (int a = 0; a < 3; ++a) {
                    B[a] = dt * Dm[a];
                    C[a] = dt * De[a];
                    inc[a] = dt * (dv[a] + (A[a] + 2.0f * B[a]) * (1.0f / 6.0f));
                    const float w = k.dS[a] + inc[a];
                    u[a] = w;
                    nn += w * w;
                }
                const float rn = rsqrtf(nn);
                const float rem = (float)(N - n - 1);
                for (int a = 0; a < 3; ++a) {
                    u[a] *= rn;
                    prefix[a] += u[a];
                    const float rbp = rb[a] + lenb * u[a];                       // adjoint of r_{n+1}
                    const float vb1 = vbN[a] + dt * rem * rb[a] + dt * lenb * (usum[a] - prefix[a]);
                    const float Ab = (dt * (1.0f / 6.0f)) * rbp + vb1 * (1.0f / 6.0f);
                    const float Bb = (dt * (1.0f / 3.0f)) * rbp + vb1 * (4.0f / 6.0f);
                    const float Cb = vb1 * (1.0f / 6.0f);
                    dtb += rbp * (dv[a] + (A[a] + 2.0f * B[a]) * (1.0f / 6.0f)) + Ab * (A[a] / dt) + Bb * Dm[a] +
                           Cb * De[a];
                    Db0[a] = carry[a] + dt * Ab;      // start sample: this step's A and the previous C
                    Dbm[a] = dt * Bb;
                    carry[a] = dt * Cb;
                    dv[a] += (A[a] + 4.0f * B[a] + C[a]) * (1.0f / 6.0f);
                    A[a] = C[a];
                }
            }
            float4 Q = make_float4(0, 0, 0, 0), Qm = make_float4(0, 0, 0, 0);
            if (a_) {
                Q = line_corner_record(p0.v, Db0);
                Qm = line_corner_record(pm.v, Dbm);
            }
            // the step's two samples share a cell more often than not: one row update
            const bool same = a_ && pm.key == p0.key;
            accumulate_dual(rows, a_, p0.key, p0.cf, Q, same, pm.cf, Qm, ca, acc, nx, nxy);
            accumulate(rows, a_ && !same, pm.key, pm.cf, Qm, ca, acc, nx, nxy);
            if (a_) p0 = pe;
        }
        // the end sample of the last step, then eta_in = 1 + deta(r_in)
        float4 Q = make_float4(0, 0, 0, 0);
        if (act) Q = line_corner_record(p0.v, carry);
        accumulate(rows, act, p0.key, p0.cf, Q, ca, acc, nx, nxy);
        int ci[3] = {0, 0, 0};
        float cf[3] = {0, 0, 0};
        if (act) {
            etab -= (double)dtb * (double)dt / eta_in;
            comp_cell(F, st.U, zero, ci, cf);
        }
        accumulate(rows, act, cell_key_of(F, ci), cf, make_float4((float)etab, 0.0f, 0.0f, 0.0f), ca, acc, nx, nxy);
    }
}

template <class E, int MINB>
__global__ void __launch_bounds__(kAdjWarps * 32, MINB)
    adjoint_quasi_kernel(SceneDev S, CkptDev ck, AdjDev adj, WorkDev wk) {
    extern __shared__ float4 smem4[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* rows = reinterpret_cast<float*>(smem4) + (size_t)warp * 32 * kRow;
    {
        float4* row = reinterpret_cast<float4*>(rows + lane * kRow);
        for (int c = 0; c < 8; ++c) row[c] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncwarp();
    const CompField<E> F = comp_field<E>(S.g);
    const TileShape ts = tile_shape(S.cam.width, S.cam.height, S.cam.spp);
    const int ntiles = tile_count(S, ts);
    float* acc = reinterpret_cast<float*>(adj.acc);
    CellAcc ca = {kNoKey, (uint32_t)S.g.n[0] * S.g.n[1] * S.g.n[2], S.g.err};
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(wk.tile_counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        adjoint_quasi_tile<E>(S, ck, adj, F, ts, t, lane, rows, acc, ca);
    }
    flush_rows(rows, ca.key != kNoKey, ca, acc, S.g.n[0], S.g.n[0] * S.g.n[1]);
}

// ---- float64 adjoint (FP64 store and tracer, Sharma RKN) -------------------------------------
//
// The same discrete adjoint in float64 throughout, for the plain float64 tracer: the state
// is the absolute (r, v), kept every K steps by the forward render (six doubles); each
// segment is recomputed into this warp's slice of global memory and reversed; every stage's
// corner sensitivities go to float64 node accumulators.  GB300 runs float64 at 1/64 of the
// float32 rate, so this path is for accuracy, not speed: it separates the method's own error
// from float32 rounding.

struct D4Grad {
    D4 v, d0, d1, d2;   // value and derivatives with respect to the three fractions
};

__device__ __forceinline__ D4 dsub4(D4 a, D4 b) {
    D4 r;
    r.x = a.x - b.x;
    r.y = a.y - b.y;
    r.z = a.z - b.z;
    r.w = a.w - b.w;
    return r;
}

// Value (the operations of trilinear_d, so bit-identical) and fraction derivatives.
__device__ __forceinline__ D4Grad trilinear_grad_d(const D4* s, uint32_t o, double f0, double f1, double f2) {
    const D4 c000 = load_d4(s, o), c100 = load_d4(s, o + 1), c010 = load_d4(s, o + 9), c110 = load_d4(s, o + 10);
    const D4 c001 = load_d4(s, o + 81), c101 = load_d4(s, o + 82), c011 = load_d4(s, o + 90), c111 = load_d4(s, o + 91);
    const D4 a0 = dlerp(c000, c100, f0), a1 = dlerp(c010, c110, f0), a2 = dlerp(c001, c101, f0),
             a3 = dlerp(c011, c111, f0);
    const D4 b0 = dlerp(a0, a1, f1), b1 = dlerp(a2, a3, f1);
    D4Grad r;
    r.v = dlerp(b0, b1, f2);
    r.d2 = dsub4(b1, b0);
    r.d1 = dlerp(dsub4(a1, a0), dsub4(a3, a2), f2);
    r.d0 = dlerp(dlerp(dsub4(c100, c000), dsub4(c110, c010), f1), dlerp(dsub4(c101, c001), dsub4(c111, c011), f1), f2);
    return r;
}

struct DStage {
    int i[3];       // base cell
    double f[3];    // fractions (unclamped at the edge cells)
    D4Grad g;
};

// Field value and gradient at absolute position x: the cell and fractions of field_at.
__device__ __forceinline__ void dstage_eval(const GridDev& g, const double x[3], DStage& s) {
    for (int a = 0; a < 3; ++a) {
        const double u = (x[a] - g.origin[a]) / g.h[a] - 0.5;
        split_coord(u, g.n[a], s.i[a], s.f[a]);
    }
    uint32_t o = bounded(brick_offset(s.i[0], s.i[1], s.i[2]) + 91u, g.store_elems, g.err);
    o = o ? o - 91u : 0u;
    s.g = trilinear_grad_d(static_cast<const D4*>(g.store), o, s.f[0], s.f[1], s.f[2]);
}

__device__ __forceinline__ void drhs(const DStage& s, double D[3]) {
    const double eta = 1.0 + s.g.v.x;
    D[0] = eta * s.g.v.y;
    D[1] = eta * s.g.v.z;
    D[2] = eta * s.g.v.w;
}

// Adjoint of D = (1 + deta) grad at a stage for Db: the position adjoint pb, and the
// record adjoint Q scattered to the 8 corners with the trilinear weights.
__device__ __forceinline__ void drhs_adjoint_scatter(const GridDev& g, const DStage& s, const double Db[3], double pb[3],
                                                     double* acc, bool act) {
    const double eta = 1.0 + s.g.v.x;
    const double Dg = Db[0] * s.g.v.y + Db[1] * s.g.v.z + Db[2] * s.g.v.w;
    const D4 dv[3] = {s.g.d0, s.g.d1, s.g.d2};
    for (int a = 0; a < 3; ++a)
        pb[a] = g.inv_h[a] * (dv[a].x * Dg + eta * (Db[0] * dv[a].y + Db[1] * dv[a].z + Db[2] * dv[a].w));
    if (!act) return;
    const double Q[4] = {Dg, eta * Db[0], eta * Db[1], eta * Db[2]};
    const size_t nx = (size_t)g.n[0], nxy = (size_t)g.n[0] * g.n[1];
    const size_t base = (size_t)s.i[0] + (size_t)s.i[1] * nx + (size_t)s.i[2] * nxy;
    for (int c = 0; c < 8; ++c) {
        const double w = ((c & 1) ? s.f[0] : 1.0 - s.f[0]) * ((c & 2) ? s.f[1] : 1.0 - s.f[1]) *
                         ((c & 4) ? s.f[2] : 1.0 - s.f[2]);
        const size_t node = base + (size_t)(c & 1) + (size_t)((c >> 1) & 1) * nx + (size_t)(c >> 2) * nxy;
        const size_t nd = bounded(node, (size_t)g.n[0] * g.n[1] * g.n[2], g.err);
        for (int ch = 0; ch < 4; ++ch) atomicAdd(acc + nd * 4 + ch, w * Q[ch]);
    }
}

// G = the seed's type: float (bos_backward) or double (bos_backward_f64).
template <class G>
__global__ void __launch_bounds__(kAdjWarps * 32) adjoint_fp64_kernel(SceneDev S, CkptDev ck, AdjDev adj, WorkDev wk) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = ck.every;
    // [K][6][32] step states (r, v) of the segment being reversed (this warp's slice)
    double* buf = reinterpret_cast<double*>(adj.seg) + ((size_t)blockIdx.x * kAdjWarps + warp) * ((size_t)K * 6 * 32);
    const double* ckd = reinterpret_cast<const double*>(ck.state);
    double* acc = reinterpret_cast<double*>(adj.acc);
    const GridDev& g = S.g;
    const FullField<double> F = {S.g};
    const int W = S.cam.width, H = S.cam.height, spp = S.cam.spp;
    const TileShape ts = tile_shape(W, H, spp);
    const int ntiles = tile_count(S, ts);
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(wk.tile_counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        const int sl = lane % ts.G;
        const TilePix tp = tile_pixel(S, ts, t, lane);
        for (int qs = 0; qs < ts.samples_per_lane; ++qs) {
            const int s = ts.samples_per_lane == 1 ? sl : qs;
            const long long slot = ((long long)t * 32 + lane) * ts.samples_per_lane + qs;
            Ray R;
            R.N = 0;
            R.wall = false;
            double Ib = 0.0;
            if (tp.valid) {
                R = ray_setup(S, tp.px, tp.py, s);
                Ib = (double)reinterpret_cast<const G*>(adj.dLdI)[(size_t)tp.out] / spp;
            }
            const bool act = tp.valid && R.wall && R.N > 0 && Ib != 0.0;
            // entry state as the forward forms it: r_in, eta_in, v0 = eta_in d, dt = ell / (N eta_in)
            double rin[3] = {0.0, 0.0, 0.0}, eta_in = 1.0, dt = 0.0;
            if (act) {
                for (int a = 0; a < 3; ++a) rin[a] = S.cam.pos[a] + R.t_in * R.d[a];
                eta_in = F.eta(rin);
                dt = R.ell / ((double)R.N * eta_in);
            }
            const int N = act ? R.N : 0;
            const int nseg = (N + K - 1) / K;
            const int nseg_max = __reduce_max_sync(0xffffffffu, (unsigned)nseg);
            double rb[3] = {0, 0, 0}, vb[3] = {0, 0, 0}, dtb = 0.0, lenb = 0.0;
            for (int c = nseg_max - 1; c >= 0; --c) {
                const int n0 = c * K, n1 = min(n0 + K, N);
                const bool seg = act && n0 < N;
                if (seg) {
                    // ---- recompute the segment from its checkpoint (full_step's operations)
                    double r[3], v[3];
                    const size_t cc = bounded((size_t)c, (size_t)ck.max_ckpt, ck.err);
                    for (int q = 0; q < 3; ++q) {
                        r[q] = ckd[(cc * 6 + q) * ck.nrays + slot];
                        v[q] = ckd[(cc * 6 + 3 + q) * ck.nrays + slot];
                    }
                    for (int n = n0; n < n1; ++n) {
                        double* p = buf + (size_t)(n - n0) * 6 * 32 + lane;
                        for (int q = 0; q < 3; ++q) {
                            p[32 * q] = r[q];
                            p[32 * (3 + q)] = v[q];
                        }
                        full_step<double, 0>(F, r, v, dt);
                    }
                    if (c == nseg - 1) {
                        double lb = 0.0;
                        const double len_before = R.t_in + reinterpret_cast<const double*>(ck.excess)[slot];
                        wall_adjoint(S, r, v, len_before, Ib, rb, vb, lb);
                        lenb = lb;
                    }
                }
                __syncwarp();
                // ---- reverse the segment's steps
                const int n_hi = __reduce_max_sync(0xffffffffu, (unsigned)(seg ? n1 : 0));
                for (int n = n_hi - 1; n >= n0; --n) {
                    const bool a_ = seg && n < n1;
                    if (!a_) continue;
                    const double* p = buf + (size_t)(n - n0) * 6 * 32 + lane;
                    double r[3], v[3], A[3], B[3], D1[3], D2[3], D3[3], q[3];
                    for (int a = 0; a < 3; ++a) {
                        r[a] = p[32 * a];
                        v[a] = p[32 * (3 + a)];
                    }
                    DStage s1, s2, s3;
                    dstage_eval(g, r, s1);
                    drhs(s1, D1);
                    for (int a = 0; a < 3; ++a) A[a] = dt * D1[a];
                    for (int a = 0; a < 3; ++a) q[a] = r[a] + (dt * 0.5) * v[a] + (dt * 0.125) * A[a];
                    dstage_eval(g, q, s2);
                    drhs(s2, D2);
                    for (int a = 0; a < 3; ++a) B[a] = dt * D2[a];
                    for (int a = 0; a < 3; ++a) q[a] = r[a] + dt * v[a] + (dt * 0.5) * B[a];
                    dstage_eval(g, q, s3);
                    drhs(s3, D3);
                    // r' = r + dt (v + (A + 2B)/6), |r' - r| enters the path length
                    double inc[3], nn = 0.0, u[3];
                    for (int a = 0; a < 3; ++a) {
                        inc[a] = dt * (v[a] + (A[a] + 2.0 * B[a]) / 6.0);
                        nn += inc[a] * inc[a];
                    }
                    const double rn = 1.0 / sqrt(nn);
                    double rbs[3], Ab[3], Bb[3], Cb[3], rn_[3], vn_[3], Db[3], pb[3];
                    for (int a = 0; a < 3; ++a) {
                        u[a] = inc[a] * rn;
                        rbs[a] = rb[a] + lenb * u[a];
                    }
                    for (int a = 0; a < 3; ++a) {
                        Ab[a] = (dt / 6.0) * rbs[a] + vb[a] / 6.0;
                        Bb[a] = (dt / 3.0) * rbs[a] + vb[a] * (4.0 / 6.0);
                        Cb[a] = vb[a] / 6.0;
                        rn_[a] = rbs[a];
                        vn_[a] = vb[a] + dt * rbs[a];
                        dtb += rbs[a] * (v[a] + (A[a] + 2.0 * B[a]) / 6.0);
                    }
                    // C = dt D(p3), p3 = r + dt v + dt/2 B
                    for (int a = 0; a < 3; ++a) {
                        dtb += Cb[a] * D3[a];
                        Db[a] = dt * Cb[a];
                    }
                    drhs_adjoint_scatter(g, s3, Db, pb, acc, true);
                    for (int a = 0; a < 3; ++a) {
                        rn_[a] += pb[a];
                        vn_[a] += dt * pb[a];
                        Bb[a] += (0.5 * dt) * pb[a];
                        dtb += pb[a] * (v[a] + 0.5 * B[a]);
                    }
                    // B = dt D(p2), p2 = r + dt/2 v + dt/8 A
                    for (int a = 0; a < 3; ++a) {
                        dtb += Bb[a] * D2[a];
                        Db[a] = dt * Bb[a];
                    }
                    drhs_adjoint_scatter(g, s2, Db, pb, acc, true);
                    for (int a = 0; a < 3; ++a) {
                        rn_[a] += pb[a];
                        vn_[a] += (0.5 * dt) * pb[a];
                        Ab[a] += (0.125 * dt) * pb[a];
                        dtb += pb[a] * (0.5 * v[a] + 0.125 * A[a]);
                    }
                    // A = dt D(p1), p1 = r
                    for (int a = 0; a < 3; ++a) {
                        dtb += Ab[a] * D1[a];
                        Db[a] = dt * Ab[a];
                    }
                    drhs_adjoint_scatter(g, s1, Db, pb, acc, true);
                    for (int a = 0; a < 3; ++a) {
                        rb[a] = rn_[a] + pb[a] - lenb * u[a];
                        vb[a] = vn_[a];
                    }
                }
                __syncwarp();
            }
            // ---- entry: v0 = eta_in d, dt = ell / (N eta_in), eta_in = 1 + deta(r_in)
            if (act) {
                const double etab = vb[0] * R.d[0] + vb[1] * R.d[1] + vb[2] * R.d[2] - dtb * dt / eta_in;
                DStage se;
                dstage_eval(g, rin, se);
                const size_t nx = (size_t)g.n[0], nxy = (size_t)g.n[0] * g.n[1];
                const size_t base = (size_t)se.i[0] + (size_t)se.i[1] * nx + (size_t)se.i[2] * nxy;
                for (int c = 0; c < 8; ++c) {
                    const double w = ((c & 1) ? se.f[0] : 1.0 - se.f[0]) * ((c & 2) ? se.f[1] : 1.0 - se.f[1]) *
                                     ((c & 4) ? se.f[2] : 1.0 - se.f[2]);
                    const size_t node = base + (size_t)(c & 1) + (size_t)((c >> 1) & 1) * nx + (size_t)(c >> 2) * nxy;
                    atomicAdd(acc + bounded(node, (size_t)g.n[0] * g.n[1] * g.n[2], g.err) * 4, w * etab);
                }
            }
        }
    }
}

// dL/dT per node: transpose of the difference stencil of grad eta, plus d L/d deta, times
// d deta/dT = -K / T^2.
__device__ __forceinline__ double acc_channel(const float4* acc, long long m, int ch) {
    const float4 v = acc[m];
    return (double)(ch == 0 ? v.x : ch == 1 ? v.y : ch == 2 ? v.z : v.w);
}
__device__ __forceinline__ double acc_channel(const double* acc, long long m, int ch) { return acc[m * 4 + ch]; }

template <class A, class O = float>
__global__ void gradient_kernel(GridDev g, const A* __restrict__ acc, const float* __restrict__ T,
                                O* __restrict__ dLdT) {
    const long long n = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int idx[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((long long)g.n[0] * g.n[1]))};
        const long long stride[3] = {1, g.n[0], (long long)g.n[0] * g.n[1]};
        double tot = acc_channel(acc, c, 0);
        for (int a = 0; a < 3; ++a) {
            const int i = idx[a], na = g.n[a];
            const double ih = g.inv_h[a], ih2 = 0.5 * g.inv_h[a];
            if (i - 1 >= 0) tot += acc_channel(acc, c - stride[a], 1 + a) * (i - 1 == 0 ? ih : ih2);        // node i-1 reads i as hi
            if (i + 1 <= na - 1) tot -= acc_channel(acc, c + stride[a], 1 + a) * (i + 1 == na - 1 ? ih : ih2);  // node i+1 reads i as lo
            if (i == 0) tot -= acc_channel(acc, c, 1 + a) * ih;                                             // one-sided at the faces
            if (i == na - 1) tot += acc_channel(acc, c, 1 + a) * ih;
        }
        if constexpr (sizeof(A) == 8) {
            const double Tc = (double)T[c];
            dLdT[c] = (O)(tot * (-g.K / (Tc * Tc)));
        } else {
            const float Tc = T[c];
            dLdT[c] = (float)tot * (-(float)g.K / (Tc * Tc));
        }
    }
}

// Batched adjoints (the request server): one launch covers warp tiles of several jobs,
// indexed as in render_batch_kernel.  The lane rows belong to one job's accumulators at a
// time, so they are flushed whenever a warp moves on to another job's tile.  The Sharma
// form's segment slices come from seg_base with room for k_max steps.
template <class E, bool QUASI>
__global__ void __launch_bounds__(kAdjWarps * 32, QUASI ? BOS_ADJ_QUASI_MIN_BLOCKS : BOS_ADJ_MIN_BLOCKS)
    adjoint_batch_kernel(const BatchJob* __restrict__ jobs, int njobs, int total, int* counter, float* seg_base,
                         int k_max) {
    extern __shared__ float4 smem4[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* rows = reinterpret_cast<float*>(smem4) + (size_t)warp * 32 * kRow;
    float* st_buf = seg_base + ((size_t)blockIdx.x * kAdjWarps + warp) * ((size_t)k_max * kSegFloats * 32);
    {
        float4* row = reinterpret_cast<float4*>(rows + lane * kRow);
        for (int c = 0; c < 8; ++c) row[c] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncwarp();
    CellAcc ca = {kNoKey, 0u, nullptr};
    int cur = -1;                      // job whose accumulators the rows belong to
    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(counter, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= total) break;
        const int j = batch_job_of(jobs, njobs, g);
        if (j != cur && cur >= 0) {
            const BatchJob& P = jobs[cur];
            flush_rows(rows, ca.key != kNoKey, ca, reinterpret_cast<float*>(P.adj.acc), P.S.g.n[0],
                       P.S.g.n[0] * P.S.g.n[1]);
        }
        cur = j;
        const BatchJob& J = jobs[j];
        ca.ncells = (uint32_t)J.S.g.n[0] * J.S.g.n[1] * J.S.g.n[2];
        ca.err = J.S.g.err;
        const CompField<E> F = comp_field<E>(J.S.g);
        const TileShape ts = tile_shape(J.S.cam.width, J.S.cam.height, J.S.cam.spp);
        float* acc = reinterpret_cast<float*>(J.adj.acc);
        if constexpr (QUASI)
            adjoint_quasi_tile<E>(J.S, J.ck, J.adj, F, ts, J.tile0 + (g - J.first), lane, rows, acc, ca);
        else
            adjoint_tile<E, false>(J.S, J.ck, J.adj, F, ts, J.tile0 + (g - J.first), lane, rows, st_buf, acc, ca,
                                   nullptr);
    }
    if (cur >= 0) {
        const BatchJob& P = jobs[cur];
        flush_rows(rows, ca.key != kNoKey, ca, reinterpret_cast<float*>(P.adj.acc), P.S.g.n[0], P.S.g.n[0] * P.S.g.n[1]);
    }
}

template <class E, bool QUASI>
static cudaError_t launch_adjoint_batch_c(const BatchJob* jobs, int njobs, int total, int* counter, float* seg_base,
                                          int k_max, int num_sms, cudaStream_t st) {
    const size_t smem = (size_t)kAdjWarps * 32 * kRow * sizeof(float);
    int per_sm = 0;
    cudaError_t e = occupancy_prefer_l1(adjoint_batch_kernel<E, QUASI>, kAdjWarps * 32, smem, per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int blocks = num_sms * per_sm < kAdjMaxBlocks ? num_sms * per_sm : kAdjMaxBlocks;
    adjoint_batch_kernel<E, QUASI><<<blocks, kAdjWarps * 32, smem, st>>>(jobs, njobs, total, counter, seg_base, k_max);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_batch(int mode, int integ, const BatchJob* jobs, int njobs, int total, int* counter,
                                 float* seg_base, int k_max, int num_sms, cudaStream_t st) {
    if (k_max > 64 || (integ != 0 && integ != 2)) return cudaErrorNotSupported;
    if (mode == 1) return integ == 2 ? launch_adjoint_batch_c<F4P, true>(jobs, njobs, total, counter, seg_base, k_max, num_sms, st)
                                     : launch_adjoint_batch_c<F4P, false>(jobs, njobs, total, counter, seg_base, k_max, num_sms, st);
    if (mode == 2) return integ == 2 ? launch_adjoint_batch_c<B4P, true>(jobs, njobs, total, counter, seg_base, k_max, num_sms, st)
                                     : launch_adjoint_batch_c<B4P, false>(jobs, njobs, total, counter, seg_base, k_max, num_sms, st);
    return cudaErrorNotSupported;
}

cudaError_t launch_gradient(const GridDev& g, const float4* acc, const float* T, float* dLdT, int num_sms,
                            cudaStream_t st) {
    gradient_kernel<float4><<<num_sms * 8, 256, 0, st>>>(g, acc, T, dLdT);
    return cudaGetLastError();
}

template <class E, bool CONN>
static cudaError_t launch_adjoint_c(const SceneDev& S, const CkptDev& ck, const AdjDev& adj, const WorkDev& w,
                                    int num_sms, cudaStream_t st) {
    size_t smem = (size_t)kAdjWarps * adj_warp_floats(ck.every) * sizeof(float);
    cudaError_t e =
        cudaFuncSetAttribute(adjoint_kernel<E, CONN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = occupancy_prefer_l1(adjoint_kernel<E, CONN>, kAdjWarps * 32, smem, per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1 || adj.seg == nullptr) return cudaErrorInvalidConfiguration;
    const int blocks = num_sms * per_sm < kAdjMaxBlocks ? num_sms * per_sm : kAdjMaxBlocks;
    adjoint_kernel<E, CONN><<<blocks, kAdjWarps * 32, smem, st>>>(S, ck, adj, w);
    return cudaGetLastError();
}

// The refracted projector connection (light mode 2) reverses each sample's projector ray
// too; it has its own instantiation so that the other modes do not carry it.
template <class E>
static cudaError_t launch_adjoint_t(const SceneDev& S, const CkptDev& ck, const AdjDev& adj, const WorkDev& w,
                                    int num_sms, cudaStream_t st) {
    if (S.L.mode == 2) {
        if (ck.pstate == nullptr || ck.conn == nullptr) return cudaErrorInvalidValue;
        return launch_adjoint_c<E, true>(S, ck, adj, w, num_sms, st);
    }
    return launch_adjoint_c<E, false>(S, ck, adj, w, num_sms, st);
}

template <class E, int MINB>
static cudaError_t launch_adjoint_quasi_b(const SceneDev& S, const CkptDev& ck, const AdjDev& adj, const WorkDev& w,
                                          int num_sms, cudaStream_t st) {
    size_t smem = (size_t)kAdjWarps * 32 * kRow * sizeof(float);
    int per_sm = 0;
    cudaError_t e = occupancy_prefer_l1(adjoint_quasi_kernel<E, MINB>, kAdjWarps * 32, smem, per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    adjoint_quasi_kernel<E, MINB><<<num_sms * per_sm, kAdjWarps * 32, smem, st>>>(S, ck, adj, w);
    return cudaGetLastError();
}

// Two register budgets of the quasi-linear adjoint: with more than 12 warp tiles per SM,
// the 128-register form's 16 resident warps per SM hide more latency; with fewer (a
// 5000-pixel minibatch is ~300 tiles) the GPU is not full either way, and the form without
// a register cap (180-200 registers, no spills) finishes each ray sooner.
template <class E>
static cudaError_t launch_adjoint_quasi_t(const SceneDev& S, const CkptDev& ck, const AdjDev& adj, const WorkDev& w,
                                          int num_sms, cudaStream_t st) {
    const int ntiles = tile_count(S, tile_shape(S.cam.width, S.cam.height, S.cam.spp));
    if (ntiles > num_sms * 12) return launch_adjoint_quasi_b<E, BOS_ADJ_QUASI_MIN_BLOCKS>(S, ck, adj, w, num_sms, st);
    return launch_adjoint_quasi_b<E, BOS_ADJ_QUASI_SMALL_MIN_BLOCKS>(S, ck, adj, w, num_sms, st);
}

// Float64 store and tracer: Sharma RKN, float64 accumulators; seed and dL/dT in float32 or
// (f64) float64.
cudaError_t launch_backward_fp64(const SceneDev& S, const CkptDev& ck, const AdjDev& adj, const WorkDev& w,
                                 const float* T, void* dLdT, bool f64, int num_sms, cudaStream_t st) {
    if (S.it.integrator != 0 || S.L.mode == 2 || adj.seg == nullptr || ck.every > 64) return cudaErrorNotSupported;
    const int blocks = num_sms * 8 < kAdjMaxBlocks ? num_sms * 8 : kAdjMaxBlocks;
    if (f64) adjoint_fp64_kernel<double><<<blocks, kAdjWarps * 32, 0, st>>>(S, ck, adj, w);
    else adjoint_fp64_kernel<float><<<blocks, kAdjWarps * 32, 0, st>>>(S, ck, adj, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double* acc = reinterpret_cast<const double*>(adj.acc);
    if (f64) gradient_kernel<double, double><<<num_sms * 8, 256, 0, st>>>(S.g, acc, T, static_cast<double*>(dLdT));
    else gradient_kernel<double, float><<<num_sms * 8, 256, 0, st>>>(S.g, acc, T, static_cast<float*>(dLdT));
    return cudaGetLastError();
}

cudaError_t launch_backward(int mode, const SceneDev& S, const CkptDev& ck, const AdjDev& adj, const WorkDev& w,
                            const float* T, float* dLdT, int num_sms, cudaStream_t st) {
    const bool quasi = S.it.integrator == 2;
    if (!quasi && ck.every > 64) return cudaErrorNotSupported;
    cudaError_t e;
    if (mode == 4) return launch_backward_fp64(S, ck, adj, w, T, dLdT, false, num_sms, st);
    if (mode == 1) e = quasi ? launch_adjoint_quasi_t<F4P>(S, ck, adj, w, num_sms, st)
                             : launch_adjoint_t<F4P>(S, ck, adj, w, num_sms, st);
    else if (mode == 2) e = quasi ? launch_adjoint_quasi_t<B4P>(S, ck, adj, w, num_sms, st)
                                  : launch_adjoint_t<B4P>(S, ck, adj, w, num_sms, st);
    else return cudaErrorNotSupported;
    if (e != cudaSuccess) return e;
    gradient_kernel<float4><<<num_sms * 8, 256, 0, st>>>(S.g, adj.acc, T, dLdT);
    return cudaGetLastError();
}

}  // namespace bos
