// Precision policies of the DEM timestep (device code shared by the force kernels):
// how a particle's state is loaded and stored, the contact decision and overlap, the
// wall geometry, the cell map CM and the update of Sec. 4.2 step 1, for
//   PF64  every quantity in FP64 (the reference formulas);
//   PF32  FP32 velocities, spins, forces and springs, positions as hi + lo float pairs.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dem_dev.cuh"

// Paired FP32 instructions (two IEEE operations per instruction) in the float-float
// contact test: 2% faster force pass on GB300, the same bits.
// List entries whose prefilter loads are in flight together (phase 1 of the list pass).
#ifndef DEM_SCAN_UNROLL
#define DEM_SCAN_UNROLL 2
#endif
#ifndef DEM_PACKED_FF
#define DEM_PACKED_FF 1
#endif

namespace demgb {

// L1 prefetch (PTX prefetch.global.L1): starts a line fill without holding a register.
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// ======================================================================= FP64 policy
struct PF64 {
    using T = double;
    using State = StateF64;
    struct Self {
        double x, y, z;
        float r;
        V3<double> v, w;
        uint32_t id;
    };
    static __device__ __forceinline__ Self load(const State& s, uint32_t q) {
        Self m;
        m.x = s.x[q]; m.y = s.y[q]; m.z = s.z[q];
        m.r = s.r[q];
        m.v = mk(s.vx[q], s.vy[q], s.vz[q]);
        m.w = mk(s.wx[q], s.wy[q], s.wz[q]);
        m.id = s.id[q];
        return m;
    }
    static __device__ __forceinline__ void store(const State& s, uint32_t q, const Self& m) {
        s.x[q] = m.x; s.y[q] = m.y; s.z[q] = m.z;
        s.r[q] = m.r;
        s.vx[q] = m.v.x; s.vy[q] = m.v.y; s.vz[q] = m.v.z;
        s.wx[q] = m.w.x; s.wy[q] = m.w.y; s.wz[q] = m.w.z;
        s.id[q] = m.id;
    }
    static __device__ __forceinline__ void load_vw(const State& s, uint32_t j, V3<double>& v, V3<double>& w) {
        v = mk(__ldg(&s.vx[j]), __ldg(&s.vy[j]), __ldg(&s.vz[j]));
        w = mk(__ldg(&s.wx[j]), __ldg(&s.wy[j]), __ldg(&s.wz[j]));
    }
    // Contact iff d^2 < R^2 with d^2 = fma(dz,dz, fma(dy,dy, dx*dx)), R = r_i + r_j (exact).
    static __device__ __forceinline__ bool touches(const Self& me, double xj, double yj, double zj, float rjf) {
        const double dx = __dsub_rn(xj, me.x), dy = __dsub_rn(yj, me.y), dz = __dsub_rn(zj, me.z);
        const double d2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
        const double R = __dadd_rn((double)me.r, (double)rjf);
        return d2 < __dmul_rn(R, R);
    }
    // Phase 1 of the walk: append to the near list every particle of [j0, j1) in contact.
    static __device__ __forceinline__ void scan_row(const State& s, const Self& me, const SceneDev&, uint32_t j0,
                                                    uint32_t j1, uint32_t q, uint32_t* lst, uint32_t bd, uint32_t tid,
                                                    uint32_t maxc, uint32_t& cnt) {
        for (uint32_t j = j0; j < j1; ++j) {
            if (j == q) continue;
            if (touches(me, __ldg(&s.x[j]), __ldg(&s.y[j]), __ldg(&s.z[j]), __ldg(&s.r[j]))) {
                if (cnt < maxc) lst[cnt * bd + tid] = j;
                ++cnt;
            }
        }
    }
    // Phase 1 from a neighbour list built at the last sort: bit k of the returned mask
    // marks list entry k as in contact.
    static __device__ __forceinline__ uint64_t scan_list(const State& s, const Self& me, const SceneDev&,
                                                         const uint32_t* nl, uint32_t m, size_t cap, uint32_t q) {
        uint64_t mask = 0;
        for (uint32_t k = 0; k < m; ++k) {
            const uint32_t j = __ldg(&nl[k * cap + q]);
            if (touches(me, __ldg(&s.x[j]), __ldg(&s.y[j]), __ldg(&s.z[j]), __ldg(&s.r[j]))) mask |= 1ull << k;
        }
        return mask;
    }
    // Neighbour-list test: j may come within contact of i while both move less than
    // skin/2 (FP32 on the rounded positions, conservative by eps).
    static __device__ __forceinline__ bool within(const State& s, const Self& me, uint32_t j, float reach_extra) {
        const float ax = (float)__ldg(&s.x[j]) - (float)me.x, ay = (float)__ldg(&s.y[j]) - (float)me.y,
                    az = (float)__ldg(&s.z[j]) - (float)me.z;
        const float Re = (__ldg(&s.r[j]) + me.r) + reach_extra;
        return ax * ax + ay * ay + az * az < Re * Re;
    }
    static __device__ __forceinline__ float4 pos_f(const Self& m) {
        return make_float4((float)m.x, (float)m.y, (float)m.z, 0.f);
    }
    struct Partner {
        uint32_t j;
        uint32_t id;
        V3<double> v, w;
    };
    static __device__ __forceinline__ Partner load_partner(const State& s, uint32_t j) {
        Partner o;
        o.j = j;
        o.id = __ldg(&s.id[j]);
        load_vw(s, j, o.v, o.w);
        return o;
    }
    static __device__ __forceinline__ void partner_vw(const Partner& o, V3<double>& v, V3<double>& w) {
        v = o.v;
        w = o.w;
    }
    static __device__ __forceinline__ bool exact_p(const State& s, const Partner& o, const Self& me,
                                                   V3<double>& n, double& delta, float& rj) {
        return exact_j(s, me, o.j, n, delta, rj);
    }
    // Phase 2: geometry of a listed contact (the decision is the same as in scan_row).
    static __device__ __forceinline__ bool exact(const State& s, const Self& me, uint32_t j, const SceneDev&,
                                                 V3<double>& n, double& delta, float& rj) {
        return exact_j(s, me, j, n, delta, rj);
    }
    static __device__ __forceinline__ bool exact_j(const State& s, const Self& me, uint32_t j, V3<double>& n,
                                                   double& delta, float& rj) {
        const double dx = __dsub_rn(__ldg(&s.x[j]), me.x);
        const double dy = __dsub_rn(__ldg(&s.y[j]), me.y);
        const double dz = __dsub_rn(__ldg(&s.z[j]), me.z);
        const float rjf = __ldg(&s.r[j]);
        const double d2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
        const double R = __dadd_rn((double)me.r, (double)rjf);
        if (!(d2 < __dmul_rn(R, R))) return false;
        const double d = sqrt(d2);
        n = mk(dx / d, dy / d, dz / d);
        delta = R - d;
        rj = rjf;
        return true;
    }
    // Wall geometry: n from the sphere toward the wall, overlap, and c - p (contact point
    // relative to the wall's reference point).
    static __device__ __forceinline__ bool wall(const WallDev& W, const Self& me, const SceneDev&, V3<double>& n,
                                                double& delta, V3<double>& cp) {
        const V3<double> x = mk(me.x, me.y, me.z);
        const V3<double> p = mk(W.p[0], W.p[1], W.p[2]);
        const V3<double> a = mk(W.n[0], W.n[1], W.n[2]);
        const double r = (double)me.r;
        if (W.kind == 0) {
            const double s = dot(x - p, a);
            const double d = r - s;
            if (!(d > 0.0)) return false;
            n = a * -1.0;
            delta = d;
            cp = (x - a * s) - p;
            return true;
        }
        if (W.kind == 2) {
            // half-plate: the nearest plate point is the projection of the centre, or the
            // edge point beside it when the projection falls off the plate
            const V3<double> u = mk(W.u[0], W.u[1], W.u[2]);
            const V3<double> q = x - p;
            const double h = dot(q, a), s = dot(q, u);
            V3<double> e = a * -h;
            if (s < 0.0) e = e + u * -s;
            const double dist = sqrt(dot(e, e));
            const double d = r - dist;
            if (!(d > 0.0)) return false;
            n = dist > 0.0 ? e * (1.0 / dist) : a * -1.0;
            delta = d;
            cp = q + e;
            return true;
        }
        const V3<double> q = x - p;
        const double ax = dot(q, a);
        const V3<double> rho = q - a * ax;
        const double rr = sqrt(dot(rho, rho));
        const double d = rr + r - W.radius;
        if (!(d > 0.0) || !(rr > 0.0)) return false;
        n = rho * (1.0 / rr);
        delta = d;
        cp = a * ax + n * W.radius;
        return true;
    }
    static __device__ __forceinline__ V3<double> wall_omega(const WallDev& W) {
        return mk(W.omega[0], W.omega[1], W.omega[2]);
    }
    static __device__ __forceinline__ V3<double> wall_vel(const WallDev& W, V3<double> cp) {
        return mk(W.vel[0], W.vel[1], W.vel[2]) + cross(mk(W.omega[0], W.omega[1], W.omega[2]), cp);
    }
    static __device__ __forceinline__ double mass(const SceneDev& S, float r) {
        const double rd = (double)r;
        return S.cmass * rd * rd * rd;
    }
    static __device__ __forceinline__ uint32_t axis_cell(const SceneDev& S, int a, double xa, bool& clamped) {
        const double c = floor(__ddiv_rn(__dsub_rn(xa, S.origin[a]), S.h));
        if (!(c >= 0.0)) { clamped = true; return 0; }
        if (c >= (double)S.dims[a]) { clamped = true; return (uint32_t)(S.dims[a] - 1); }
        return (uint32_t)c;
    }
    static __device__ __forceinline__ uint32_t cell_key(const SceneDev& S, double x, double y, double z, bool& clamped) {
        const uint32_t i = axis_cell(S, 0, x, clamped), j = axis_cell(S, 1, y, clamped), k = axis_cell(S, 2, z, clamped);
        return S.c0 + cell_index(S, i, j, k);
    }
    static __device__ __forceinline__ uint32_t key_of(const State& s, const SceneDev& S, uint32_t q, bool& clamped) {
        return cell_key(S, s.x[q], s.y[q], s.z[q], clamped);
    }
    // Semi-implicit Euler (Sec. 4.2 step 1): v' = v + F dt/m, w' = w + T dt/I, x' = x + v' dt.
    static __device__ __forceinline__ uint32_t integrate(const State& B, uint32_t q, const Self& me, V3<double> F,
                                                         V3<double> Tq, const SceneDev& S, double m, bool& clamped,
                                                         bool& finite, float4& pnew) {
        const double r = (double)me.r;
        const double I = 0.4 * m * r * r;
        const V3<double> vn = me.v + F * (S.dt / m);
        const V3<double> wn = me.w + Tq * (S.dt / I);
        const double xn = me.x + vn.x * S.dt, yn = me.y + vn.y * S.dt, zn = me.z + vn.z * S.dt;
        B.x[q] = xn; B.y[q] = yn; B.z[q] = zn;
        B.r[q] = me.r;
        B.vx[q] = vn.x; B.vy[q] = vn.y; B.vz[q] = vn.z;
        B.wx[q] = wn.x; B.wy[q] = wn.y; B.wz[q] = wn.z;
        B.id[q] = me.id;
        finite = isfinite(xn) && isfinite(yn) && isfinite(zn) && isfinite(vn.x) && isfinite(vn.y) && isfinite(vn.z);
        pnew = make_float4((float)xn, (float)yn, (float)zn, (float)(dot(vn, vn) * (S.dt * S.dt)));
        return cell_key(S, xn, yn, zn, clamped);
    }
    static __device__ __forceinline__ V3<double> pos(const Self& m) { return mk(m.x, m.y, m.z); }
    static __device__ __forceinline__ V3<double> vel(const Self& m) { return m.v; }
    static __device__ __forceinline__ V3<double> spin(const Self& m) { return m.w; }
};

// ======================================================================= FP32 policy
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// Positions are hi + lo (two floats per coordinate, hi = fl32(hi + lo)).
__device__ __forceinline__ void ff_diff(float hi, float lo, float phi, float plo, float& u, float& ul) {
    float e;
    two_sum(hi, -phi, u, e);
    ul = __fadd_rn(__fsub_rn(lo, plo), e);
}

struct PF32 {
    using T = float;
    using State = StateF32;
    struct Self {
        float hx, hy, hz, r, lx, ly, lz;
        V3<float> v, w;
        uint32_t id;
    };
    static __device__ __forceinline__ Self load(const State& s, uint32_t q) {
        Self m;
        const float4 p0 = __ldg(&s.P0[q]), p1 = __ldg(&s.P1[q]), v = __ldg(&s.V[q]), w = __ldg(&s.W[q]);
        m.hx = p0.x; m.hy = p0.y; m.hz = p0.z; m.r = p0.w;
        m.lx = p1.x; m.ly = p1.y; m.lz = p1.z;
        m.v = mk(v.x, v.y, v.z);
        m.w = mk(w.x, w.y, w.z);
        m.id = __float_as_uint(p1.w);
        return m;
    }
    // P1.w carries the bits of the particle's id (also kept in the id plane), so a partner's
    // id arrives with its low position words.
    static __device__ __forceinline__ void store(const State& s, uint32_t q, const Self& m) {
        s.P0[q] = make_float4(m.hx, m.hy, m.hz, m.r);
        s.P1[q] = make_float4(m.lx, m.ly, m.lz, __uint_as_float(m.id));
        s.V[q] = make_float4(m.v.x, m.v.y, m.v.z, 0.f);
        s.W[q] = make_float4(m.w.x, m.w.y, m.w.z, 0.f);
        s.id[q] = m.id;
    }
    static __device__ __forceinline__ void load_vw(const State& s, uint32_t j, V3<float>& v, V3<float>& w) {
        const float4 a = __ldg(&s.V[j]), b = __ldg(&s.W[j]);
        v = mk(a.x, a.y, a.z);
        w = mk(b.x, b.y, b.z);
    }
    // FP32 prefilter on hi: conservative by eps_f (it bounds the FP32 error of hi_j - hi_i
    // and of the squared distance), so no pair in contact is ever rejected.
    static __device__ __forceinline__ bool near(const Self& me, float4 pj, float eps) {
        const float ax = pj.x - me.hx, ay = pj.y - me.hy, az = pj.z - me.hz;
        const float Re = (pj.w + me.r) + eps;
        return ax * ax + ay * ay + az * az < Re * Re;
    }
    // Phase 1 of the walk: append to the near list every particle of [j0, j1) that passes
    // the prefilter (two candidates in flight per iteration).
    static __device__ __forceinline__ void scan_row(const State& s, const Self& me, const SceneDev& S, uint32_t j0,
                                                    uint32_t j1, uint32_t q, uint32_t* lst, uint32_t bd, uint32_t tid,
                                                    uint32_t maxc, uint32_t& cnt) {
        const float eps = S.eps_f;
        uint32_t j = j0;
        for (; j + 2 <= j1; j += 2) {
            const float4 a = __ldg(&s.P0[j]), b = __ldg(&s.P0[j + 1]);
            if (j != q && near(me, a, eps)) {
                if (cnt < maxc) lst[cnt * bd + tid] = j;
                ++cnt;
            }
            if (j + 1 != q && near(me, b, eps)) {
                if (cnt < maxc) lst[cnt * bd + tid] = j + 1;
                ++cnt;
            }
        }
        if (j < j1 && j != q && near(me, __ldg(&s.P0[j]), eps)) {
            if (cnt < maxc) lst[cnt * bd + tid] = j;
            ++cnt;
        }
    }
    // Phase 1 from a neighbour list built at the last sort: bit k of the returned mask
    // marks list entry k as passing the prefilter (two candidates in flight).
    static __device__ __forceinline__ uint64_t scan_list(const State& s, const Self& me, const SceneDev& S,
                                                         const uint32_t* nl, uint32_t m, size_t cap, uint32_t q) {
        const float eps = S.eps_f;
        uint64_t mask = 0;
        uint32_t k = 0;
        // (no L1 prefetch of the near candidates' payload: measured 9% slower here and 4%
        // in the walk; the prefetched lines are evicted before phase 2 reads them)
        for (; k + DEM_SCAN_UNROLL <= m; k += DEM_SCAN_UNROLL) {
            uint32_t j[DEM_SCAN_UNROLL];
            float4 pj[DEM_SCAN_UNROLL];
#pragma unroll
            for (int u = 0; u < DEM_SCAN_UNROLL; ++u) j[u] = __ldg(&nl[(k + u) * cap + q]);
#pragma unroll
            for (int u = 0; u < DEM_SCAN_UNROLL; ++u) pj[u] = __ldg(&s.P0[j[u]]);
#pragma unroll
            for (int u = 0; u < DEM_SCAN_UNROLL; ++u)
                if (near(me, pj[u], eps)) mask |= 1ull << (k + u);
        }
        for (; k < m; ++k) {
            const uint32_t j0 = __ldg(&nl[k * cap + q]);
            if (near(me, __ldg(&s.P0[j0]), eps)) mask |= 1ull << k;
        }
        return mask;
    }
    // Neighbour-list test: j may come within contact of i while both move less than
    // skin/2 (FP32 on hi, conservative by eps).
    static __device__ __forceinline__ bool within(const State& s, const Self& me, uint32_t j, float reach_extra) {
        const float4 pj = __ldg(&s.P0[j]);
        const float ax = pj.x - me.hx, ay = pj.y - me.hy, az = pj.z - me.hz;
        const float Re = (pj.w + me.r) + reach_extra;
        return ax * ax + ay * ay + az * az < Re * Re;
    }
    static __device__ __forceinline__ float4 pos_f(const Self& m) { return make_float4(m.hx, m.hy, m.hz, 0.f); }
    // Everything phase 2 reads of a candidate, loaded together so the latencies overlap.
    struct Partner {
        float4 p0, p1, v, w;
        uint32_t id;
    };
    static __device__ __forceinline__ Partner load_partner(const State& s, uint32_t j) {
        Partner o;
        o.p0 = __ldg(&s.P0[j]);
        o.p1 = __ldg(&s.P1[j]);
        o.v = __ldg(&s.V[j]);
        o.w = __ldg(&s.W[j]);
        o.id = __float_as_uint(o.p1.w);
        return o;
    }
    static __device__ __forceinline__ void partner_vw(const Partner& o, V3<float>& v, V3<float>& w) {
        v = mk(o.v.x, o.v.y, o.v.z);
        w = mk(o.w.x, o.w.y, o.w.z);
    }
    static __device__ __forceinline__ bool exact_p(const State&, const Partner& o, const Self& me, V3<float>& n,
                                                   float& delta, float& rj) {
        return exact_xy(o.p0, o.p1, me, n, delta, rj);
    }
    // Phase 2: the sign of R^2 - d^2 evaluated with error-free transformations (about
    // 2^-46 relative to R^2), then delta = (R^2 - d^2)/(R + d) and the unit normal.
    static __device__ __forceinline__ bool exact(const State& s, const Self& me, uint32_t j, const SceneDev&,
                                                 V3<float>& n, float& delta, float& rj) {
        return exact_xy(__ldg(&s.P0[j]), __ldg(&s.P1[j]), me, n, delta, rj);
    }
    static __device__ __forceinline__ bool exact_xy(const float4 pj, const float4 lj, const Self& me, V3<float>& n,
                                                    float& delta, float& rj) {
        float sx, tx, sy, ty, sz, tz;
        float px, pex, py, pey, pz, pez;
#if DEM_PACKED_FF
        // x and y in the two lanes of the paired FP32 instructions (each lane rounds like
        // the scalar operation, so the bits are those of the scalar code below)
        {
            // TwoSum(hi_j, -hi_i) and the low-word difference, as in ff_diff
            const float2 a = make_float2(pj.x, pj.y), b = make_float2(-me.hx, -me.hy);
            const float2 s = __fadd2_rn(a, b);
            const float2 bb = __fadd2_rn(s, neg2(a));
            const float2 u = __fadd2_rn(s, neg2(bb));
            const float2 e = __fadd2_rn(__fadd2_rn(a, neg2(u)), __fadd2_rn(b, neg2(bb)));
            const float2 t = __fadd2_rn(__fadd2_rn(make_float2(lj.x, lj.y), make_float2(-me.lx, -me.ly)), e);
            // TwoProd(s, s)
            const float2 p = __fmul2_rn(s, s);
            const float2 pe = __ffma2_rn(s, s, neg2(p));
            sx = s.x; sy = s.y; tx = t.x; ty = t.y;
            px = p.x; py = p.y; pex = pe.x; pey = pe.y;
        }
#else
        ff_diff(pj.x, lj.x, me.hx, me.lx, sx, tx);
        ff_diff(pj.y, lj.y, me.hy, me.ly, sy, ty);
        two_prod(sx, sx, px, pex);
        two_prod(sy, sy, py, pey);
#endif
        ff_diff(pj.z, lj.z, me.hz, me.lz, sz, tz);
        two_prod(sz, sz, pz, pez);
        float Rh, Rl;
        two_sum(me.r, pj.w, Rh, Rl);
        float qh, qe;
        two_prod(Rh, Rh, qh, qe);
        float a1, e1, a2, e2, a3, e3;
        two_sum(qh, -px, a1, e1);
        two_sum(a1, -py, a2, e2);
        two_sum(a2, -pz, a3, e3);
        const float cx = __fmaf_rn(2.f * sx, tx, __fmul_rn(tx, tx));
        const float cy = __fmaf_rn(2.f * sy, ty, __fmul_rn(ty, ty));
        const float cz = __fmaf_rn(2.f * sz, tz, __fmul_rn(tz, tz));
        const float rr = __fmaf_rn(2.f * Rh, Rl, __fmul_rn(Rl, Rl));
        float low = __fadd_rn(__fadd_rn(e1, e2), e3);
        low = __fadd_rn(low, __fadd_rn(qe, rr));
        low = __fsub_rn(low, __fadd_rn(__fadd_rn(pex, pey), pez));
        low = __fsub_rn(low, __fadd_rn(__fadd_rn(cx, cy), cz));
        const float D = __fadd_rn(a3, low);
        if (!(D > 0.f)) return false;
        const float d = law_sqrt(__fadd_rn(__fadd_rn(px, py), pz));
        delta = law_div(D, __fadd_rn(Rh, d));
        const float dc = __fadd_rn(__fsub_rn(Rh, delta), Rl);
        const float inv = law_div(1.f, dc);
        n = mk(__fmul_rn(__fadd_rn(sx, tx), inv), __fmul_rn(__fadd_rn(sy, ty), inv), __fmul_rn(__fadd_rn(sz, tz), inv));
        rj = pj.w;
        return true;
    }
    static __device__ __forceinline__ float hic(const Self& m, int a) { return a == 0 ? m.hx : (a == 1 ? m.hy : m.hz); }
    static __device__ __forceinline__ float loc(const Self& m, int a) { return a == 0 ? m.lx : (a == 1 ? m.ly : m.lz); }
    // Half-plate whose normal (axis na) and edge-to-plate direction u (axis ua) are
    // coordinate axes. Height h and the distance s from the edge line are float-float;
    // over the plate (s >= 0) delta = r - |h|, beside it the nearest point is on the edge
    // and delta = (r^2 - dist^2) / (r + dist) with dist^2 = s^2 + h^2.
    static __device__ __noinline__ bool half_plate(const WallDev& W, const Self& me, const SceneDev& S,
                                                      V3<float>& n, float& delta, V3<float>& cp) {
        const float r = me.r;
        const int na = W.axis, ua = W.uaxis, oa = 3 - W.axis - W.uaxis;
        const float sn = W.n_hi[na], su = W.uf[ua];
        if (fabsf(sn * (hic(me, na) - W.pf[na])) >= r + S.eps_f) return false;
        float hh, hl, sh, sl;
        ff_diff(hic(me, na), loc(me, na), W.p_hi[na], W.p_lo[na], hh, hl);
        ff_diff(hic(me, ua), loc(me, ua), W.p_hi[ua], W.p_lo[ua], sh, sl);
        hh *= sn; hl *= sn; sh *= su; sl *= su;
        const float th = sh, tl = sl;
        float c[3];
        c[oa] = __fadd_rn(hic(me, oa) - W.pf[oa], loc(me, oa) - W.p_lo[oa]);
        c[na] = 0.f;
        float nn[3] = {0.f, 0.f, 0.f};
        if (sh > 0.f || (sh == 0.f && sl >= 0.f)) {
            const bool up = hh > 0.f || (hh == 0.f && hl >= 0.f);
            float dh, de;
            two_sum(r, up ? -hh : hh, dh, de);
            const float d = __fadd_rn(dh, __fsub_rn(de, up ? hl : -hl));
            if (!(d > 0.f)) return false;
            delta = d;
            nn[na] = up ? -sn : sn;
            c[ua] = su * __fadd_rn(sh, sl);
        } else {
            float pt, pte, ph, phe, s1, e1, rr, rre, a, ae;
            two_prod(th, th, pt, pte);
            two_prod(hh, hh, ph, phe);
            two_sum(pt, ph, s1, e1);
            float rlo = __fadd_rn(e1, __fadd_rn(pte, phe));
            rlo = __fadd_rn(rlo, __fadd_rn(__fmaf_rn(2.f * th, tl, __fmul_rn(tl, tl)),
                                           __fmaf_rn(2.f * hh, hl, __fmul_rn(hl, hl))));
            two_prod(r, r, rr, rre);
            two_sum(rr, -s1, a, ae);
            const float D = __fadd_rn(a, __fadd_rn(ae, __fsub_rn(rre, rlo)));
            if (!(D > 0.f)) return false;
            delta = __fdiv_rn(D, __fadd_rn(r, sqrtf(s1)));
            const float dist = __fsub_rn(r, delta);
            if (dist > 0.f) {
                const float inv = __fdiv_rn(1.f, dist);
                nn[ua] = -su * __fmul_rn(__fadd_rn(th, tl), inv);
                nn[na] = -sn * __fmul_rn(__fadd_rn(hh, hl), inv);
            } else {
                nn[na] = -sn;
            }
            c[ua] = 0.f;
        }
        n = mk(nn[0], nn[1], nn[2]);
        cp = mk(c[0], c[1], c[2]);
        return true;
    }
    static __device__ __forceinline__ bool wall(const WallDev& W, const Self& me, const SceneDev& S, V3<float>& n,
                                                float& delta, V3<float>& cp) {
        const float r = me.r;
        if (W.kind == 0) {
            // prefilter: centre farther than r + eps from the plane
            const float sf = W.nf[0] * (me.hx - W.pf[0]) + W.nf[1] * (me.hy - W.pf[1]) + W.nf[2] * (me.hz - W.pf[2]);
            if (sf >= r + S.eps_f) return false;
            float u[3], ul[3];
            for (int a = 0; a < 3; ++a) ff_diff(hic(me, a), loc(me, a), W.p_hi[a], W.p_lo[a], u[a], ul[a]);
            float sh, sl;
            if (W.axis >= 0) {
                const float sg = W.n_hi[W.axis];
                sh = u[W.axis] * sg;
                sl = ul[W.axis] * sg;
            } else {
                float m0, e0, m1, e1, m2, e2;
                two_prod(W.n_hi[0], u[0], m0, e0);
                two_prod(W.n_hi[1], u[1], m1, e1);
                two_prod(W.n_hi[2], u[2], m2, e2);
                float s01, f01, s012, f012;
                two_sum(m0, m1, s01, f01);
                two_sum(s01, m2, s012, f012);
                float lw = __fadd_rn(__fadd_rn(e0, e1), e2);
                lw = __fadd_rn(lw, __fadd_rn(f01, f012));
                for (int a = 0; a < 3; ++a)
                    lw = __fadd_rn(lw, __fadd_rn(__fmul_rn(W.n_hi[a], ul[a]), __fmul_rn(W.n_lo[a], u[a])));
                sh = s012;
                sl = lw;
            }
            float dh, de;
            two_sum(r, -sh, dh, de);
            const float d = __fadd_rn(dh, __fsub_rn(de, sl));
            if (!(d > 0.f)) return false;
            n = mk(-W.nf[0], -W.nf[1], -W.nf[2]);
            delta = d;
            const float s = __fadd_rn(sh, sl);
            cp = mk((u[0] + ul[0]) - s * W.nf[0], (u[1] + ul[1]) - s * W.nf[1], (u[2] + ul[2]) - s * W.nf[2]);
            return true;
        }
        if (W.kind == 2) return half_plate(W, me, S, n, delta, cp);
        // cylinder interior with a coordinate axis
        const int ax = W.axis, b = (ax + 1) % 3, c = (ax + 2) % 3;
        const float gf = W.rad_hi - r;
        {
            const float ub = hic(me, b) - W.pf[b], uc = hic(me, c) - W.pf[c];
            const float lim = gf - S.eps_f;
            if (lim > 0.f && ub * ub + uc * uc <= lim * lim) return false;
        }
        float ub, ubl, uc, ucl;
        ff_diff(hic(me, b), loc(me, b), W.p_hi[b], W.p_lo[b], ub, ubl);
        ff_diff(hic(me, c), loc(me, c), W.p_hi[c], W.p_lo[c], uc, ucl);
        float pb, peb, pc, pec;
        two_prod(ub, ub, pb, peb);
        two_prod(uc, uc, pc, pec);
        float s1, e1;
        two_sum(pb, pc, s1, e1);
        float rlo = __fadd_rn(e1, __fadd_rn(peb, pec));
        rlo = __fadd_rn(rlo, __fadd_rn(__fmaf_rn(2.f * ub, ubl, __fmul_rn(ubl, ubl)),
                                       __fmaf_rn(2.f * uc, ucl, __fmul_rn(ucl, ucl))));
        float g, ge;
        two_sum(W.rad_hi, -r, g, ge);
        const float gl = __fadd_rn(ge, W.rad_lo);
        float gg, gge;
        two_prod(g, g, gg, gge);
        const float glo = __fadd_rn(gge, __fmaf_rn(2.f * g, gl, __fmul_rn(gl, gl)));
        float a, ae;
        two_sum(s1, -gg, a, ae);
        const float D = __fadd_rn(a, __fadd_rn(ae, __fsub_rn(rlo, glo)));
        if (!(D > 0.f)) return false;
        const float rho = sqrtf(s1);
        if (!(rho > 0.f)) return false;
        delta = __fdiv_rn(D, __fadd_rn(rho, g));
        const float rc = __fadd_rn(__fadd_rn(g, gl), delta);
        const float inv = __fdiv_rn(1.f, rc);
        float nn[3];
        nn[ax] = 0.f;
        nn[b] = __fmul_rn(__fadd_rn(ub, ubl), inv);
        nn[c] = __fmul_rn(__fadd_rn(uc, ucl), inv);
        n = mk(nn[0], nn[1], nn[2]);
        float cpp[3];
        cpp[ax] = hic(me, ax) - W.pf[ax] + (loc(me, ax) - W.p_lo[ax]);
        cpp[b] = W.rad_hi * nn[b];
        cpp[c] = W.rad_hi * nn[c];
        cp = mk(cpp[0], cpp[1], cpp[2]);
        return true;
    }
    static __device__ __forceinline__ V3<float> wall_omega(const WallDev& W) {
        return mk(W.omegaf[0], W.omegaf[1], W.omegaf[2]);
    }
    static __device__ __forceinline__ V3<float> wall_vel(const WallDev& W, V3<float> cp) {
        return mk(W.velf[0], W.velf[1], W.velf[2]) + cross(mk(W.omegaf[0], W.omegaf[1], W.omegaf[2]), cp);
    }
    static __device__ __forceinline__ float mass(const SceneDev& S, float r) { return S.cmass_f * (r * r * r); }
    static __device__ __forceinline__ uint32_t axis_cell(const SceneDev& S, int a, float hi, bool& clamped) {
        const float c = floorf(__fdiv_rn(__fsub_rn(hi, S.origin_f[a]), S.h_f));
        if (!(c >= 0.f)) { clamped = true; return 0; }
        if (c >= (float)S.dims[a]) { clamped = true; return (uint32_t)(S.dims[a] - 1); }
        return (uint32_t)c;
    }
    static __device__ __forceinline__ uint32_t cell_key(const SceneDev& S, float x, float y, float z, bool& clamped) {
        const uint32_t i = axis_cell(S, 0, x, clamped), j = axis_cell(S, 1, y, clamped), k = axis_cell(S, 2, z, clamped);
        return S.c0 + cell_index(S, i, j, k);
    }
    static __device__ __forceinline__ uint32_t key_of(const State& s, const SceneDev& S, uint32_t q, bool& clamped) {
        const float4 p = s.P0[q];
        return cell_key(S, p.x, p.y, p.z, clamped);
    }
    // position += dt * v' with compensated summation: TwoSum(hi, dx), lo += err, renormalise
    static __device__ __forceinline__ void advance(float& hi, float& lo, float dx) {
        float s, e;
        two_sum(hi, dx, s, e);
        const float l2 = __fadd_rn(lo, e);
        two_sum(s, l2, hi, lo);
    }
    static __device__ __forceinline__ uint32_t integrate(const State& B, uint32_t q, const Self& me, V3<float> F,
                                                         V3<float> Tq, const SceneDev& S, float m, bool& clamped,
                                                         bool& finite, float4& pnew) {
        const float r = me.r;
        const float I = 0.4f * m * r * r;
        const V3<float> vn = me.v + F * (S.dt_f / m);
        const V3<float> wn = me.w + Tq * (S.dt_f / I);
        float hx = me.hx, hy = me.hy, hz = me.hz, lx = me.lx, ly = me.ly, lz = me.lz;
        advance(hx, lx, __fmul_rn(vn.x, S.dt_f));
        advance(hy, ly, __fmul_rn(vn.y, S.dt_f));
        advance(hz, lz, __fmul_rn(vn.z, S.dt_f));
        B.P0[q] = make_float4(hx, hy, hz, r);
        B.P1[q] = make_float4(lx, ly, lz, __uint_as_float(me.id));
        B.V[q] = make_float4(vn.x, vn.y, vn.z, 0.f);
        B.W[q] = make_float4(wn.x, wn.y, wn.z, 0.f);
        B.id[q] = me.id;
        finite = isfinite(hx) && isfinite(hy) && isfinite(hz) && isfinite(vn.x) && isfinite(vn.y) && isfinite(vn.z);
        pnew = make_float4(hx, hy, hz, dot(vn, vn) * (S.dt_f * S.dt_f));
        return cell_key(S, hx, hy, hz, clamped);
    }
    static __device__ __forceinline__ V3<double> pos(const Self& m) {
        return mk((double)m.hx + (double)m.lx, (double)m.hy + (double)m.ly, (double)m.hz + (double)m.lz);
    }
    static __device__ __forceinline__ V3<double> vel(const Self& m) { return mk((double)m.v.x, (double)m.v.y, (double)m.v.z); }
    static __device__ __forceinline__ V3<double> spin(const Self& m) { return mk((double)m.w.x, (double)m.w.y, (double)m.w.z); }
};

// Load the stored tangential spring of slot k (partner ids are in shared memory).
template <class T>
__device__ __forceinline__ V3<T> find_spring(const uint32_t* s_oid, uint32_t bd, uint32_t tid, uint32_t cnt_old,
                                             uint32_t gid, const T* hin_d, size_t maxc, size_t cap, uint32_t src) {
    for (uint32_t k = 0; k < cnt_old; ++k)
        if (s_oid[k * bd + tid] == gid)
            return mk(__ldg(&hin_d[(0 * maxc + k) * cap + src]), __ldg(&hin_d[(1 * maxc + k) * cap + src]),
                      __ldg(&hin_d[(2 * maxc + k) * cap + src]));
    return mk(T(0), T(0), T(0));
}

}  // namespace demgb
