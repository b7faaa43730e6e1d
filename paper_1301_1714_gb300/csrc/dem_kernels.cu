// Kernels of the GB300 DEM timestep and their launchers.
//
//   k_force      steps 5-8 + 1 + 2: 27-cell contact search (Eq. 12) or neighbour list,
//                contact laws (Eq. 1 or Eqs. 2-10), walls, gravity, semi-implicit Euler,
//                then the new cell key CM and its rank within the cell (sort every step)
//                or the displacement test that decides a sort (neighbour lists)
//   k_hash       step 2 for a sort step in list mode
//   k_scan_*     exclusive scan of per-cell counts -> dense cell-start table
//   k_scatter    particles into cell-major slots (order within a cell still arbitrary)
//   k_reorder    step 4: (cell, id) order (Eq. 11) and gather of every property
//   k_nlist      neighbour lists of the sorted state (list mode)
//   k_end_step   per-step bookkeeping of the device-side step control
//   k_import / k_export / k_diag* / k_hist_canon / k_repack   set-up, read-out,
//                diagnostics, batch repacking
#include <algorithm>

#include <cuda_runtime.h>

#include "dem_domain.h"

// Minimum resident 256-thread blocks per SM requested for the force kernel, which caps
// its registers at 65536 / (256 * value): 64 registers in both modes (measured on
// GB300: the list-mode pass is 11% faster at 64 than at 80; the walk-mode pass, once it
// stopped prefetching its candidates' payload, 10% faster; 48 spills and is 19% slower).
#ifndef DEM_FORCE_MIN_BLOCKS
#define DEM_FORCE_MIN_BLOCKS 4
#endif
#ifndef DEM_FORCE_MIN_BLOCKS_LIST
#define DEM_FORCE_MIN_BLOCKS_LIST 4
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
        return S.c0 + (k * (uint32_t)S.dims[1] + j) * (uint32_t)S.dims[0] + i;
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
        for (; k + 2 <= m; k += 2) {
            const uint32_t j0 = __ldg(&nl[k * cap + q]), j1 = __ldg(&nl[(k + 1) * cap + q]);
            const float4 a = __ldg(&s.P0[j0]), b = __ldg(&s.P0[j1]);
            if (near(me, a, eps)) mask |= 1ull << k;
            if (near(me, b, eps)) mask |= 1ull << (k + 1);
        }
        if (k < m) {
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
        ff_diff(pj.x, lj.x, me.hx, me.lx, sx, tx);
        ff_diff(pj.y, lj.y, me.hy, me.ly, sy, ty);
        ff_diff(pj.z, lj.z, me.hz, me.lz, sz, tz);
        float px, pex, py, pey, pz, pez;
        two_prod(sx, sx, px, pex);
        two_prod(sy, sy, py, pey);
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
        return S.c0 + (k * (uint32_t)S.dims[1] + j) * (uint32_t)S.dims[0] + i;
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

// ======================================================================= force pass
template <class PR>
struct ForceArgs {
    const SceneDev* scenes;
    int nscenes;
    uint32_t n, cap;
    int maxc, stiffness;
    typename PR::State S0, S1;   // the two state sets; ctrl->cur names the current one
    CtrlDev* ctrl;
    const uint32_t* ncnt;        // list mode: neighbour lists of the last sort
    const uint32_t* nl;
    const float4* ref;           // list mode: positions at the last sort
    float thresh2;               // list mode: squared displacement that forces a sort
    int interval;                // list mode: sort at least every `interval` steps (0: never forced)
    const uint32_t* skey;
    const uint32_t* cs;
    const uint32_t* perm;
    const uint32_t* hin_cnt;
    const uint32_t* hin_pid;
    const typename PR::T* hin_d;
    uint32_t* hout_cnt;
    uint32_t* hout_pid;
    typename PR::T* hout_d;
    uint32_t* key;
    uint32_t* rank;
    uint32_t* cnt;
    StatusDev* st;
    double* dbgF;
    double* dbgT;
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

// One thread per cell-sorted particle. Phase 1 walks the 27 cells (Eq. 12) as 9 rows of
// three x-adjacent cells and keeps the candidates that may touch in a per-thread list in
// shared memory; phase 2 runs the lanes of a warp in lockstep over their lists (the warp
// iterates max-list-length times instead of once per candidate), taking the contact
// decision, the law (Eq. 1 or Eqs. 2-10) and the springs; then walls, gravity, the
// update (step 1) and the new cell key with its rank in the cell (step 2).
// MODEL: 0 the practical law, 1 the simple law (Eq. 1), 2 the practical law with the
// scene's optional terms (no attraction, rolling resistance).
template <class PR, int MODEL, bool EVAL, bool LIST>
__global__ void __launch_bounds__(256, LIST ? DEM_FORCE_MIN_BLOCKS_LIST : DEM_FORCE_MIN_BLOCKS) k_force(ForceArgs<PR> a) {
    using T = typename PR::T;
    constexpr bool PRACT = MODEL != 1;
    constexpr bool TERMS = MODEL == 2;
    extern __shared__ uint32_t smem[];
    const int cur = a.ctrl->cur;
    const typename PR::State A = cur ? a.S1 : a.S0;
    const typename PR::State B = cur ? a.S0 : a.S1;
    const bool pv = a.ctrl->perm_valid != 0;
    if (LIST && !EVAL && blockIdx.x == 0 && threadIdx.x == 0 && a.interval > 0 && a.ctrl->since + 1 >= a.interval)
        atomicOr(&a.ctrl->rebuild, 1);
    const uint32_t tid = threadIdx.x;
    const uint32_t bd = blockDim.x;
    const uint32_t maxc = (uint32_t)a.maxc;
    uint32_t* s_oid = smem;               // [maxc][bd] partner ids of the stored springs
    uint32_t* s_near = smem + maxc * bd;  // [maxc][bd] near candidates of phase 1 (walk mode)
    uint64_t near_mask = 0;               // list mode: list entries that passed phase 1
    const uint32_t q = blockIdx.x * bd + tid;
    const size_t cap = a.cap;
    uint32_t c_pp = 0, c_wc = 0, c_clamp = 0, c_nnew = 0;
    float c_maxov = 0.f, c_disp2 = 0.f;
    const bool valid = q < a.n;
    const SceneDev& S = a.scenes[valid ? scene_of(a.scenes, a.nscenes, q) : 0];
    const bool live = valid && S.active;
    typename PR::Self me{};
    uint32_t src = 0, cnt_old = 0, nnear = 0;
    if (valid) {
        me = PR::load(A, q);
        src = pv ? __ldg(&a.perm[q]) : q;
        if (PRACT || !S.active) {
            cnt_old = min(__ldg(&a.hin_cnt[src]), maxc);
            // the stored springs are streamed from DRAM: start their loads now so they are
            // in L1 when phase 2 matches contacts against them
            for (uint32_t k = 0; k < cnt_old; ++k)
                for (int c = 0; c < 3; ++c) prefetch_l1(&a.hin_d[(c * (size_t)maxc + k) * cap + src]);
            for (uint32_t k = 0; k < cnt_old; ++k) s_oid[k * bd + tid] = __ldg(&a.hin_pid[k * cap + src]);
        }
    }
    if (valid && !live) {
        // frozen scene: carry state and springs unchanged
        if (!EVAL) {
            PR::store(B, q, me);
            for (uint32_t k = 0; k < cnt_old; ++k) {
                a.hout_pid[k * cap + q] = s_oid[k * bd + tid];
                for (int c = 0; c < 3; ++c)
                    a.hout_d[(c * (size_t)maxc + k) * cap + q] = a.hin_d[(c * (size_t)maxc + k) * cap + src];
            }
            a.hout_cnt[q] = cnt_old;
            if (!LIST) {
                const uint32_t kk = a.skey[q];
                a.key[q] = kk;
                a.rank[q] = atomicAdd(&a.cnt[kk], 1u);
            }
        } else {
            a.hout_cnt[q] = 0;
        }
    }
    // ---- phase 1: candidates that may touch. The 18 cell-start loads of the 9 rows are
    // issued together before any candidate is read.
    if (live && LIST) {
        near_mask = PR::scan_list(A, me, S, a.nl, min(__ldg(&a.ncnt[q]), 2 * maxc), cap, q);
        nnear = __popcll(near_mask);
    } else if (live) {
        const int nx = S.dims[0], ny = S.dims[1], nz = S.dims[2];
        const uint32_t local = a.skey[q] - S.c0;
        const int ix = (int)(local % (uint32_t)nx);
        const uint32_t t1 = local / (uint32_t)nx;
        const int iy = (int)(t1 % (uint32_t)ny);
        const int iz = (int)(t1 / (uint32_t)ny);
        const uint32_t xlo = (uint32_t)max(ix - 1, 0), xhi = (uint32_t)min(ix + 1, nx - 1) + 1;
        uint32_t rlo[9], rhi[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            const int z2 = iz + r / 3 - 1, y2 = iy + r % 3 - 1;
            const bool ok = z2 >= 0 && z2 < nz && y2 >= 0 && y2 < ny;
            const uint32_t rowbase = S.c0 + (uint32_t)((z2 * ny + y2) * nx);
            rlo[r] = ok ? __ldg(&a.cs[rowbase + xlo]) : 0u;
            rhi[r] = ok ? __ldg(&a.cs[rowbase + xhi]) : 0u;
        }
#pragma unroll
        for (int r = 0; r < 9; ++r)
            PR::scan_row(A, me, S, rlo[r], rhi[r], q, s_near, bd, tid, maxc, nnear);
        if (nnear > maxc) raise_status(a.st, ST_CAPACITY, (int32_t)q);
    }
    // ---- phase 2: contacts, in lockstep over the lists
    const uint32_t mylen = LIST ? nnear : min(nnear, maxc);
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, mylen);
    V3<T> F = mk(T(0), T(0), T(0)), Tq = mk(T(0), T(0), T(0));
    uint32_t nnew = 0;
    T mi = T(0);
    const T ri = (T)me.r;
    Law<T> L{};
    if (live) {
        L = law_of(S, a.stiffness, T());
        mi = PR::mass(S, me.r);
    }
    uint64_t mask_left = near_mask;
    for (uint32_t k = 0; k < kmax; ++k) {
        if (!(live && k < mylen)) continue;
        uint32_t j;
        if (LIST) {
            const int e = __ffsll((long long)mask_left) - 1;
            mask_left &= mask_left - 1;
            j = __ldg(&a.nl[(size_t)e * cap + q]);
        } else {
            j = s_near[k * bd + tid];
        }
        V3<T> n;
        T delta;
        float rj;
        const typename PR::Partner o = PR::load_partner(A, j);
        if (!PR::exact_p(A, o, me, n, delta, rj)) continue;
        const uint32_t gid = o.id;
        V3<T> vj, wj;
        PR::partner_vw(o, vj, wj);
        const V3<T> v = me.v - vj;
        if (PRACT) {
            const T rjT = (T)rj;
            const V3<T> rw = mk(sym_madd(ri, me.w.x, rjT, wj.x), sym_madd(ri, me.w.y, rjT, wj.y),
                                sym_madd(ri, me.w.z, rjT, wj.z));
            const T mj = PR::mass(S, rj);
            const T meff = law_div(mi * mj, mi + mj);
            const T Reff = law_div(ri * rjT, ri + rjT);
            const V3<T> dold = find_spring(s_oid, bd, tid, cnt_old, gid, a.hin_d, (size_t)maxc, cap, src);
            V3<T> Fc, Ftc, dnew, Mr;
            law_practical<TERMS>(L, n, delta, v, rw, Reff, meff, dold, Fc, Ftc, dnew, me.w - wj, Mr);
            F = F + Fc;
            Tq = Tq + cross(n, Ftc) * ri;
            if (TERMS) Tq = Tq + Mr;
            if (nnew < maxc) {
                a.hout_pid[nnew * cap + q] = gid;
                a.hout_d[(0 * (size_t)maxc + nnew) * cap + q] = dnew.x;
                a.hout_d[(1 * (size_t)maxc + nnew) * cap + q] = dnew.y;
                a.hout_d[(2 * (size_t)maxc + nnew) * cap + q] = dnew.z;
            }
        } else {
            F = F + law_simple(L, n, delta, v);
            if (EVAL && nnew < maxc) a.hout_pid[nnew * cap + q] = gid;
        }
        ++nnew;
        ++c_pp;
        c_maxov = fmaxf(c_maxov, (float)delta);
    }
    if (live) {
        // ---- walls (step 8)
        for (int w = 0; w < S.nwalls; ++w) {
            const WallDev& W = S.walls[w];
            V3<T> n, cp;
            T delta;
            if (!PR::wall(W, me, S, n, delta, cp)) continue;
            const V3<T> v = me.v - PR::wall_vel(W, cp);
            const uint32_t gid = DEM_WALL_BASE + (uint32_t)w;
            if (PRACT) {
                const V3<T> rw = me.w * ri;
                const V3<T> dold = find_spring(s_oid, bd, tid, cnt_old, gid, a.hin_d, (size_t)maxc, cap, src);
                V3<T> Fc, Ftc, dnew, Mr;
                law_practical<TERMS>(L, n, delta, v, rw, ri, mi, dold, Fc, Ftc, dnew, me.w - PR::wall_omega(W), Mr);
                F = F + Fc;
                Tq = Tq + cross(n, Ftc) * ri;
                if (TERMS) Tq = Tq + Mr;
                if (nnew < maxc) {
                    a.hout_pid[nnew * cap + q] = gid;
                    a.hout_d[(0 * (size_t)maxc + nnew) * cap + q] = dnew.x;
                    a.hout_d[(1 * (size_t)maxc + nnew) * cap + q] = dnew.y;
                    a.hout_d[(2 * (size_t)maxc + nnew) * cap + q] = dnew.z;
                }
            } else {
                F = F + law_simple(L, n, delta, v);
                if (EVAL && nnew < maxc) a.hout_pid[nnew * cap + q] = gid;
            }
            ++nnew;
            ++c_wc;
            c_maxov = fmaxf(c_maxov, (float)delta);
        }
        if (nnew > maxc) raise_status(a.st, ST_CAPACITY, (int32_t)q);
        c_nnew = nnew;
        if (PRACT || EVAL) a.hout_cnt[q] = min(nnew, maxc);
        // gravity, once per particle
        {
            const T gx = sizeof(T) == 8 ? (T)S.g[0] : (T)S.g_f[0];
            const T gy = sizeof(T) == 8 ? (T)S.g[1] : (T)S.g_f[1];
            const T gz = sizeof(T) == 8 ? (T)S.g[2] : (T)S.g_f[2];
            F = F + mk(gx, gy, gz) * mi;
        }
        if (EVAL) {
            const size_t o = 3 * (size_t)me.id;
            if (a.dbgF) { a.dbgF[o] = F.x; a.dbgF[o + 1] = F.y; a.dbgF[o + 2] = F.z; }
            if (a.dbgT) { a.dbgT[o] = Tq.x; a.dbgT[o + 1] = Tq.y; a.dbgT[o + 2] = Tq.z; }
        } else {
            bool clamped = false, finite = true;
            float4 pnew;
            const uint32_t kk = PR::integrate(B, q, me, F, Tq, S, mi, clamped, finite, pnew);
            if (!finite) raise_status(a.st, ST_NONFINITE, (int32_t)q);
            c_clamp = clamped ? 1u : 0u;
            c_disp2 = pnew.w;
            if (LIST) {
                // a particle that moved skin/2 (less the FP32 margin) since the last sort
                // makes this step end with a sort and new lists
                const float4 r0 = __ldg(&a.ref[q]);
                const float ex = pnew.x - r0.x, ey = pnew.y - r0.y, ez = pnew.z - r0.z;
                if (ex * ex + ey * ey + ez * ez > a.thresh2 || !finite) atomicOr(&a.ctrl->rebuild, 1);
            } else {
                a.key[q] = kk;
                a.rank[q] = atomicAdd(&a.cnt[kk], 1u);
            }
        }
    }
    // warp-aggregated counters (every lane reaches this point)
    const unsigned full = 0xffffffffu;
    const uint32_t s_pp = __reduce_add_sync(full, c_pp);
    const uint32_t s_wc = __reduce_add_sync(full, c_wc);
    const uint32_t s_cl = __reduce_add_sync(full, c_clamp);
    const uint32_t s_mx = __reduce_max_sync(full, c_nnew);
    const uint32_t s_ov = __reduce_max_sync(full, __float_as_uint(c_maxov));
    const uint32_t s_dp = __reduce_max_sync(full, __float_as_uint(c_disp2));
    if ((tid & 31) == 0) {
        if (s_pp) atomicAdd(&a.st->live.ncontacts, s_pp);
        if (s_wc) atomicAdd(&a.st->live.nwallc, s_wc);
        if (s_cl) atomicAdd(&a.st->live.clamped, s_cl);
        if (s_mx) atomicMax(&a.st->live.max_nnew, s_mx);
        if (s_ov) atomicMax(&a.st->live.max_overlap_bits, s_ov);
        if (s_dp) atomicMax(&a.st->live.max_disp2_bits, s_dp);
    }
}

// ======================================================================= counting sort
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Every kernel of the sort takes the step control and does nothing when this step does
// not sort (list mode between sorts).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t* __restrict__ cnt, uint32_t m,
                                                              uint32_t ntiles, uint32_t* __restrict__ part,
                                                              const CtrlDev* ctrl) {
    if (!ctrl->rebuild) return;
    __shared__ uint32_t ws[SCAN_THREADS / 32];
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t base = tile * SCAN_TILE;
        uint32_t s = 0;
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            const uint32_t k = base + i * SCAN_THREADS + threadIdx.x;
            if (k < m) s += cnt[k];
        }
        s = __reduce_add_sync(0xffffffffu, s);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < SCAN_THREADS / 32; ++w) t += ws[w];
            part[tile] = t;
        }
        __syncthreads();
    }
}

// exclusive scan of part[0..nb) in one block of 1024 threads
__global__ void __launch_bounds__(1024) k_scan_spine(uint32_t* part, uint32_t nb, const CtrlDev* ctrl) {
    if (!ctrl->rebuild) return;
    __shared__ uint32_t sh[1024];
    const uint32_t per = (nb + 1023) / 1024;
    const uint32_t b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (uint32_t k = 0; k < per; ++k)
        if (b0 + k < nb) s += part[b0 + k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = threadIdx.x >= (uint32_t)off ? sh[threadIdx.x - off] : 0u;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = sh[threadIdx.x] - s;   // exclusive prefix of this thread's chunk
    for (uint32_t k = 0; k < per; ++k)
        if (b0 + k < nb) {
            const uint32_t v = part[b0 + k];
            part[b0 + k] = run;
            run += v;
        }
}

// cs[k] = exclusive prefix of cnt; cnt[k] = 0 for the next sort
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(uint32_t* __restrict__ cnt, uint32_t m, uint32_t ntiles,
                                                            const uint32_t* __restrict__ part, uint32_t* __restrict__ cs,
                                                            const CtrlDev* ctrl) {
    if (!ctrl->rebuild) return;
    __shared__ uint32_t ws[SCAN_THREADS / 32];
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t base = tile * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
        uint32_t v[SCAN_ITEMS];
        uint32_t s = 0;
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            const uint32_t k = base + i;
            v[i] = k < m ? cnt[k] : 0u;
            s += v[i];
        }
        // block-exclusive scan of the thread sums
        uint32_t inc = s;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= (uint32_t)off) inc += t;
        }
        if (lane == 31) ws[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            uint32_t w = lane < SCAN_THREADS / 32 ? ws[lane] : 0u;
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= (uint32_t)off) w += t;
            }
            if (lane < SCAN_THREADS / 32) ws[lane] = w;
        }
        __syncthreads();
        uint32_t run = part[tile] + (inc - s) + (wid > 0 ? ws[wid - 1] : 0u);
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            const uint32_t k = base + i;
            if (k < m) {
                cs[k] = run;
                cnt[k] = 0u;
            }
            run += v[i];
        }
        __syncthreads();
    }
}

__global__ void k_scatter(uint32_t n, const uint32_t* __restrict__ key, const uint32_t* __restrict__ rank,
                          const uint32_t* __restrict__ cs, uint32_t* __restrict__ tmp, const CtrlDev* ctrl) {
    if (!ctrl->rebuild) return;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        tmp[cs[key[q]] + rank[q]] = q;
}

// (cell, id) order: a particle's place in its cell is the number of cell-mates with a
// smaller id. Gathers the state from the next set (pre-sort order) into the current one,
// records the permutation, the cell of each sorted particle and (list mode) its position.
template <class PR>
__device__ __forceinline__ void reorder_one(uint32_t s, const typename PR::State& A, const typename PR::State& B,
                                            const uint32_t* __restrict__ key, const uint32_t* __restrict__ cs,
                                            const uint32_t* __restrict__ tmp, uint32_t* __restrict__ perm,
                                            uint32_t* __restrict__ skey, float4* __restrict__ ref) {
    const uint32_t p = tmp[s];
    const uint32_t c = key[p];
    const uint32_t lo = cs[c], hi = cs[c + 1];
    const uint32_t idp = B.id[p];
    uint32_t r = 0;
    for (uint32_t k = lo; k < hi; ++k) r += (B.id[tmp[k]] < idp) ? 1u : 0u;
    const uint32_t q = lo + r;
    const typename PR::Self m = PR::load(B, p);
    PR::store(A, q, m);
    perm[q] = p;
    skey[q] = c;
    if (ref) ref[q] = PR::pos_f(m);
}

template <class PR>
__global__ void k_reorder(uint32_t n, typename PR::State S0, typename PR::State S1, const CtrlDev* ctrl,
                          const uint32_t* __restrict__ key, const uint32_t* __restrict__ cs,
                          const uint32_t* __restrict__ tmp, uint32_t* __restrict__ perm, uint32_t* __restrict__ skey,
                          float4* __restrict__ ref) {
    if (!ctrl->rebuild) return;
    const int cur = ctrl->cur;
    const typename PR::State A = cur ? S1 : S0;
    const typename PR::State B = cur ? S0 : S1;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        reorder_one<PR>(s, A, B, key, cs, tmp, perm, skey, ref);
}

// List mode stores the sorted particles in (cell, id) order within windows of the force
// pass's block size, each window ordered by the particles' contact counts in the step
// just finished (descending; ties keep the (cell, id) order). The lanes of a warp run
// their candidate lists in lockstep, so grouping similar counts shortens the longest
// lane's loop; a particle's own sums keep their order, so results do not change.
// Three passes replace k_reorder: the (cell, id) position of every particle, its final
// position in its window, and the gather to the final position.
template <class PR>
__global__ void k_rank_cell(uint32_t n, typename PR::State S0, typename PR::State S1, const CtrlDev* ctrl,
                            const uint32_t* __restrict__ key, const uint32_t* __restrict__ cs,
                            const uint32_t* __restrict__ tmp, const uint32_t* __restrict__ hcnt_last,
                            uint32_t* __restrict__ canon, uint32_t* __restrict__ wkey) {
    if (!ctrl->rebuild) return;
    const typename PR::State B = ctrl->cur ? S0 : S1;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const uint32_t p = tmp[s];
        const uint32_t c = key[p];
        const uint32_t lo = cs[c], hi = cs[c + 1];
        const uint32_t idp = B.id[p];
        uint32_t r = 0;
        for (uint32_t k = lo; k < hi; ++k) r += (B.id[tmp[k]] < idp) ? 1u : 0u;
        canon[lo + r] = p;
        wkey[lo + r] = hcnt_last[p];
    }
}

// One block per window of blockDim.x (cell, id) positions: fin[q] = final position.
__global__ void __launch_bounds__(256) k_window(uint32_t n, const CtrlDev* ctrl, const uint32_t* __restrict__ wkey,
                                                uint32_t* __restrict__ fin) {
    if (!ctrl->rebuild) return;
    __shared__ uint32_t s_key[256];
    const uint32_t w = blockDim.x;
    for (uint32_t base = blockIdx.x * w; base < n; base += gridDim.x * w) {
        const uint32_t q = base + threadIdx.x;
        const uint32_t key = q < n ? min(wkey[q], 0xFFFFu) : 0u;
        __syncthreads();
        s_key[threadIdx.x] = key;
        __syncthreads();
        uint32_t rank = 0;
        for (uint32_t t = 0; t < w; ++t) {
            const uint32_t kt = s_key[t];
            rank += (kt > key || (kt == key && t < threadIdx.x)) ? 1u : 0u;
        }
        if (q < n) fin[q] = base + rank;
    }
}

template <class PR>
__global__ void k_gather(uint32_t n, typename PR::State S0, typename PR::State S1, const CtrlDev* ctrl,
                         const uint32_t* __restrict__ key, const uint32_t* __restrict__ canon,
                         const uint32_t* __restrict__ fin, uint32_t* __restrict__ perm, uint32_t* __restrict__ skey,
                         float4* __restrict__ ref) {
    if (!ctrl->rebuild) return;
    const typename PR::State A = ctrl->cur ? S1 : S0;
    const typename PR::State B = ctrl->cur ? S0 : S1;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const uint32_t p = canon[q], f = fin[q];
        const typename PR::Self m = PR::load(B, p);
        PR::store(A, f, m);
        perm[f] = p;
        skey[f] = key[p];
        ref[f] = PR::pos_f(m);
    }
}

// Neighbour lists of the sorted state (list mode): every particle of the 27 cells around
// each particle (Eq. 12) that lies within r_i + r_j + skin (+ the FP32 margin). With
// cells of edge >= 2 r_max + skin, no pair that comes into contact before some particle
// has moved skin/2 is missed.
template <class PR>
__device__ __forceinline__ uint32_t nlist_one(uint32_t q, const SceneDev* scenes, int nscenes,
                                              const typename PR::State& A, const uint32_t* __restrict__ skey,
                                              const uint32_t* __restrict__ cs, const uint32_t* __restrict__ fin,
                                              uint32_t* __restrict__ nl, size_t cap, uint32_t maxn, float skin,
                                              StatusDev* st) {
    const SceneDev& S = scenes[scene_of(scenes, nscenes, q)];
    const typename PR::Self me = PR::load(A, q);
    const float extra = skin + S.eps_f;
    const int nx = S.dims[0], ny = S.dims[1], nz = S.dims[2];
    const uint32_t local = skey[q] - S.c0;
    const int ix = (int)(local % (uint32_t)nx);
    const uint32_t t1 = local / (uint32_t)nx;
    const int iy = (int)(t1 % (uint32_t)ny);
    const int iz = (int)(t1 / (uint32_t)ny);
    const uint32_t xlo = (uint32_t)max(ix - 1, 0), xhi = (uint32_t)min(ix + 1, nx - 1) + 1;
    uint32_t rlo[9], rhi[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int z2 = iz + r / 3 - 1, y2 = iy + r % 3 - 1;
        const bool ok = z2 >= 0 && z2 < nz && y2 >= 0 && y2 < ny;
        const uint32_t rowbase = S.c0 + (uint32_t)((z2 * ny + y2) * nx);
        rlo[r] = ok ? __ldg(&cs[rowbase + xlo]) : 0u;
        rhi[r] = ok ? __ldg(&cs[rowbase + xhi]) : 0u;
    }
    uint32_t m = 0;
#pragma unroll
    for (int r = 0; r < 9; ++r)
        for (uint32_t jc = rlo[r]; jc < rhi[r]; ++jc) {
            const uint32_t j = fin[jc];   // the cell table holds (cell, id) positions
            if (j == q || !PR::within(A, me, j, extra)) continue;
            if (m < maxn) nl[m * cap + q] = j;
            ++m;
        }
    if (m > maxn) raise_status(st, ST_CAPACITY, (int32_t)q);
    return min(m, maxn);
}

template <class PR>
__global__ void __launch_bounds__(256) k_nlist(uint32_t n, const SceneDev* scenes, int nscenes, typename PR::State S0,
                                                typename PR::State S1, const CtrlDev* ctrl,
                                                const uint32_t* __restrict__ skey, const uint32_t* __restrict__ cs,
                                                const uint32_t* __restrict__ fin, uint32_t* __restrict__ ncnt,
                                                uint32_t* __restrict__ nl, size_t cap, uint32_t maxn, float skin,
                                                StatusDev* st) {
    if (!ctrl->rebuild) return;
    const typename PR::State A = ctrl->cur ? S1 : S0;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        ncnt[q] = nlist_one<PR>(q, scenes, nscenes, A, skey, cs, fin, nl, cap, maxn, skin, st);
}

// Step bookkeeping (one thread): after a sort the current set stays and springs are read
// through the permutation next step; otherwise the next set becomes current.
__global__ void k_end_step(CtrlDev* ctrl, StatusDev* st, int walk_mode) {
    if (ctrl->rebuild) {
        ctrl->perm_valid = 1;
        ctrl->since = 0;
        ctrl->nsorts += 1;
    } else {
        ctrl->cur ^= 1;
        ctrl->perm_valid = 0;
        ctrl->since += 1;
    }
    ctrl->rebuild = walk_mode;
    st->last = st->live;
    st->live = CountersDev{};
}

// ======================================================================= set-up / read-out
template <class PR>
__global__ void k_import(uint32_t n, typename PR::State B, const double* __restrict__ x, const double* __restrict__ v,
                         const double* __restrict__ w, const float* __restrict__ r);

template <>
__global__ void k_import<PF64>(uint32_t n, StateF64 B, const double* __restrict__ x, const double* __restrict__ v,
                               const double* __restrict__ w, const float* __restrict__ r) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    B.x[k] = x[3 * (size_t)k]; B.y[k] = x[3 * (size_t)k + 1]; B.z[k] = x[3 * (size_t)k + 2];
    B.vx[k] = v[3 * (size_t)k]; B.vy[k] = v[3 * (size_t)k + 1]; B.vz[k] = v[3 * (size_t)k + 2];
    B.wx[k] = w[3 * (size_t)k]; B.wy[k] = w[3 * (size_t)k + 1]; B.wz[k] = w[3 * (size_t)k + 2];
    B.r[k] = r[k];
    B.id[k] = k;
}

__device__ __forceinline__ void split_ff(double x, float& hi, float& lo) {
    const float h = (float)x;
    const float l = (float)(x - (double)h);
    two_sum(h, l, hi, lo);
}

template <>
__global__ void k_import<PF32>(uint32_t n, StateF32 B, const double* __restrict__ x, const double* __restrict__ v,
                               const double* __restrict__ w, const float* __restrict__ r) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float h[3], l[3];
    for (int a = 0; a < 3; ++a) split_ff(x[3 * (size_t)k + a], h[a], l[a]);
    B.P0[k] = make_float4(h[0], h[1], h[2], r[k]);
    B.P1[k] = make_float4(l[0], l[1], l[2], __uint_as_float(k));
    B.V[k] = make_float4((float)v[3 * (size_t)k], (float)v[3 * (size_t)k + 1], (float)v[3 * (size_t)k + 2], 0.f);
    B.W[k] = make_float4((float)w[3 * (size_t)k], (float)w[3 * (size_t)k + 1], (float)w[3 * (size_t)k + 2], 0.f);
    B.id[k] = k;
}

// Cell key CM (step 2) and the rank of each particle within its cell, for the next set.
template <class PR>
__global__ void k_hash(uint32_t n, const SceneDev* scenes, int nscenes, typename PR::State S0, typename PR::State S1,
                       const CtrlDev* ctrl, uint32_t* __restrict__ key, uint32_t* __restrict__ rank,
                       uint32_t* __restrict__ cnt, StatusDev* st) {
    if (!ctrl->rebuild) return;
    const typename PR::State B = ctrl->cur ? S0 : S1;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const SceneDev& S = scenes[scene_of(scenes, nscenes, q)];
        bool clamped = false;
        const uint32_t kk = PR::key_of(B, S, q, clamped);
        if (clamped) atomicAdd(&st->live.clamped, 1u);
        key[q] = kk;
        rank[q] = atomicAdd(&cnt[kk], 1u);
    }
}

template <class PR>
__global__ void k_export(uint32_t n, typename PR::State S0, typename PR::State S1, const CtrlDev* ctrl, double* x,
                         double* v, double* w);

template <>
__global__ void k_export<PF64>(uint32_t n, StateF64 S0, StateF64 S1, const CtrlDev* ctrl, double* x, double* v,
                               double* w) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const StateF64 A = ctrl->cur ? S1 : S0;
    const size_t o = 3 * (size_t)A.id[q];
    if (x) { x[o] = A.x[q]; x[o + 1] = A.y[q]; x[o + 2] = A.z[q]; }
    if (v) { v[o] = A.vx[q]; v[o + 1] = A.vy[q]; v[o + 2] = A.vz[q]; }
    if (w) { w[o] = A.wx[q]; w[o + 1] = A.wy[q]; w[o + 2] = A.wz[q]; }
}

template <>
__global__ void k_export<PF32>(uint32_t n, StateF32 S0, StateF32 S1, const CtrlDev* ctrl, double* x, double* v,
                               double* w) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const StateF32 A = ctrl->cur ? S1 : S0;
    const size_t o = 3 * (size_t)A.id[q];
    if (x) {
        const float4 h = A.P0[q], l = A.P1[q];
        x[o] = (double)h.x + (double)l.x;
        x[o + 1] = (double)h.y + (double)l.y;
        x[o + 2] = (double)h.z + (double)l.z;
    }
    if (v) { const float4 a = A.V[q]; v[o] = a.x; v[o + 1] = a.y; v[o + 2] = a.z; }
    if (w) { const float4 a = A.W[q]; w[o] = a.x; w[o + 1] = a.y; w[o + 2] = a.z; }
}

// ---------------------------------------------------------------- diagnostics (FP64)
constexpr int DIAG_THREADS = 256;
constexpr int NDIAG = 10;

template <class PR>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag(uint32_t n, const SceneDev* scenes, int nscenes,
                                                       typename PR::State S0, typename PR::State S1,
                                                       const CtrlDev* ctrl, double* __restrict__ part) {
    __shared__ double sh[NDIAG][DIAG_THREADS];
    const typename PR::State A = ctrl->cur ? S1 : S0;
    const uint32_t tid = threadIdx.x;
    const uint32_t q = blockIdx.x * DIAG_THREADS + tid;
    double val[NDIAG];
    for (int k = 0; k < NDIAG; ++k) val[k] = 0.0;
    if (q < n) {
        const SceneDev& S = scenes[scene_of(scenes, nscenes, q)];
        const typename PR::Self m = PR::load(A, q);
        const V3<double> x = PR::pos(m), v = PR::vel(m), w = PR::spin(m);
        const double r = (double)m.r;
        const double mass = S.cmass * r * r * r;
        const double I = 0.4 * mass * r * r;
        val[0] = 0.5 * mass * dot(v, v);
        val[1] = 0.5 * I * dot(w, w);
        val[2] = mass * v.x; val[3] = mass * v.y; val[4] = mass * v.z;
        const V3<double> L = cross(x, v) * mass + w * I;
        val[5] = L.x; val[6] = L.y; val[7] = L.z;
        val[8] = -mass * dot(mk(S.g[0], S.g[1], S.g[2]), x);
        val[9] = mass;
    }
    for (int k = 0; k < NDIAG; ++k) sh[k][tid] = val[k];
    __syncthreads();
    for (uint32_t s = DIAG_THREADS / 2; s > 0; s >>= 1) {
        if (tid < s)
            for (int k = 0; k < NDIAG; ++k) sh[k][tid] += sh[k][tid + s];
        __syncthreads();
    }
    if (tid == 0)
        for (int k = 0; k < NDIAG; ++k) part[(size_t)blockIdx.x * NDIAG + k] = sh[k][0];
}

// one block: fixed-order reduction of the per-block partial sums
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_final(const double* __restrict__ part, uint32_t nb,
                                                             double* __restrict__ out) {
    __shared__ double sh[NDIAG][DIAG_THREADS];
    const uint32_t tid = threadIdx.x;
    double val[NDIAG];
    for (int k = 0; k < NDIAG; ++k) val[k] = 0.0;
    for (uint32_t b = tid; b < nb; b += DIAG_THREADS)
        for (int k = 0; k < NDIAG; ++k) val[k] += part[(size_t)b * NDIAG + k];
    for (int k = 0; k < NDIAG; ++k) sh[k][tid] = val[k];
    __syncthreads();
    for (uint32_t s = DIAG_THREADS / 2; s > 0; s >>= 1) {
        if (tid < s)
            for (int k = 0; k < NDIAG; ++k) sh[k][tid] += sh[k][tid + s];
        __syncthreads();
    }
    if (tid == 0)
        for (int k = 0; k < NDIAG; ++k) out[k] = sh[k][0];
}


// ======================================================================= batch repacking
// Springs of the current state rewritten in cell-sorted order (index q), into the free
// history buffer: afterwards slot lists sit at the same index as the particle.
template <class T>
__global__ void k_hist_canon(uint32_t n, const CtrlDev* ctrl, const uint32_t* __restrict__ perm,
                             const uint32_t* __restrict__ cin, const uint32_t* __restrict__ pin,
                             const T* __restrict__ din, uint32_t* __restrict__ cout, uint32_t* __restrict__ pout,
                             T* __restrict__ dout, size_t cap, uint32_t maxc) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint32_t src = ctrl->perm_valid ? perm[q] : q;
    const uint32_t c = min(cin[src], maxc);
    cout[q] = c;
    for (uint32_t k = 0; k < c; ++k) {
        pout[k * cap + q] = pin[k * cap + src];
        for (int a = 0; a < 3; ++a) dout[(a * (size_t)maxc + k) * cap + q] = din[(a * (size_t)maxc + k) * cap + src];
    }
}

// New packed layout: particle p of the new domain takes the old current-state particle
// map[p] (with its springs, already in sorted order) or, for map[p] == ~0, starts with
// no springs (its state is imported separately).
template <class PR>
__global__ void k_repack(uint32_t n_new, const uint32_t* __restrict__ map, typename PR::State oS0,
                         typename PR::State oS1, const CtrlDev* octrl, const uint32_t* __restrict__ ocnt,
                         const uint32_t* __restrict__ opid, const typename PR::T* __restrict__ od, size_t ocap,
                         typename PR::State nB, uint32_t* __restrict__ ncnt, uint32_t* __restrict__ npid,
                         typename PR::T* __restrict__ nd, size_t ncap, uint32_t maxc) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_new) return;
    const uint32_t m = map[p];
    if (m == 0xFFFFFFFFu) {
        ncnt[p] = 0;
        return;
    }
    const typename PR::State A = octrl->cur ? oS1 : oS0;
    PR::store(nB, p, PR::load(A, m));
    const uint32_t c = min(ocnt[m], maxc);
    ncnt[p] = c;
    for (uint32_t k = 0; k < c; ++k) {
        npid[k * ncap + p] = opid[k * ocap + m];
        for (int a = 0; a < 3; ++a) nd[(a * (size_t)maxc + k) * ncap + p] = od[(a * (size_t)maxc + k) * ocap + m];
    }
}

static inline StateF64 shifted(StateF64 s, uint32_t p0) {
    s.x += p0; s.y += p0; s.z += p0; s.vx += p0; s.vy += p0; s.vz += p0; s.wx += p0; s.wy += p0; s.wz += p0;
    s.r += p0; s.id += p0;
    return s;
}
static inline StateF32 shifted(StateF32 s, uint32_t p0) {
    s.P0 += p0; s.P1 += p0; s.V += p0; s.W += p0; s.id += p0;
    return s;
}

// ======================================================================= launchers
static inline uint32_t nblk(uint32_t n, uint32_t b) { return (n + b - 1) / b; }
// Grid of the sort-phase kernels: they loop over their items, so a grid of a few blocks
// per SM does the work of a sort, and a step that does not sort pays for few blocks.
static inline uint32_t sgrid(const Domain& d, uint32_t n) {
    return std::max(1u, std::min(nblk(n, 256), (uint32_t)std::max(d.sort_blocks, 1)));
}

#define DEM_LAUNCH_CHECK()                          \
    do {                                            \
        ++d.launches;                               \
        cudaError_t e_ = cudaGetLastError();        \
        if (e_ != cudaSuccess) return e_;           \
    } while (0)

cudaError_t run_import(Domain& d, const double* x, const double* v, const double* w, const float* r) {
    // the caller has set ctrl->cur = 0, so set 1 is the "next" set that the sort gathers from
    if (d.n == 0) return cudaSuccess;
    if (d.precision == 0) k_import<PF64><<<nblk(d.n, 256), 256, 0, d.stream>>>(d.n, d.S64[1], x, v, w, r);
    else k_import<PF32><<<nblk(d.n, 256), 256, 0, d.stream>>>(d.n, d.S32[1], x, v, w, r);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_hash(Domain& d) {
    if (d.n == 0) return cudaSuccess;
    if (d.precision == 0)
        k_hash<PF64><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.d_scenes, d.nscenes, d.S64[0], d.S64[1], d.ctrl,
                                                            d.key, d.rank, d.cnt, d.st);
    else
        k_hash<PF32><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.d_scenes, d.nscenes, d.S32[0], d.S32[1], d.ctrl,
                                                            d.key, d.rank, d.cnt, d.st);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_rebuild(Domain& d) {
    if (d.n == 0) return cudaSuccess;
    const uint32_t m = d.ncells + 1;
    const uint32_t nb = nblk(m, SCAN_TILE);
    const uint32_t gb = std::min(nb, (uint32_t)std::max(d.sort_blocks, 1));
    k_scan_reduce<<<gb, SCAN_THREADS, 0, d.stream>>>(d.cnt, m, nb, d.part, d.ctrl);
    DEM_LAUNCH_CHECK();
    k_scan_spine<<<1, 1024, 0, d.stream>>>(d.part, nb, d.ctrl);
    DEM_LAUNCH_CHECK();
    k_scan_down<<<gb, SCAN_THREADS, 0, d.stream>>>(d.cnt, m, nb, d.part, d.cs, d.ctrl);
    DEM_LAUNCH_CHECK();
    k_scatter<<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.key, d.rank, d.cs, d.tmp, d.ctrl);
    DEM_LAUNCH_CHECK();
    if (!d.list_mode) {
        if (d.precision == 0)
            k_reorder<PF64><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.S64[0], d.S64[1], d.ctrl, d.key, d.cs,
                                                                   d.tmp, d.perm, d.skey, nullptr);
        else
            k_reorder<PF32><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.S32[0], d.S32[1], d.ctrl, d.key, d.cs,
                                                                   d.tmp, d.perm, d.skey, nullptr);
        DEM_LAUNCH_CHECK();
    } else {
        // (cell, id) positions, the window order by last contact count, the gather
        const uint32_t* hc = d.hcnt[d.h_cur];   // contact counts of the step just finished (pre-sort order)
        const uint32_t wb = (uint32_t)d.block;
        const uint32_t wg = std::max(1u, std::min(nblk(d.n, wb), (uint32_t)std::max(d.sort_blocks, 1)));
        if (d.precision == 0)
            k_rank_cell<PF64><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.S64[0], d.S64[1], d.ctrl, d.key, d.cs,
                                                                     d.tmp, hc, d.canon, d.rank);
        else
            k_rank_cell<PF32><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.S32[0], d.S32[1], d.ctrl, d.key, d.cs,
                                                                     d.tmp, hc, d.canon, d.rank);
        DEM_LAUNCH_CHECK();
        k_window<<<wg, wb, 0, d.stream>>>(d.n, d.ctrl, d.rank, d.fin);
        DEM_LAUNCH_CHECK();
        if (d.precision == 0)
            k_gather<PF64><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.S64[0], d.S64[1], d.ctrl, d.key, d.canon,
                                                                  d.fin, d.perm, d.skey, d.ref);
        else
            k_gather<PF32><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.S32[0], d.S32[1], d.ctrl, d.key, d.canon,
                                                                  d.fin, d.perm, d.skey, d.ref);
        DEM_LAUNCH_CHECK();
        if (d.precision == 0)
            k_nlist<PF64><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.d_scenes, d.nscenes, d.S64[0], d.S64[1], d.ctrl,
                                                                 d.skey, d.cs, d.fin, d.ncnt, d.nl, d.cap,
                                                                 (uint32_t)d.maxn, d.skin_f, d.st);
        else
            k_nlist<PF32><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.d_scenes, d.nscenes, d.S32[0], d.S32[1], d.ctrl,
                                                                 d.skey, d.cs, d.fin, d.ncnt, d.nl, d.cap,
                                                                 (uint32_t)d.maxn, d.skin_f, d.st);
        DEM_LAUNCH_CHECK();
    }
    return cudaSuccess;
}

// Sets the condition of the step graph's sort node from the device-side decision, and
// counts the sorts that run that way (one thread).
__global__ void k_sort_cond(cudaGraphConditionalHandle h, CtrlDev* ctrl) {
    const unsigned int go = ctrl->rebuild ? 1u : 0u;
    ctrl->cond_sorts += go;
    cudaGraphSetConditional(h, go);
}

cudaError_t run_sort_cond(Domain& d, cudaGraphConditionalHandle h) {
    k_sort_cond<<<1, 1, 0, d.stream>>>(h, d.ctrl);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_end_step(Domain& d) {
    k_end_step<<<1, 1, 0, d.stream>>>(d.ctrl, d.st, d.list_mode ? 0 : 1);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

template <class PR>
static cudaError_t force_impl(Domain& d, const typename PR::State& S0, const typename PR::State& S1, bool eval,
                              double* dbgF, double* dbgT) {
    ForceArgs<PR> a;
    a.scenes = d.d_scenes;
    a.nscenes = d.nscenes;
    a.n = d.n;
    a.cap = d.cap;
    a.maxc = d.maxc;
    a.stiffness = d.stiffness;
    a.S0 = S0;
    a.S1 = S1;
    a.ctrl = d.ctrl;
    a.ncnt = d.ncnt;
    a.nl = d.nl;
    a.ref = d.ref;
    a.thresh2 = d.thresh2;
    a.interval = d.interval;
    a.skey = d.skey;
    a.cs = d.cs;
    a.perm = d.perm;
    const int hi = d.h_cur, ho = 1 - d.h_cur;
    a.hin_cnt = d.hcnt[hi];
    a.hin_pid = d.hpid[hi];
    a.hin_d = (const typename PR::T*)d.hd[hi];
    a.hout_cnt = d.hcnt[ho];
    a.hout_pid = d.hpid[ho];
    a.hout_d = (typename PR::T*)d.hd[ho];
    a.key = d.key;
    a.rank = d.rank;
    a.cnt = d.cnt;
    a.st = d.st;
    a.dbgF = dbgF;
    a.dbgT = dbgT;
    const uint32_t b = (uint32_t)d.block;
    const size_t smem = (d.list_mode ? 1 : 2) * (size_t)d.maxc * b * sizeof(uint32_t);
    const uint32_t g = nblk(d.n, b);
    auto launch = [&](auto kern) -> cudaError_t {
        // lists of 2 x maxc ids per thread may exceed the 48 KB default of dynamic shared memory
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<g, b, smem, d.stream>>>(a);
        return cudaSuccess;
    };
    cudaError_t e;
    const int model = d.model != 0 ? 1 : (d.terms != 0 ? 2 : 0);
    if (d.list_mode) {
        if (model == 0) e = eval ? launch(k_force<PR, 0, true, true>) : launch(k_force<PR, 0, false, true>);
        else if (model == 2) e = eval ? launch(k_force<PR, 2, true, true>) : launch(k_force<PR, 2, false, true>);
        else e = eval ? launch(k_force<PR, 1, true, true>) : launch(k_force<PR, 1, false, true>);
    } else {
        if (model == 0) e = eval ? launch(k_force<PR, 0, true, false>) : launch(k_force<PR, 0, false, false>);
        else if (model == 2) e = eval ? launch(k_force<PR, 2, true, false>) : launch(k_force<PR, 2, false, false>);
        else e = eval ? launch(k_force<PR, 1, true, false>) : launch(k_force<PR, 1, false, false>);
    }
    if (e != cudaSuccess) return e;
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_force(Domain& d, bool eval, double* dbgF, double* dbgT) {
    if (d.n == 0) return cudaSuccess;
    if (d.precision == 0) return force_impl<PF64>(d, d.S64[0], d.S64[1], eval, dbgF, dbgT);
    return force_impl<PF32>(d, d.S32[0], d.S32[1], eval, dbgF, dbgT);
}

cudaError_t run_export(Domain& d, double* x, double* v, double* w) {
    if (d.n == 0) return cudaSuccess;
    if (d.precision == 0)
        k_export<PF64><<<nblk(d.n, 256), 256, 0, d.stream>>>(d.n, d.S64[0], d.S64[1], d.ctrl, x, v, w);
    else
        k_export<PF32><<<nblk(d.n, 256), 256, 0, d.stream>>>(d.n, d.S32[0], d.S32[1], d.ctrl, x, v, w);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}


cudaError_t run_hist_canon(Domain& d) {
    if (d.n == 0) return cudaSuccess;
    const int hi = d.h_cur, ho = 1 - d.h_cur;
    if (d.precision == 0)
        k_hist_canon<double><<<nblk(d.n, 256), 256, 0, d.stream>>>(
            d.n, d.ctrl, d.perm, d.hcnt[hi], d.hpid[hi], (const double*)d.hd[hi], d.hcnt[ho], d.hpid[ho],
            (double*)d.hd[ho], d.cap, (uint32_t)d.maxc);
    else
        k_hist_canon<float><<<nblk(d.n, 256), 256, 0, d.stream>>>(
            d.n, d.ctrl, d.perm, d.hcnt[hi], d.hpid[hi], (const float*)d.hd[hi], d.hcnt[ho], d.hpid[ho],
            (float*)d.hd[ho], d.cap, (uint32_t)d.maxc);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_repack(Domain& od, Domain& d, const uint32_t* map, uint32_t n_new) {
    if (n_new == 0) return cudaSuccess;
    const int ho = 1 - od.h_cur;   // canonical springs of the old domain (run_hist_canon)
    if (d.precision == 0)
        k_repack<PF64><<<nblk(n_new, 256), 256, 0, d.stream>>>(
            n_new, map, od.S64[0], od.S64[1], od.ctrl, od.hcnt[ho], od.hpid[ho], (const double*)od.hd[ho], od.cap,
            d.S64[1], d.hcnt[0], d.hpid[0], (double*)d.hd[0], d.cap, (uint32_t)d.maxc);
    else
        k_repack<PF32><<<nblk(n_new, 256), 256, 0, d.stream>>>(
            n_new, map, od.S32[0], od.S32[1], od.ctrl, od.hcnt[ho], od.hpid[ho], (const float*)od.hd[ho], od.cap,
            d.S32[1], d.hcnt[0], d.hpid[0], (float*)d.hd[0], d.cap, (uint32_t)d.maxc);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_import_at(Domain& d, uint32_t p0, uint32_t np, const double* x, const double* v, const double* w,
                          const float* r) {
    if (np == 0) return cudaSuccess;
    if (d.precision == 0) k_import<PF64><<<nblk(np, 256), 256, 0, d.stream>>>(np, shifted(d.S64[1], p0), x, v, w, r);
    else k_import<PF32><<<nblk(np, 256), 256, 0, d.stream>>>(np, shifted(d.S32[1], p0), x, v, w, r);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_export_range(Domain& d, uint32_t p0, uint32_t np, double* x, double* v, double* w) {
    if (np == 0) return cudaSuccess;
    if (d.precision == 0)
        k_export<PF64><<<nblk(np, 256), 256, 0, d.stream>>>(np, shifted(d.S64[0], p0), shifted(d.S64[1], p0), d.ctrl,
                                                             x, v, w);
    else
        k_export<PF32><<<nblk(np, 256), 256, 0, d.stream>>>(np, shifted(d.S32[0], p0), shifted(d.S32[1], p0), d.ctrl,
                                                             x, v, w);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_diag(Domain& d) {
    const uint32_t nb = d.n ? nblk(d.n, DIAG_THREADS) : 1;
    if (d.n) {
        if (d.precision == 0)
            k_diag<PF64><<<nb, DIAG_THREADS, 0, d.stream>>>(d.n, d.d_scenes, d.nscenes, d.S64[0], d.S64[1], d.ctrl,
                                                             d.diag_part);
        else
            k_diag<PF32><<<nb, DIAG_THREADS, 0, d.stream>>>(d.n, d.d_scenes, d.nscenes, d.S32[0], d.S32[1], d.ctrl,
                                                             d.diag_part);
        DEM_LAUNCH_CHECK();
        k_diag_final<<<1, DIAG_THREADS, 0, d.stream>>>(d.diag_part, nb, d.diag_out);
        DEM_LAUNCH_CHECK();
    } else {
        cudaError_t e = cudaMemsetAsync(d.diag_out, 0, NDIAG * sizeof(double), d.stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace demgb
