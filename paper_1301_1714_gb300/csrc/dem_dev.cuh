// Device-side definitions of the GB300 DEM timestep: scene table, state layouts,
// compensated (float-float) arithmetic, contact geometry and the contact laws.
//
// Layout in HBM (all arrays in cell-sorted particle order, "SoA"):
//   FP64 mode: x,y,z / vx,vy,vz / wx,wy,wz planes of doubles, r (float), id (u32).
//   FP32 mode: P0 = float4(hi.x, hi.y, hi.z, r), P1 = float4(lo.x, lo.y, lo.z, 0),
//              V = float4(v, 0), W = float4(w, 0), id (u32). Position = hi + lo exactly,
//              with hi = fl32(hi + lo) kept by every update (FastTwoSum renormalisation).
//   History (per particle, slot-major): cnt[p], pid[k*cap + p] (partner global id, or
//   DEM_WALL_BASE + wall), d[(c*maxc + k)*cap + p] for c = x,y,z (T = float or double).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define DEM_MAX_WALLS 8
#define DEM_WALL_BASE 0xFFFFFF00u

// Neighbour lists of list mode: at most DEM_LIST_CAP candidates per particle (one bit each
// in the force pass's 64-bit mask); a fuller list is reported, never truncated silently.
#define DEM_LIST_CAP 64
// Cell order of list mode: bricks of 2^s x 2^s x 2^s cells, s at most DEM_LIST_BRICK_SHIFT
// (0 = row-major). Each grid takes the largest s whose padding to whole bricks adds at most
// 1/8 to its cell count.
#ifndef DEM_LIST_BRICK_SHIFT
#define DEM_LIST_BRICK_SHIFT 4
#endif

namespace demgb {

// ------------------------------------------------------------------ scene table
struct WallDev {
    int32_t kind;       // 0 plane, 1 cylinder interior, 2 half-plate
    int32_t axis;       // cylinder axis / plane or plate normal index when it is a coordinate axis, else -1
    int32_t uaxis;      // half-plate: index of u when it is a coordinate axis, else -1
    int32_t pad;
    double p[3], n[3], radius, omega[3], vel[3], u[3];
    float uf[3];
    float p_hi[3], p_lo[3];     // p split into hi + lo (FP32 mode)
    float n_hi[3], n_lo[3];     // n split into hi + lo
    float rad_hi, rad_lo;       // radius split
    float nf[3], omegaf[3], velf[3], pf[3];
};

struct SceneDev {
    uint32_t p0, np;            // particles [p0, p0 + np) of the packed arrays
    uint32_t c0, ncell;         // cell keys [c0, c0 + ncell)
    int32_t dims[3];
    int32_t nwalls;
    int32_t active;             // 0: frozen (state is carried, no forces)
    int32_t pad;
    double origin[3], h;
    float origin_f[3], h_f;
    double dt, g[3], kn, kt, cn, ct, alpha, mu, ksp, kda, ksh, cmass;   // cmass = rho*4/3*pi
    float dt_f, g_f[3], kn_f, kt_f, cn_f, ct_f, alpha_f, mu_f, ksp_f, kda_f, ksh_f, cmass_f;
    float eps_f;                // FP32 prefilter margin [m]
    int32_t terms;              // optional force terms (DEM_TERM_*)
    int32_t bshift;             // cell order: 0 row-major; s > 0 bricks of (2^s)^3 cells (list mode)
    int32_t bdims[3];           // bricks per axis (bshift > 0)
    float skin_f;               // list mode: Verlet skin [m] of the scene's neighbour lists
    float thresh2_f;            // list mode: squared displacement since the last sort that forces a sort
    float pad4;
    double mu_roll;             // rolling resistance coefficient
    double alpha_t;             // tangential damping factor
    double kcoh_pi;             // pi * cohesion energy density
    float mu_roll_f, alpha_t_f, kcoh_pi_f;
    float pad3;
    WallDev walls[DEM_MAX_WALLS];
};

// Per-pass counters (accumulated by the force pass, rotated into `last` by the sort).
struct CountersDev {
    uint32_t ncontacts;          // particle-particle contact records (each pair counted from both sides)
    uint32_t nwallc;             // particle-wall contacts
    uint32_t max_overlap_bits;   // bits of the largest overlap as a non-negative float
    uint32_t clamped;            // particles whose new cell index was clamped to the grid
    uint32_t max_nnew;           // largest per-particle contact count
    uint32_t max_disp2_bits;     // bits of the largest squared displacement of the step (|v'| dt)^2
    uint32_t pad[2];
};
// Status word: the first error raised on the device (sticky until the host reads it).
struct StatusDev {
    int32_t code;
    int32_t where;
    int32_t pad[2];
    CountersDev live, last;
};

enum : int32_t { ST_OK = 0, ST_CAPACITY = 4, ST_LIST = 5, ST_NONFINITE = 6 };
#define DEM_HALT 2

// Step control, read and written only by kernels (the host never needs to know, while
// stepping, whether a step sorted).
struct CtrlDev {
    int32_t cur;         // state set holding the current cell-sorted state (the other is "next")
    int32_t rebuild;     // bit 0: this step ends with a cell sort (and, in list mode, new lists);
                         // bit 1 (DEM_HALT): a particle overflowed its contact slots this step, so
                         // the step is void: no sort, no swap, and the later steps of the launch
                         // sequence do nothing (the host grows the slots and runs it again)
    int32_t perm_valid;  // 1: the last step sorted, so stored springs are read through perm
    int32_t since;       // steps since the last sort
    uint32_t nsorts;     // sorts performed since the particles were set
    uint32_t cond_sorts; // sorts run as the conditional body of a step graph (launch accounting)
    uint32_t steps_done; // steps completed (not void) since the control block was set
    int32_t pad;
};

__device__ __forceinline__ void raise_status(StatusDev* st, int32_t code, int32_t where) {
    if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

// Key of cell (i, j, k) of scene S, relative to the scene's first cell. Row-major
// ((k ny + j) nx + i) or, with bshift = s > 0, bricks of 2^s x 2^s x 2^s cells: bricks in
// row-major order, cells row-major within their brick. A run of consecutive keys is then
// a compact block of space, so the particles a thread block holds are mostly each
// other's neighbours (list mode stores particles in this order).
__device__ __forceinline__ uint32_t cell_index(const SceneDev& S, uint32_t i, uint32_t j, uint32_t k) {
    if (S.bshift == 0) return (k * (uint32_t)S.dims[1] + j) * (uint32_t)S.dims[0] + i;
    const uint32_t sh = (uint32_t)S.bshift, m = (1u << sh) - 1u;
    const uint32_t brick = ((k >> sh) * (uint32_t)S.bdims[1] + (j >> sh)) * (uint32_t)S.bdims[0] + (i >> sh);
    return (brick << (3 * sh)) | ((((k & m) << sh) | (j & m)) << sh) | (i & m);
}
// Inverse of cell_index.
__device__ __forceinline__ void cell_coords(const SceneDev& S, uint32_t local, int& i, int& j, int& k) {
    if (S.bshift == 0) {
        i = (int)(local % (uint32_t)S.dims[0]);
        const uint32_t t = local / (uint32_t)S.dims[0];
        j = (int)(t % (uint32_t)S.dims[1]);
        k = (int)(t / (uint32_t)S.dims[1]);
        return;
    }
    const uint32_t sh = (uint32_t)S.bshift, m = (1u << sh) - 1u;
    const uint32_t brick = local >> (3 * sh), in = local & ((1u << (3 * sh)) - 1u);
    const uint32_t bi = brick % (uint32_t)S.bdims[0], bt = brick / (uint32_t)S.bdims[0];
    const uint32_t bj = bt % (uint32_t)S.bdims[1], bk = bt / (uint32_t)S.bdims[1];
    i = (int)((bi << sh) | (in & m));
    j = (int)((bj << sh) | ((in >> sh) & m));
    k = (int)((bk << sh) | (in >> (2 * sh)));
}

// Scene of packed particle index q (scenes are contiguous, in order).
__device__ __forceinline__ int scene_of(const SceneDev* sc, int nscenes, uint32_t q) {
    if (nscenes == 1) return 0;
    int lo = 0, hi = nscenes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&sc[mid].p0) <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------ 3-vectors
template <class T>
struct V3 { T x, y, z; };
template <class T> __device__ __forceinline__ V3<T> mk(T x, T y, T z) { return V3<T>{x, y, z}; }
template <class T> __device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> __device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> __device__ __forceinline__ V3<T> operator*(V3<T> a, T s) { return {a.x * s, a.y * s, a.z * s}; }
template <class T> __device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> __device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }

// Quotient and square root of the contact law. FP64 mode: IEEE operations. FP32 mode: the
// hardware approximations (PTX div.approx / sqrt.approx, relative error about 2^-22),
// well inside the FP32 mode's force tolerance; both are deterministic functions of their
// arguments, so the two evaluations of a pair stay exact mirrors of each other.
__device__ __forceinline__ double law_div(double a, double b) { return a / b; }
__device__ __forceinline__ double law_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float law_div(float a, float b) {
    float r;
    asm("div.approx.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float law_sqrt(float a) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// Symmetric in (a1, b1) <-> (a2, b2): products rounded first, then one rounded sum, so the
// two threads that evaluate the same pair get the same bits.
__device__ __forceinline__ float sym_madd(float a1, float b1, float a2, float b2) {
    return __fadd_rn(__fmul_rn(a1, b1), __fmul_rn(a2, b2));
}
__device__ __forceinline__ double sym_madd(double a1, double b1, double a2, double b2) {
    return __dadd_rn(__dmul_rn(a1, b1), __dmul_rn(a2, b2));
}

// ------------------------------------------------- error-free transformations
// Knuth TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Dekker FastTwoSum (|a| >= |b| or a == 0): s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// TwoProd with FMA: p + e == a * b exactly.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// ----------------------------------------------------------- law parameters
template <class T>
struct Law {
    T dt, kn, kt, cn, ct, alpha, mu, ksp, kda, ksh, mu_roll, alpha_t, kcoh_pi;
    int stiffness;  // 0 linear, 1 Hertz
    int terms;      // 1: no attractive normal force, 2: rolling resistance
};
__device__ __forceinline__ Law<double> law_of(const SceneDev& s, int stiffness, double) {
    return Law<double>{s.dt,  s.kn,  s.kt,  s.cn,      s.ct,      s.alpha,   s.mu,
                       s.ksp, s.kda, s.ksh, s.mu_roll, s.alpha_t, s.kcoh_pi, stiffness, s.terms};
}
__device__ __forceinline__ Law<float> law_of(const SceneDev& s, int stiffness, float) {
    return Law<float>{s.dt_f,  s.kn_f,  s.kt_f,  s.cn_f,      s.ct_f,      s.alpha_f,   s.mu_f,
                      s.ksp_f, s.kda_f, s.ksh_f, s.mu_roll_f, s.alpha_t_f, s.kcoh_pi_f, stiffness, s.terms};
}

// Practical contact law (Eqs. 2-10) for body i against partner j, seen from i:
//   n      unit normal from i to j; delta overlap (> 0); v = v_i - v_j (or - wall velocity)
//   rw     r_i w_i + r_j w_j (walls: r_i w_i)
//   Reff   1/(1/r_i + 1/r_j) (walls: r_i); meff 1/(1/m_i + 1/m_j) (walls: m_i)
//   dold   stored tangential spring from i's side (0 for a new contact)
// Outputs: F (force on i, Eq. 2), Ft (tangential part after Eq. 5), dnew (Eq. 7 spring,
// reset after a cap so that Eq. 4 holds).
// Optional terms, compiled in with TERMS and switched by P.terms: 1 = the normal force
// never attracts (F_n = 0 when it would pull i toward j); 2 = rolling resistance, a torque
// -mu_roll R_eff |F_n| w_rel/|w_rel| returned in Mroll (w_rel = w_i - w_j, or minus the
// wall's angular velocity); 4 = eta_t = alpha_t sqrt(k_t m_eff) in the tangential part;
// 8 = cohesion k_coh pi R_eff delta n added after the Coulomb cap.
template <bool TERMS, class T>
__device__ __forceinline__ void law_practical(const Law<T>& P, V3<T> n, T delta, V3<T> v, V3<T> rw, T Reff, T meff,
                                              V3<T> dold, V3<T>& F, V3<T>& Ft, V3<T>& dnew, V3<T> wrel,
                                              V3<T>& Mroll) {
    const T vn_s = dot(v, n);                                    // Eq. 6
    const V3<T> vn = n * vn_s;
    const V3<T> vt = (v - vn) + cross(rw, n);
    const T dn = dot(dold, n);                                   // Eq. 7
    V3<T> dt = (dold - n * dn) + vt * P.dt;
    T kn, kt;                                                    // Eqs. 8-9
    if (P.stiffness == 0) { kn = P.kn; kt = P.kt; }
    else {
        const T s = law_sqrt(delta * Reff);
        kn = P.cn * s;
        kt = P.ct * s;
    }
    const T eta = P.alpha * law_sqrt(kn * meff);                 // Eq. 10
    V3<T> Fn = n * (-kn * delta) - vn * eta;                     // Eq. 4
    if (TERMS && (P.terms & 1) && dot(Fn, n) > T(0)) Fn = mk(T(0), T(0), T(0));
    T eta_t = eta;
    if (TERMS && (P.terms & 4)) eta_t = P.alpha_t * law_sqrt(kt * meff);
    V3<T> Ftt = dt * (-kt) - vt * eta_t;
    // Eq. 5, compared on squared lengths; the lengths are taken only when the cap applies
    const T ft2 = dot(Ftt, Ftt), fn2 = dot(Fn, Fn);
    if (ft2 > (P.mu * P.mu) * fn2 && ft2 > T(0)) {
        const T ftn = law_sqrt(ft2), fnn = law_sqrt(fn2);
        if (ftn > P.mu * fnn) {
            Ftt = Ftt * law_div(P.mu * fnn, ftn);
            if (kt > T(0)) dt = (Ftt + vt * eta_t) * law_div(T(-1), kt);
        }
    }
    F = Fn + Ftt;                                                // Eq. 2
    if (TERMS && (P.terms & 8)) F = F + n * (P.kcoh_pi * Reff * delta);
    Ft = Ftt;
    dnew = dt;
    Mroll = mk(T(0), T(0), T(0));
    if (TERMS && (P.terms & 2)) {
        const T wn2 = dot(wrel, wrel);
        if (wn2 > T(0)) Mroll = wrel * law_div(-P.mu_roll * Reff * law_sqrt(fn2), law_sqrt(wn2));
    }
}

// Simple law (Eq. 1): -k_sp delta n - k_da v - k_sh v_t, v_t = v - (v.n) n.
template <class T>
__device__ __forceinline__ V3<T> law_simple(const Law<T>& P, V3<T> n, T delta, V3<T> v) {
    const V3<T> vt = v - n * dot(v, n);
    return (n * (-P.ksp * delta) - v * P.kda) - vt * P.ksh;
}

}  // namespace demgb
