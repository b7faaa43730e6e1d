/*
 * FP64 CPU ORACLE of one soft-sphere DEM timestep -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline leg load
 * this library. It shares no code, header, table or helper with the CUDA library; the
 * two meet only in the seeded input arrays. It is written to be read against the paper
 * (Washizawa & Nakahara, "Parallel Computing of Discrete Element Method on GPU"):
 * straight-line FP64 arithmetic, one pair at a time, no blocking, no fusion.
 *
 *   cell map CM ............ Sec. 4.1, Sec. 4.2 step 2         orc_cell_keys
 *   sort by cell (SCM/SCCM)  Sec. 4.2 steps 3-4, Eq. 11         orc_sort_by_cell
 *   cell start table ....... implied by steps 3-6               orc_cell_start
 *   27-cell neighbourhood .. Sec. 4.2 step 6, Eq. 12            orc_pairs_grid
 *   contact pairs .......... Sec. 4.2 step 7 (detection)        orc_pairs_brute / orc_pairs_grid
 *   simple force ........... Eq. 1                              law_simple
 *   practical force ........ Eqs. 2-10                          law_practical
 *   one state's forces ..... steps 5-8                          orc_forces
 *   walls .................. Sec. 4.2 step 8                    wall_geometry
 *   update of properties ... Sec. 4.2 step 1                    integrate
 *
 * Readings where the paper is silent or ambiguous:
 *  - n is the unit vector from particle i to its partner j; v = v_i - v_j; the normal
 *    overlap is delta = r_i + r_j - |x_j - x_i| and delta_n = delta * n, so -k_n delta_n
 *    pushes i away from j (Eq. 4). Contact iff delta > 0, decided as d^2 < R^2 with
 *    d^2 = fma(dz,dz, fma(dy,dy, dx*dx)) and R = r_i + r_j (exact in FP64 for FP32 radii).
 *  - One eta serves both components (Eq. 4 as printed); eta = alpha*sqrt(k_n*m_eff) with
 *    m_eff = 1/(1/m_i + 1/m_j) (Eq. 10).
 *  - Eq. 5 caps iff |F_t| > mu|F_n| (strict, skipped when |F_t| = 0), where
 *    |F_n| is the length of the vector F_n of Eq. 4. After capping the stored spring
 *    is reset so that Eq. 4 still holds: delta_t = -(F_t + eta v_t)/k_t.
 *  - Eq. 7 is applied literally (projection onto the new tangent plane, no rescaling).
 *  - The history of a pair starts at zero on first contact and is dropped when the pair
 *    separates. It is stored once per pair (i < j) from i's side; j sees its negative.
 *  - Walls (step 8: a wall is a particle of infinite radius): R_eff = r_i, m_eff = m_i,
 *    n points from the particle to the wall, and the wall's surface velocity at the
 *    contact point replaces v_j + r_j omega_j x n in Eq. 6. The contact point is the
 *    point of the wall surface nearest the sphere centre.
 *  - Eq. 1 (simple model): F_i += -k_sp delta n - k_da v - k_sh v_t with
 *    v_t = v - (v.n) n; no spin, no torque, no history; walls use the same law.
 *  - Gravity m g is added once per particle (not per pair).
 *  - Moment of inertia of a solid sphere, I = (2/5) m r^2; m = rho (4/3) pi r^3.
 *  - Time integration (step 1 names no scheme): semi-implicit Euler,
 *    v' = v + dt F/m, w' = w + dt T/I, x' = x + dt v'.
 *  - Per-particle force sums run over partners in ascending global id, walls after
 *    particles (in wall order), gravity last.
 *  - Cell of a position: (i,j,k) = clamp(floor((x - o)/h), 0, dims-1) per axis. In
 *    hash mode 0 the subtraction and the division are IEEE FP64; in hash mode 1 they are
 *    IEEE FP32 on fl32(x), fl32(o), fl32(h) (the mixed-precision GPU mode hashes this
 *    way, and both sides must take the integer decision in the same precision).
 *    Key = (k*ny + j)*nx + i. Ties in the sort are broken by global id.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fused multiply-add unless
 * written as fma()).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_WALL_BASE 0xFFFFFF00u
#define ORC_PI 3.14159265358979323846

typedef struct {
    int32_t model;      /* 0 practical (Eqs. 2-10), 1 simple (Eq. 1) */
    int32_t stiffness;  /* 0 linear (constant k_n, k_t), 1 Hertz (Eqs. 8-9) */
    int32_t hash_mode;  /* 0 FP64 division, 1 FP32 division on fl32(x) */
    int32_t pad;
    double dt, rho, g[3];
    double kn, kt, cn, ct, alpha, mu;
    double ksp, kda, ksh;
    double origin[3], h;
    int64_t dims[3];
    int32_t terms;      /* optional force terms (see law_practical) */
    int32_t pad2;
    double mu_roll;     /* rolling resistance coefficient (terms & 2) */
    double alpha_t;     /* tangential damping factor (terms & 4) */
    double k_coh;       /* cohesion energy density [N/m^2] (terms & 8) */
} orc_params;

typedef struct {
    int32_t kind;       /* 0 plane (n = unit normal into the domain), 1 cylinder interior (n = unit axis),
                           2 half-plate: zero-thickness half-plane through p with unit normal n,
                           covering the side (y - p).u >= 0 of its edge (u unit, in the plane) */
    int32_t pad;
    double p[3], n[3], radius, omega[3], vel[3], u[3];
} orc_wall;

/* Sizes of the parameter and wall records (checked against the Python mirrors). */
void orc_struct_sizes(int64_t* out) {
    out[0] = (int64_t)sizeof(orc_params);
    out[1] = (int64_t)sizeof(orc_wall);
}

/* ------------------------------------------------------------- 3-vectors */
typedef struct { double x, y, z; } vec3;
static vec3 v3(double x, double y, double z) { vec3 r = {x, y, z}; return r; }
static vec3 vadd(vec3 a, vec3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static vec3 vsub(vec3 a, vec3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static vec3 vscale(vec3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
static double vdot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec3 vcross(vec3 a, vec3 b) {
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double vnorm(vec3 a) { return sqrt(vdot(a, a)); }
static vec3 load3(const double* p, int64_t k) { return v3(p[3 * k], p[3 * k + 1], p[3 * k + 2]); }
static void store3(double* p, int64_t k, vec3 a) { p[3 * k] = a.x; p[3 * k + 1] = a.y; p[3 * k + 2] = a.z; }
static void add3(double* p, int64_t k, vec3 a) { p[3 * k] += a.x; p[3 * k + 1] += a.y; p[3 * k + 2] += a.z; }

static double sphere_mass(const orc_params* P, double r) { return P->rho * (4.0 / 3.0) * ORC_PI * r * r * r; }

/* ------------------------------------------------ cell map (Sec. 4.1, step 2) */
static int64_t cell_coord(const orc_params* P, int a, double xa) {
    double q;
    if (P->hash_mode == 0) {
        q = floor((xa - P->origin[a]) / P->h);
    } else {
        float xf = (float)xa, of = (float)P->origin[a], hf = (float)P->h;
        float t = xf - of;
        float u = t / hf;
        q = floor((double)u);
    }
    int64_t i;
    if (q < 0.0) i = 0;
    else if (q >= (double)P->dims[a]) i = P->dims[a] - 1;
    else i = (int64_t)q;
    return i;
}

/* CM[j] = cell key of particle j; ijk optional (3 per particle) */
void orc_cell_keys(const orc_params* P, int64_t n, const double* x, int64_t* ijk, uint64_t* key) {
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = cell_coord(P, 0, x[3 * k]), j = cell_coord(P, 1, x[3 * k + 1]), l = cell_coord(P, 2, x[3 * k + 2]);
        if (ijk) { ijk[3 * k] = i; ijk[3 * k + 1] = j; ijk[3 * k + 2] = l; }
        key[k] = (uint64_t)((l * P->dims[1] + j) * P->dims[0] + i);
    }
}

/* --------------------------------------- sort by cell (steps 3-4, Eq. 11) */
typedef struct { uint64_t key; uint32_t id; } keyid;
static int cmp_keyid(const void* a, const void* b) {
    const keyid* p = (const keyid*)a; const keyid* q = (const keyid*)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    if (p->id != q->id) return p->id < q->id ? -1 : 1;
    return 0;
}
/* SCCM (order) and SCM (sorted_key) with SCM[j] = CM[SCCM[j]] */
int orc_sort_by_cell(int64_t n, const uint64_t* key, uint32_t* order, uint64_t* sorted_key) {
    keyid* t = (keyid*)malloc(sizeof(keyid) * (n > 0 ? n : 1));
    if (!t) return -1;
    for (int64_t k = 0; k < n; ++k) { t[k].key = key[k]; t[k].id = (uint32_t)k; }
    qsort(t, (size_t)n, sizeof(keyid), cmp_keyid);
    for (int64_t k = 0; k < n; ++k) { order[k] = t[k].id; if (sorted_key) sorted_key[k] = t[k].key; }
    free(t);
    return 0;
}

/* start[c] = number of particles in cells < c, for c = 0..ncells (so cell c holds sorted
 * positions start[c] .. start[c+1]-1) */
void orc_cell_start(int64_t n, const uint64_t* sorted_key, int64_t ncells, int64_t* start) {
    for (int64_t c = 0; c <= ncells; ++c) start[c] = 0;
    for (int64_t k = 0; k < n; ++k) start[sorted_key[k] + 1] += 1;
    for (int64_t c = 0; c < ncells; ++c) start[c + 1] += start[c];
}

/* ------------------------------------------------------ contact predicate */
static int in_contact(const double* x, const float* r, int64_t i, int64_t j) {
    double dx = x[3 * j] - x[3 * i];
    double dy = x[3 * j + 1] - x[3 * i + 1];
    double dz = x[3 * j + 2] - x[3 * i + 2];
    double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
    double R = (double)r[i] + (double)r[j];
    return d2 < R * R;
}

typedef struct { uint32_t i, j; } pairij;
static int cmp_pair(const void* a, const void* b) {
    const pairij* p = (const pairij*)a; const pairij* q = (const pairij*)b;
    if (p->i != q->i) return p->i < q->i ? -1 : 1;
    if (p->j != q->j) return p->j < q->j ? -1 : 1;
    return 0;
}

/* All pairs i < j in contact, by testing every pair (O(N^2)). pairs holds 2*cap u32.
 * Returns the number of pairs (may exceed cap: only the first cap are written). */
int64_t orc_pairs_brute(int64_t n, const double* x, const float* r, int64_t cap, uint32_t* pairs) {
    int64_t np = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (in_contact(x, r, i, j)) {
                if (np < cap) { pairs[2 * np] = (uint32_t)i; pairs[2 * np + 1] = (uint32_t)j; }
                ++np;
            }
    return np;
}

/* The same set found through the cell map: for each particle, the particles of the 3x3x3
 * block of cells around its own (Eq. 12, clipped at the grid's faces). Returns the count
 * (sorted by (i, j)), or -1 on allocation failure. ncand (optional) receives, per
 * particle, how many other particles its 27 cells hold (candidates). */
int64_t orc_pairs_grid(const orc_params* P, int64_t n, const double* x, const float* r, int64_t cap,
                       uint32_t* pairs, int64_t* ncand) {
    const int64_t ncells = P->dims[0] * P->dims[1] * P->dims[2];
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    uint64_t* skey = (uint64_t*)malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
    int64_t* ijk = (int64_t*)malloc(sizeof(int64_t) * 3 * (n > 0 ? n : 1));
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (ncells + 1));
    size_t pcap = 64;
    pairij* found = (pairij*)malloc(sizeof(pairij) * pcap);
    if (!key || !skey || !order || !ijk || !start || !found) {
        free(key); free(skey); free(order); free(ijk); free(start); free(found);
        return -1;
    }
    orc_cell_keys(P, n, x, ijk, key);
    orc_sort_by_cell(n, key, order, skey);
    orc_cell_start(n, skey, ncells, start);
    int64_t np = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = ijk[3 * i + a] - 1; if (lo[a] < 0) lo[a] = 0;
            hi[a] = ijk[3 * i + a] + 1; if (hi[a] > P->dims[a] - 1) hi[a] = P->dims[a] - 1;
        }
        int64_t cand = 0;
        for (int64_t cz = lo[2]; cz <= hi[2]; ++cz)
            for (int64_t cy = lo[1]; cy <= hi[1]; ++cy)
                for (int64_t cx = lo[0]; cx <= hi[0]; ++cx) {
                    int64_t c = (cz * P->dims[1] + cy) * P->dims[0] + cx;
                    for (int64_t s = start[c]; s < start[c + 1]; ++s) {
                        int64_t j = order[s];
                        if (j == i) continue;
                        ++cand;
                        if (j < i) continue;
                        if (in_contact(x, r, i, j)) {
                            if ((size_t)np == pcap) {
                                pcap *= 2;
                                pairij* g = (pairij*)realloc(found, sizeof(pairij) * pcap);
                                if (!g) { free(key); free(skey); free(order); free(ijk); free(start); free(found); return -1; }
                                found = g;
                            }
                            found[np].i = (uint32_t)i; found[np].j = (uint32_t)j; ++np;
                        }
                    }
                }
        if (ncand) ncand[i] = cand;
    }
    qsort(found, (size_t)np, sizeof(pairij), cmp_pair);
    for (int64_t k = 0; k < np && k < cap; ++k) { pairs[2 * k] = found[k].i; pairs[2 * k + 1] = found[k].j; }
    free(key); free(skey); free(order); free(ijk); free(start); free(found);
    return np;
}

/* ------------------------------------------------------------- history */
/* One tangential spring per contact: (i, j) with j > i a particle id, or j =
 * ORC_WALL_BASE + wall index. Arrays are kept sorted by (i, j). */
typedef struct { uint32_t i, j; double d[3]; } orc_hist_rec;
typedef orc_hist_rec hrec;
static int cmp_hrec(const void* a, const void* b) {
    const hrec* p = (const hrec*)a; const hrec* q = (const hrec*)b;
    if (p->i != q->i) return p->i < q->i ? -1 : 1;
    if (p->j != q->j) return p->j < q->j ? -1 : 1;
    return 0;
}
static vec3 hist_lookup(const hrec* h, int64_t nh, uint32_t i, uint32_t j) {
    hrec key; key.i = i; key.j = j;
    const hrec* f = (const hrec*)bsearch(&key, h, (size_t)nh, sizeof(hrec), cmp_hrec);
    if (!f) return v3(0.0, 0.0, 0.0);
    return v3(f->d[0], f->d[1], f->d[2]);
}

/* ------------------------------------------------- practical pair (Eqs. 2-10)
 * Computes, for the contact of i with partner j seen from i, the force F on i and the
 * torque factor F_t (torques: T_i = r_i n x F_t, T_j = r_j n x F_t by Eq. 3), and the new
 * tangential spring. ri_wi and rj_wj are r omega of each body (for a wall, the partner's
 * term is folded into v via its surface velocity and rj_wj = 0). */
typedef struct { vec3 F, Ft, dt_new, Mroll; double overlap; } contact_out;

/* Optional terms beyond Eqs. 2-10 (the paper builds its force from separable terms so
 * that terms can be added or removed, Sec. 3; none of these is in the paper):
 *  terms & 1  the normal force never attracts: if F_n . n > 0 on i, F_n = 0 (the Coulomb
 *             cap then uses |F_n| = 0);
 *  terms & 2  rolling resistance: a torque -mu_roll R_eff |F_n| w_rel/|w_rel| on i (and
 *             its negative on j), w_rel = w_i - w_j (a wall's angular velocity for walls);
 *  terms & 4  a separate tangential damping coefficient eta_t = alpha_t sqrt(k_t m_eff)
 *             in place of eta in the tangential part of Eq. 4 and in the spring reset;
 *  terms & 8  cohesion: a force k_coh pi R_eff delta n on i (toward j; contact area of
 *             a Hertzian contact, pi a^2 = pi R_eff delta) added after Eq. 5, so the
 *             Coulomb cap and the rolling torque use the spring-dashpot |F_n| alone. */
static contact_out law_practical(const orc_params* P, vec3 n, double delta, vec3 v, vec3 ri_wi, vec3 rj_wj,
                                 double Reff, double meff, vec3 dt_old, vec3 wrel) {
    contact_out o;
    /* Eq. 6 */
    double vn_s = vdot(v, n);
    vec3 vn = vscale(n, vn_s);
    vec3 vt = vadd(vsub(v, vn), vcross(vadd(ri_wi, rj_wj), n));
    /* Eq. 7 */
    vec3 dt = vadd(vsub(dt_old, vscale(n, vdot(dt_old, n))), vscale(vt, P->dt));
    /* Eqs. 8-9 */
    double kn, kt;
    if (P->stiffness == 0) { kn = P->kn; kt = P->kt; }
    else {
        double s = sqrt(fabs(delta) * Reff);   /* |delta_n| / (1/r_i + 1/r_j) */
        kn = P->cn * s;
        kt = P->ct * s;
    }
    /* Eq. 10 */
    double eta = P->alpha * sqrt(kn * meff);
    /* Eq. 4 */
    vec3 Fn = vsub(vscale(n, -kn * delta), vscale(vn, eta));
    if ((P->terms & 1) && vdot(Fn, n) > 0.0) Fn = v3(0.0, 0.0, 0.0);
    double eta_t = eta;
    if (P->terms & 4) eta_t = P->alpha_t * sqrt(kt * meff);
    vec3 Ft = vsub(vscale(dt, -kt), vscale(vt, eta_t));
    /* Eq. 5 */
    double ftn = vnorm(Ft), fnn = vnorm(Fn);
    if (ftn > P->mu * fnn && ftn > 0.0) {
        Ft = vscale(Ft, P->mu * fnn / ftn);
        if (kt > 0.0) dt = vscale(vadd(Ft, vscale(vt, eta_t)), -1.0 / kt);
    }
    /* Eq. 2 */
    o.F = vadd(Fn, Ft);
    if (P->terms & 8) o.F = vadd(o.F, vscale(n, P->k_coh * ORC_PI * Reff * delta));
    o.Ft = Ft;
    o.dt_new = dt;
    o.overlap = delta;
    o.Mroll = v3(0.0, 0.0, 0.0);
    if (P->terms & 2) {
        double wn = vnorm(wrel);
        if (wn > 0.0) o.Mroll = vscale(wrel, -P->mu_roll * Reff * fnn / wn);
    }
    return o;
}

/* -------------------------------------------------------- simple pair (Eq. 1) */
static contact_out law_simple(const orc_params* P, vec3 n, double delta, vec3 v) {
    contact_out o;
    vec3 vt = vsub(v, vscale(n, vdot(v, n)));
    vec3 F = vscale(n, -P->ksp * delta);
    F = vsub(F, vscale(v, P->kda));
    F = vsub(F, vscale(vt, P->ksh));
    o.F = F;
    o.Ft = v3(0.0, 0.0, 0.0);
    o.dt_new = v3(0.0, 0.0, 0.0);
    o.Mroll = v3(0.0, 0.0, 0.0);
    o.overlap = delta;
    return o;
}

/* ------------------------------------------------------- wall geometry (step 8)
 * For sphere (x, r) and wall W: returns 1 if in contact (delta > 0) and fills the unit
 * normal n from the sphere toward the wall, the overlap delta and the contact point c. */
static int wall_geometry(const orc_wall* W, vec3 x, double r, vec3* n, double* delta, vec3* c) {
    vec3 p = v3(W->p[0], W->p[1], W->p[2]);
    vec3 a = v3(W->n[0], W->n[1], W->n[2]);
    if (W->kind == 0) {
        double s = vdot(vsub(x, p), a);          /* distance of the centre from the plane */
        double d = r - s;
        if (!(d > 0.0)) return 0;
        *n = vscale(a, -1.0);
        *delta = d;
        *c = vsub(x, vscale(a, s));
        return 1;
    } else if (W->kind == 2) {
        /* Half-plate (two of them with opposite u make a slit, the bottom of the paper's
         * benchmark box, Sec. 5): touched from either side. The nearest plate point to
         * the centre is its projection when that lies on the plate (s >= 0), else the
         * point of the edge line (s = 0) beside it. */
        vec3 u = v3(W->u[0], W->u[1], W->u[2]);
        vec3 q = vsub(x, p);
        double h = vdot(q, a);                  /* height above the plate's plane */
        double s = vdot(q, u);                  /* distance from the edge line into the plate */
        vec3 e = vscale(a, -h);                 /* from the centre to the nearest plate point */
        if (s < 0.0) e = vadd(e, vscale(u, -s));
        double dist = vnorm(e);
        double d = r - dist;
        if (!(d > 0.0)) return 0;
        if (dist > 0.0) *n = vscale(e, 1.0 / dist);
        else *n = vscale(a, -1.0);
        *delta = d;
        *c = vadd(x, e);
        return 1;
    } else {
        vec3 q = vsub(x, p);
        double ax = vdot(q, a);
        vec3 rho = vsub(q, vscale(a, ax));
        double rr = vnorm(rho);
        double d = rr + r - W->radius;
        if (!(d > 0.0) || !(rr > 0.0)) return 0;
        *n = vscale(rho, 1.0 / rr);
        *delta = d;
        *c = vadd(vadd(p, vscale(a, ax)), vscale(*n, W->radius));
        return 1;
    }
}
static vec3 wall_velocity(const orc_wall* W, vec3 c) {
    vec3 p = v3(W->p[0], W->p[1], W->p[2]);
    vec3 om = v3(W->omega[0], W->omega[1], W->omega[2]);
    return vadd(v3(W->vel[0], W->vel[1], W->vel[2]), vcross(om, vsub(c, p)));
}

/* ----------------------------------------------------- forces of one state
 * Evaluates every contact of the state (x, v, w, r) and returns per-particle force F and
 * torque T (gravity included). hist_in (sorted, nh_in records) gives delta_t,old; the
 * springs of this step's contacts are written to hist_out (sorted; capacity cap_out).
 * Returns the number of records written to hist_out, -1 on allocation failure, or -2 if
 * hist_out is too small. pair_mode 0 = brute-force pair search, 1 = cell grid.
 * stats (optional, 4 doubles): number of particle pairs, number of wall contacts,
 * maximum overlap, sum of overlaps. */
int64_t orc_forces(const orc_params* P, int32_t nwalls, const orc_wall* walls, int64_t n, const double* x,
                   const double* v, const double* w, const float* r, const orc_hist_rec* hist_in, int64_t nh_in,
                   int32_t pair_mode, double* F, double* T, orc_hist_rec* hist_out, int64_t cap_out, double* stats) {
    const hrec* hin = hist_in;
    hrec* hout = hist_out;
    int64_t pcap = 16 * (n > 0 ? n : 1);
    uint32_t* pairs = NULL;
    int64_t np;
    for (;;) {
        pairs = (uint32_t*)malloc(sizeof(uint32_t) * 2 * pcap);
        if (!pairs) return -1;
        np = pair_mode == 0 ? orc_pairs_brute(n, x, r, pcap, pairs) : orc_pairs_grid(P, n, x, r, pcap, pairs, NULL);
        if (np < 0) { free(pairs); return -1; }
        if (np <= pcap) break;
        free(pairs);
        pcap = np;
    }
    for (int64_t k = 0; k < 3 * n; ++k) { F[k] = 0.0; T[k] = 0.0; }
    int64_t nout = 0, nwallc = 0;
    double maxov = 0.0, sumov = 0.0;
    /* Particle pairs in (i, j) order: every particle receives its partners' contributions
     * in ascending partner id. */
    for (int64_t k = 0; k < np; ++k) {
        uint32_t i = pairs[2 * k], j = pairs[2 * k + 1];
        double dxv = x[3 * j] - x[3 * i], dyv = x[3 * j + 1] - x[3 * i + 1], dzv = x[3 * j + 2] - x[3 * i + 2];
        double d2 = fma(dzv, dzv, fma(dyv, dyv, dxv * dxv));
        double d = sqrt(d2);
        double R = (double)r[i] + (double)r[j];
        vec3 n = v3(dxv / d, dyv / d, dzv / d);
        double delta = R - d;
        vec3 vrel = vsub(load3(v, i), load3(v, j));
        double ri = (double)r[i], rj = (double)r[j];
        contact_out o;
        if (P->model == 0) {
            double mi = sphere_mass(P, ri), mj = sphere_mass(P, rj);
            double Reff = 1.0 / (1.0 / ri + 1.0 / rj);
            double meff = 1.0 / (1.0 / mi + 1.0 / mj);
            vec3 dold = hist_lookup(hin, nh_in, i, j);
            o = law_practical(P, n, delta, vrel, vscale(load3(w, i), ri), vscale(load3(w, j), rj), Reff, meff, dold,
                              vsub(load3(w, i), load3(w, j)));
            if (nout >= cap_out) { free(pairs); return -2; }
            hout[nout].i = i; hout[nout].j = j;
            hout[nout].d[0] = o.dt_new.x; hout[nout].d[1] = o.dt_new.y; hout[nout].d[2] = o.dt_new.z;
            ++nout;
        } else {
            o = law_simple(P, n, delta, vrel);
        }
        add3(F, i, o.F);
        add3(F, j, vscale(o.F, -1.0));
        vec3 tq = vcross(n, o.Ft);
        add3(T, i, vadd(vscale(tq, ri), o.Mroll));
        add3(T, j, vsub(vscale(tq, rj), o.Mroll));
        if (delta > maxov) maxov = delta;
        sumov += delta;
    }
    /* walls (step 8), then gravity */
    for (int64_t i = 0; i < n; ++i) {
        double ri = (double)r[i];
        double mi = sphere_mass(P, ri);
        for (int32_t wi = 0; wi < nwalls; ++wi) {
            vec3 nn, c; double delta;
            if (!wall_geometry(&walls[wi], load3(x, i), ri, &nn, &delta, &c)) continue;
            vec3 vrel = vsub(load3(v, i), wall_velocity(&walls[wi], c));
            contact_out o;
            uint32_t jw = ORC_WALL_BASE + (uint32_t)wi;
            if (P->model == 0) {
                vec3 dold = hist_lookup(hin, nh_in, (uint32_t)i, jw);
                vec3 wwall = v3(walls[wi].omega[0], walls[wi].omega[1], walls[wi].omega[2]);
                o = law_practical(P, nn, delta, vrel, vscale(load3(w, i), ri), v3(0.0, 0.0, 0.0), ri, mi, dold,
                                  vsub(load3(w, i), wwall));
                if (nout >= cap_out) { free(pairs); return -2; }
                hout[nout].i = (uint32_t)i; hout[nout].j = jw;
                hout[nout].d[0] = o.dt_new.x; hout[nout].d[1] = o.dt_new.y; hout[nout].d[2] = o.dt_new.z;
                ++nout;
            } else {
                o = law_simple(P, nn, delta, vrel);
            }
            add3(F, i, o.F);
            add3(T, i, vadd(vscale(vcross(nn, o.Ft), ri), o.Mroll));
            ++nwallc;
            if (delta > maxov) maxov = delta;
            sumov += delta;
        }
        add3(F, i, vscale(v3(P->g[0], P->g[1], P->g[2]), mi));
    }
    qsort(hout, (size_t)nout, sizeof(hrec), cmp_hrec);
    if (stats) { stats[0] = (double)np; stats[1] = (double)nwallc; stats[2] = maxov; stats[3] = sumov; }
    free(pairs);
    return nout;
}

/* ----------------------------------------------- update of properties (step 1) */
static void integrate(const orc_params* P, int64_t n, double* x, double* v, double* w, const float* r,
                      const double* F, const double* T) {
    for (int64_t i = 0; i < n; ++i) {
        double ri = (double)r[i];
        double m = sphere_mass(P, ri);
        double I = 0.4 * m * ri * ri;
        vec3 vn = vadd(load3(v, i), vscale(load3(F, i), P->dt / m));
        vec3 wn = vadd(load3(w, i), vscale(load3(T, i), P->dt / I));
        vec3 xn = vadd(load3(x, i), vscale(vn, P->dt));
        store3(v, i, vn);
        store3(w, i, wn);
        store3(x, i, xn);
    }
}

/* nsteps full timesteps in place. hist (capacity cap, *nh records on entry and exit) is
 * the persistent tangential history. F, T (3n each, may be NULL) receive the forces of
 * the last step. Returns 0, -1 (allocation) or -2 (history capacity). */
int orc_run(const orc_params* P, int32_t nwalls, const orc_wall* walls, int64_t n, double* x, double* v, double* w,
            const float* r, orc_hist_rec* hist, int64_t* nh, int64_t cap, int32_t pair_mode, int64_t nsteps,
            double* Fout, double* Tout, double* stats) {
    double* F = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double* T = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    orc_hist_rec* tmp = (orc_hist_rec*)malloc(sizeof(orc_hist_rec) * (cap > 0 ? cap : 1));
    if (!F || !T || !tmp) { free(F); free(T); free(tmp); return -1; }
    for (int64_t s = 0; s < nsteps; ++s) {
        int64_t no = orc_forces(P, nwalls, walls, n, x, v, w, r, hist, *nh, pair_mode, F, T, tmp, cap, stats);
        if (no < 0) { free(F); free(T); free(tmp); return (int)no; }
        integrate(P, n, x, v, w, r, F, T);
        memcpy(hist, tmp, sizeof(orc_hist_rec) * (size_t)no);
        *nh = no;
    }
    if (Fout) memcpy(Fout, F, sizeof(double) * 3 * n);
    if (Tout) memcpy(Tout, T, sizeof(double) * 3 * n);
    free(F); free(T); free(tmp);
    return 0;
}

/* ------------------------------------------------------------ diagnostics
 * out[0] translational KE, out[1] rotational KE, out[2..4] linear momentum,
 * out[5..7] angular momentum about the origin (m x cross v + I w), out[8] gravitational
 * potential energy (-m g.x), out[9] total mass. */
void orc_diagnostics(const orc_params* P, int64_t n, const double* x, const double* v, const double* w,
                     const float* r, double* out) {
    for (int k = 0; k < 10; ++k) out[k] = 0.0;
    vec3 g = v3(P->g[0], P->g[1], P->g[2]);
    for (int64_t i = 0; i < n; ++i) {
        double ri = (double)r[i];
        double m = sphere_mass(P, ri);
        double I = 0.4 * m * ri * ri;
        vec3 xi = load3(x, i), vi = load3(v, i), wi = load3(w, i);
        out[0] += 0.5 * m * vdot(vi, vi);
        out[1] += 0.5 * I * vdot(wi, wi);
        out[2] += m * vi.x; out[3] += m * vi.y; out[4] += m * vi.z;
        vec3 L = vadd(vscale(vcross(xi, vi), m), vscale(wi, I));
        out[5] += L.x; out[6] += L.y; out[7] += L.z;
        out[8] += -m * vdot(g, xi);
        out[9] += m;
    }
}
