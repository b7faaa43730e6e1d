/*
 * Seeded synthetic DEM scenes: initial particle positions, radii and velocities.
 *
 * This file generates INPUTS only. It holds none of the contact-force, hashing,
 * sorting or integration arithmetic of the method; both the CUDA library and the
 * CPU oracle receive the arrays it fills.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through SplitMix64
 * (Steele, Lea & Flood, 2014), both written here from their published definitions.
 * Normal variates use the Box-Muller transform. Every generator is a pure function of
 * its seed and arguments, so the same call gives the same bytes on x86-64 and aarch64
 * (IEEE double arithmetic, no fused multiply-add: compile with -ffp-contract=off).
 *
 * Scene families (the shapes of the paper's workloads; the paper's own hopper geometry
 * is not given, Sec. 5):
 *   scn_lattice_box  jittered simple-cubic lattice in a walled box
 *   scn_rsa_box      random sequential addition (loose fill) in a walled box
 *   scn_drum_fill    dense layered deposition in the lower part of a horizontal drum
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- PRNG */
typedef struct { uint64_t s[4]; } scn_rng;

static uint64_t splitmix64(uint64_t* x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static uint64_t rotl64(uint64_t v, int k) { return (v << k) | (v >> (64 - k)); }
static void rng_seed(scn_rng* r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}
static uint64_t rng_next(scn_rng* r) {
    uint64_t* s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl64(s[3], 45);
    return result;
}
/* uniform in [0,1) with 53 random bits */
static double rng_u01(scn_rng* r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }
static double rng_uniform(scn_rng* r, double a, double b) { return a + (b - a) * rng_u01(r); }
/* standard normal via Box-Muller (one value per call; the sine branch is discarded) */
static double rng_normal(scn_rng* r) {
    double u1 = rng_u01(r), u2 = rng_u01(r);
    if (u1 < 0x1.0p-60) u1 = 0x1.0p-60;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* exported for the tests that pin the generator itself */
uint64_t scn_xoshiro_first(uint64_t seed, int k, uint64_t* out) {
    scn_rng r; rng_seed(&r, seed);
    for (int i = 0; i < k; ++i) out[i] = rng_next(&r);
    return (uint64_t)k;
}

void scn_uniform(uint64_t seed, int64_t n, double a, double b, double* out) {
    scn_rng r; rng_seed(&r, seed);
    for (int64_t i = 0; i < n; ++i) out[i] = rng_uniform(&r, a, b);
}

void scn_normal(uint64_t seed, int64_t n, double sigma, double* out) {
    scn_rng r; rng_seed(&r, seed);
    for (int64_t i = 0; i < n; ++i) out[i] = sigma * rng_normal(&r);
}

/* log-uniform integers in [lo, hi] (used for scene-size mixes) */
void scn_loguniform_int(uint64_t seed, int64_t n, double lo, double hi, int64_t* out) {
    scn_rng r; rng_seed(&r, seed);
    double a = log(lo), b = log(hi);
    for (int64_t i = 0; i < n; ++i) {
        double v = exp(rng_uniform(&r, a, b));
        int64_t k = (int64_t)floor(v + 0.5);
        if (k < (int64_t)lo) k = (int64_t)lo;
        if (k > (int64_t)hi) k = (int64_t)hi;
        out[i] = k;
    }
}

/* ------------------------------------------------ jittered lattice in a box
 * nx*ny*nz particles on a simple-cubic lattice of the given spacing, the first site at
 * `first` (x,y,z), each coordinate jittered by U(-jitter, +jitter); radius r for all;
 * velocity components N(0, vsigma); spin zero. Particle k = (iz*ny + iy)*nx + ix.
 */
void scn_lattice_box(uint64_t seed, int nx, int ny, int nz, double spacing, double jitter,
                     const double first[3], double r, double vsigma,
                     double* x, double* v, double* w, float* rad) {
    scn_rng g; rng_seed(&g, seed);
    int64_t k = 0;
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix, ++k) {
                x[3 * k + 0] = first[0] + ix * spacing + rng_uniform(&g, -jitter, jitter);
                x[3 * k + 1] = first[1] + iy * spacing + rng_uniform(&g, -jitter, jitter);
                x[3 * k + 2] = first[2] + iz * spacing + rng_uniform(&g, -jitter, jitter);
                rad[k] = (float)r;
            }
    for (int64_t i = 0; i < 3 * k; ++i) v[i] = vsigma * rng_normal(&g);
    for (int64_t i = 0; i < 3 * k; ++i) w[i] = 0.0;
}

/* ---------------------------------------------- helper: 3-D occupancy grid */
typedef struct {
    double lo[3], h;
    int64_t dims[3];
    int64_t* head;   /* per cell: first particle, -1 if none */
    int64_t* next;   /* per particle: next particle in the same cell */
} scn_grid;

static int scn_grid_init(scn_grid* G, const double lo[3], const double hi[3], double h, int64_t cap) {
    G->h = h;
    int64_t nc = 1;
    for (int a = 0; a < 3; ++a) {
        G->lo[a] = lo[a];
        G->dims[a] = (int64_t)ceil((hi[a] - lo[a]) / h);
        if (G->dims[a] < 1) G->dims[a] = 1;
        nc *= G->dims[a];
    }
    G->head = (int64_t*)malloc(sizeof(int64_t) * nc);
    G->next = (int64_t*)malloc(sizeof(int64_t) * (cap > 0 ? cap : 1));
    if (!G->head || !G->next) { free(G->head); free(G->next); return -1; }
    for (int64_t c = 0; c < nc; ++c) G->head[c] = -1;
    return 0;
}
static void scn_grid_free(scn_grid* G) { free(G->head); free(G->next); }
static int64_t scn_grid_coord(const scn_grid* G, int a, double p) {
    int64_t i = (int64_t)floor((p - G->lo[a]) / G->h);
    if (i < 0) i = 0;
    if (i >= G->dims[a]) i = G->dims[a] - 1;
    return i;
}
static void scn_grid_insert(scn_grid* G, int64_t k, const double* p) {
    int64_t ix = scn_grid_coord(G, 0, p[0]), iy = scn_grid_coord(G, 1, p[1]), iz = scn_grid_coord(G, 2, p[2]);
    int64_t c = (iz * G->dims[1] + iy) * G->dims[0] + ix;
    G->next[k] = G->head[c];
    G->head[c] = k;
}
/* 1 if a sphere (p, rp) overlaps (or touches within `gap`) any inserted sphere */
static int scn_grid_hits(const scn_grid* G, const double* x, const float* rad, const double* p, double rp, double gap) {
    int64_t c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
        c0[a] = scn_grid_coord(G, a, p[a] - G->h);
        c1[a] = scn_grid_coord(G, a, p[a] + G->h);
    }
    for (int64_t iz = c0[2]; iz <= c1[2]; ++iz)
        for (int64_t iy = c0[1]; iy <= c1[1]; ++iy)
            for (int64_t ix = c0[0]; ix <= c1[0]; ++ix) {
                int64_t c = (iz * G->dims[1] + iy) * G->dims[0] + ix;
                for (int64_t k = G->head[c]; k >= 0; k = G->next[k]) {
                    double dx = x[3 * k] - p[0], dy = x[3 * k + 1] - p[1], dz = x[3 * k + 2] - p[2];
                    double s = (double)rad[k] + rp + gap;
                    if (dx * dx + dy * dy + dz * dz < s * s) return 1;
                }
            }
    return 0;
}

/* ---------------------------------------- random sequential addition (loose fill)
 * n spheres with radii U[rmin, rmax] placed one by one at uniform random positions in
 * the region [lo, hi] (wall clearance r), rejecting any that would overlap a placed
 * sphere. If one sphere needs more than max_tries attempts the region's top (z) grows
 * by 1% of its height and the attempts continue. Velocities and spins are zero.
 * Returns the number of grow events (>= 0), or -1 on allocation failure.
 */
int64_t scn_rsa_box(uint64_t seed, int64_t n, double rmin, double rmax,
                    const double lo[3], const double hi_in[3], int64_t max_tries,
                    double* x, double* v, double* w, float* rad) {
    scn_rng g; rng_seed(&g, seed);
    double hi[3] = {hi_in[0], hi_in[1], hi_in[2]};
    /* the grid spans a generous height so that growth never leaves it */
    double ghi[3] = {hi[0], hi[1], lo[2] + 4.0 * (hi[2] - lo[2]) + 4.0 * rmax};
    scn_grid G;
    if (scn_grid_init(&G, lo, ghi, 2.0 * rmax, n) != 0) return -1;
    int64_t grows = 0;
    for (int64_t k = 0; k < n; ++k) {
        double rk = rng_uniform(&g, rmin, rmax);
        rad[k] = (float)rk;
        double rr = (double)rad[k];
        int64_t tries = 0;
        for (;;) {
            double p[3];
            for (int a = 0; a < 3; ++a) p[a] = rng_uniform(&g, lo[a] + rr, hi[a] - rr);
            if (!scn_grid_hits(&G, x, rad, p, rr, 0.0)) {
                x[3 * k] = p[0]; x[3 * k + 1] = p[1]; x[3 * k + 2] = p[2];
                scn_grid_insert(&G, k, p);
                break;
            }
            if (++tries >= max_tries) {
                hi[2] += 0.01 * (hi_in[2] - lo[2]);
                if (hi[2] > ghi[2] - rmax) hi[2] = ghi[2] - rmax;
                ++grows;
                tries = 0;
            }
        }
    }
    for (int64_t i = 0; i < 3 * n; ++i) { v[i] = 0.0; w[i] = 0.0; }
    scn_grid_free(&G);
    return grows;
}

/* ------------------------------------ layered deposition in a horizontal drum
 * Drum: axis along x through (0, 0, 0), radius Rd, end caps at x = 0 and x = L;
 * gravity along -z. Radii U[rmin, rmax]. Lateral sites form a triangular lattice of
 * spacing a = 2*rmax*(1 + 1e-9) in the x-y plane, with the A/B/C stacking offset cycling
 * from pass to pass. Pass k visits every site (in a seeded random order) and drops a new
 * sphere vertically onto what is already placed: its height is the lowest z that
 * clears every placed sphere within lateral reach and the drum shell. The sphere is kept
 * only if that height lies below the pass's slab top, -Rd + (k+1)*slab, so the bed grows
 * from the bottom up with a nearly flat top. Deposition stops at n spheres. Velocities
 * and spins are zero.
 * Returns the number of passes used, or -1 (allocation) / -2 (did not fit).
 */
typedef struct { int64_t cnt; int64_t top[12]; } scn_col;

int64_t scn_drum_fill(uint64_t seed, int64_t n, double rmin, double rmax, double Rd, double L,
                      double slab, double* x, double* v, double* w, float* rad) {
    scn_rng g; rng_seed(&g, seed);
    const double a = 2.0 * rmax * (1.0 + 1e-9);
    const double row = a * 0.8660254037844386;          /* a*sqrt(3)/2 */
    const int64_t nsx = (int64_t)floor(L / a) + 1;
    const int64_t nsy = (int64_t)floor(2.0 * Rd / row) + 2;
    const int64_t nsites = nsx * nsy;
    /* lateral columns of size a x a keep the highest few spheres each */
    const double ch = a;
    const int64_t ncx = (int64_t)ceil(L / ch) + 1, ncy = (int64_t)ceil(2.0 * Rd / ch) + 1;
    scn_col* col = (scn_col*)calloc((size_t)(ncx * ncy), sizeof(scn_col));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * nsites);
    if (!col || !order) { free(col); free(order); return -1; }
    int64_t placed = 0, pass = 0;
    const int64_t max_pass = (int64_t)(2.0 * Rd / slab) + 8;
    /* radius for the next sphere (drawn once, kept until it is placed) */
    double rk = (double)(float)rng_uniform(&g, rmin, rmax);
    while (placed < n && pass < max_pass) {
        const double zmax = -Rd + (double)(pass + 1) * slab;
        const double offx = (double)(pass % 3) * 0.5 * a;
        const double offy = (double)(pass % 3) * a * 0.28867513459481287;  /* a*sqrt(3)/6 */
        for (int64_t s = 0; s < nsites; ++s) order[s] = s;
        for (int64_t s = nsites - 1; s > 0; --s) {          /* Fisher-Yates */
            int64_t t = (int64_t)(rng_u01(&g) * (double)(s + 1));
            if (t > s) t = s;
            int64_t tmp = order[s]; order[s] = order[t]; order[t] = tmp;
        }
        for (int64_t si = 0; si < nsites && placed < n; ++si) {
            const int64_t s = order[si];
            const int64_t sx = s % nsx, sy = s / nsx;
            const double px = offx + (double)sx * a + ((sy & 1) ? 0.5 * a : 0.0) + rmax;
            const double py = -Rd + offy + (double)sy * row + rmax;
            if (px < rk || px > L - rk) continue;
            const double rin = (Rd - rk) * (1.0 - 1e-10);     /* clear of the shell by rounding */
            if (fabs(py) >= rin) continue;
            double z = -sqrt(rin * rin - py * py);            /* drum shell below */
            const int64_t cx = (int64_t)floor(px / ch), cy = (int64_t)floor((py + Rd) / ch);
            for (int64_t jy = cy - 2; jy <= cy + 2; ++jy)
                for (int64_t jx = cx - 2; jx <= cx + 2; ++jx) {
                    if (jx < 0 || jy < 0 || jx >= ncx || jy >= ncy) continue;
                    const scn_col* C = &col[jy * ncx + jx];
                    for (int64_t t = 0; t < C->cnt; ++t) {
                        const int64_t j = C->top[t];
                        const double dx = x[3 * j] - px, dy = x[3 * j + 1] - py;
                        const double s2 = (double)rad[j] + rk;
                        const double dl2 = dx * dx + dy * dy;
                        if (dl2 < s2 * s2) {
                            const double zt = x[3 * j + 2] + sqrt(s2 * s2 - dl2) * (1.0 + 1e-9);
                            if (zt > z) z = zt;
                        }
                    }
                }
            if (z > zmax) continue;
            if (py * py + z * z > rin * rin) continue;       /* must stay inside the shell */
            x[3 * placed] = px; x[3 * placed + 1] = py; x[3 * placed + 2] = z;
            rad[placed] = (float)rk;
            /* keep the column's highest spheres */
            scn_col* C = &col[cy * ncx + cx];
            if (C->cnt < 12) C->top[C->cnt++] = placed;
            else {
                int64_t lowest = 0;
                for (int64_t t = 1; t < 12; ++t)
                    if (x[3 * C->top[t] + 2] < x[3 * C->top[lowest] + 2]) lowest = t;
                C->top[lowest] = placed;
            }
            ++placed;
            rk = (double)(float)rng_uniform(&g, rmin, rmax);
        }
        ++pass;
    }
    free(col); free(order);
    if (placed < n) return -2;
    for (int64_t i = 0; i < 3 * n; ++i) { v[i] = 0.0; w[i] = 0.0; }
    return pass;
}

/* ------------------------------------------------------ overlap audit (inputs)
 * Counts sphere pairs whose centre distance is below r_i + r_j (a check that a
 * generated scene has no initial overlaps). O(N) with a grid. Returns -1 on failure.
 */
int64_t scn_count_overlaps(int64_t n, const double* x, const float* rad, double rmax) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t k = 0; k < n; ++k)
        for (int a = 0; a < 3; ++a) {
            if (x[3 * k + a] < lo[a]) lo[a] = x[3 * k + a];
            if (x[3 * k + a] > hi[a]) hi[a] = x[3 * k + a];
        }
    for (int a = 0; a < 3; ++a) hi[a] += 1e-12;
    scn_grid G;
    if (scn_grid_init(&G, lo, hi, 2.0 * rmax, n) != 0) return -1;
    int64_t cnt = 0;
    for (int64_t k = 0; k < n; ++k) {
        cnt += 0;
        int64_t ix = scn_grid_coord(&G, 0, x[3 * k]), iy = scn_grid_coord(&G, 1, x[3 * k + 1]),
                iz = scn_grid_coord(&G, 2, x[3 * k + 2]);
        for (int64_t jz = iz - 1; jz <= iz + 1; ++jz)
            for (int64_t jy = iy - 1; jy <= iy + 1; ++jy)
                for (int64_t jx = ix - 1; jx <= ix + 1; ++jx) {
                    if (jx < 0 || jy < 0 || jz < 0 || jx >= G.dims[0] || jy >= G.dims[1] || jz >= G.dims[2]) continue;
                    int64_t c = (jz * G.dims[1] + jy) * G.dims[0] + jx;
                    for (int64_t j = G.head[c]; j >= 0; j = G.next[j]) {
                        double dx = x[3 * j] - x[3 * k], dy = x[3 * j + 1] - x[3 * k + 1], dz = x[3 * j + 2] - x[3 * k + 2];
                        double s = (double)rad[j] + (double)rad[k];
                        if (dx * dx + dy * dy + dz * dz < s * s) ++cnt;
                    }
                }
        scn_grid_insert(&G, k, &x[3 * k]);
    }
    scn_grid_free(&G);
    return cnt;
}
