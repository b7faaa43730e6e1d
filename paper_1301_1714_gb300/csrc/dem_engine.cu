// Host engine behind the C ABI of include/dem.h: validation, device buffers, the
// per-step launch sequence and the read-out paths.
//
// One dem_step = force pass (steps 5-8 and step 1, which also computes the new cell map
// CM of step 2 and each particle's rank within its cell) followed by the cell sort
// (steps 3-4: scan of the cell counts, scatter, (cell, id) order and gather).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "dem.h"
#include "dem_domain.h"
#include "dem_halo.h"

using namespace demgb;

struct dem_handle {
    Domain d;
    dem_config cfg{};
    int device = 0;
    std::vector<dem_wall> walls;
    double rmax = 0.0;
    double origin[3] = {0, 0, 0};
    double h = 0.0;
    int64_t dims[3] = {1, 1, 1};
    int bshift = 0;                    // cell order of the sort: 0 row-major, s > 0 bricks of (2^s)^3 cells (list mode)
    int64_t bdims[3] = {1, 1, 1};      // bricks per axis
    bool has_particles = false;
    bool broken = false;
    bool eval_valid = false;
    int64_t steps = 0;
    std::string err;
    StepGraph graph;   // replayed by dem_step when timing is off and the stream is not the legacy one
    // phase timing (events around force passes and sorts)
    bool timing = false;
    std::vector<cudaEvent_t> events;
    double t_force_ms = 0.0, t_sort_ms = 0.0;
    int64_t n_force = 0, n_sort = 0;
    // staging for host <-> device transfers (x, v, w: 3n doubles each; r: n floats)
    double* stage = nullptr;
    float* stage_r = nullptr;
    uint32_t stage_cap = 0;
    // input check of dem_set_particles: flags and the largest radius (device, pinned host);
    // chk_host[2]: the device's count of completed steps when a dem_step attempt began
    uint32_t* chk_dev = nullptr;
    uint32_t* chk_host = nullptr;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

dem_status fail(dem_handle* h, dem_status s, const std::string& msg) {
    if (h) h->err = msg;
    return s;
}

dem_status cuda_fail(dem_handle* h, cudaError_t e, const char* what) {
    if (h) {
        h->broken = true;
        h->err = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return DEM_ERR_CUDA;
}

#define CK(h, expr)                                                        \
    do {                                                                   \
        cudaError_t e__ = (expr);                                          \
        if (e__ != cudaSuccess) return cuda_fail((h), e__, #expr);         \
    } while (0)

template <class P>
cudaError_t dmalloc(Domain& d, P** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) return e;
    d.allocations.push_back(q);
    *p = (P*)q;
    return cudaSuccess;
}

void free_particle_buffers(Domain& d) {
    for (void* p : d.allocations) cudaFree(p);
    d.allocations.clear();
    d.S64[0] = d.S64[1] = StateF64{};
    d.S32[0] = d.S32[1] = StateF32{};
    d.ncnt = d.nl = d.wmask = nullptr;
    d.ref = nullptr;
    d.canon = d.fin = nullptr;
    for (int i = 0; i < 2; ++i) { d.hcnt[i] = nullptr; d.hpid[i] = nullptr; d.hd[i] = nullptr; }
    d.key = d.rank = d.tmp = d.perm = d.skey = d.cnt = d.cs = d.part = nullptr;
    d.diag_part = nullptr;
    d.cap = 0;
    d.cells_cap = 0;
    d.part_cap = 0;
    d.diag_part_cap = 0;
}

bool finite3(const double* a) { return std::isfinite(a[0]) && std::isfinite(a[1]) && std::isfinite(a[2]); }

void split_f(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// Fill a WallDev from a dem_wall.
// Blocks of 256 threads for the sort-phase kernels: eight per SM fill the SM.
int sort_blocks_of(int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 152;
    }
    return 8 * sms;
}

WallDev make_wall(const dem_wall& w) {
    WallDev W{};
    W.kind = w.kind;
    W.axis = -1;
    for (int a = 0; a < 3; ++a) {
        W.p[a] = w.p[a];
        W.n[a] = w.n[a];
        W.omega[a] = w.omega[a];
        W.vel[a] = w.vel[a];
        split_f(w.p[a], W.p_hi[a], W.p_lo[a]);
        split_f(w.n[a], W.n_hi[a], W.n_lo[a]);
        W.nf[a] = (float)w.n[a];
        W.omegaf[a] = (float)w.omega[a];
        W.velf[a] = (float)w.vel[a];
        W.pf[a] = (float)w.p[a];
    }
    W.radius = w.radius;
    split_f(w.radius, W.rad_hi, W.rad_lo);
    W.uaxis = -1;
    for (int a = 0; a < 3; ++a) {
        W.u[a] = w.u[a];
        W.uf[a] = (float)w.u[a];
    }
    // coordinate-axis normal / axis (and the plate's axis across the slit)
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        if (std::fabs(w.n[a]) == 1.0 && w.n[b] == 0.0 && w.n[c] == 0.0) W.axis = a;
        if (w.kind == DEM_HALF_PLATE && std::fabs(w.u[a]) == 1.0 && w.u[b] == 0.0 && w.u[c] == 0.0) W.uaxis = a;
    }
    return W;
}

bool check_wall(const dem_wall& w, int precision, std::string& why) {
    if (w.kind != DEM_PLANE && w.kind != DEM_CYLINDER_IN && w.kind != DEM_HALF_PLATE) { why = "wall kind"; return false; }
    if (!finite3(w.p) || !finite3(w.n) || !finite3(w.omega) || !finite3(w.vel) || !finite3(w.u)) {
        why = "wall vectors must be finite";
        return false;
    }
    const double nn = w.n[0] * w.n[0] + w.n[1] * w.n[1] + w.n[2] * w.n[2];
    if (std::fabs(nn - 1.0) > 1e-12) { why = "wall n must be a unit vector"; return false; }
    if (w.kind == DEM_CYLINDER_IN) {
        if (!(w.radius > 0.0) || !std::isfinite(w.radius)) { why = "cylinder radius must be > 0"; return false; }
        if (precision == DEM_FP32 && make_wall(w).axis < 0) {
            why = "in DEM_FP32 mode a cylinder axis must be a coordinate axis";
            return false;
        }
    }
    if (w.kind == DEM_HALF_PLATE) {
        const double uu = w.u[0] * w.u[0] + w.u[1] * w.u[1] + w.u[2] * w.u[2];
        const double un = w.u[0] * w.n[0] + w.u[1] * w.n[1] + w.u[2] * w.n[2];
        if (std::fabs(uu - 1.0) > 1e-12 || std::fabs(un) > 1e-12) {
            why = "half-plate u must be a unit vector orthogonal to n";
            return false;
        }
        const WallDev W = make_wall(w);
        if (precision == DEM_FP32 && (W.axis < 0 || W.uaxis < 0)) {
            why = "in DEM_FP32 mode a half-plate's n and u must be coordinate axes";
            return false;
        }
    }
    return true;
}

void fill_scene(dem_handle* h, SceneDev& S, uint32_t p0, uint32_t np, uint32_t c0) {
    const dem_config& c = h->cfg;
    S = SceneDev{};
    S.p0 = p0;
    S.np = np;
    S.c0 = c0;
    S.bshift = h->bshift;
    S.ncell = h->bshift ? (uint32_t)((h->bdims[0] * h->bdims[1] * h->bdims[2]) << (3 * h->bshift))
                        : (uint32_t)(h->dims[0] * h->dims[1] * h->dims[2]);
    for (int a = 0; a < 3; ++a) {
        S.bdims[a] = (int32_t)h->bdims[a];
        S.dims[a] = (int32_t)h->dims[a];
        S.origin[a] = h->origin[a];
        S.origin_f[a] = (float)h->origin[a];
        S.g[a] = c.g[a];
        S.g_f[a] = (float)c.g[a];
    }
    S.h = h->h;
    S.h_f = (float)h->h;
    S.active = 1;
    S.nwalls = (int32_t)h->walls.size();
    S.dt = c.dt; S.kn = c.kn; S.kt = c.kt; S.cn = c.cn; S.ct = c.ct; S.alpha = c.alpha; S.mu = c.mu;
    S.ksp = c.ksp; S.kda = c.kda; S.ksh = c.ksh;
    S.cmass = c.rho * (4.0 / 3.0) * 3.14159265358979323846;
    S.dt_f = (float)c.dt; S.kn_f = (float)c.kn; S.kt_f = (float)c.kt; S.cn_f = (float)c.cn; S.ct_f = (float)c.ct;
    S.alpha_f = (float)c.alpha; S.mu_f = (float)c.mu; S.ksp_f = (float)c.ksp; S.kda_f = (float)c.kda;
    S.ksh_f = (float)c.ksh; S.cmass_f = (float)S.cmass;
    S.terms = c.terms;
    S.mu_roll = c.mu_roll;
    S.mu_roll_f = (float)c.mu_roll;
    S.alpha_t = c.alpha_t;
    S.alpha_t_f = (float)c.alpha_t;
    S.kcoh_pi = c.k_coh * 3.14159265358979323846;
    S.kcoh_pi_f = (float)S.kcoh_pi;
    // FP32 prefilter margin: bounds the FP32 error of |hi_j - hi_i| for coordinates up to X
    double X = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double ext = c.domain_hi[a] - c.domain_lo[a];
        X = std::max(X, std::max(std::fabs(c.domain_lo[a]), std::fabs(c.domain_hi[a])) + ext);
    }
    S.eps_f = (float)(std::ldexp(1.0, -20) * (X + 2.0 * h->rmax));
    if (c.resort_interval != 1) {
        // a particle that moved skin/2 less the FP32 position margin forces a sort
        const double t = std::max(0.5 * c.skin - (double)S.eps_f, 0.0);
        S.skin_f = (float)c.skin;
        S.thresh2_f = (float)(t * t);
    }
    for (size_t k = 0; k < h->walls.size(); ++k) S.walls[k] = make_wall(h->walls[k]);
}

dem_status validate_config(const dem_config* c, std::string& why) {
    if (!c) { why = "cfg is NULL"; return DEM_ERR_INVALID_ARG; }
    if (c->model != DEM_PRACTICAL && c->model != DEM_SIMPLE) { why = "model"; return DEM_ERR_INVALID_ARG; }
    if (c->stiffness != DEM_LINEAR && c->stiffness != DEM_HERTZ) { why = "stiffness"; return DEM_ERR_INVALID_ARG; }
    if (c->precision != DEM_FP64 && c->precision != DEM_FP32) { why = "precision"; return DEM_ERR_INVALID_ARG; }
    if (!(c->dt > 0.0) || !std::isfinite(c->dt)) { why = "dt must be > 0"; return DEM_ERR_INVALID_ARG; }
    if (!(c->rho > 0.0) || !std::isfinite(c->rho)) { why = "rho must be > 0"; return DEM_ERR_INVALID_ARG; }
    if (!finite3(c->g)) { why = "g"; return DEM_ERR_INVALID_ARG; }
    const double nonneg[] = {c->kn, c->kt, c->cn, c->ct, c->alpha, c->mu, c->ksp, c->kda, c->ksh, c->skin, c->cell_size};
    for (double v : nonneg)
        if (!(v >= 0.0) || !std::isfinite(v)) { why = "stiffness, damping, friction, skin and cell_size must be finite and >= 0"; return DEM_ERR_INVALID_ARG; }
    for (int a = 0; a < 3; ++a)
        if (!(c->domain_hi[a] > c->domain_lo[a]) || !std::isfinite(c->domain_lo[a]) || !std::isfinite(c->domain_hi[a])) {
            why = "domain_hi must exceed domain_lo on every axis";
            return DEM_ERR_INVALID_ARG;
        }
    if (c->resort_interval < 0) { why = "resort_interval"; return DEM_ERR_INVALID_ARG; }
    if (c->resort_interval != 1 && !(c->skin > 0.0)) {
        why = "resort_interval != 1 needs a skin > 0";
        return DEM_ERR_INVALID_ARG;
    }
    if (c->block_size != 0 && (c->block_size < 32 || c->block_size > 256 || c->block_size % 32)) {
        why = "block_size must be 0 or a multiple of 32 in [32, 256]";
        return DEM_ERR_INVALID_ARG;
    }
    if (c->max_contacts < 0 || c->max_contacts > 64) { why = "max_contacts must be in [0, 64]"; return DEM_ERR_INVALID_ARG; }
    if (c->terms & ~(DEM_TERM_NO_ATTRACTION | DEM_TERM_ROLLING | DEM_TERM_ETA_T | DEM_TERM_COHESION)) {
        why = "unknown terms";
        return DEM_ERR_INVALID_ARG;
    }
    if (c->terms && c->model != DEM_PRACTICAL) { why = "optional terms need the practical model"; return DEM_ERR_INVALID_ARG; }
    for (double q : {c->mu_roll, c->alpha_t, c->k_coh})
        if (!(q >= 0.0) || !std::isfinite(q)) { why = "mu_roll, alpha_t and k_coh must be finite and >= 0"; return DEM_ERR_INVALID_ARG; }
    return DEM_OK;
}

// (Re)allocate particle and cell buffers for n particles and ncells cells.
// Device buffers of a domain for n particles and ncells cells (reused when large enough).
dem_status alloc_domain(Domain& d, uint32_t n, uint32_t ncells, std::string& err) {
    const uint32_t need = std::max<uint32_t>(n, 1);
    if (need <= d.cap && ncells <= d.cells_cap) return DEM_OK;
    // host-side fault injection for tests: DEM_FAULT=alloc makes every allocation of
    // particle buffers fail as if the device were out of memory
    const char* fault = std::getenv("DEM_FAULT");
    if (fault && std::strstr(fault, "alloc")) {
        err = "injected allocation failure (DEM_FAULT=alloc)";
        return DEM_ERR_OOM;
    }
    free_particle_buffers(d);
    const uint32_t cap = std::max<uint32_t>(need, 64);
    const uint32_t ccap = std::max<uint32_t>(ncells, 1);
    const size_t N = cap;
    const size_t T = d.precision == 0 ? sizeof(double) : sizeof(float);
    cudaError_t e = cudaSuccess;
#define AL(ptr, bytes) do { if ((e = dmalloc(d, &(ptr), (bytes))) != cudaSuccess) { free_particle_buffers(d); cudaGetLastError(); err = std::string("cudaMalloc failed: ") + cudaGetErrorString(e); return DEM_ERR_OOM; } } while (0)
    for (int s = 0; s < 2; ++s) {
        if (d.precision == 0) {
            StateF64& S = d.S64[s];
            AL(S.x, N * 8); AL(S.y, N * 8); AL(S.z, N * 8);
            AL(S.vx, N * 8); AL(S.vy, N * 8); AL(S.vz, N * 8);
            AL(S.wx, N * 8); AL(S.wy, N * 8); AL(S.wz, N * 8);
            AL(S.r, N * 4); AL(S.id, N * 4);
        } else {
            StateF32& S = d.S32[s];
            AL(S.P0, N * 16); AL(S.P1, N * 16); AL(S.V, N * 16); AL(S.W, N * 16); AL(S.id, N * 4);
        }
        AL(d.hcnt[s], N * 4);
        AL(d.hpid[s], N * 4 * (size_t)d.maxc);
        AL(d.hd[s], N * T * 3 * (size_t)d.maxc);
    }
    AL(d.key, N * 4); AL(d.rank, N * 4); AL(d.tmp, N * 4); AL(d.perm, N * 4); AL(d.skey, N * 4);
    if (d.list_mode) {
        AL(d.ncnt, N * 4);
        AL(d.nl, N * 4 * (size_t)DEM_LIST_CAP);
        AL(d.wmask, N * 4);
        AL(d.ref, N * 16);
        AL(d.canon, N * 4);
        AL(d.fin, N * 4);
    }
    AL(d.cnt, ((size_t)ccap + 1) * 4);
    AL(d.cs, ((size_t)ccap + 1) * 4);
    const uint32_t nb = (ccap + 1 + 2047) / 2048;
    AL(d.part, (size_t)nb * 4);
    const uint32_t db = (cap + 255) / 256;
    AL(d.diag_part, (size_t)db * 10 * 8);
#undef AL
    d.cap = cap;
    d.cells_cap = ccap;
    d.part_cap = nb;
    d.diag_part_cap = db;
    e = cudaMemsetAsync(d.cnt, 0, ((size_t)ccap + 1) * 4, d.stream);
    if (e != cudaSuccess) {
        err = std::string("cudaMemsetAsync(cnt): ") + cudaGetErrorString(e);
        return DEM_ERR_CUDA;
    }
    return DEM_OK;
}

dem_status ensure_buffers(dem_handle* h, uint32_t n, uint32_t ncells) {
    std::string err;
    dem_status s = alloc_domain(h->d, n, ncells, err);
    if (s == DEM_ERR_CUDA) h->broken = true;
    if (s != DEM_OK) h->err = err;
    return s;
}

dem_status ensure_stage(dem_handle* h, uint32_t n) {
    if (n <= h->stage_cap && h->stage) return DEM_OK;
    if (h->stage) cudaFree(h->stage);
    if (h->stage_r) cudaFree(h->stage_r);
    h->stage = nullptr;
    h->stage_r = nullptr;
    h->stage_cap = 0;
    const uint32_t cap = std::max<uint32_t>(n, 64);
    if (cudaMalloc(&h->stage, (size_t)cap * 9 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->stage_r, (size_t)cap * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, DEM_ERR_OOM, "cudaMalloc of the staging buffer failed");
    }
    h->stage_cap = cap;
    return DEM_OK;
}

dem_status sync_status(dem_handle* h) {
    Domain& d = h->d;
    CK(h, cudaMemcpyAsync(d.st_host, d.st, sizeof(StatusDev), cudaMemcpyDeviceToHost, d.stream));
    CK(h, cudaStreamSynchronize(d.stream));
    if (d.st_host->code != 0) {
        const int code = d.st_host->code, where = d.st_host->where;
        CK(h, cudaMemsetAsync(d.st, 0, 2 * sizeof(int32_t), d.stream));
        CK(h, cudaStreamSynchronize(d.stream));
        char buf[160];
        if (code == ST_CAPACITY) {
            snprintf(buf, sizeof buf, "particle at sorted position %d has more than max_contacts=%d contacts", where,
                     d.maxc);
            return fail(h, DEM_ERR_CAPACITY, buf);
        }
        if (code == ST_LIST) {
            snprintf(buf, sizeof buf,
                     "neighbour list of the particle at sorted position %d is full (more than %d candidates "
                     "within r_i + r_j + skin); use a smaller skin",
                     where, DEM_LIST_CAP);
            return fail(h, DEM_ERR_CAPACITY, buf);
        }
        snprintf(buf, sizeof buf, "non-finite position or velocity at sorted position %d", where);
        return fail(h, DEM_ERR_NONFINITE, buf);
    }
    return DEM_OK;
}

dem_status read_ctrl(dem_handle* h, CtrlDev& c) {
    Domain& d = h->d;
    CK(h, cudaMemcpyAsync(d.ctrl_host, d.ctrl, sizeof(CtrlDev), cudaMemcpyDeviceToHost, d.stream));
    CK(h, cudaStreamSynchronize(d.stream));
    c = *d.ctrl_host;
    return DEM_OK;
}

// Contact slots of a handle grown to newmaxc: new history buffers, the springs of the
// buffer the next step reads copied in (the partner-id planes keep their places; the
// three component blocks move to the new stride); the other buffer is written by the
// next step. On failure the old buffers stay.
dem_status regrow_slots(dem_handle* h, int newmaxc) {
    Domain& d = h->d;
    const size_t N = d.cap, M = (size_t)d.maxc, M2 = (size_t)newmaxc;
    const size_t T = d.precision == 0 ? sizeof(double) : sizeof(float);
    void* npid[2] = {nullptr, nullptr};
    void* nhd[2] = {nullptr, nullptr};
    bool ok = true;
    for (int s = 0; s < 2 && ok; ++s)
        ok = cudaMalloc(&npid[s], N * 4 * M2) == cudaSuccess && cudaMalloc(&nhd[s], N * T * 3 * M2) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        for (int s = 0; s < 2; ++s) {
            if (npid[s]) cudaFree(npid[s]);
            if (nhd[s]) cudaFree(nhd[s]);
        }
        return fail(h, DEM_ERR_OOM, "cudaMalloc of the grown contact slots failed");
    }
    const int hi = d.h_cur;
    CK(h, cudaMemcpyAsync(npid[hi], d.hpid[hi], N * 4 * M, cudaMemcpyDeviceToDevice, d.stream));
    for (size_t c = 0; c < 3; ++c)
        CK(h, cudaMemcpyAsync((char*)nhd[hi] + c * M2 * N * T, (const char*)d.hd[hi] + c * M * N * T, M * N * T,
                              cudaMemcpyDeviceToDevice, d.stream));
    CK(h, cudaStreamSynchronize(d.stream));
    for (int s = 0; s < 2; ++s) {
        for (void*& p : d.allocations) {
            if (p == (void*)d.hpid[s]) p = npid[s];
            else if (p == d.hd[s]) p = nhd[s];
        }
        cudaFree(d.hpid[s]);
        cudaFree(d.hd[s]);
        d.hpid[s] = (uint32_t*)npid[s];
        d.hd[s] = nhd[s];
    }
    d.maxc = newmaxc;
    return DEM_OK;
}

dem_status rotate_counters(dem_handle* h) {
    Domain& d = h->d;
    CK(h, cudaMemcpyAsync(&d.st->last, &d.st->live, sizeof(CountersDev), cudaMemcpyDeviceToDevice, d.stream));
    CK(h, cudaMemsetAsync(&d.st->live, 0, sizeof(CountersDev), d.stream));
    return DEM_OK;
}

// Cell order of a list-mode grid of dims cells (nc of them): consecutive stored particles
// form compact blocks of space when cells are numbered brick by brick (the grid padded to
// whole bricks). Returns the largest brick shift s <= DEM_LIST_BRICK_SHIFT whose padding
// adds at most 1/8 to the cell count (0 = row-major), the bricks per axis and the padded
// cell count. Measured on the 4,194,304-sphere drum (88 x 254 x 254 cells): 16^3 bricks are
// 3% faster per step than 4^3, with the same bits.
int choose_bricks(const int64_t dims[3], int64_t nc, int64_t bdims[3], int64_t& padded) {
    for (int s = DEM_LIST_BRICK_SHIFT; s >= 1; --s) {
        const int64_t B = (int64_t)1 << s;
        double p = 1.0;
        for (int a = 0; a < 3; ++a) p *= (double)(((dims[a] + B - 1) / B) * B);
        if (p > 1.125 * (double)nc || p > 2147483647.0) continue;
        padded = 1;
        for (int a = 0; a < 3; ++a) {
            bdims[a] = (dims[a] + B - 1) / B;
            padded *= bdims[a] * B;
        }
        return s;
    }
    bdims[0] = bdims[1] = bdims[2] = 1;
    padded = nc;
    return 0;
}

// Grid of Sec. 4.1 over the configured domain: cell edge >= one diameter of the largest
// sphere (+ a 2^-10 margin, + skin), or the configured cell size.
dem_status set_grid(dem_handle* h, bool any, double rmax, int64_t& nc) {
    const dem_config& c = h->cfg;
    const double hmin = 2.0 * rmax * (1.0 + std::ldexp(1.0, -10)) + c.skin;
    double hc = c.cell_size > 0.0 ? c.cell_size : hmin;
    if (any && hc < hmin * (1.0 - 1e-12))
        return fail(h, DEM_ERR_INVALID_ARG, "cell_size is smaller than 2 r_max (1 + 2^-10) + skin");
    if (!any && !(hc > 0.0)) hc = 1.0;
    nc = 1;
    for (int a = 0; a < 3; ++a) {
        h->origin[a] = c.domain_lo[a];
        h->dims[a] = std::max<int64_t>(1, (int64_t)std::ceil((c.domain_hi[a] - c.domain_lo[a]) / hc));
        if (h->dims[a] > (int64_t)0x7FFFFFFF) return fail(h, DEM_ERR_INVALID_ARG, "grid has more than 2^31 cells");
        nc *= h->dims[a];
        if (nc > (int64_t)0x7FFFFFFF) return fail(h, DEM_ERR_INVALID_ARG, "grid has more than 2^31 cells");
    }
    // list mode numbers cells brick by brick
    h->bshift = 0;
    h->bdims[0] = h->bdims[1] = h->bdims[2] = 1;
    if (h->d.list_mode) {
        h->bshift = choose_bricks(h->dims, nc, h->bdims, nc);
        if (nc > (int64_t)0x7FFFFFFF) return fail(h, DEM_ERR_INVALID_ARG, "grid has more than 2^31 cells");
    }
    h->h = hc;
    h->rmax = rmax;
    return DEM_OK;
}

// Upload (or take from the device) particle arrays, build the grid and do the first sort.
dem_status load_particles(dem_handle* h, int64_t n64, const double* x, const double* v, const double* w,
                          const float* r, int where) {
    Domain& d = h->d;
    if (n64 < 0 || n64 > (int64_t)0x7FFFFF00) return fail(h, DEM_ERR_INVALID_ARG, "n out of range");
    const uint32_t n = (uint32_t)n64;
    if (where != DEM_HOST && where != DEM_DEVICE) return fail(h, DEM_ERR_INVALID_ARG, "where");
    h->graph.reset();
    if (n > 0 && (!x || !v || !w || !r)) return fail(h, DEM_ERR_INVALID_ARG, "x, v, w and r are required");
    // host input goes to the staging buffers first; the arrays are checked (radii finite
    // and > 0, finite x, v, w) and r_max is found on the device, before anything of the
    // handle's state changes
    const double *xd = x, *vd = v, *wd = w;
    const float* rd = r;
    double rmax = 0.0;
    dem_status s;
    if (n > 0) {
        if (where == DEM_HOST) {
            s = ensure_stage(h, n);
            if (s != DEM_OK) return s;
            CK(h, cudaMemcpyAsync(h->stage, x, (size_t)n * 24, cudaMemcpyHostToDevice, d.stream));
            CK(h, cudaMemcpyAsync(h->stage + 3 * (size_t)n, v, (size_t)n * 24, cudaMemcpyHostToDevice, d.stream));
            CK(h, cudaMemcpyAsync(h->stage + 6 * (size_t)n, w, (size_t)n * 24, cudaMemcpyHostToDevice, d.stream));
            CK(h, cudaMemcpyAsync(h->stage_r, r, (size_t)n * 4, cudaMemcpyHostToDevice, d.stream));
            xd = h->stage; vd = h->stage + 3 * (size_t)n; wd = h->stage + 6 * (size_t)n; rd = h->stage_r;
        }
        CK(h, run_check_input(d, n, xd, vd, wd, rd, h->chk_dev));
        CK(h, cudaMemcpyAsync(h->chk_host, h->chk_dev, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, d.stream));
        CK(h, cudaStreamSynchronize(d.stream));
        if (h->chk_host[0] & 1u) return fail(h, DEM_ERR_INVALID_ARG, "radii must be finite and > 0");
        if (h->chk_host[0] & 2u) return fail(h, DEM_ERR_INVALID_ARG, "non-finite position, velocity or spin in the input");
        float rm;
        std::memcpy(&rm, &h->chk_host[1], sizeof rm);
        rmax = (double)rm;
    }
    const dem_config& c = h->cfg;
    int64_t nc = 1;
    s = set_grid(h, n > 0, rmax, nc);
    if (s != DEM_OK) return s;
    d.n = n;
    d.ncells = (uint32_t)nc;
    s = ensure_buffers(h, n, (uint32_t)nc);
    if (s != DEM_OK) return s;
    // scene table (one scene)
    d.nscenes = 1;
    d.h_scenes.assign(1, SceneDev{});
    fill_scene(h, d.h_scenes[0], 0, n, 0);
    if (!d.d_scenes) {
        if (cudaMalloc(&d.d_scenes, sizeof(SceneDev)) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, DEM_ERR_OOM, "cudaMalloc(scene table) failed");
        }
        d.scenes_cap = 1;
    }
    CK(h, cudaMemcpyAsync(d.d_scenes, d.h_scenes.data(), sizeof(SceneDev), cudaMemcpyHostToDevice, d.stream));
    CK(h, cudaMemsetAsync(d.st, 0, sizeof(StatusDev), d.stream));
    CK(h, cudaMemsetAsync(d.cnt, 0, ((size_t)d.ncells + 1) * 4, d.stream));
    // step control: current set 0, the first step after the import sorts
    *d.ctrl_host = CtrlDev{};
    d.ctrl_host->rebuild = 1;
    CK(h, cudaMemcpyAsync(d.ctrl, d.ctrl_host, sizeof(CtrlDev), cudaMemcpyHostToDevice, d.stream));
    d.h_cur = 0;
    if (n > 0) {
        CK(h, cudaMemsetAsync(d.hcnt[0], 0, (size_t)n * 4, d.stream));
        CK(h, cudaMemsetAsync(d.hcnt[1], 0, (size_t)n * 4, d.stream));
        CK(h, run_import(d, xd, vd, wd, rd));
        CK(h, run_hash(d));
        CK(h, run_rebuild(d));
        CK(h, run_end_step(d));
    }
    h->has_particles = true;
    h->eval_valid = false;
    h->steps = 0;
    return DEM_OK;
}


// One timestep enqueued on d.stream: force pass, then (when this step sorts) hash, scan,
// scatter, gather, lists, then the bookkeeping kernel.
cudaError_t enqueue_step(Domain& d) {
    cudaError_t e;
    if ((e = run_force(d, false, nullptr, nullptr)) != cudaSuccess) return e;
    d.h_cur = 1 - d.h_cur;
    if (d.list_mode && (e = run_hash(d)) != cudaSuccess) return e;
    if ((e = run_rebuild(d)) != cudaSuccess) return e;
    return run_end_step(d);
}

// One step for a graph in list mode: force pass, the kernel that sets the condition, a
// conditional node whose body (captured on the side stream) is the sort and the new
// lists, then the bookkeeping. A step that does not sort launches three kernels.
// The part of a list-mode step after the force pass, while d.stream is capturing: the
// condition kernel, the conditional sort node (body captured on g->side), bookkeeping.
cudaError_t capture_sort_tail(Domain& d, StepGraph* g, int64_t& body) {
    cudaError_t e;
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if ((e = cudaStreamGetCaptureInfo(d.stream, &cs, nullptr, &graph, &deps, nullptr, &ndeps)) != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphConditionalHandle hc;
    if ((e = cudaGraphConditionalHandleCreate(&hc, graph, 0, 0)) != cudaSuccess) return e;
    if ((e = run_sort_cond(d, hc)) != cudaSuccess) return e;
    if ((e = cudaStreamGetCaptureInfo(d.stream, &cs, nullptr, &graph, &deps, nullptr, &ndeps)) != cudaSuccess) return e;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hc;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &p)) != cudaSuccess) return e;
    if ((e = cudaStreamUpdateCaptureDependencies(d.stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return e;
    cudaGraph_t bg = p.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(g->side, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return e;
    const cudaStream_t main = d.stream;
    const int64_t l0 = d.launches;
    d.stream = g->side;
    cudaError_t e1 = run_hash(d);
    if (e1 == cudaSuccess) e1 = run_rebuild(d);
    d.stream = main;
    body = d.launches - l0;
    d.launches = l0;
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(g->side, &out);
    if (e1 != cudaSuccess) return e1;
    if (e != cudaSuccess) return e;
    return run_end_step(d);
}

cudaError_t capture_step_cond(Domain& d, StepGraph* g, int64_t& body) {
    cudaError_t e;
    if ((e = run_force(d, false, nullptr, nullptr)) != cudaSuccess) return e;
    d.h_cur = 1 - d.h_cur;
    return capture_sort_tail(d, g, body);
}

// Phase timing in list mode: the sort tail of a step as its own graph, one per history
// parity (the tail reads the contact counts of the buffer the force pass just wrote).
cudaError_t capture_sort_graphs(Domain& d, StepGraph* g) {
    cudaError_t e;
    if (!g->side && (e = cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking)) != cudaSuccess) {
        g->side = nullptr;
        return e;
    }
    const int64_t l0 = d.launches;
    const int hc0 = d.h_cur;
    for (int par = 0; par < 2; ++par) {
        d.h_cur = par;
        if ((e = cudaStreamBeginCapture(d.stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
        int64_t b = 0;
        cudaError_t e1 = capture_sort_tail(d, g, b);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(d.stream, &graph);
        if (e1 == cudaSuccess && e == cudaSuccess) e = cudaGraphInstantiate(&g->sort_exec[par], graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e1 != cudaSuccess) e = e1;
        if (e != cudaSuccess) break;
        g->body_launches = b;
        g->sort_launches = d.launches - l0;
        d.launches = l0;
    }
    d.h_cur = hc0;
    d.launches = l0;
    if (e != cudaSuccess) {
        for (int par = 0; par < 2; ++par)
            if (g->sort_exec[par]) cudaGraphExecDestroy(g->sort_exec[par]);
        g->sort_exec[0] = g->sort_exec[1] = nullptr;
    }
    return e;
}

// Two timesteps captured once as a CUDA graph (two, so that the history buffers return
// to their starting roles) and replayed; plain launches on the legacy default stream.
// In list mode the sort of each step is a conditional node (see capture_step_cond); if
// the driver refuses conditional nodes the plain two-step graph is used.
cudaError_t capture_cond_graph(Domain& d, StepGraph* g) {
    cudaError_t e;
    if (!g->side && (e = cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking)) != cudaSuccess) {
        g->side = nullptr;
        return e;
    }
    const int64_t l0 = d.launches;
    const int hc0 = d.h_cur;
    if ((e = cudaStreamBeginCapture(d.stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    int64_t b1 = 0, b2 = 0;
    cudaError_t e1 = capture_step_cond(d, g, b1);
    cudaError_t e2 = e1 == cudaSuccess ? capture_step_cond(d, g, b2) : e1;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(d.stream, &graph);
    if (e1 == cudaSuccess && e2 == cudaSuccess && e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    const cudaError_t bad = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e);
    if (bad != cudaSuccess) {
        g->exec = nullptr;
        d.launches = l0;
        d.h_cur = hc0;
        return bad;
    }
    g->launches = d.launches - l0;
    g->body_launches = b1;
    d.launches = l0;
    return cudaSuccess;
}

cudaError_t run_steps(Domain& d, StepGraph* g, int64_t nsteps) {
    cudaError_t e;
    if (!g || !d.stream || d.n == 0) {
        for (int64_t k = 0; k < nsteps; ++k)
            if ((e = enqueue_step(d)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    if (d.h_cur == 1 && nsteps > 0) {
        if ((e = enqueue_step(d)) != cudaSuccess) return e;
        --nsteps;
    }
    if (nsteps >= 2 && !g->exec && d.list_mode) {
        const cudaError_t ce = capture_cond_graph(d, g);
        if (ce != cudaSuccess) {
            cudaGetLastError();   // conditional nodes unavailable: fall back to the plain graph
            g->reset();
            static bool said = false;
            if (!said) {
                said = true;
                fprintf(stderr, "dem: step graph with a conditional sort node unavailable (%s); using the plain graph\n",
                        cudaGetErrorString(ce));
            }
        }
    }
    if (nsteps >= 2 && !g->exec) {
        const int64_t l0 = d.launches;
        if ((e = cudaStreamBeginCapture(d.stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
        cudaError_t e1 = enqueue_step(d);
        cudaError_t e2 = e1 == cudaSuccess ? enqueue_step(d) : e1;
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(d.stream, &graph);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e);
        }
        g->launches = d.launches - l0;
        d.launches = l0;
        e = cudaGraphInstantiate(&g->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g->exec = nullptr;
            return e;
        }
    }
    for (; nsteps >= 2; nsteps -= 2) {
        if ((e = cudaGraphLaunch(g->exec, d.stream)) != cudaSuccess) return e;
        d.launches += g->launches;
    }
    if (nsteps == 1 && (e = enqueue_step(d)) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace

// =========================================================================== C ABI
extern "C" {

dem_status dem_create(const dem_config* cfg, int device, void* cuda_stream, dem_handle** out) {
    if (!out) return DEM_ERR_INVALID_ARG;
    *out = nullptr;
    std::string why;
    dem_status s = validate_config(cfg, why);
    if (s != DEM_OK) return s;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DEM_ERR_INVALID_ARG;
    }
    DeviceGuard g(device);
    dem_handle* h = new dem_handle();
    h->cfg = *cfg;
    h->device = device;
    Domain& d = h->d;
    d.precision = cfg->precision;
    d.model = cfg->model;
    d.terms = cfg->terms;
    d.stiffness = cfg->stiffness;
    d.maxc = cfg->max_contacts > 0 ? cfg->max_contacts : 32;
    d.block = cfg->block_size > 0 ? cfg->block_size : 256;
    d.sort_blocks = sort_blocks_of(device);
    d.list_mode = cfg->resort_interval != 1 ? 1 : 0;
    d.regrow = 1;   // a contact-slot overflow voids the step; dem_step grows the slots and reruns it
    d.interval = cfg->resort_interval;
    d.maxn = DEM_LIST_CAP;
    d.stream = (cudaStream_t)cuda_stream;
    if (cudaMalloc(&d.st, sizeof(StatusDev)) != cudaSuccess ||
        cudaMallocHost(&d.st_host, sizeof(StatusDev)) != cudaSuccess ||
        cudaMalloc(&d.ctrl, sizeof(CtrlDev)) != cudaSuccess ||
        cudaMallocHost(&d.ctrl_host, sizeof(CtrlDev)) != cudaSuccess ||
        cudaMemset(d.ctrl, 0, sizeof(CtrlDev)) != cudaSuccess ||
        cudaMalloc(&d.diag_out, 16 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->chk_dev, 2 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&h->chk_host, 4 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(d.st, 0, sizeof(StatusDev)) != cudaSuccess) {
        cudaGetLastError();
        dem_destroy(h);
        return DEM_ERR_OOM;
    }
    *out = h;
    return DEM_OK;
}

dem_status dem_set_particles(dem_handle* h, int64_t n, const uint32_t* id, const double* x, const double* v,
                             const double* w, const float* r, int where) {
    if (!h) return DEM_ERR_INVALID_ARG;
    if (h->broken) return fail(h, DEM_ERR_STATE, "handle is unusable after a CUDA error");
    if (id) return fail(h, DEM_ERR_INVALID_ARG, "id must be NULL (particle k has id k)");
    DeviceGuard g(h->device);
    dem_status s = load_particles(h, n, x, v, w, r, where);
    if (s != DEM_OK) { h->has_particles = false; return s; }
    CK(h, cudaStreamSynchronize(h->d.stream));
    h->err.clear();
    return DEM_OK;
}

dem_status dem_set_walls(dem_handle* h, int nwalls, const dem_wall* walls) {
    if (!h) return DEM_ERR_INVALID_ARG;
    if (h->broken) return fail(h, DEM_ERR_STATE, "handle is unusable after a CUDA error");
    if (nwalls < 0 || nwalls > DEM_MAX_WALLS || (nwalls > 0 && !walls))
        return fail(h, DEM_ERR_INVALID_ARG, "nwalls must be in [0, 8]");
    for (int k = 0; k < nwalls; ++k) {
        std::string why;
        if (!check_wall(walls[k], h->cfg.precision, why)) return fail(h, DEM_ERR_INVALID_ARG, why.c_str());
    }
    DeviceGuard g(h->device);
    h->walls.assign(walls, walls + nwalls);
    if (h->has_particles && !h->d.h_scenes.empty()) {
        Domain& d = h->d;
        for (auto& S : d.h_scenes) {
            S.nwalls = nwalls;
            for (int k = 0; k < nwalls; ++k) S.walls[k] = make_wall(h->walls[k]);
        }
        CK(h, cudaMemcpyAsync(d.d_scenes, d.h_scenes.data(), sizeof(SceneDev) * d.h_scenes.size(),
                              cudaMemcpyHostToDevice, d.stream));
        // list mode: which walls each particle can reach is known from the last sort;
        // recompute it for the new walls before the next step
        if (d.list_mode) CK(h, run_wall_masks(d));
        CK(h, cudaStreamSynchronize(d.stream));
    }
    return DEM_OK;
}

dem_status dem_step(dem_handle* h, int64_t nsteps) {
    if (!h) return DEM_ERR_INVALID_ARG;
    if (h->broken) return fail(h, DEM_ERR_STATE, "handle is unusable after a CUDA error");
    if (!h->has_particles) return fail(h, DEM_ERR_STATE, "dem_step before dem_set_particles");
    if (nsteps < 0) return fail(h, DEM_ERR_INVALID_ARG, "nsteps < 0");
    DeviceGuard g(h->device);
    Domain& d = h->d;
    const bool timed = h->timing && d.n > 0;
    int64_t left = nsteps;
    for (;;) {
        if (timed) {
            const size_t need = 3 * (size_t)left;
            while (h->events.size() < need) {
                cudaEvent_t e;
                CK(h, cudaEventCreate(&e));
                h->events.push_back(e);
            }
        }
        // the device's count of completed steps as this attempt begins (read back with the
        // status, so that a void step can be located without another synchronisation)
        const int hc0 = d.h_cur;
        CK(h, cudaMemcpyAsync(&h->chk_host[2], &d.ctrl->steps_done, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                              d.stream));
        if (timed) {
            // list mode on a capturable stream: the sort tail runs as a small graph whose sort
            // node executes only when the device decided to sort
            if (d.list_mode && d.stream && !h->graph.sort_exec[0] && capture_sort_graphs(d, &h->graph) != cudaSuccess)
                cudaGetLastError();
            for (int64_t s = 0; s < left; ++s) {
                CK(h, cudaEventRecord(h->events[3 * s], d.stream));
                CK(h, run_force(d, false, nullptr, nullptr));
                CK(h, cudaEventRecord(h->events[3 * s + 1], d.stream));
                d.h_cur = 1 - d.h_cur;
                if (h->graph.sort_exec[d.h_cur]) {
                    CK(h, cudaGraphLaunch(h->graph.sort_exec[d.h_cur], d.stream));
                    d.launches += h->graph.sort_launches;
                } else {
                    if (d.list_mode) CK(h, run_hash(d));   // (sort steps only; fused into the force pass otherwise)
                    CK(h, run_rebuild(d));
                    CK(h, run_end_step(d));
                }
                CK(h, cudaEventRecord(h->events[3 * s + 2], d.stream));
            }
        } else {
            CK(h, run_steps(d, &h->graph, left));
        }
        dem_status st = sync_status(h);
        // a particle with more contacts than slots voided its step (and the later ones of
        // this attempt did nothing): the state is the one at the start of that step
        int64_t done = left;
        bool void_step = false;
        if (st == DEM_ERR_CAPACITY && d.st_host->code == ST_CAPACITY && d.regrow) {
            CtrlDev c;
            dem_status s2 = read_ctrl(h, c);
            if (s2 != DEM_OK) return s2;
            if (c.rebuild & DEM_HALT) {
                void_step = true;
                done = (int64_t)(uint32_t)(c.steps_done - h->chk_host[2]);
            }
        }
        h->steps += done;
        if (done > 0) h->eval_valid = false;
        if (timed) {
            for (int64_t s = 0; s < done; ++s) {
                float a = 0.f, b = 0.f;
                CK(h, cudaEventElapsedTime(&a, h->events[3 * s], h->events[3 * s + 1]));
                CK(h, cudaEventElapsedTime(&b, h->events[3 * s + 1], h->events[3 * s + 2]));
                h->t_force_ms += a;
                h->t_sort_ms += b;
            }
            h->n_force += done;
            h->n_sort += done;
        }
        if (!void_step) return st;
        // resume at the void step: its history buffers (the parity of the steps done), the
        // step control as at its start, no counters, no cell counts of its new keys
        d.h_cur = hc0 ^ (int)(done & 1);
        CtrlDev c;
        CK(h, cudaMemcpyAsync(&c, d.ctrl, sizeof c, cudaMemcpyDeviceToHost, d.stream));
        CK(h, cudaStreamSynchronize(d.stream));
        c.rebuild = d.list_mode ? 0 : 1;
        *d.ctrl_host = c;
        CK(h, cudaMemcpyAsync(d.ctrl, d.ctrl_host, sizeof(CtrlDev), cudaMemcpyHostToDevice, d.stream));
        CK(h, cudaMemsetAsync(&d.st->live, 0, sizeof(CountersDev), d.stream));
        CK(h, cudaMemsetAsync(d.cnt, 0, ((size_t)d.ncells + 1) * 4, d.stream));
        CK(h, cudaStreamSynchronize(d.stream));
        h->graph.reset();
        if (d.maxc >= 64) {
            char buf[200];
            snprintf(buf, sizeof buf,
                     "particle at sorted position %d has more than 64 contacts (the largest capacity); the state is "
                     "the one before the step that overflowed",
                     d.st_host->where);
            return fail(h, DEM_ERR_CAPACITY, buf);
        }
        const dem_status sg = regrow_slots(h, std::min(64, 2 * d.maxc));
        if (sg != DEM_OK) return sg;
        h->err.clear();
        left -= done;
    }
}

dem_status dem_run_until(dem_handle* h, int64_t max_steps, double disp_threshold, int64_t check_every,
                         int64_t* steps_done, double* last_max_disp, int* settled) {
    if (!h) return DEM_ERR_INVALID_ARG;
    if (max_steps < 0 || check_every < 1 || !(disp_threshold >= 0.0))
        return fail(h, DEM_ERR_INVALID_ARG, "max_steps >= 0, check_every >= 1 and disp_threshold >= 0 are required");
    int64_t done = 0;
    double disp = 0.0;
    int ok = 0;
    while (done < max_steps) {
        const int64_t k = std::min(check_every, max_steps - done);
        const int64_t s0 = h->steps;
        const dem_status st = dem_step(h, k);
        if (st != DEM_OK) {
            // the steps dem_step took (fewer than k when a step was voided by a capacity
            // overflow it could not grow past)
            if (steps_done) *steps_done = done + (h->steps - s0);
            return st;
        }
        done += k;
        uint32_t bits = h->d.st_host->last.max_disp2_bits;
        float d2;
        std::memcpy(&d2, &bits, sizeof d2);
        disp = std::sqrt((double)d2);
        if (disp < disp_threshold) {
            ok = 1;
            break;
        }
    }
    if (steps_done) *steps_done = done;
    if (last_max_disp) *last_max_disp = disp;
    if (settled) *settled = ok;
    return DEM_OK;
}

dem_status dem_set_timing(dem_handle* h, int enable) {
    if (!h) return DEM_ERR_INVALID_ARG;
    h->timing = enable != 0;
    if (h->timing) {
        h->t_force_ms = h->t_sort_ms = 0.0;
        h->n_force = h->n_sort = 0;
    }
    return DEM_OK;
}

dem_status dem_get_phase_times(const dem_handle* h, double* out) {
    if (!h || !out) return DEM_ERR_INVALID_ARG;
    out[0] = h->t_force_ms;
    out[1] = h->t_sort_ms;
    out[2] = (double)h->n_force;
    out[3] = (double)h->n_sort;
    return DEM_OK;
}

dem_status dem_get_state(dem_handle* h, double* x, double* v, double* w, int where) {
    if (!h) return DEM_ERR_INVALID_ARG;
    if (h->broken) return fail(h, DEM_ERR_STATE, "handle is unusable after a CUDA error");
    if (!h->has_particles) return fail(h, DEM_ERR_STATE, "no particles");
    if (where != DEM_HOST && where != DEM_DEVICE) return fail(h, DEM_ERR_INVALID_ARG, "where");
    DeviceGuard g(h->device);
    Domain& d = h->d;
    const size_t n = d.n;
    if (n == 0) return DEM_OK;
    if (where == DEM_DEVICE) {
        CK(h, run_export(d, x, v, w));
    } else {
        dem_status s = ensure_stage(h, d.n);
        if (s != DEM_OK) return s;
        CK(h, run_export(d, x ? h->stage : nullptr, v ? h->stage + 3 * n : nullptr, w ? h->stage + 6 * n : nullptr));
        if (x) CK(h, cudaMemcpyAsync(x, h->stage, n * 24, cudaMemcpyDeviceToHost, d.stream));
        if (v) CK(h, cudaMemcpyAsync(v, h->stage + 3 * n, n * 24, cudaMemcpyDeviceToHost, d.stream));
        if (w) CK(h, cudaMemcpyAsync(w, h->stage + 6 * n, n * 24, cudaMemcpyDeviceToHost, d.stream));
    }
    CK(h, cudaStreamSynchronize(d.stream));
    return DEM_OK;
}

dem_status dem_get_forces(dem_handle* h, double* F, double* T, int where) {
    if (!h) return DEM_ERR_INVALID_ARG;
    if (h->broken) return fail(h, DEM_ERR_STATE, "handle is unusable after a CUDA error");
    if (!h->has_particles) return fail(h, DEM_ERR_STATE, "no particles");
    if (where != DEM_HOST && where != DEM_DEVICE) return fail(h, DEM_ERR_INVALID_ARG, "where");
    DeviceGuard g(h->device);
    Domain& d = h->d;
    const size_t n = d.n;
    if (n == 0) return DEM_OK;
    double *Fd = F, *Td = T;
    if (where == DEM_HOST) {
        dem_status s = ensure_stage(h, d.n);
        if (s != DEM_OK) return s;
        Fd = h->stage;
        Td = h->stage + 3 * n;
    }
    CK(h, cudaMemsetAsync(&d.st->live, 0, sizeof(CountersDev), d.stream));
    CK(h, run_force(d, true, Fd, Td));
    dem_status s = rotate_counters(h);
    if (s != DEM_OK) return s;
    if (where == DEM_HOST) {
        if (F) CK(h, cudaMemcpyAsync(F, Fd, n * 24, cudaMemcpyDeviceToHost, d.stream));
        if (T) CK(h, cudaMemcpyAsync(T, Td, n * 24, cudaMemcpyDeviceToHost, d.stream));
    }
    h->eval_valid = true;
    return sync_status(h);
}

// Used spring slots of a particle from its count word.
static uint32_t slots_of(const Domain& d, uint32_t raw) { return std::min<uint32_t>(raw, (uint32_t)d.maxc); }

static dem_status download_u32(dem_handle* h, std::vector<uint32_t>& out, const uint32_t* src, size_t count) {
    out.resize(count);
    if (count) CK(h, cudaMemcpyAsync(out.data(), src, count * 4, cudaMemcpyDeviceToHost, h->d.stream));
    return DEM_OK;
}

dem_status dem_get_history(dem_handle* h, int64_t cap, uint32_t* oi, uint32_t* oj, double* od, int64_t* nout) {
    if (!h || !nout || cap < 0) return DEM_ERR_INVALID_ARG;
    if (h->broken) return fail(h, DEM_ERR_STATE, "handle is unusable after a CUDA error");
    if (!h->has_particles) return fail(h, DEM_ERR_STATE, "no particles");
    DeviceGuard g(h->device);
    Domain& d = h->d;
    const size_t n = d.n, N = d.cap, M = d.maxc;
    *nout = 0;
    if (n == 0 || d.model != 0) return DEM_OK;
    std::vector<uint32_t> perm, ids, cnt;
    dem_status s;
    CtrlDev ctl;
    if ((s = read_ctrl(h, ctl)) != DEM_OK) return s;
    if ((s = download_u32(h, perm, d.perm, n)) != DEM_OK) return s;
    if ((s = download_u32(h, ids, d.precision == 0 ? d.S64[ctl.cur].id : d.S32[ctl.cur].id, n)) != DEM_OK) return s;
    if ((s = download_u32(h, cnt, d.hcnt[d.h_cur], N)) != DEM_OK) return s;
    CK(h, cudaStreamSynchronize(d.stream));
    if (!ctl.perm_valid)
        for (size_t q = 0; q < n; ++q) perm[q] = (uint32_t)q;
    uint32_t mx = 0;
    for (size_t q = 0; q < n; ++q) mx = std::max(mx, slots_of(d, cnt[perm[q]]));
    std::vector<uint32_t> pid((size_t)mx * N);
    std::vector<double> dv((size_t)3 * mx * N);
    if (mx) {
        CK(h, cudaMemcpyAsync(pid.data(), d.hpid[d.h_cur], (size_t)mx * N * 4, cudaMemcpyDeviceToHost, d.stream));
        for (int c = 0; c < 3; ++c) {
            if (d.precision == 0) {
                CK(h, cudaMemcpyAsync(dv.data() + (size_t)c * mx * N, (const double*)d.hd[d.h_cur] + (size_t)c * M * N,
                                      (size_t)mx * N * 8, cudaMemcpyDeviceToHost, d.stream));
            } else {
                std::vector<float> tmp((size_t)mx * N);
                CK(h, cudaMemcpyAsync(tmp.data(), (const float*)d.hd[d.h_cur] + (size_t)c * M * N, (size_t)mx * N * 4,
                                      cudaMemcpyDeviceToHost, d.stream));
                CK(h, cudaStreamSynchronize(d.stream));
                for (size_t k = 0; k < tmp.size(); ++k) dv[(size_t)c * mx * N + k] = tmp[k];
            }
        }
        CK(h, cudaStreamSynchronize(d.stream));
    }
    struct Rec { uint32_t i, j; double d[3]; };
    std::vector<Rec> recs;
    for (size_t q = 0; q < n; ++q) {
        const uint32_t src = perm[q], owner = ids[q];
        const uint32_t c = slots_of(d, cnt[src]);
        for (uint32_t k = 0; k < c; ++k) {
            const uint32_t p = pid[(size_t)k * N + src];
            if (p >= DEM_WALL_BASE || owner < p) {
                Rec r{owner, p, {dv[(size_t)0 * mx * N + (size_t)k * N + src], dv[(size_t)1 * mx * N + (size_t)k * N + src],
                                 dv[(size_t)2 * mx * N + (size_t)k * N + src]}};
                recs.push_back(r);
            }
        }
    }
    std::sort(recs.begin(), recs.end(), [](const Rec& a, const Rec& b) { return a.i != b.i ? a.i < b.i : a.j < b.j; });
    *nout = (int64_t)recs.size();
    for (size_t k = 0; k < recs.size() && (int64_t)k < cap; ++k) {
        if (oi) oi[k] = recs[k].i;
        if (oj) oj[k] = recs[k].j;
        if (od) { od[3 * k] = recs[k].d[0]; od[3 * k + 1] = recs[k].d[1]; od[3 * k + 2] = recs[k].d[2]; }
    }
    return DEM_OK;
}

dem_status dem_restore(dem_handle* h, int64_t n, const double* x, const double* v, const double* w, const float* r,
                       int64_t nrec, const uint32_t* ri, const uint32_t* rj, const double* rd) {
    if (!h || nrec < 0 || (nrec > 0 && (!ri || !rj || !rd))) return DEM_ERR_INVALID_ARG;
    if (h->broken) return fail(h, DEM_ERR_STATE, "handle is unusable after a CUDA error");
    DeviceGuard g(h->device);
    dem_status s = load_particles(h, n, x, v, w, r, DEM_HOST);
    if (s != DEM_OK) { h->has_particles = false; return s; }
    Domain& d = h->d;
    if (nrec == 0 || d.model != 0) {
        CK(h, cudaStreamSynchronize(d.stream));
        return DEM_OK;
    }
    // per-particle lists in id order; after the first sort perm[q] is the id position
    const size_t N = d.cap, M = d.maxc;
    std::vector<uint32_t> cnt(N, 0), pid(M * N, 0);
    std::vector<double> dv(3 * M * N, 0.0);
    auto add = [&](uint32_t owner, uint32_t partner, double a, double b, double c) -> bool {
        if (owner >= (uint32_t)n) return false;
        const uint32_t k = cnt[owner];
        if (k >= M) return false;
        pid[(size_t)k * N + owner] = partner;
        dv[(0 * M + k) * N + owner] = a;
        dv[(1 * M + k) * N + owner] = b;
        dv[(2 * M + k) * N + owner] = c;
        cnt[owner] = k + 1;
        return true;
    };
    const int nw = (int)h->walls.size();
    for (int64_t k = 0; k < nrec; ++k) {
        const uint32_t i = ri[k], j = rj[k];
        const double* dd = rd + 3 * k;
        bool ok;
        if (j >= DEM_WALL_BASE) ok = (int)(j - DEM_WALL_BASE) < nw && add(i, j, dd[0], dd[1], dd[2]);
        else ok = i < j && j < (uint32_t)n && add(i, j, dd[0], dd[1], dd[2]) && add(j, i, -dd[0], -dd[1], -dd[2]);
        if (!ok) { h->has_particles = false; return fail(h, DEM_ERR_INVALID_ARG, "invalid or excess history record"); }
    }
    CK(h, cudaMemcpyAsync(d.hcnt[d.h_cur], cnt.data(), N * 4, cudaMemcpyHostToDevice, d.stream));
    CK(h, cudaMemcpyAsync(d.hpid[d.h_cur], pid.data(), M * N * 4, cudaMemcpyHostToDevice, d.stream));
    if (d.precision == 0) {
        CK(h, cudaMemcpyAsync(d.hd[d.h_cur], dv.data(), 3 * M * N * 8, cudaMemcpyHostToDevice, d.stream));
        CK(h, cudaStreamSynchronize(d.stream));
    } else {
        std::vector<float> f(dv.size());
        for (size_t k = 0; k < dv.size(); ++k) f[k] = (float)dv[k];
        CK(h, cudaMemcpyAsync(d.hd[d.h_cur], f.data(), f.size() * 4, cudaMemcpyHostToDevice, d.stream));
        CK(h, cudaStreamSynchronize(d.stream));
    }
    return DEM_OK;
}

dem_status dem_get_diagnostics(dem_handle* h, double* out) {
    if (!h || !out) return DEM_ERR_INVALID_ARG;
    if (h->broken) return fail(h, DEM_ERR_STATE, "handle is unusable after a CUDA error");
    if (!h->has_particles) return fail(h, DEM_ERR_STATE, "no particles");
    DeviceGuard g(h->device);
    Domain& d = h->d;
    CK(h, run_diag(d));
    double tmp[10];
    CK(h, cudaMemcpyAsync(tmp, d.diag_out, 10 * sizeof(double), cudaMemcpyDeviceToHost, d.stream));
    CK(h, cudaMemcpyAsync(d.st_host, d.st, sizeof(StatusDev), cudaMemcpyDeviceToHost, d.stream));
    CK(h, cudaMemcpyAsync(d.ctrl_host, d.ctrl, sizeof(CtrlDev), cudaMemcpyDeviceToHost, d.stream));
    CK(h, cudaStreamSynchronize(d.stream));
    for (int k = 0; k < 10; ++k) out[k] = tmp[k];
    const CountersDev& c = d.st_host->last;
    float mo;
    std::memcpy(&mo, &c.max_overlap_bits, 4);
    out[10] = (double)c.ncontacts / 2.0;
    out[11] = (double)c.nwallc;
    out[12] = (double)mo;
    out[13] = (double)h->steps;
    out[14] = (double)d.ctrl_host->nsorts;
    out[15] = (double)c.clamped;
    return DEM_OK;
}

// Row-major key ((k ny + j) nx + i) of a cell key of the handle's sort order.
static uint32_t row_major_key(const dem_handle* h, uint32_t key) {
    if (h->bshift == 0) return key;
    const uint32_t sh = (uint32_t)h->bshift, m = (1u << sh) - 1u;
    const uint32_t brick = key >> (3 * sh), in = key & ((1u << (3 * sh)) - 1u);
    const uint32_t bi = brick % (uint32_t)h->bdims[0], bt = brick / (uint32_t)h->bdims[0];
    const uint32_t bj = bt % (uint32_t)h->bdims[1], bk = bt / (uint32_t)h->bdims[1];
    const uint32_t i = (bi << sh) | (in & m), j = (bj << sh) | ((in >> sh) & m), k = (bk << sh) | (in >> (2 * sh));
    return (uint32_t)(((uint64_t)k * (uint64_t)h->dims[1] + j) * (uint64_t)h->dims[0] + i);
}

dem_status dem_debug_snapshot(dem_handle* h, uint32_t* cell, uint32_t* order, int64_t pair_cap, uint32_t* pairs,
                              int64_t* npairs) {
    if (!h) return DEM_ERR_INVALID_ARG;
    if (h->broken) return fail(h, DEM_ERR_STATE, "handle is unusable after a CUDA error");
    if (!h->has_particles) return fail(h, DEM_ERR_STATE, "no particles");
    DeviceGuard g(h->device);
    Domain& d = h->d;
    const size_t n = d.n, N = d.cap;
    std::vector<uint32_t> ids, skey;
    dem_status s;
    CtrlDev ctl;
    if ((s = read_ctrl(h, ctl)) != DEM_OK) return s;
    if ((s = download_u32(h, ids, d.precision == 0 ? d.S64[ctl.cur].id : d.S32[ctl.cur].id, n)) != DEM_OK) return s;
    if ((s = download_u32(h, skey, d.skey, n)) != DEM_OK) return s;
    CK(h, cudaStreamSynchronize(d.stream));
    // keys in row-major numbering ((k ny + j) nx + i), whatever order the sort used
    for (size_t q = 0; q < n; ++q) skey[q] = row_major_key(h, skey[q]);
    if (cell)
        for (size_t q = 0; q < n; ++q) cell[ids[q]] = skey[q];
    if (order) {
        // storage order; list mode keeps windows ordered by contact count, so the
        // (cell, id) order is recovered here
        std::vector<size_t> pos(n);
        for (size_t q = 0; q < n; ++q) pos[q] = q;
        if (d.list_mode)
            std::sort(pos.begin(), pos.end(), [&](size_t a, size_t b) {
                return skey[a] != skey[b] ? skey[a] < skey[b] : ids[a] < ids[b];
            });
        for (size_t q = 0; q < n; ++q) order[q] = ids[pos[q]];
    }
    if (npairs) *npairs = 0;
    if (pairs || npairs) {
        if (!h->eval_valid) return fail(h, DEM_ERR_STATE, "pairs need a dem_get_forces call on the current state");
        const int ho = 1 - d.h_cur;
        std::vector<uint32_t> cnt;
        if ((s = download_u32(h, cnt, d.hcnt[ho], n)) != DEM_OK) return s;
        CK(h, cudaStreamSynchronize(d.stream));
        uint32_t mx = 0;
        for (size_t q = 0; q < n; ++q) mx = std::max(mx, slots_of(d, cnt[q]));
        std::vector<uint32_t> pid((size_t)mx * N);
        if (mx) {
            CK(h, cudaMemcpyAsync(pid.data(), d.hpid[ho], (size_t)mx * N * 4, cudaMemcpyDeviceToHost, d.stream));
            CK(h, cudaStreamSynchronize(d.stream));
        }
        std::vector<std::pair<uint32_t, uint32_t>> pr;
        for (size_t q = 0; q < n; ++q) {
            const uint32_t c = slots_of(d, cnt[q]);
            for (uint32_t k = 0; k < c; ++k) {
                const uint32_t p = pid[(size_t)k * N + q];
                if (p < DEM_WALL_BASE && ids[q] < p) pr.emplace_back(ids[q], p);
            }
        }
        std::sort(pr.begin(), pr.end());
        if (npairs) *npairs = (int64_t)pr.size();
        if (pairs)
            for (size_t k = 0; k < pr.size() && (int64_t)k < pair_cap; ++k) {
                pairs[2 * k] = pr[k].first;
                pairs[2 * k + 1] = pr[k].second;
            }
    }
    return DEM_OK;
}

dem_status dem_get_grid(const dem_handle* h, double* origin, double* cell, int64_t* dims) {
    if (!h) return DEM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) {
        if (origin) origin[a] = h->origin[a];
        if (dims) dims[a] = h->dims[a];
    }
    if (cell) *cell = h->h;
    return DEM_OK;
}

int64_t dem_device_bytes(const dem_handle* h) {
    if (!h) return 0;
    const Domain& d = h->d;
    const size_t N = d.cap, M = d.maxc, C = (size_t)d.cells_cap + 1;
    const size_t T = d.precision == 0 ? 8 : 4;
    size_t state = d.precision == 0 ? N * (9 * 8 + 8) : N * (4 * 16 + 4);
    size_t b = 2 * state + 2 * (N * 4 + N * 4 * M + N * T * 3 * M) + 5 * N * 4 + 2 * C * 4 + (size_t)d.part_cap * 4 +
               (size_t)d.diag_part_cap * 80 + sizeof(StatusDev) + 128 + sizeof(SceneDev) * d.scenes_cap;
    b += (size_t)h->stage_cap * (9 * 8 + 4);
    if (d.list_mode) b += N * (4 + 4 * (size_t)DEM_LIST_CAP + 4 + 16 + 8);
    return (int64_t)b;
}

int64_t dem_max_contacts_seen(const dem_handle* h) {
    return (h && h->d.st_host) ? (int64_t)h->d.st_host->last.max_nnew : 0;
}

int64_t dem_launch_count(const dem_handle* h) {
    if (!h) return 0;
    int64_t n = h->d.launches;
    if (h->graph.body_launches > 0 && h->d.ctrl) {
        // sorts that ran as conditional graph bodies (counted on the device)
        CtrlDev c{};
        DeviceGuard g(h->device);
        if (cudaMemcpyAsync(&c, h->d.ctrl, sizeof c, cudaMemcpyDeviceToHost, h->d.stream) == cudaSuccess &&
            cudaStreamSynchronize(h->d.stream) == cudaSuccess)
            n += h->graph.body_launches * (int64_t)c.cond_sorts;
        else
            cudaGetLastError();
    }
    return n;
}

const char* dem_last_error(const dem_handle* h) { return h ? h->err.c_str() : "null handle"; }

void dem_destroy(dem_handle* h) {
    if (!h) return;
    DeviceGuard g(h->device);
    if (h->d.stream) cudaStreamSynchronize(h->d.stream);
    else cudaDeviceSynchronize();
    free_particle_buffers(h->d);
    if (h->d.d_scenes) cudaFree(h->d.d_scenes);
    if (h->d.st) cudaFree(h->d.st);
    if (h->d.st_host) cudaFreeHost(h->d.st_host);
    if (h->d.ctrl) cudaFree(h->d.ctrl);
    if (h->d.ctrl_host) cudaFreeHost(h->d.ctrl_host);
    if (h->d.diag_out) cudaFree(h->d.diag_out);
    if (h->chk_dev) cudaFree(h->chk_dev);
    if (h->chk_host) cudaFreeHost(h->chk_host);
    if (h->stage) cudaFree(h->stage);
    if (h->stage_r) cudaFree(h->stage_r);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    h->graph.reset();
    cudaGetLastError();
    delete h;
}

}  // extern "C"

// =========================================================================== batches
// Many independent scenes packed end to end in one domain: every kernel launch of a step
// covers all of them (each particle finds its scene's parameters, grid and walls in the
// scene table), so uneven scenes advance together in one launch sequence, replayed as a
// CUDA graph. Scenes are added as arrays and enter at the next dem_batch_run, when the
// domain is repacked (kept scenes keep their state and springs, finished or removed
// scenes leave). Each scene advances until its own step budget; then it is frozen
// (carried unchanged) until it is removed.
namespace {

struct BatchScene {
    int slot = -1;
    dem_config cfg{};
    std::vector<dem_wall> walls;
    int64_t n = 0, budget = 0, done = 0;
    bool in_domain = false, removed = false;
    std::vector<double> x, v, w;   // staged input until the scene enters the domain
    std::vector<float> r;
    double rmax = 0.0, origin[3] = {0, 0, 0}, h = 0.0;
    int64_t dims[3] = {1, 1, 1};
    int bshift = 0;                    // list mode: cells in bricks of (2^bshift)^3
    int64_t bdims[3] = {1, 1, 1};
    uint32_t p0 = 0, c0 = 0, ncell = 1;
};

}  // namespace

struct dem_batch {
    Domain d;
    int device = 0;
    std::vector<BatchScene> scenes;
    int next_slot = 0;
    bool dirty = false;
    bool broken = false;
    std::string err;
    StepGraph graph;
    double* stage = nullptr;
    float* stage_r = nullptr;
    size_t stage_cap = 0;
    uint32_t* d_map = nullptr;
    size_t map_cap = 0;
    int resort_interval = -1;   // sort policy of every scene (set by the first scene added)
};

namespace {

dem_status bfail(dem_batch* b, dem_status s, const std::string& m) {
    if (b) b->err = m;
    return s;
}
dem_status bcuda(dem_batch* b, cudaError_t e, const char* what) {
    if (b) {
        b->broken = true;
        b->err = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return DEM_ERR_CUDA;
}
#define BCK(b, expr)                                                   \
    do {                                                               \
        cudaError_t e__ = (expr);                                      \
        if (e__ != cudaSuccess) return bcuda((b), e__, #expr);         \
    } while (0)

// Scene table entry of a batch scene (the same fields a handle fills for its one scene).
void fill_batch_scene(const BatchScene& sc, SceneDev& S) {
    dem_handle tmp;
    tmp.cfg = sc.cfg;
    tmp.walls = sc.walls;
    tmp.rmax = sc.rmax;
    tmp.h = sc.h;
    tmp.bshift = sc.bshift;
    for (int a = 0; a < 3; ++a) {
        tmp.origin[a] = sc.origin[a];
        tmp.dims[a] = sc.dims[a];
        tmp.bdims[a] = sc.bdims[a];
    }
    fill_scene(&tmp, S, sc.p0, (uint32_t)sc.n, sc.c0);
}

// Rebuild the packed domain: kept scenes (state + springs), then the staged ones.
dem_status repack(dem_batch* b) {
    Domain& od = b->d;
    std::vector<BatchScene*> kept, fresh;
    for (auto& sc : b->scenes) {
        if (sc.removed) continue;
        (sc.in_domain ? kept : fresh).push_back(&sc);
    }
    // new layout
    uint64_t n_new = 0, c_new = 0;
    std::vector<uint32_t> map;
    for (BatchScene* sc : kept) {
        for (int64_t k = 0; k < sc->n; ++k) map.push_back(sc->p0 + (uint32_t)k);
    }
    uint32_t p = 0, c = 0;
    for (BatchScene* sc : kept) {
        sc->p0 = p;
        sc->c0 = c;
        p += (uint32_t)sc->n;
        c += sc->ncell;
    }
    for (BatchScene* sc : fresh) {
        sc->p0 = p;
        sc->c0 = c;
        p += (uint32_t)sc->n;
        c += sc->ncell;
        for (int64_t k = 0; k < sc->n; ++k) map.push_back(0xFFFFFFFFu);
    }
    n_new = p;
    c_new = c;
    if (n_new > 0x7FFFFF00ull || c_new > 0x7FFFFFFFull) return bfail(b, DEM_ERR_INVALID_ARG, "batch too large");
    // springs of the current state into sorted order (old domain), then the new domain
    if (od.n > 0) BCK(b, run_hist_canon(od));
    Domain nd;
    nd.precision = od.precision;
    nd.model = od.model;
    nd.terms = 0;
    for (BatchScene* sc : kept) nd.terms |= sc->cfg.terms;
    for (BatchScene* sc : fresh) nd.terms |= sc->cfg.terms;
    nd.stiffness = od.stiffness;
    nd.maxc = od.maxc;
    nd.maxn = od.maxn;
    nd.block = od.block;
    nd.sort_blocks = od.sort_blocks;
    nd.stream = od.stream;
    nd.list_mode = (b->resort_interval >= 0 && b->resort_interval != 1) ? 1 : 0;
    nd.interval = b->resort_interval < 0 ? 1 : b->resort_interval;
    nd.st = od.st;
    nd.st_host = od.st_host;
    nd.ctrl = od.ctrl;
    nd.ctrl_host = od.ctrl_host;
    nd.diag_out = od.diag_out;
    nd.launches = od.launches;
    nd.n = (uint32_t)n_new;
    nd.ncells = (uint32_t)std::max<uint64_t>(c_new, 1);
    std::string err;
    dem_status s = alloc_domain(nd, nd.n, nd.ncells, err);
    if (s != DEM_OK) return bfail(b, s, err);
    // scene table
    const int ns = (int)(kept.size() + fresh.size());
    nd.nscenes = ns;
    nd.h_scenes.assign(std::max(ns, 1), SceneDev{});
    int k = 0;
    for (BatchScene* sc : kept) fill_batch_scene(*sc, nd.h_scenes[k++]);
    for (BatchScene* sc : fresh) fill_batch_scene(*sc, nd.h_scenes[k++]);
    for (k = 0; k < ns; ++k) {
        BatchScene* sc = k < (int)kept.size() ? kept[k] : fresh[k - kept.size()];
        nd.h_scenes[k].active = sc->done < sc->budget ? 1 : 0;
    }
    if (cudaMalloc(&nd.d_scenes, sizeof(SceneDev) * std::max(ns, 1)) != cudaSuccess) {
        cudaGetLastError();
        free_particle_buffers(nd);
        return bfail(b, DEM_ERR_OOM, "cudaMalloc(scene table) failed");
    }
    nd.scenes_cap = std::max(ns, 1);
    BCK(b, cudaMemcpyAsync(nd.d_scenes, nd.h_scenes.data(), sizeof(SceneDev) * ns, cudaMemcpyHostToDevice, nd.stream));
    // old -> new particle map, kept springs and state
    if (n_new > 0) {
        if (b->map_cap < n_new) {
            if (b->d_map) cudaFree(b->d_map);
            b->d_map = nullptr;
            if (cudaMalloc(&b->d_map, n_new * 4) != cudaSuccess) {
                cudaGetLastError();
                return bfail(b, DEM_ERR_OOM, "cudaMalloc(map) failed");
            }
            b->map_cap = n_new;
        }
        BCK(b, cudaMemcpyAsync(b->d_map, map.data(), n_new * 4, cudaMemcpyHostToDevice, nd.stream));
        BCK(b, run_repack(od, nd, b->d_map, (uint32_t)n_new));
    }
    // staged scenes
    for (BatchScene* sc : fresh) {
        const size_t n = (size_t)sc->n;
        if (n == 0) continue;
        if (b->stage_cap < n) {
            if (b->stage) cudaFree(b->stage);
            if (b->stage_r) cudaFree(b->stage_r);
            b->stage = nullptr;
            b->stage_r = nullptr;
            if (cudaMalloc(&b->stage, n * 72) != cudaSuccess || cudaMalloc(&b->stage_r, n * 4) != cudaSuccess) {
                cudaGetLastError();
                return bfail(b, DEM_ERR_OOM, "cudaMalloc(stage) failed");
            }
            b->stage_cap = n;
        }
        BCK(b, cudaMemcpyAsync(b->stage, sc->x.data(), n * 24, cudaMemcpyHostToDevice, nd.stream));
        BCK(b, cudaMemcpyAsync(b->stage + 3 * n, sc->v.data(), n * 24, cudaMemcpyHostToDevice, nd.stream));
        BCK(b, cudaMemcpyAsync(b->stage + 6 * n, sc->w.data(), n * 24, cudaMemcpyHostToDevice, nd.stream));
        BCK(b, cudaMemcpyAsync(b->stage_r, sc->r.data(), n * 4, cudaMemcpyHostToDevice, nd.stream));
        BCK(b, run_import_at(nd, sc->p0, (uint32_t)n, b->stage, b->stage + 3 * n, b->stage + 6 * n, b->stage_r));
        BCK(b, cudaStreamSynchronize(nd.stream));   // the stage is reused by the next scene
        sc->in_domain = true;
        std::vector<double>().swap(sc->x);
        std::vector<double>().swap(sc->v);
        std::vector<double>().swap(sc->w);
        std::vector<float>().swap(sc->r);
    }
    // first sort of the new layout
    *nd.ctrl_host = CtrlDev{};
    nd.ctrl_host->rebuild = 1;
    BCK(b, cudaStreamSynchronize(nd.stream));
    BCK(b, cudaMemcpyAsync(nd.ctrl, nd.ctrl_host, sizeof(CtrlDev), cudaMemcpyHostToDevice, nd.stream));
    BCK(b, cudaMemsetAsync(nd.cnt, 0, ((size_t)nd.ncells + 1) * 4, nd.stream));
    nd.h_cur = 0;
    BCK(b, run_hash(nd));
    BCK(b, run_rebuild(nd));
    BCK(b, run_end_step(nd));
    BCK(b, cudaStreamSynchronize(nd.stream));
    // swap in
    b->graph.reset();
    free_particle_buffers(od);
    if (od.d_scenes) cudaFree(od.d_scenes);
    od.d_scenes = nullptr;
    Domain keep_shared = od;   // status, ctrl and diag buffers are shared
    (void)keep_shared;
    b->d = nd;
    // drop removed scenes from the list
    std::vector<BatchScene> left;
    for (auto& sc : b->scenes)
        if (!sc.removed) left.push_back(std::move(sc));
    b->scenes = std::move(left);
    b->dirty = false;
    return DEM_OK;
}

BatchScene* find_slot(dem_batch* b, int slot) {
    for (auto& sc : b->scenes)
        if (sc.slot == slot && !sc.removed) return &sc;
    return nullptr;
}

}  // namespace

extern "C" {

dem_status dem_batch_create(int precision, int model, int stiffness, int max_contacts, int block_size, int device,
                            void* cuda_stream, dem_batch** out) {
    if (!out) return DEM_ERR_INVALID_ARG;
    *out = nullptr;
    if ((precision != DEM_FP64 && precision != DEM_FP32) || (model != DEM_PRACTICAL && model != DEM_SIMPLE) ||
        (stiffness != DEM_LINEAR && stiffness != DEM_HERTZ) || max_contacts < 0 || max_contacts > 64 ||
        (block_size != 0 && (block_size < 32 || block_size > 256 || block_size % 32)))
        return DEM_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DEM_ERR_INVALID_ARG;
    }
    DeviceGuard g(device);
    dem_batch* b = new dem_batch();
    b->device = device;
    Domain& d = b->d;
    d.precision = precision;
    d.model = model;
    d.stiffness = stiffness;
    d.maxc = max_contacts > 0 ? max_contacts : 32;
    d.maxn = DEM_LIST_CAP;
    d.block = block_size > 0 ? block_size : 256;
    d.sort_blocks = sort_blocks_of(device);
    d.stream = (cudaStream_t)cuda_stream;
    if (cudaMalloc(&d.st, sizeof(StatusDev)) != cudaSuccess || cudaMallocHost(&d.st_host, sizeof(StatusDev)) != cudaSuccess ||
        cudaMalloc(&d.ctrl, sizeof(CtrlDev)) != cudaSuccess || cudaMallocHost(&d.ctrl_host, sizeof(CtrlDev)) != cudaSuccess ||
        cudaMalloc(&d.diag_out, 16 * sizeof(double)) != cudaSuccess || cudaMemset(d.st, 0, sizeof(StatusDev)) != cudaSuccess ||
        cudaMemset(d.ctrl, 0, sizeof(CtrlDev)) != cudaSuccess) {
        cudaGetLastError();
        dem_batch_destroy(b);
        return DEM_ERR_OOM;
    }
    *out = b;
    return DEM_OK;
}

dem_status dem_batch_add(dem_batch* b, const dem_config* cfg, int nwalls, const dem_wall* walls, int64_t n,
                         const double* x, const double* v, const double* w, const float* r, int64_t step_budget,
                         int* slot) {
    if (!b || !slot) return DEM_ERR_INVALID_ARG;
    if (b->broken) return bfail(b, DEM_ERR_STATE, "batch is unusable after a CUDA error");
    std::string why;
    if (validate_config(cfg, why) != DEM_OK) return bfail(b, DEM_ERR_INVALID_ARG, why);
    if (cfg->precision != b->d.precision || cfg->model != b->d.model || cfg->stiffness != b->d.stiffness)
        return bfail(b, DEM_ERR_INVALID_ARG, "precision, model and stiffness must match the batch");
    // the batch's sort policy is its first scene's: every scene sorts every step, or every
    // scene keeps neighbour lists (each with its own skin) under one resort_interval
    if (b->resort_interval < 0) b->resort_interval = cfg->resort_interval;
    if (cfg->resort_interval != b->resort_interval)
        return bfail(b, DEM_ERR_INVALID_ARG, "every scene of a batch must have the batch's resort_interval");
    if (nwalls < 0 || nwalls > DEM_MAX_WALLS || (nwalls > 0 && !walls)) return bfail(b, DEM_ERR_INVALID_ARG, "nwalls");
    if (n < 0 || n > 0x7FFFFF00 || step_budget < 0) return bfail(b, DEM_ERR_INVALID_ARG, "n or step_budget");
    if (n > 0 && (!x || !v || !w || !r)) return bfail(b, DEM_ERR_INVALID_ARG, "x, v, w and r are required");
    for (int k = 0; k < nwalls; ++k)
        if (!check_wall(walls[k], cfg->precision, why)) return bfail(b, DEM_ERR_INVALID_ARG, why);
    BatchScene sc;
    sc.slot = b->next_slot++;
    sc.cfg = *cfg;
    sc.walls.assign(walls, walls + nwalls);
    sc.n = n;
    sc.budget = step_budget;
    double rmax = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        if (!(r[k] > 0.f) || !std::isfinite(r[k])) return bfail(b, DEM_ERR_INVALID_ARG, "radii must be finite and > 0");
        if (!finite3(x + 3 * k) || !finite3(v + 3 * k) || !finite3(w + 3 * k))
            return bfail(b, DEM_ERR_INVALID_ARG, "non-finite input");
        rmax = std::max(rmax, (double)r[k]);
    }
    const double hmin = 2.0 * rmax * (1.0 + std::ldexp(1.0, -10)) + cfg->skin;
    double hc = cfg->cell_size > 0.0 ? cfg->cell_size : hmin;
    if (n > 0 && hc < hmin * (1.0 - 1e-12)) return bfail(b, DEM_ERR_INVALID_ARG, "cell_size too small");
    if (!(hc > 0.0)) hc = 1.0;
    int64_t nc = 1;
    for (int a = 0; a < 3; ++a) {
        sc.origin[a] = cfg->domain_lo[a];
        sc.dims[a] = std::max<int64_t>(1, (int64_t)std::ceil((cfg->domain_hi[a] - cfg->domain_lo[a]) / hc));
        nc *= sc.dims[a];
        if (nc > (int64_t)0x7FFFFFFF) return bfail(b, DEM_ERR_INVALID_ARG, "grid has more than 2^31 cells");
    }
    if (b->resort_interval != 1) sc.bshift = choose_bricks(sc.dims, nc, sc.bdims, nc);
    sc.h = hc;
    sc.rmax = rmax;
    sc.ncell = (uint32_t)nc;
    sc.x.assign(x, x + 3 * n);
    sc.v.assign(v, v + 3 * n);
    sc.w.assign(w, w + 3 * n);
    sc.r.assign(r, r + n);
    *slot = sc.slot;
    b->scenes.push_back(std::move(sc));
    b->dirty = true;
    return DEM_OK;
}

dem_status dem_batch_remove(dem_batch* b, int slot) {
    if (!b) return DEM_ERR_INVALID_ARG;
    BatchScene* sc = find_slot(b, slot);
    if (!sc) return bfail(b, DEM_ERR_INVALID_ARG, "no such slot");
    sc->removed = true;
    b->dirty = true;
    return DEM_OK;
}

dem_status dem_batch_run(dem_batch* b, int64_t max_steps, int* finished, int cap, int* nfinished) {
    if (!b || max_steps < 0 || (cap > 0 && !finished)) return DEM_ERR_INVALID_ARG;
    if (b->broken) return bfail(b, DEM_ERR_STATE, "batch is unusable after a CUDA error");
    DeviceGuard g(b->device);
    if (nfinished) *nfinished = 0;
    if (b->dirty) {
        dem_status s = repack(b);
        if (s != DEM_OK) return s;
    }
    Domain& d = b->d;
    int64_t left = max_steps;
    int nfin = 0;
    while (left > 0) {
        int64_t s = left;
        bool any = false;
        for (auto& sc : b->scenes)
            if (sc.in_domain && sc.done < sc.budget) {
                any = true;
                s = std::min(s, sc.budget - sc.done);
            }
        if (!any) break;
        BCK(b, run_steps(d, &b->graph, s));
        left -= s;
        bool changed = false;
        for (size_t k = 0; k < b->scenes.size(); ++k) {
            BatchScene& sc = b->scenes[k];
            if (!sc.in_domain || sc.done >= sc.budget) continue;
            sc.done += s;
            if (sc.done >= sc.budget) {
                if (nfin < cap) finished[nfin] = sc.slot;
                ++nfin;
                changed = true;
            }
        }
        if (changed) {
            // freeze the finished scenes (the scene table is device memory, so the
            // captured graph stays valid)
            for (size_t k = 0; k < b->scenes.size(); ++k)
                d.h_scenes[k].active = b->scenes[k].done < b->scenes[k].budget ? 1 : 0;
            BCK(b, cudaMemcpyAsync(d.d_scenes, d.h_scenes.data(), sizeof(SceneDev) * b->scenes.size(),
                                   cudaMemcpyHostToDevice, d.stream));
            break;   // hand control back so that the caller can read, remove and admit
        }
    }
    if (nfinished) *nfinished = nfin;
    BCK(b, cudaMemcpyAsync(d.st_host, d.st, sizeof(StatusDev), cudaMemcpyDeviceToHost, d.stream));
    BCK(b, cudaStreamSynchronize(d.stream));
    if (d.st_host->code != 0) {
        const int code = d.st_host->code;
        BCK(b, cudaMemsetAsync(d.st, 0, 2 * sizeof(int32_t), d.stream));
        return bfail(b, code == ST_CAPACITY ? DEM_ERR_CAPACITY : DEM_ERR_NONFINITE, "device status raised");
    }
    return DEM_OK;
}

dem_status dem_batch_get_state(dem_batch* b, int slot, double* x, double* v, double* w, int where) {
    if (!b || (where != DEM_HOST && where != DEM_DEVICE)) return DEM_ERR_INVALID_ARG;
    if (b->broken) return bfail(b, DEM_ERR_STATE, "batch is unusable after a CUDA error");
    BatchScene* sc = find_slot(b, slot);
    if (!sc) return bfail(b, DEM_ERR_INVALID_ARG, "no such slot");
    const size_t n = (size_t)sc->n;
    if (!sc->in_domain) {
        if (where != DEM_HOST) return bfail(b, DEM_ERR_STATE, "scene not yet in the domain: host read only");
        if (x) std::copy(sc->x.begin(), sc->x.end(), x);
        if (v) std::copy(sc->v.begin(), sc->v.end(), v);
        if (w) std::copy(sc->w.begin(), sc->w.end(), w);
        return DEM_OK;
    }
    DeviceGuard g(b->device);
    Domain& d = b->d;
    if (n == 0) return DEM_OK;
    if (where == DEM_DEVICE) {
        BCK(b, run_export_range(d, sc->p0, (uint32_t)n, x, v, w));
    } else {
        if (b->stage_cap < n) {
            if (b->stage) cudaFree(b->stage);
            if (b->stage_r) cudaFree(b->stage_r);
            b->stage = nullptr;
            b->stage_r = nullptr;
            if (cudaMalloc(&b->stage, n * 72) != cudaSuccess || cudaMalloc(&b->stage_r, n * 4) != cudaSuccess) {
                cudaGetLastError();
                return bfail(b, DEM_ERR_OOM, "cudaMalloc(stage) failed");
            }
            b->stage_cap = n;
        }
        BCK(b, run_export_range(d, sc->p0, (uint32_t)n, x ? b->stage : nullptr, v ? b->stage + 3 * n : nullptr,
                                w ? b->stage + 6 * n : nullptr));
        if (x) BCK(b, cudaMemcpyAsync(x, b->stage, n * 24, cudaMemcpyDeviceToHost, d.stream));
        if (v) BCK(b, cudaMemcpyAsync(v, b->stage + 3 * n, n * 24, cudaMemcpyDeviceToHost, d.stream));
        if (w) BCK(b, cudaMemcpyAsync(w, b->stage + 6 * n, n * 24, cudaMemcpyDeviceToHost, d.stream));
    }
    BCK(b, cudaStreamSynchronize(d.stream));
    return DEM_OK;
}

dem_status dem_batch_info(const dem_batch* b, int slot, int64_t* n, int64_t* steps_done, int64_t* budget) {
    if (!b) return DEM_ERR_INVALID_ARG;
    for (const auto& sc : b->scenes)
        if (sc.slot == slot && !sc.removed) {
            if (n) *n = sc.n;
            if (steps_done) *steps_done = sc.done;
            if (budget) *budget = sc.budget;
            return DEM_OK;
        }
    return DEM_ERR_INVALID_ARG;
}

int64_t dem_batch_device_bytes(const dem_batch* b) {
    if (!b) return 0;
    const Domain& d = b->d;
    const size_t N = d.cap, M = d.maxc, C = (size_t)d.cells_cap + 1;
    const size_t T = d.precision == 0 ? 8 : 4;
    const size_t state = d.precision == 0 ? N * (9 * 8 + 8) : N * (4 * 16 + 4);
    size_t bytes = 2 * state + 2 * (N * 4 + N * 4 * M + N * T * 3 * M) + 5 * N * 4 + 2 * C * 4 +
                   b->stage_cap * 76 + b->map_cap * 4;
    if (d.list_mode) bytes += N * (4 + 4 * (size_t)DEM_LIST_CAP + 4 + 16 + 8);
    return (int64_t)bytes;
}

int64_t dem_batch_launch_count(const dem_batch* b) { return b ? b->d.launches : 0; }

const char* dem_batch_last_error(const dem_batch* b) { return b ? b->err.c_str() : "null batch"; }

void dem_batch_destroy(dem_batch* b) {
    if (!b) return;
    DeviceGuard g(b->device);
    if (b->d.stream) cudaStreamSynchronize(b->d.stream);
    else cudaDeviceSynchronize();
    b->graph.reset();
    free_particle_buffers(b->d);
    if (b->d.d_scenes) cudaFree(b->d.d_scenes);
    if (b->d.st) cudaFree(b->d.st);
    if (b->d.st_host) cudaFreeHost(b->d.st_host);
    if (b->d.ctrl) cudaFree(b->d.ctrl);
    if (b->d.ctrl_host) cudaFreeHost(b->d.ctrl_host);
    if (b->d.diag_out) cudaFree(b->d.diag_out);
    if (b->stage) cudaFree(b->stage);
    if (b->stage_r) cudaFree(b->stage_r);
    if (b->d_map) cudaFree(b->d_map);
    cudaGetLastError();
    delete b;
}

}  // extern "C"

// =========================================================================== slabs
// One scene divided along one axis into slabs (sub-domains), each a handle with its own
// particle buffers and cell table on the scene's global grid and a ghost layer one cell
// edge wide on each side (dem_halo.h). A step runs the force pass of every slab, one
// exchange launch (migration of owned particles with their springs, fresh ghost copies),
// the flip of every slab's current set (the exchange wrote into the set the force pass
// read), and the cell sort of every slab's new layout.
struct dem_slabs {
    dem_config cfg{};
    int device = 0;
    int nslabs = 0;
    int axis = 2;
    cudaStream_t stream = nullptr;
    std::vector<dem_handle*> sl;
    std::vector<int> cur;              // host mirror of each slab's ctrl->cur
    HaloGeom geom{};
    uint8_t* owner[2] = {nullptr, nullptr};   // slab of every particle id, double-buffered
    int own_cur = 0;                   // owner[own_cur] holds the current owners
    uint32_t owner_cap = 0;
    HaloCounters* hc = nullptr;        // device: counters of the exchange in flight
    HaloCounters* hc_host = nullptr;   // pinned: counters of the last exchange
    std::vector<uint8_t> io_table;     // SlabIO table of the exchange (host; passed by value)
    void* io_host = nullptr;
    double* stage = nullptr;           // host input / output staging: x, v, w (3n doubles each)
    float* stage_r = nullptr;
    uint32_t stage_cap = 0;
    uint32_t n = 0;
    bool has_particles = false;
    bool broken = false;
    int64_t steps = 0;
    int64_t migrated = 0;
    int64_t launches = 0;              // exchange, flip and export launches
    std::string err;
};

namespace {

dem_status sfail(dem_slabs* S, dem_status st, const std::string& m) {
    if (S) S->err = m;
    return st;
}

dem_status scuda(dem_slabs* S, cudaError_t e, const char* what) {
    S->broken = true;
    S->err = std::string(what) + ": " + cudaGetErrorString(e);
    return DEM_ERR_CUDA;
}

#define SCK(S, expr)                                                       \
    do {                                                                   \
        cudaError_t e__ = (expr);                                          \
        if (e__ != cudaSuccess) return scuda((S), e__, #expr);             \
    } while (0)

// A slab's error (from its handle) becomes the slabs' error.
dem_status from_slab(dem_slabs* S, int k, dem_status st) {
    if (st == DEM_OK) return st;
    if (S->sl[k]->broken) S->broken = true;
    S->err = "slab " + std::to_string(k) + ": " + S->sl[k]->err;
    return st;
}

// Buffers of an empty slab for up to cap particles on the scene's grid, a scene table,
// cleared status and spring counts, and a step control that sorts next.
dem_status slab_prepare(dem_handle* h, uint32_t cap, double rmax) {
    Domain& d = h->d;
    h->graph.reset();
    int64_t nc = 1;
    dem_status s = set_grid(h, cap > 0, rmax, nc);
    if (s != DEM_OK) return s;
    d.n = 0;
    d.ncells = (uint32_t)nc;
    s = ensure_buffers(h, cap, (uint32_t)nc);
    if (s != DEM_OK) return s;
    d.nscenes = 1;
    d.h_scenes.assign(1, SceneDev{});
    fill_scene(h, d.h_scenes[0], 0, cap, 0);
    if (!d.d_scenes) {
        if (cudaMalloc(&d.d_scenes, sizeof(SceneDev)) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, DEM_ERR_OOM, "cudaMalloc(scene table) failed");
        }
        d.scenes_cap = 1;
    }
    CK(h, cudaMemcpyAsync(d.d_scenes, d.h_scenes.data(), sizeof(SceneDev), cudaMemcpyHostToDevice, d.stream));
    CK(h, cudaMemsetAsync(d.st, 0, sizeof(StatusDev), d.stream));
    CK(h, cudaMemsetAsync(d.cnt, 0, ((size_t)d.ncells + 1) * 4, d.stream));
    *d.ctrl_host = CtrlDev{};
    d.ctrl_host->rebuild = 1;
    CK(h, cudaMemcpyAsync(d.ctrl, d.ctrl_host, sizeof(CtrlDev), cudaMemcpyHostToDevice, d.stream));
    d.h_cur = 0;
    CK(h, cudaMemsetAsync(d.hcnt[0], 0, (size_t)d.cap * 4, d.stream));
    CK(h, cudaMemsetAsync(d.hcnt[1], 0, (size_t)d.cap * 4, d.stream));
    h->has_particles = true;
    h->eval_valid = false;
    h->steps = 0;
    return DEM_OK;
}

// Exchange table: sources are the sets and springs the force pass just wrote; each
// destination is the set the force pass read (import: the set the first sort gathers
// from) and the spring buffer not holding the sources.
template <class St, class T>
void fill_io(dem_slabs* S, bool import, uint32_t& ntotal) {
    auto* io = (SlabIO<St, T>*)S->io_host;
    uint32_t p0 = 0;
    for (int k = 0; k < S->nslabs; ++k) {
        Domain& d = S->sl[k]->d;
        SlabIO<St, T> e{};
        const int c = S->cur[k];
        St sets[2];
        if constexpr (sizeof(T) == 8) { sets[0] = d.S64[0]; sets[1] = d.S64[1]; }
        else { sets[0] = d.S32[0]; sets[1] = d.S32[1]; }
        const int hs = d.h_cur;            // springs written by the force pass
        const int hd = import ? d.h_cur : 1 - d.h_cur;
        e.src = sets[1 - c];
        e.dst = import ? sets[1 - c] : sets[c];
        e.hcnt_src = d.hcnt[hs];
        e.hpid_src = d.hpid[hs];
        e.hd_src = (const T*)d.hd[hs];
        e.hcnt_dst = d.hcnt[hd];
        e.hpid_dst = d.hpid[hd];
        e.hd_dst = (T*)d.hd[hd];
        e.n = import ? 0u : d.n;
        e.p0 = p0;
        e.cap = d.cap;
        p0 += e.n;
        io[k] = e;
    }
    ntotal = p0;
}

// The exchange table (passed to the exchange kernel by value) and cleared counters.
dem_status prepare_exchange(dem_slabs* S, bool import, uint32_t& ntotal) {
    if (S->cfg.precision == 0) fill_io<StateF64, double>(S, import, ntotal);
    else fill_io<StateF32, float>(S, import, ntotal);
    SCK(S, cudaMemsetAsync(S->hc, 0, sizeof(HaloCounters), S->stream));
    return DEM_OK;
}

// After an exchange: its counters on the host, the new particle count of every slab.
dem_status take_counts(dem_slabs* S) {
    SCK(S, cudaMemcpyAsync(S->hc_host, S->hc, sizeof(HaloCounters), cudaMemcpyDeviceToHost, S->stream));
    SCK(S, cudaStreamSynchronize(S->stream));
    if (S->hc_host->overflow)
        return sfail(S, DEM_ERR_CAPACITY, "slab exchange overflowed a slab's capacity");
    for (int k = 0; k < S->nslabs; ++k) S->sl[k]->d.n = S->hc_host->fill[k];
    return DEM_OK;
}

// Cell sort of every slab's new layout (the set that is "next" for its step control).
dem_status sort_slabs(dem_slabs* S) {
    for (int k = 0; k < S->nslabs; ++k) {
        dem_handle* h = S->sl[k];
        Domain& d = h->d;
        // cell counts from scratch (the force pass counted the layout before the exchange)
        cudaError_t e = cudaMemsetAsync(d.cnt, 0, ((size_t)d.ncells + 1) * 4, d.stream);
        if (e == cudaSuccess && d.n > 0) e = run_hash(d);
        if (e == cudaSuccess && d.n > 0) e = run_rebuild(d);
        if (e == cudaSuccess) e = run_end_step(d);
        if (e != cudaSuccess) return from_slab(S, k, cuda_fail(h, e, "slab sort"));
    }
    return DEM_OK;
}

dem_status slabs_one_step(dem_slabs* S) {
    for (int k = 0; k < S->nslabs; ++k) {
        Domain& d = S->sl[k]->d;
        if (d.n > 0) {
            cudaError_t e = run_force(d, false, nullptr, nullptr);
            if (e != cudaSuccess) return from_slab(S, k, cuda_fail(S->sl[k], e, "slab force pass"));
        }
        d.h_cur = 1 - d.h_cur;   // springs just written
    }
    uint32_t ntotal = 0;
    dem_status st = prepare_exchange(S, false, ntotal);
    if (st != DEM_OK) return st;
    SCK(S, run_halo_route(S->cfg.precision, S->io_host, S->geom, ntotal, (uint32_t)S->sl[0]->d.maxc,
                          S->owner[S->own_cur], S->owner[1 - S->own_cur], S->hc, S->sl[0]->d.sort_blocks, S->stream));
    CtrlTable t{};
    t.n = S->nslabs;
    for (int k = 0; k < S->nslabs; ++k) t.c[k] = S->sl[k]->d.ctrl;
    SCK(S, run_halo_flip(t, S->stream));
    S->launches += ntotal ? 2 : 1;
    st = take_counts(S);
    if (st != DEM_OK) return st;
    S->own_cur ^= 1;
    S->migrated += S->hc_host->migrated;
    for (int k = 0; k < S->nslabs; ++k) {
        S->cur[k] ^= 1;
        S->sl[k]->d.h_cur = 1 - S->sl[k]->d.h_cur;   // the exchanged springs
    }
    return sort_slabs(S);
}

}  // namespace

extern "C" {

dem_status dem_slab_bounds(int64_t n, const double* z, int nslabs, double* bounds) {
    if (nslabs < 1 || nslabs > DEM_MAX_SLABS || n < 0 || !bounds || (n > 0 && !z)) return DEM_ERR_INVALID_ARG;
    std::vector<double> v(z, z + n);
    for (double a : v)
        if (!std::isfinite(a)) return DEM_ERR_INVALID_ARG;
    const double inf = std::numeric_limits<double>::infinity();
    bounds[0] = -inf;
    bounds[nslabs] = inf;
    size_t lo = 0;
    for (int k = 1; k < nslabs; ++k) {
        const size_t idx = (size_t)((n * (int64_t)k) / nslabs);
        if (n == 0) {
            bounds[k] = inf;
            continue;
        }
        if (idx >= lo) std::nth_element(v.begin() + lo, v.begin() + idx, v.end());
        bounds[k] = v[idx];
        lo = idx + 1;
    }
    return DEM_OK;
}

dem_status dem_slabs_create(const dem_config* cfg, int nslabs, int axis, int device, void* cuda_stream,
                            dem_slabs** out) {
    if (!out) return DEM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || nslabs < 1 || nslabs > DEM_MAX_SLABS || axis < -1 || axis > 2) return DEM_ERR_INVALID_ARG;
    if (cfg->resort_interval != 1) return DEM_ERR_INVALID_ARG;   // the walk mode only
    std::string why;
    dem_status st = validate_config(cfg, why);
    if (st != DEM_OK) return st;
    if (axis < 0) {
        axis = 0;
        for (int a = 1; a < 3; ++a)
            if (cfg->domain_hi[a] - cfg->domain_lo[a] >= cfg->domain_hi[axis] - cfg->domain_lo[axis]) axis = a;
    }
    dem_slabs* S = new dem_slabs();
    S->cfg = *cfg;
    S->device = device;
    S->nslabs = nslabs;
    S->axis = axis;
    S->stream = (cudaStream_t)cuda_stream;
    for (int k = 0; k < nslabs; ++k) {
        dem_handle* h = nullptr;
        st = dem_create(cfg, device, cuda_stream, &h);
        if (st != DEM_OK) {
            dem_slabs_destroy(S);
            return st;
        }
        h->d.regrow = 0;   // a slab's overflow is reported (its step is part of the exchange)
        S->sl.push_back(h);
    }
    S->cur.assign(nslabs, 0);
    DeviceGuard g(device);
    const size_t iob = std::max(sizeof(SlabIO<StateF64, double>), sizeof(SlabIO<StateF32, float>)) * DEM_MAX_SLABS;
    S->io_table.assign(iob, 0);
    S->io_host = S->io_table.data();
    if (cudaMalloc(&S->hc, sizeof(HaloCounters)) != cudaSuccess ||
        cudaMallocHost(&S->hc_host, sizeof(HaloCounters)) != cudaSuccess) {
        cudaGetLastError();
        dem_slabs_destroy(S);
        return DEM_ERR_OOM;
    }
    std::memset(S->hc_host, 0, sizeof(HaloCounters));
    *out = S;
    return DEM_OK;
}

dem_status dem_slabs_set_walls(dem_slabs* S, int nwalls, const dem_wall* walls) {
    if (!S) return DEM_ERR_INVALID_ARG;
    if (S->broken) return sfail(S, DEM_ERR_STATE, "slabs are unusable after a CUDA error");
    for (int k = 0; k < S->nslabs; ++k) {
        dem_status st = dem_set_walls(S->sl[k], nwalls, walls);
        if (st != DEM_OK) return from_slab(S, k, st);
    }
    return DEM_OK;
}

dem_status dem_slabs_set_particles(dem_slabs* S, int64_t n64, const double* x, const double* v, const double* w,
                                   const float* r, int where) {
    if (!S) return DEM_ERR_INVALID_ARG;
    if (S->broken) return sfail(S, DEM_ERR_STATE, "slabs are unusable after a CUDA error");
    // every slab holds at most n particles, so the exchange's launch indices over all
    // slabs (32-bit) cannot overflow
    if (n64 < 0 || n64 > (int64_t)(0x7FFFFF00 / DEM_MAX_SLABS)) return sfail(S, DEM_ERR_INVALID_ARG, "n out of range");
    if (where != DEM_HOST && where != DEM_DEVICE) return sfail(S, DEM_ERR_INVALID_ARG, "where");
    const uint32_t n = (uint32_t)n64;
    if (n > 0 && (!x || !v || !w || !r)) return sfail(S, DEM_ERR_INVALID_ARG, "x, v, w and r are required");
    DeviceGuard g(S->device);
    S->has_particles = false;
    // radii and the coordinates along the axis on the host (boundaries, grid)
    std::vector<float> rh;
    std::vector<double> xh;
    const float* rr = r;
    const double* xx = x;
    if (n > 0 && where == DEM_DEVICE) {
        rh.resize(n);
        xh.resize(3 * (size_t)n);
        SCK(S, cudaMemcpy(rh.data(), r, (size_t)n * 4, cudaMemcpyDeviceToHost));
        SCK(S, cudaMemcpy(xh.data(), x, (size_t)n * 24, cudaMemcpyDeviceToHost));
        rr = rh.data();
        xx = xh.data();
    }
    double rmax = 0.0;
    for (uint32_t k = 0; k < n; ++k) {
        if (!(rr[k] > 0.f) || !std::isfinite(rr[k])) return sfail(S, DEM_ERR_INVALID_ARG, "radii must be finite and > 0");
        rmax = std::max(rmax, (double)rr[k]);
    }
    if (where == DEM_HOST)
        for (uint32_t k = 0; k < n; ++k)
            if (!finite3(x + 3 * (size_t)k) || !finite3(v + 3 * (size_t)k) || !finite3(w + 3 * (size_t)k))
                return sfail(S, DEM_ERR_INVALID_ARG, "non-finite position, velocity or spin in the input");
    std::vector<double> za(n);
    for (uint32_t k = 0; k < n; ++k) za[k] = xx[3 * (size_t)k + S->axis];
    HaloGeom geom{};
    geom.nslabs = S->nslabs;
    geom.axis = S->axis;
    if (dem_slab_bounds(n, za.data(), S->nslabs, geom.zb) != DEM_OK)
        return sfail(S, DEM_ERR_INVALID_ARG, "non-finite coordinate along the slab axis");
    for (int k = 0; k < S->nslabs; ++k) {
        dem_status st = slab_prepare(S->sl[k], n, rmax);
        if (st != DEM_OK) return from_slab(S, k, st);
        S->cur[k] = 0;
    }
    geom.G = S->sl[0]->h;
    set_keys(geom);
    S->geom = geom;
    S->n = n;
    if (n > S->owner_cap) {
        for (auto& o : S->owner) {
            if (o) cudaFree(o);
            o = nullptr;
        }
        S->owner_cap = 0;
        if (cudaMalloc(&S->owner[0], n) != cudaSuccess || cudaMalloc(&S->owner[1], n) != cudaSuccess) {
            cudaGetLastError();
            return sfail(S, DEM_ERR_OOM, "cudaMalloc(owner map) failed");
        }
        S->owner_cap = n;
    }
    S->own_cur = 0;
    const double *xd = x, *vd = v, *wd = w;
    const float* rd = r;
    if (n > 0 && where == DEM_HOST) {
        if (n > S->stage_cap) {
            if (S->stage) cudaFree(S->stage);
            if (S->stage_r) cudaFree(S->stage_r);
            S->stage = nullptr;
            S->stage_r = nullptr;
            S->stage_cap = 0;
            if (cudaMalloc(&S->stage, (size_t)n * 72) != cudaSuccess || cudaMalloc(&S->stage_r, (size_t)n * 4) != cudaSuccess) {
                cudaGetLastError();
                return sfail(S, DEM_ERR_OOM, "cudaMalloc(stage) failed");
            }
            S->stage_cap = n;
        }
        SCK(S, cudaMemcpyAsync(S->stage, x, (size_t)n * 24, cudaMemcpyHostToDevice, S->stream));
        SCK(S, cudaMemcpyAsync(S->stage + 3 * (size_t)n, v, (size_t)n * 24, cudaMemcpyHostToDevice, S->stream));
        SCK(S, cudaMemcpyAsync(S->stage + 6 * (size_t)n, w, (size_t)n * 24, cudaMemcpyHostToDevice, S->stream));
        SCK(S, cudaMemcpyAsync(S->stage_r, r, (size_t)n * 4, cudaMemcpyHostToDevice, S->stream));
        xd = S->stage; vd = S->stage + 3 * (size_t)n; wd = S->stage + 6 * (size_t)n; rd = S->stage_r;
    }
    uint32_t ntotal = 0;
    dem_status st = prepare_exchange(S, true, ntotal);
    if (st != DEM_OK) return st;
    SCK(S, run_halo_import(S->cfg.precision, S->io_host, S->geom, n, xd, vd, wd, rd, S->owner[0], S->hc,
                           S->sl[0]->d.sort_blocks, S->stream));
    if (n > 0) S->launches += 1;
    st = take_counts(S);
    if (st != DEM_OK) return st;
    st = sort_slabs(S);
    if (st != DEM_OK) return st;
    SCK(S, cudaStreamSynchronize(S->stream));
    for (int k = 0; k < S->nslabs; ++k) {
        st = sync_status(S->sl[k]);
        if (st != DEM_OK) return from_slab(S, k, st);
    }
    S->has_particles = true;
    S->steps = 0;
    S->migrated = 0;
    S->err.clear();
    return DEM_OK;
}

dem_status dem_slabs_step(dem_slabs* S, int64_t nsteps) {
    if (!S) return DEM_ERR_INVALID_ARG;
    if (S->broken) return sfail(S, DEM_ERR_STATE, "slabs are unusable after a CUDA error");
    if (!S->has_particles) return sfail(S, DEM_ERR_STATE, "dem_slabs_step before dem_slabs_set_particles");
    if (nsteps < 0) return sfail(S, DEM_ERR_INVALID_ARG, "nsteps < 0");
    DeviceGuard g(S->device);
    for (int64_t i = 0; i < nsteps; ++i) {
        dem_status st = slabs_one_step(S);
        if (st != DEM_OK) return st;
        ++S->steps;
    }
    SCK(S, cudaStreamSynchronize(S->stream));
    for (int k = 0; k < S->nslabs; ++k) {
        S->sl[k]->steps = S->steps;
        dem_status st = sync_status(S->sl[k]);
        if (st != DEM_OK) return from_slab(S, k, st);
    }
    return DEM_OK;
}

dem_status dem_slabs_get_state(dem_slabs* S, double* x, double* v, double* w, int where) {
    if (!S) return DEM_ERR_INVALID_ARG;
    if (S->broken) return sfail(S, DEM_ERR_STATE, "slabs are unusable after a CUDA error");
    if (!S->has_particles) return sfail(S, DEM_ERR_STATE, "no particles");
    if (where != DEM_HOST && where != DEM_DEVICE) return sfail(S, DEM_ERR_INVALID_ARG, "where");
    DeviceGuard g(S->device);
    const size_t n = S->n;
    if (n == 0) return DEM_OK;
    double *xo = x, *vo = v, *wo = w;
    if (where == DEM_HOST) {
        if (S->n > S->stage_cap) {
            if (S->stage) cudaFree(S->stage);
            if (S->stage_r) cudaFree(S->stage_r);
            S->stage = nullptr;
            S->stage_r = nullptr;
            S->stage_cap = 0;
            if (cudaMalloc(&S->stage, n * 72) != cudaSuccess || cudaMalloc(&S->stage_r, n * 4) != cudaSuccess) {
                cudaGetLastError();
                return sfail(S, DEM_ERR_OOM, "cudaMalloc(stage) failed");
            }
            S->stage_cap = S->n;
        }
        xo = x ? S->stage : nullptr;
        vo = v ? S->stage + 3 * n : nullptr;
        wo = w ? S->stage + 6 * n : nullptr;
    }
    for (int k = 0; k < S->nslabs; ++k) {
        Domain& d = S->sl[k]->d;
        if (d.n == 0) continue;
        SCK(S, run_halo_export(d, k, S->owner[S->own_cur], xo, vo, wo));
        S->launches += 1;
    }
    if (where == DEM_HOST) {
        if (x) SCK(S, cudaMemcpyAsync(x, xo, n * 24, cudaMemcpyDeviceToHost, S->stream));
        if (v) SCK(S, cudaMemcpyAsync(v, vo, n * 24, cudaMemcpyDeviceToHost, S->stream));
        if (w) SCK(S, cudaMemcpyAsync(w, wo, n * 24, cudaMemcpyDeviceToHost, S->stream));
    }
    SCK(S, cudaStreamSynchronize(S->stream));
    return DEM_OK;
}

dem_status dem_slabs_info(const dem_slabs* S, int64_t* owned, int64_t* ghosts, double* bounds, int64_t* migrated,
                          int64_t* steps) {
    if (!S) return DEM_ERR_INVALID_ARG;
    for (int k = 0; k < S->nslabs; ++k) {
        const int64_t f = S->has_particles ? S->hc_host->fill[k] : 0;
        const int64_t o = S->has_particles ? S->hc_host->owned[k] : 0;
        if (owned) owned[k] = o;
        if (ghosts) ghosts[k] = f - o;
    }
    if (bounds)
        for (int k = 0; k <= S->nslabs; ++k) bounds[k] = S->geom.zb[k];
    if (migrated) *migrated = S->migrated;
    if (steps) *steps = S->steps;
    return DEM_OK;
}

int64_t dem_slabs_launch_count(const dem_slabs* S) {
    if (!S) return 0;
    int64_t L = S->launches;
    for (dem_handle* h : S->sl) L += h->d.launches;
    return L;
}

const char* dem_slabs_last_error(const dem_slabs* S) { return S ? S->err.c_str() : "null slabs"; }

void dem_slabs_destroy(dem_slabs* S) {
    if (!S) return;
    {
        DeviceGuard g(S->device);
        if (S->stream) cudaStreamSynchronize(S->stream);
        else cudaDeviceSynchronize();
        for (auto& o : S->owner)
            if (o) cudaFree(o);
        if (S->hc) cudaFree(S->hc);
        if (S->hc_host) cudaFreeHost(S->hc_host);
        if (S->stage) cudaFree(S->stage);
        if (S->stage_r) cudaFree(S->stage_r);
        cudaGetLastError();
    }
    for (dem_handle* h : S->sl) dem_destroy(h);
    delete S;
}

}  // extern "C"
