/*
 * dem.h -- C ABI of the GB300 soft-sphere DEM timestep library (libdemgb.so).
 *
 * The library advances spherical particles by the method of Washizawa & Nakahara,
 * "Parallel Computing of Discrete Element Method on GPU": each timestep
 *   1. updates all particle properties (Sec. 4.2 step 1; semi-implicit Euler here),
 *   2. maps every particle to a cell of a uniform grid, CM (Sec. 4.1; step 2),
 *   3. sorts particles by cell, giving SCM and the permutation SCCM (Eq. 11; step 3),
 *   4. reorders every particle property into that order (step 4),
 *   5-7. evaluates the contact force of each particle against the 27 surrounding cells
 *      (Eq. 12) with the simple model (Eq. 1) or the practical model (Eqs. 2-10),
 *   8. adds particle-wall contacts (a wall is a particle of infinite radius).
 *
 * Conventions for every function:
 *  - Return a dem_status; never abort the process. On failure a message is available
 *    from dem_last_error(h). A failed call leaves the handle usable unless the status is
 *    DEM_ERR_CUDA (a CUDA error), after which only dem_destroy is valid.
 *  - Arrays passed in or out are owned by the caller. Inputs are copied; the library
 *    keeps no pointer after the call returns.
 *  - `where` says whether a pointer is host memory (DEM_HOST) or device memory on the
 *    handle's device (DEM_DEVICE). Device pointers are read or written in order on the
 *    handle's CUDA stream.
 *  - Per-particle arrays are in GLOBAL-ID order: element k belongs to particle id k.
 *    Vectors are interleaved (x0 y0 z0 x1 y1 z1 ...), SI units, double precision.
 *  - Functions that return data synchronise the handle's stream before returning.
 *    dem_step enqueues its work and synchronises once at its end to read the status word.
 *  - The library is not thread-safe per handle; distinct handles may be used from
 *    distinct threads.
 */
#ifndef DEM_GB300_H
#define DEM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DEM_OK = 0,
    DEM_ERR_INVALID_ARG = 1,  /* a pointer, size or parameter is out of range */
    DEM_ERR_OOM = 2,          /* a device or host allocation failed */
    DEM_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    DEM_ERR_CAPACITY = 4,     /* a particle had more contacts than 64 (or, for batches and
                                 slabs, than max_contacts), or a neighbour list overflowed */
    DEM_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    DEM_ERR_NONFINITE = 6,    /* a position or velocity became NaN/Inf */
    DEM_ERR_STATE = 7         /* call order: e.g. dem_step before dem_set_particles */
} dem_status;

enum { DEM_PRACTICAL = 0, DEM_SIMPLE = 1 };   /* contact model: Eqs. 2-10 or Eq. 1 */
enum { DEM_LINEAR = 0, DEM_HERTZ = 1 };       /* stiffness: constant k, or Eqs. 8-9 */
enum { DEM_FP64 = 0, DEM_FP32 = 1 };          /* precision mode, see dem_config */
enum { DEM_HOST = 0, DEM_DEVICE = 1 };
enum { DEM_PLANE = 0, DEM_CYLINDER_IN = 1, DEM_HALF_PLATE = 2 };
enum { DEM_TERM_NO_ATTRACTION = 1, DEM_TERM_ROLLING = 2, DEM_TERM_ETA_T = 4, DEM_TERM_COHESION = 8 };

/* Parameters of one scene (Sec. 3 "particle properties" and the grid of Sec. 4.1).
 *  model       DEM_PRACTICAL: F = F_t + F_n (Eq. 2), torque r_i n x F_t (Eq. 3),
 *              spring-dashpots (Eq. 4) with Coulomb cap (Eq. 5), slip velocity (Eq. 6),
 *              tangential spring history (Eq. 7), stiffness (Eqs. 8-9), damping (Eq. 10).
 *              DEM_SIMPLE: F = -k_sp delta n - k_da v - k_sh v_t (Eq. 1), no torque.
 *  stiffness   DEM_LINEAR: k_n = kn, k_t = kt. DEM_HERTZ: k = C sqrt(delta R_eff) with
 *              C = cn (normal) or ct (tangential), Eqs. 8-9.
 *  precision   DEM_FP64: every quantity and operation in FP64; contact and cell
 *              decisions are the FP64 ones of the reference formulas.
 *              DEM_FP32: velocities, spins, forces, torques and tangential springs in
 *              FP32; positions as an unevaluated sum of two FP32 numbers (compensated,
 *              about 48 significant bits); the overlap delta and the contact decision
 *              are computed with error-free transformations; cells are hashed in FP32.
 *  dt          timestep [s]; rho density [kg/m^3] (m = rho 4/3 pi r^3, I = 2/5 m r^2)
 *  g           gravitational acceleration [m/s^2], added as m g once per particle
 *  kn, kt      linear stiffnesses [N/m]; cn, ct Hertz coefficients [N/m^1.5... see Eqs. 8-9]
 *  alpha       restitution parameter of Eq. 10: eta = alpha sqrt(k_n m_eff)
 *  mu          kinetic friction coefficient of Eq. 5
 *  ksp,kda,ksh spring, damping and shear coefficients of Eq. 1
 *  skin        Verlet skin [m] (>= 0). The cell edge grows by skin.
 *  cell_size   grid cell edge [m]; 0 = 2 r_max (1 + 2^-10) + skin, r_max the largest
 *              radius passed to dem_set_particles. Must be >= that value.
 *  domain_lo/hi  box covered by the grid; particles outside use the nearest face cell.
 *  resort_interval  1 = sort by cell every step and walk the 27 cells every step
 *              (Sec. 4.2 as printed). 0 = sort (steps 2-4) only after some particle has
 *              moved skin/2 since the last sort; at each sort a neighbour list of every
 *              particle within r_i + r_j + skin is built from the 27 cells and the force
 *              pass reads it instead of walking. K > 1 = as 0, and also at least every K
 *              steps. 0 and K > 1 need skin > 0; they find exactly the same contacts.
 *              In these modes the library numbers grid cells in cubic bricks internally
 *              (the largest edge of 2, 4, 8 or 16 cells that pads the grid by at most 1/8;
 *              row-major cells when none does) and stores each window of four blocks
 *              of consecutive (cell, id) positions (at most 1,024) ordered by the
 *              particles' last contact counts, so the force kernel's warps get similar
 *              amounts of work; a list holds at most 64
 *              candidates in ascending partner id (a fuller one makes dem_step return
 *              DEM_ERR_CAPACITY), so a particle's contacts are summed in that order and
 *              results do not depend on when the sorts happened.
 *  block_size  threads per block of the force kernel (32..256); 0 = automatic (256)
 *  terms       optional force terms added to Eqs. 2-10 (none is in the paper; its force
 *              is built from separable terms so that terms can be added, Sec. 3), an OR of:
 *              DEM_TERM_NO_ATTRACTION  the normal force never pulls: F_n = 0 when
 *                                      F_n . n > 0 on i;
 *              DEM_TERM_ROLLING        rolling resistance: torque -mu_roll R_eff |F_n|
 *                                      w_rel/|w_rel| on i and its negative on j, w_rel =
 *                                      w_i - w_j (or minus the wall's angular velocity);
 *              DEM_TERM_ETA_T          eta_t = alpha_t sqrt(k_t m_eff) replaces eta in the
 *                                      tangential part of Eq. 4;
 *              DEM_TERM_COHESION       k_coh pi R_eff delta n on i, added after Eq. 5.
 *              0 = the paper's law. Any nonzero value selects a separate compiled
 *              variant of the force kernel; the paper's law runs without these terms.
 *  mu_roll     rolling resistance coefficient (DEM_TERM_ROLLING)
 *  alpha_t     tangential damping factor (DEM_TERM_ETA_T)
 *  k_coh       cohesion energy density [N/m^2] (DEM_TERM_COHESION)
 *  max_contacts  starting per-particle capacity of the contact/history list (incl.
 *              walls); 0 = 32. A step in which a particle has more contacts is voided
 *              on the device and dem_step runs it again with twice the capacity, up to
 *              64 (a handle keeps the capacity it grew to); past 64 dem_step returns
 *              DEM_ERR_CAPACITY. Batches and slabs keep max_contacts and report an
 *              overflow. Neighbour lists (resort_interval != 1) hold 64 candidates
 *              whatever max_contacts is; a fuller list makes dem_step return
 *              DEM_ERR_CAPACITY. No contact is dropped silently.
 */
typedef struct {
    int32_t model;
    int32_t stiffness;
    int32_t precision;
    int32_t resort_interval;
    double dt, rho, g[3];
    double kn, kt, cn, ct, alpha, mu;
    double ksp, kda, ksh;
    double skin, cell_size;
    double domain_lo[3], domain_hi[3];
    int32_t block_size;
    int32_t max_contacts;
    int32_t terms;
    int32_t pad;
    double mu_roll;
    double alpha_t;
    double k_coh;
} dem_config;

/* A wall (Sec. 4.2 step 8): a body of infinite radius and mass.
 *  DEM_PLANE        plane through p with unit normal n pointing INTO the domain;
 *                   a sphere touches it when its centre is closer than r.
 *  DEM_CYLINDER_IN  inside of a cylinder of the given radius whose axis passes through
 *                   p along the unit vector n (in DEM_FP32 mode n must be a coordinate
 *                   axis); a sphere touches it when its centre is farther than
 *                   radius - r from the axis.
 *  DEM_HALF_PLATE   a plate of zero thickness: the half-plane through p with unit normal
 *                   n on the side (y - p) . u >= 0 of its edge line (the line through p
 *                   along n x u; u a unit vector orthogonal to n). Touched from either
 *                   side: a sphere touches the nearest plate point (the projection of its
 *                   centre, or the edge point beside it when the projection falls off the
 *                   plate) when that point is closer than r. Two half-plates with opposite
 *                   u make a plate with a slit: the paper's benchmark drains a box through
 *                   a slit in its bottom onto a floor (Sec. 5; the geometry is not given).
 *                   In DEM_FP32 mode n and u must be coordinate axes. radius is unused.
 *  omega, vel       the wall surface moves with velocity vel + omega x (c - p) at a
 *                   point c; this velocity replaces the partner's in Eq. 6.
 */
typedef struct {
    int32_t kind;
    int32_t pad;
    double p[3], n[3];
    double radius;
    double omega[3], vel[3];
    double u[3];
} dem_wall;

typedef struct dem_handle dem_handle;

/* Creates a handle on CUDA device `device` whose work runs on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). Validates cfg. */
dem_status dem_create(const dem_config* cfg, int device, void* cuda_stream, dem_handle** out);

/* Sets n particles (Sec. 3 particle properties): positions x, velocities v, spins w
 * (3n doubles each, id order) and radii r (n floats, > 0). id must be NULL: particle k
 * has global id k. Clears the tangential history. Allocates device memory as needed
 * and performs the first cell sort (steps 2-4). n may be 0. The arrays are checked on
 * the device, host and device inputs alike (host inputs after their upload):
 * DEM_ERR_INVALID_ARG for a radius that is not finite and > 0 or a non-finite x, v or w,
 * and the handle then holds no particles. */
dem_status dem_set_particles(dem_handle* h, int64_t n, const uint32_t* id, const double* x, const double* v,
                             const double* w, const float* r, int where);

/* Replaces the walls (at most 8). Keeps particle state; clears wall histories. */
dem_status dem_set_walls(dem_handle* h, int nwalls, const dem_wall* walls);

/* Advances nsteps timesteps (each: forces of steps 5-8 at the current state, update of
 * step 1, then steps 2-4 for the new positions). A step that overflows the contact
 * capacity is voided and run again with the capacity doubled (see max_contacts); if 64
 * contacts are still too few, DEM_ERR_CAPACITY is returned with the state from before
 * that step. Other errors raised on the device (DEM_ERR_NONFINITE, a full neighbour
 * list) are returned with the state reached at the end of the call. */
dem_status dem_step(dem_handle* h, int64_t nsteps);

/* Runs until the particles come to rest: the paper continues its benchmark until every
 * particle moves less than a set amount (Sec. 5). Steps in chunks of check_every (>= 1)
 * through dem_step; after each chunk reads the largest displacement of any particle in
 * the chunk's last step, max |v'| dt (FP32 in DEM_FP32 mode), and stops when it is below
 * disp_threshold or when max_steps (>= 0) steps have run. Outputs (any may be NULL):
 * steps_done, last_max_disp (the displacement read after the last chunk, 0 when no step
 * ran) and settled (1 if the threshold was met). Errors as dem_step. */
dem_status dem_run_until(dem_handle* h, int64_t max_steps, double disp_threshold, int64_t check_every,
                         int64_t* steps_done, double* last_max_disp, int* settled);

/* Copies the current state out in id order (any pointer may be NULL to skip it). */
dem_status dem_get_state(dem_handle* h, double* x, double* v, double* w, int where);

/* Evaluates the force and torque on every particle at the current state (steps 5-8 and
 * gravity) without advancing time; 3n doubles each in id order (NULL skips). The
 * contact pairs found are kept for dem_debug_snapshot. */
dem_status dem_get_forces(dem_handle* h, double* F, double* T, int where);

/* Tangential springs currently stored, one record per contact: particle pairs as
 * (i, j) with i < j and the spring seen from i (n from i to j, v = v_i - v_j); wall
 * contacts as (i, 0xFFFFFF00 + wall index). Records are sorted by (i, j). Host memory.
 * *n receives the number of records; at most cap are written. */
dem_status dem_get_history(dem_handle* h, int64_t cap, uint32_t* i, uint32_t* j, double* d, int64_t* n);

/* Restores a state and its tangential springs (records as returned by dem_get_history,
 * host memory). Equivalent to dem_set_particles followed by setting the springs; a
 * restored run continues exactly as the saved one would have. */
dem_status dem_restore(dem_handle* h, int64_t n, const double* x, const double* v, const double* w, const float* r,
                       int64_t nrec, const uint32_t* i, const uint32_t* j, const double* d);

/* Diagnostics of the current state, reduced in FP64 in a fixed order (host array of 16):
 * [0] translational KE, [1] rotational KE, [2..4] linear momentum, [5..7] angular
 * momentum about the origin (m x cross v + I w), [8] gravitational potential energy
 * (-m g.x), [9] total mass, [10] number of particle-particle contacts, [11] number of
 * particle-wall contacts, [12] largest overlap (of the last force evaluation),
 * [13] steps taken since dem_set_particles, [14] cell sorts performed,
 * [15] particles whose cell index was clamped to the grid. */
dem_status dem_get_diagnostics(dem_handle* h, double* out16);

/* Parity hooks (host memory). cell: cell key of each particle (id order) as of the last
 * sort; order: particle ids in (cell, id) order (SCCM of Eq. 11); pairs: the contact
 * pairs (i < j, sorted) of the last dem_get_forces call, 2 per pair, at most pair_cap
 * pairs written; *npairs receives the count. Any output pointer may be NULL. */
dem_status dem_debug_snapshot(dem_handle* h, uint32_t* cell, uint32_t* order, int64_t pair_cap, uint32_t* pairs,
                              int64_t* npairs);

/* The grid in use: origin (3), cell edge, and cells per axis (3). */
dem_status dem_get_grid(const dem_handle* h, double* origin, double* cell, int64_t* dims);

/* Phase timing. While enabled, dem_step records a CUDA event pair around every force
 * pass (steps 5-8, 1 and the new cell map of step 2) and every cell sort (steps 3-4) on
 * the handle's stream; the device times are accumulated when dem_step synchronises.
 * dem_set_timing(h, 1) also clears the totals. out4: [0] force-pass milliseconds,
 * [1] sort milliseconds, [2] force passes timed, [3] sorts timed. */
dem_status dem_set_timing(dem_handle* h, int enable);
dem_status dem_get_phase_times(const dem_handle* h, double* out4);

/* ------------------------------------------------------------------------------ batches
 * Many independent scenes advanced together: their particles are packed end to end in
 * one domain and every kernel launch of a timestep (the force pass and the cell sort of
 * Sec. 4.2) covers all of them; each particle reads its own scene's parameters, grid and
 * walls. Scenes differ in size, dt, mu, alpha, walls and grid, but share precision,
 * model and stiffness law. A scene's result does not depend on the other scenes in the
 * batch. The first scene added sets the batch's sort policy (its resort_interval): either
 * every scene sorts every step (1), or every scene keeps neighbour lists with its own skin
 * and the whole batch sorts when a particle of any scene has moved half its scene's skin
 * (0), or also every K steps (K > 1); later scenes must have the same resort_interval.
 * In list mode a scene's results are still those of its own run, bit for bit, because
 * they do not depend on when sorts happen. */
typedef struct dem_batch dem_batch;

/* Creates an empty batch on `device` / `cuda_stream` (a non-legacy stream lets the step
 * be replayed as a CUDA graph). max_contacts and block_size as in dem_config. */
dem_status dem_batch_create(int precision, int model, int stiffness, int max_contacts, int block_size, int device,
                            void* cuda_stream, dem_batch** out);

/* Stages a scene (host arrays, id order, as dem_set_particles; walls as dem_set_walls)
 * that enters the batch at the next dem_batch_run and advances step_budget steps of its
 * own dt. *slot receives its identifier. */
dem_status dem_batch_add(dem_batch* b, const dem_config* cfg, int nwalls, const dem_wall* walls, int64_t n,
                         const double* x, const double* v, const double* w, const float* r, int64_t step_budget,
                         int* slot);

/* Advances the scenes that have steps left by up to max_steps steps, returning early
 * when some scene reaches its budget; the slots that finished during this call are
 * written to finished (at most cap; *nfinished receives the count). Scenes added or
 * removed since the last call are packed in first (kept scenes keep state and springs). */
dem_status dem_batch_run(dem_batch* b, int64_t max_steps, int* finished, int cap, int* nfinished);

/* Current state of one scene, id order (any pointer may be NULL). */
dem_status dem_batch_get_state(dem_batch* b, int slot, double* x, double* v, double* w, int where);

/* Removes a scene (it leaves the domain at the next dem_batch_run). */
dem_status dem_batch_remove(dem_batch* b, int slot);

/* Particle count, steps done and step budget of a scene. */
dem_status dem_batch_info(const dem_batch* b, int slot, int64_t* n, int64_t* steps_done, int64_t* budget);

int64_t dem_batch_device_bytes(const dem_batch* b);
int64_t dem_batch_launch_count(const dem_batch* b);
const char* dem_batch_last_error(const dem_batch* b);
void dem_batch_destroy(dem_batch* b);

/* Largest sizes dem_sort_cells_static accepts (its scratch is a fixed array). */
#define DEM_STATIC_SORT_MAX_N 262144
#define DEM_STATIC_SORT_MAX_CELLS 1048576

/* Cell map and (cell, id) sort of n positions WITHOUT allocating device memory; the
 * paper has no counterpart: it is for callers that cannot call cudaMalloc, such as a
 * process that has already reserved all of the GPU's memory for its own pool, or a
 * loop that forbids allocation after start-up because cudaMalloc/cudaFree can block or
 * synchronise the device. The result is the one a handle computes in DEM_FP64 mode:
 *   x          device, 3n doubles, particle k's position (id order)
 *   origin, cell, dims   host: grid origin (3), cell edge, cells per axis (3)
 *   cell_of    device out, n: cell key (k*ny + j)*nx + i of each particle (clamped)
 *   order      device out, n: particle ids in (cell, id) order
 *   cell_start device out, nx*ny*nz + 1: cell c holds order[cell_start[c] .. cell_start[c+1]-1]
 *   cuda_stream  stream of the work (NULL = legacy default stream); the call returns
 *              once the work is enqueued, on the calling thread's current device.
 * The caller owns all buffers. Temporary storage is one fixed array of about 6 MB in the
 * library's device memory, present on every GPU that loads the library until the
 * process exits; n > DEM_STATIC_SORT_MAX_N or more than DEM_STATIC_SORT_MAX_CELLS cells
 * returns DEM_ERR_INVALID_ARG. The first call on a device looks up that array's device
 * address and keeps it for the life of the process (so make the first call before any
 * stream capture; a device reset while the library is loaded is not supported). All
 * calls share the array: calls whose work overlaps on the GPU race and give wrong results.
 * The place of a particle within its cell is found by comparing it with every cell-mate,
 * so the time grows with the square of the cells' occupancy: a cell edge near the largest
 * diameter keeps it to a few particles per cell, while a grid of a single cell holding
 * the maximum of 262,144 particles takes seconds. */
dem_status dem_sort_cells_static(int64_t n, const double* x, const double* origin, double cell, const int64_t* dims,
                                 uint32_t* cell_of, uint32_t* order, uint32_t* cell_start, void* cuda_stream);

/* ------------------------------------------------------------------------------------
 * Slab decomposition with halo exchange (sub-domains of one scene on one device).
 *
 * The scene is cut along one axis into nslabs slabs (sub-domains) at the boundaries
 * bounds[1..nslabs-1] (bounds[0] = -inf, bounds[nslabs] = +inf). Each slab has its own
 * particle buffers and cell table on the scene's global grid (Sec. 4.1). A particle is
 * OWNED by the slab whose range [bounds[s], bounds[s+1]) holds its coordinate along the
 * axis and is a GHOST of every other slab within one cell edge h of its range. Because
 * a contact needs a distance below r_i + r_j <= 2 r_max < h, every contact partner of an
 * owned particle is present in its slab, and the 27-cell walk of Eq. 12 meets them in the
 * (cell, id) order of Eq. 11 of the undivided scene: owned particles get the same bits
 * as a dem_handle with the same configuration.
 * A step: the force pass of every slab (steps 5-8 and 1 of Sec. 4.2; the ghosts' own
 * results are discarded), one exchange launch that sends every owned particle with its
 * tangential springs (Eq. 7) to the slab that owns its new position (migration) and a
 * ghost copy to each slab whose ghost layer holds it (halo exchange), then the cell sort
 * (steps 2-4) of every slab. In a run over several devices the exchange is the step
 * that would cross devices; here the slabs share one device and one stream.
 * Only the walk mode runs this way (dem_config.resort_interval must be 1). Each slab's
 * buffers hold up to n particles, so no exchange can overflow. The exchange reads its
 * counts back to the host every step (the slabs' particle counts set the launches of
 * the sort), so dem_slabs_step synchronises the stream once per step.
 * ------------------------------------------------------------------------------------ */
typedef struct dem_slabs dem_slabs;

#define DEM_MAX_SLABS 8

/* Boundaries that split n coordinates z (host) into nslabs slabs of nearly equal counts:
 * bounds (nslabs + 1 doubles, out) = -inf, the (k n / nslabs)-th smallest z for
 * k = 1 .. nslabs - 1, +inf. Host only (no GPU needed). DEM_ERR_INVALID_ARG for nslabs
 * outside [1, DEM_MAX_SLABS], n < 0, a NULL pointer or a non-finite z. */
dem_status dem_slab_bounds(int64_t n, const double* z, int nslabs, double* bounds);

/* Slabs of one scene: cfg as for dem_create (resort_interval must be 1); axis 0, 1 or 2,
 * or -1 for the axis along which the configured domain is longest (the last of equal
 * ones). The slabs share the device and the stream. */
dem_status dem_slabs_create(const dem_config* cfg, int nslabs, int axis, int device, void* cuda_stream,
                            dem_slabs** out);

/* Walls of the scene, given to every slab (as dem_set_walls). */
dem_status dem_slabs_set_walls(dem_slabs* s, int nwalls, const dem_wall* walls);

/* Particles of the scene (as dem_set_particles, particle k has id k, n at most
 * 0x7FFFFF00 / DEM_MAX_SLABS): the boundaries
 * are chosen by dem_slab_bounds over the coordinates along the axis, every particle goes
 * to its owning slab and to the ghost layers that hold it, and every slab sorts. */
dem_status dem_slabs_set_particles(dem_slabs* s, int64_t n, const double* x, const double* v, const double* w,
                                   const float* r, int where);

/* nsteps steps of the whole scene (force passes, exchange, sorts); returns once they are
 * done. DEM_ERR_CAPACITY / DEM_ERR_NONFINITE as dem_step, from any slab. */
dem_status dem_slabs_step(dem_slabs* s, int64_t nsteps);

/* State of every particle, from its owning slab, at 3 * id (as dem_get_state). */
dem_status dem_slabs_get_state(dem_slabs* s, double* x, double* v, double* w, int where);

/* After the last exchange (or the first distribution): owned[k] and ghosts[k] particles
 * of slab k (nslabs entries each), the boundaries (nslabs + 1), the owned particles that
 * changed slab summed over all steps, and the steps done. Any pointer may be NULL. */
dem_status dem_slabs_info(const dem_slabs* s, int64_t* owned, int64_t* ghosts, double* bounds, int64_t* migrated,
                          int64_t* steps);

/* Kernel launches enqueued so far by all slabs and the exchange. */
int64_t dem_slabs_launch_count(const dem_slabs* s);

/* Last error message ("" if none). */
const char* dem_slabs_last_error(const dem_slabs* s);

/* Frees the slabs and their device memory. NULL is allowed. */
void dem_slabs_destroy(dem_slabs* s);

/* Bytes of device memory held by the handle. */
int64_t dem_device_bytes(const dem_handle* h);

/* Largest number of contacts (particles and walls) of any one particle in the last
 * step, as read at the end of the last dem_step (at most the handle's capacity, which
 * dem_step grows up to 64 as needed). */
int64_t dem_max_contacts_seen(const dem_handle* h);

/* Number of kernel launches the handle has enqueued so far (kernels that a replayed step
 * graph ran conditionally are counted from a device-side counter: the call synchronises
 * the handle's stream). */
int64_t dem_launch_count(const dem_handle* h);

/* Last error message of the handle ("" if none). Valid until the next call on h. */
const char* dem_last_error(const dem_handle* h);

/* Frees the handle and its device memory. NULL is allowed. */
void dem_destroy(dem_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* DEM_GB300_H */
