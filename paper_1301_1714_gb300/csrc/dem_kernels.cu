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
//   (list mode: the neighbour lists and the pair-once force pass are in dem_list.cu)
//   k_end_step   per-step bookkeeping of the device-side step control
//   k_import / k_export / k_diag* / k_hist_canon / k_repack   set-up, read-out,
//                diagnostics, batch repacking
#include <algorithm>

#include <cuda_runtime.h>

#include "dem_domain.h"
#include "dem_policy.cuh"

// Minimum resident 256-thread blocks per SM requested for the force kernel, which caps
// its registers at 65536 / (256 * value): 64 registers in both modes (measured on
// GB300: the list-mode pass is 11% faster at 64 than at 80; the walk-mode pass, once it
// stopped prefetching its candidates' payload, 10% faster; 48 spills and is 19% slower).
#ifndef DEM_FORCE_MIN_BLOCKS
#define DEM_FORCE_MIN_BLOCKS 4
#endif

// List mode orders windows of DEM_WINDOW_MULT force blocks (at most 1,024 positions) by
// contact count. Measured on GB300, 4,194,304-sphere drum, block 128, step with its share
// of the sorts: 0.741 / 0.724 / 0.719 / 0.720 ms for 1 / 2 / 4 / 8 blocks per window
// (narrower contact counts per warp against a longer window sort).
#ifndef DEM_WINDOW_MULT
#define DEM_WINDOW_MULT 4
#endif

namespace demgb {

// ======================================================================= force pass
template <class PR>
struct ForceArgs {
    const SceneDev* scenes;
    int nscenes;
    uint32_t n, cap;
    int maxc, stiffness;
    typename PR::State S0, S1;   // the two state sets; ctrl->cur names the current one
    CtrlDev* ctrl;
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
    int halt;                    // 1: a capacity overflow makes the step void (DEM_HALT)
};


// One thread per cell-sorted particle. Phase 1 walks the 27 cells (Eq. 12) as 9 rows of
// three x-adjacent cells and keeps the candidates that may touch in a per-thread list in
// shared memory; phase 2 runs the lanes of a warp in lockstep over their lists (the warp
// iterates max-list-length times instead of once per candidate), taking the contact
// decision, the law (Eq. 1 or Eqs. 2-10) and the springs; then walls, gravity, the
// update (step 1) and the new cell key with its rank in the cell (step 2).
// MODEL: 0 the practical law, 1 the simple law (Eq. 1), 2 the practical law with the
// scene's optional terms (no attraction, rolling resistance).
template <class PR, int MODEL, bool EVAL>
__global__ void __launch_bounds__(256, DEM_FORCE_MIN_BLOCKS) k_force(ForceArgs<PR> a) {
    using T = typename PR::T;
    constexpr bool PRACT = MODEL != 1;
    constexpr bool TERMS = MODEL == 2;
    extern __shared__ uint32_t smem[];
    // a void step (an earlier launch overflowed): nothing to do; one decision per warp
    if (!EVAL && __any_sync(0xffffffffu, (a.ctrl->rebuild & DEM_HALT) != 0)) return;
    const int cur = a.ctrl->cur;
    const typename PR::State A = cur ? a.S1 : a.S0;
    const typename PR::State B = cur ? a.S0 : a.S1;
    const bool pv = a.ctrl->perm_valid != 0;
    const uint32_t tid = threadIdx.x;
    const uint32_t bd = blockDim.x;
    const uint32_t maxc = (uint32_t)a.maxc;
    uint32_t* s_oid = smem;               // [maxc][bd] partner ids of the stored springs
    uint32_t* s_near = smem + maxc * bd;  // [maxc][bd] near candidates of phase 1
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
            const uint32_t kk = a.skey[q];
            a.key[q] = kk;
            a.rank[q] = atomicAdd(&a.cnt[kk], 1u);
        } else {
            a.hout_cnt[q] = 0;
        }
    }
    // ---- phase 1: candidates that may touch. The 18 cell-start loads of the 9 rows are
    // issued together before any candidate is read.
    if (live) {
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
        if (nnear > maxc) {
            raise_status(a.st, ST_CAPACITY, (int32_t)q);
            if (!EVAL && a.halt) atomicOr(&a.ctrl->rebuild, DEM_HALT);
        }
    }
    // ---- phase 2: contacts, in lockstep over the lists
    const uint32_t mylen = min(nnear, maxc);
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
    for (uint32_t k = 0; k < kmax; ++k) {
        if (!(live && k < mylen)) continue;
        const uint32_t j = s_near[k * bd + tid];
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
        if (nnew > maxc) {
            raise_status(a.st, ST_CAPACITY, (int32_t)q);
            if (!EVAL && a.halt) atomicOr(&a.ctrl->rebuild, DEM_HALT);
        }
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
            a.key[q] = kk;
            a.rank[q] = atomicAdd(&a.cnt[kk], 1u);
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
    if (ctrl->rebuild != 1) return;   // no sort this step (or a void step)
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
    if (ctrl->rebuild != 1) return;   // no sort this step (or a void step)
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
    if (ctrl->rebuild != 1) return;   // no sort this step (or a void step)
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
    if (ctrl->rebuild != 1) return;   // no sort this step (or a void step)
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
    if (ctrl->rebuild != 1) return;   // no sort this step (or a void step)
    const int cur = ctrl->cur;
    const typename PR::State A = cur ? S1 : S0;
    const typename PR::State B = cur ? S0 : S1;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        reorder_one<PR>(s, A, B, key, cs, tmp, perm, skey, ref);
}

// List mode stores the sorted particles in (cell, id) order within windows of
// DEM_WINDOW_MULT force blocks, each window ordered by the particles' contact counts in
// the step just finished (descending; ties keep the (cell, id) order). The lanes of a warp run
// their candidate lists in lockstep, so grouping similar counts shortens the longest
// lane's loop; a particle's own sums keep their order, so results do not change.
// Three passes replace k_reorder: the (cell, id) position of every particle, its final
// position in its window, and the gather to the final position.
template <class PR>
__global__ void k_rank_cell(uint32_t n, typename PR::State S0, typename PR::State S1, const CtrlDev* ctrl,
                            const uint32_t* __restrict__ key, const uint32_t* __restrict__ cs,
                            const uint32_t* __restrict__ tmp, const uint32_t* __restrict__ hcnt_last,
                            uint32_t* __restrict__ canon, uint32_t* __restrict__ wkey) {
    if (ctrl->rebuild != 1) return;   // no sort this step (or a void step)
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

// One block per window of wsize (cell, id) positions (blockDim.x: the power of two at or
// above wsize, at most 1,024): fin[q] = final position, the window's particles in descending order of their last
// contact count (ties in (cell, id) order), so the lanes of a force-pass warp carry similar
// numbers of contacts. A window is split where one scene ends and the next begins (scenes
// are contiguous in the (cell, id) order), so every particle stays inside its scene's range
// of positions. The order is a bitonic sort in shared memory of one 32-bit word per
// position: scene run within the window (10 bits), 63 - count (6 bits), position (10 bits).
__global__ void __launch_bounds__(1024) k_window(uint32_t n, uint32_t wsize, const SceneDev* scenes, int nscenes,
                                                 const CtrlDev* ctrl, const uint32_t* __restrict__ wkey,
                                                 uint32_t* __restrict__ fin) {
    if (ctrl->rebuild != 1) return;   // no sort this step (or a void step)
    __shared__ uint32_t s_w[1024];
    const uint32_t w = blockDim.x, t = threadIdx.x;
    for (uint32_t base = blockIdx.x * wsize; base < n; base += gridDim.x * wsize) {
        const uint32_t q = base + t;
        const int sc0 = scene_of(scenes, nscenes, base);
        uint32_t word = 0xFFFFFFFFu;   // past the window or the end: sorts last
        if (t < wsize && q < n) {
            const uint32_t run = (uint32_t)(scene_of(scenes, nscenes, q) - sc0);
            word = (run << 16) | ((63u - min(wkey[q], 63u)) << 10) | t;
        }
        __syncthreads();
        s_w[t] = word;
        __syncthreads();
        for (uint32_t k = 2; k <= w; k <<= 1)
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                const uint32_t o = t ^ j;
                if (o > t) {
                    const uint32_t a = s_w[t], b = s_w[o];
                    const bool up = (t & k) == 0;
                    if ((a > b) == up) {
                        s_w[t] = b;
                        s_w[o] = a;
                    }
                }
                __syncthreads();
            }
        const uint32_t sw = s_w[t];
        if (sw != 0xFFFFFFFFu) fin[base + (sw & 1023u)] = base + t;
    }
}

template <class PR>
__global__ void k_gather(uint32_t n, typename PR::State S0, typename PR::State S1, const CtrlDev* ctrl,
                         const uint32_t* __restrict__ key, const uint32_t* __restrict__ canon,
                         const uint32_t* __restrict__ fin, uint32_t* __restrict__ perm, uint32_t* __restrict__ skey,
                         float4* __restrict__ ref) {
    if (ctrl->rebuild != 1) return;   // no sort this step (or a void step)
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

// Step bookkeeping (one thread): after a sort the current set stays and springs are read
// through the permutation next step; otherwise the next set becomes current.
__global__ void k_end_step(CtrlDev* ctrl, StatusDev* st, int walk_mode) {
    if (ctrl->rebuild & DEM_HALT) return;   // a void step changes nothing
    ctrl->steps_done += 1;
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
    if (ctrl->rebuild != 1) return;   // no sort this step (or a void step)
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

// Input check of dem_set_particles on the device (the arrays are there anyway, and a
// host loop over them costs ~20 ms per 4M particles on one core): out[0] |= 1 for a radius
// that is not finite and > 0, |= 2 for a non-finite position, velocity or spin; out[1] =
// bits of the largest radius (radii are positive, so their bits order like their values).
__global__ void __launch_bounds__(256) k_check_input(uint32_t n, const double* __restrict__ x,
                                                     const double* __restrict__ v, const double* __restrict__ w,
                                                     const float* __restrict__ r, uint32_t* out) {
    uint32_t bad = 0, rmax = 0;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const float rq = r[q];
        if (!(rq > 0.f) || !isfinite(rq)) bad |= 1u;
        else rmax = max(rmax, __float_as_uint(rq));
        for (int c = 0; c < 3; ++c) {
            const size_t o = 3 * (size_t)q + c;
            if (!isfinite(x[o]) || !isfinite(v[o]) || !isfinite(w[o])) bad |= 2u;
        }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    rmax = __reduce_max_sync(0xffffffffu, rmax);
    if ((threadIdx.x & 31u) == 0) {
        if (bad) atomicOr(&out[0], bad);
        if (rmax) atomicMax(&out[1], rmax);
    }
}

cudaError_t run_check_input(Domain& d, uint32_t n, const double* x, const double* v, const double* w, const float* r,
                            uint32_t* out) {
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(uint32_t), d.stream);
    if (e != cudaSuccess || n == 0) return e;
    k_check_input<<<sgrid(d, n), 256, 0, d.stream>>>(n, x, v, w, r, out);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

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
        const uint32_t wsz = std::min(1024u, (uint32_t)d.block * DEM_WINDOW_MULT);
        uint32_t wb = 32;
        while (wb < wsz) wb <<= 1;
        const uint32_t wg = std::max(1u, std::min(nblk(d.n, wsz), (uint32_t)std::max(d.sort_blocks, 1)));
        if (d.precision == 0)
            k_rank_cell<PF64><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.S64[0], d.S64[1], d.ctrl, d.key, d.cs,
                                                                     d.tmp, hc, d.canon, d.rank);
        else
            k_rank_cell<PF32><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.S32[0], d.S32[1], d.ctrl, d.key, d.cs,
                                                                     d.tmp, hc, d.canon, d.rank);
        DEM_LAUNCH_CHECK();
        k_window<<<wg, wb, 0, d.stream>>>(d.n, wsz, d.d_scenes, d.nscenes, d.ctrl, d.rank, d.fin);
        DEM_LAUNCH_CHECK();
        if (d.precision == 0)
            k_gather<PF64><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.S64[0], d.S64[1], d.ctrl, d.key, d.canon,
                                                                  d.fin, d.perm, d.skey, d.ref);
        else
            k_gather<PF32><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.S32[0], d.S32[1], d.ctrl, d.key, d.canon,
                                                                  d.fin, d.perm, d.skey, d.ref);
        DEM_LAUNCH_CHECK();
        cudaError_t e = run_lists(d);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Sets the condition of the step graph's sort node from the device-side decision, and
// counts the sorts that run that way (one thread).
__global__ void k_sort_cond(cudaGraphConditionalHandle h, CtrlDev* ctrl) {
    const unsigned int go = ctrl->rebuild == 1 ? 1u : 0u;
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
    a.halt = d.regrow;
    const uint32_t b = (uint32_t)d.block;
    const size_t smem = 2 * (size_t)d.maxc * b * sizeof(uint32_t);
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
    if (model == 0) e = eval ? launch(k_force<PR, 0, true>) : launch(k_force<PR, 0, false>);
    else if (model == 2) e = eval ? launch(k_force<PR, 2, true>) : launch(k_force<PR, 2, false>);
    else e = eval ? launch(k_force<PR, 1, true>) : launch(k_force<PR, 1, false>);
    if (e != cudaSuccess) return e;
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_force(Domain& d, bool eval, double* dbgF, double* dbgT) {
    if (d.n == 0) return cudaSuccess;
    if (d.list_mode) return run_force_list(d, eval, dbgF, dbgT);
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
