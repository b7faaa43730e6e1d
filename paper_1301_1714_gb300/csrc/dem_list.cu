// List mode (re-sort only after some particle moved skin/2): the force pass over the
// neighbour lists built at each sort (the lists themselves: dem_nlist.cu).
//
//   k_list   steps 5-8 and 1 for one thread per stored particle. Phase 1 keeps the list
//            entries that pass the contact prefilter as a 64-bit mask; phase 2 runs the
//            lanes of a warp in lockstep over their masks (contact decision, Eq. 1 or
//            Eqs. 2-10, the spring); then the walls the last sort found within reach
//            (step 8), gravity, the update (step 1) and the displacement test that
//            decides whether this step ends with a sort.
//
// Every particle evaluates all of its contacts (each pair twice, once from each side, with
// arithmetic that makes the two results exact negatives), so a step is one pass with no
// exchange between particles; springs are stored per particle, keyed by partner id. No
// floating-point atomics: a particle's sums run in list order (ascending partner id), so
// results depend neither on the block size nor on when the sorts happened.
#include <algorithm>

#include <cuda_runtime.h>

#include "dem_domain.h"
#include "dem_policy.cuh"

// Minimum resident 256-thread blocks per SM of the list-mode force kernel: 4 caps it at 64
// registers (measured on GB300, 4,194,304-sphere drum: 0.71 ms per pass at 64 registers,
// 0.85 ms at 85; the kernel is bound by memory latency, so occupancy wins).
#ifndef DEM_LIST_MIN_BLOCKS
#define DEM_LIST_MIN_BLOCKS 4
#endif



namespace demgb {

template <class PR>
struct ListArgs {
    using T = typename PR::T;
    const SceneDev* scenes;
    int nscenes;
    uint32_t n, cap;
    int maxc, stiffness;
    typename PR::State S0, S1;   // the two state sets; ctrl->cur names the current one
    CtrlDev* ctrl;
    const uint32_t* ncnt;        // list lengths
    const uint32_t* nl;          // list entries (stored index), slot-major
    const float4* ref;           // positions at the last sort
    int interval;                // sort at least every `interval` steps (0: never forced)
    const uint32_t* perm;
    const uint32_t* wmask;       // walls each particle can reach until the next sort
    const uint32_t* hin_cnt;     // springs read
    const uint32_t* hin_pid;
    const T* hin_d;
    uint32_t* hout_cnt;          // springs written
    uint32_t* hout_pid;
    T* hout_d;
    StatusDev* st;
    double* dbgF;
    double* dbgT;
    int halt;                    // 1: a capacity overflow makes the step void (DEM_HALT)
};

// ------------------------------------------------------------------- force pass

// MODEL: 0 the practical law, 1 the simple law (Eq. 1), 2 the practical law with the
// scene's optional terms. EVAL: forces and torques by id instead of the update.
template <class PR, int MODEL, bool EVAL>
__global__ void __launch_bounds__(256, DEM_LIST_MIN_BLOCKS) k_list(ListArgs<PR> a) {
    using T = typename PR::T;
    constexpr bool PRACT = MODEL != 1;
    constexpr bool TERMS = MODEL == 2;
    const unsigned full = 0xffffffffu;
    extern __shared__ uint32_t smem[];
    // a void step (an earlier launch overflowed): nothing to do; one decision per warp
    if (!EVAL && __any_sync(full, (a.ctrl->rebuild & DEM_HALT) != 0)) return;
    const int cur = a.ctrl->cur;
    const typename PR::State A = cur ? a.S1 : a.S0;
    const typename PR::State B = cur ? a.S0 : a.S1;
    const bool pv = a.ctrl->perm_valid != 0;
    if (!EVAL && blockIdx.x == 0 && threadIdx.x == 0 && a.interval > 0 && a.ctrl->since + 1 >= a.interval)
        atomicOr(&a.ctrl->rebuild, 1);
    const uint32_t tid = threadIdx.x, bd = blockDim.x, lane = tid & 31u;
    const uint32_t maxc = (uint32_t)a.maxc;
    uint32_t* s_oid = smem;   // [maxc][bd] partner ids of each particle's stored springs
    const uint32_t q = blockIdx.x * bd + tid;
    const size_t cap = a.cap;
    uint32_t c_pp = 0, c_wc = 0, c_clamp = 0, c_nnew = 0;
    float c_maxov = 0.f, c_disp2 = 0.f;
    const bool valid = q < a.n;
    const int sidx = valid ? scene_of(a.scenes, a.nscenes, q) : 0;
    const SceneDev& S = a.scenes[sidx];
    const bool live = valid && S.active;
    uint32_t src = 0, cnt_old = 0, m = 0;
    if (valid) {
        src = pv ? __ldg(&a.perm[q]) : q;
        if (live) m = min(__ldg(&a.ncnt[q]), (uint32_t)DEM_LIST_CAP);
        if (PRACT || !S.active) cnt_old = min(__ldg(&a.hin_cnt[src]), maxc);
        // the list and the stored springs stream from DRAM: start every line fill now, so
        // that the loads below do not wait for them one after another
        for (uint32_t k = 0; k < m; ++k) prefetch_l1(&a.nl[k * cap + q]);
        for (uint32_t k = 0; k < cnt_old; ++k) prefetch_l1(&a.hin_pid[k * cap + src]);
        for (uint32_t k = 0; k < cnt_old; ++k)
            for (int c = 0; c < 3; ++c) prefetch_l1(&a.hin_d[(c * (size_t)maxc + k) * cap + src]);
    }
    // ---- phase 1: list entries that pass the prefilter
    uint64_t near_mask = 0;
    if (live) near_mask = PR::scan_list(A, PR::load(A, q), S, a.nl, m, cap, q);
    for (uint32_t k = 0; k < cnt_old; ++k) s_oid[k * bd + tid] = __ldg(&a.hin_pid[k * cap + src]);
    __syncwarp();
    if (valid && !live) {
        // frozen scene: carry state and springs unchanged
        if (!EVAL) {
            PR::store(B, q, PR::load(A, q));
            for (uint32_t k = 0; k < cnt_old; ++k) {
                a.hout_pid[k * cap + q] = s_oid[k * bd + tid];
                for (int c = 0; c < 3; ++c)
                    a.hout_d[(c * (size_t)maxc + k) * cap + q] = a.hin_d[(c * (size_t)maxc + k) * cap + src];
            }
            a.hout_cnt[q] = cnt_old;
        } else {
            a.hout_cnt[q] = 0;
        }
    }
    // ---- phase 2: the lanes of a warp in lockstep over their near candidates
    T mi = T(0);
    V3<T> F = mk(T(0), T(0), T(0)), Tq = mk(T(0), T(0), T(0));
    uint32_t nnew = 0;
    {
        const uint32_t nnear = (uint32_t)__popcll(near_mask);
        const uint32_t kmax = __reduce_max_sync(full, nnear);
        typename PR::Self me{};
        Law<T> L{};
        if (live) {
            me = PR::load(A, q);
            L = law_of(S, a.stiffness, T());
            mi = PR::mass(S, me.r);
        }
        const T ri = (T)me.r;
        for (uint32_t k = 0; k < kmax; ++k) {
            if (!(live && k < nnear)) continue;
            const int e = __ffsll((long long)near_mask) - 1;
            near_mask &= near_mask - 1;
            const uint32_t j = __ldg(&a.nl[(size_t)e * cap + q]);
            V3<T> n;
            T delta;
            float rj;
            const typename PR::Partner pj = PR::load_partner(A, j);
            if (!PR::exact_p(A, pj, me, n, delta, rj)) continue;
            const uint32_t gid = pj.id;
            V3<T> vj, wj;
            PR::partner_vw(pj, vj, wj);
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
    }
    if (live) {
        const typename PR::Self me = PR::load(A, q);
        const Law<T> L = law_of(S, a.stiffness, T());
        const T ri = (T)me.r;
        // ---- walls (step 8), those the last sort found within reach
        for (uint32_t wm = __ldg(&a.wmask[q]); wm; wm &= wm - 1) {
            const int w = __ffs(wm) - 1;
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
            PR::integrate(B, q, me, F, Tq, S, mi, clamped, finite, pnew);
            if (!finite) raise_status(a.st, ST_NONFINITE, (int32_t)q);
            c_clamp = clamped ? 1u : 0u;
            c_disp2 = pnew.w;
            // a particle that moved skin/2 (less the FP32 margin) since the last sort makes
            // this step end with a sort and new lists
            const float4 r0 = __ldg(&a.ref[q]);
            const float ex = pnew.x - r0.x, ey = pnew.y - r0.y, ez = pnew.z - r0.z;
            if (ex * ex + ey * ey + ez * ez > S.thresh2_f || !finite) atomicOr(&a.ctrl->rebuild, 1);
        }
    }
    // warp-aggregated counters (every lane reaches this point)
    const uint32_t s_pp = __reduce_add_sync(full, c_pp);
    const uint32_t s_wc = __reduce_add_sync(full, c_wc);
    const uint32_t s_cl = __reduce_add_sync(full, c_clamp);
    const uint32_t s_mx = __reduce_max_sync(full, c_nnew);
    const uint32_t s_ov = __reduce_max_sync(full, __float_as_uint(c_maxov));
    const uint32_t s_dp = __reduce_max_sync(full, __float_as_uint(c_disp2));
    if (lane == 0) {
        if (s_pp) atomicAdd(&a.st->live.ncontacts, s_pp);
        if (s_wc) atomicAdd(&a.st->live.nwallc, s_wc);
        if (s_cl) atomicAdd(&a.st->live.clamped, s_cl);
        if (s_mx) atomicMax(&a.st->live.max_nnew, s_mx);
        if (s_ov) atomicMax(&a.st->live.max_overlap_bits, s_ov);
        if (s_dp) atomicMax(&a.st->live.max_disp2_bits, s_dp);
    }
}

// ======================================================================= launchers
static inline uint32_t nblk(uint32_t n, uint32_t b) { return (n + b - 1) / b; }

#define DEM_LAUNCH_CHECK()                          \
    do {                                            \
        ++d.launches;                               \
        cudaError_t e_ = cudaGetLastError();        \
        if (e_ != cudaSuccess) return e_;           \
    } while (0)

template <class PR>
static cudaError_t force_list_impl(Domain& d, const typename PR::State& S0, const typename PR::State& S1, bool eval,
                                   double* dbgF, double* dbgT) {
    using T = typename PR::T;
    ListArgs<PR> a;
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
    a.interval = d.interval;
    a.perm = d.perm;
    a.wmask = d.wmask;
    const int hi = d.h_cur, ho = 1 - d.h_cur;
    a.hin_cnt = d.hcnt[hi];
    a.hin_pid = d.hpid[hi];
    a.hin_d = (const T*)d.hd[hi];
    a.hout_cnt = d.hcnt[ho];
    a.hout_pid = d.hpid[ho];
    a.hout_d = (T*)d.hd[ho];
    a.st = d.st;
    a.dbgF = dbgF;
    a.dbgT = dbgT;
    a.halt = d.regrow;
    const uint32_t b = (uint32_t)d.block;
    const size_t smem = (size_t)d.maxc * b * sizeof(uint32_t);
    const int model = d.model != 0 ? 1 : (d.terms != 0 ? 2 : 0);
    auto launch = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<nblk(d.n, b), b, smem, d.stream>>>(a);
        return cudaSuccess;
    };
    cudaError_t e;
    if (model == 0) e = eval ? launch(k_list<PR, 0, true>) : launch(k_list<PR, 0, false>);
    else if (model == 2) e = eval ? launch(k_list<PR, 2, true>) : launch(k_list<PR, 2, false>);
    else e = eval ? launch(k_list<PR, 1, true>) : launch(k_list<PR, 1, false>);
    if (e != cudaSuccess) return e;
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_force_list(Domain& d, bool eval, double* dbgF, double* dbgT) {
    if (d.n == 0) return cudaSuccess;
    if (d.precision == 0) return force_list_impl<PF64>(d, d.S64[0], d.S64[1], eval, dbgF, dbgT);
    return force_list_impl<PF32>(d, d.S32[0], d.S32[1], eval, dbgF, dbgT);
}

}  // namespace demgb
