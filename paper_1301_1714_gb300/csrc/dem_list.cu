// List mode (re-sort only after some particle moved skin/2): neighbour lists built at a
// sort, and a force pass that evaluates every contact pair once.
//
//   k_nlist_split  at a sort: the 27 cells around each particle (Eq. 12); candidates
//                  within r_i + r_j + skin go to its owned list (higher global id) or its
//                  owner list (lower id)
//   k_nlist_link   at a sort: each owned entry learns the slot its partner reserved for it
//   k_pair         steps 5-7 once per pair: the owner (lower id) of each contact takes the
//                  contact decision and the law (Eq. 1 or Eqs. 2-10) with its tangential
//                  spring, sums its own share, and writes the partner's share (-F and the
//                  partner's torque, Eq. 3) into the partner's reserved record slot
//   k_update       per particle: its own sums, then the records it received in slot order,
//                  walls (step 8), gravity, the update (step 1) and the displacement test
//                  that decides whether the step ends with a sort
//
// No floating-point atomics: a particle's force is summed in a fixed order (owned
// contacts in list order, received records in slot order, walls, gravity), and a pair's
// law is evaluated from the side of its lower global id whatever the storage order, so
// results do not depend on block size, window order or scheduling. The only atomics are
// integer ones (the record mask bits, counters, the sort flag).
#include <algorithm>

#include <cuda_runtime.h>

#include "dem_domain.h"
#include "dem_policy.cuh"

// Minimum resident 256-thread blocks per SM of the two force-pass kernels: 3 (85 registers)
// for both (measured on GB300, 4,194,304-sphere drum: the pair pass is 6% faster at 85
// registers than at 64, which spill, and 13% faster than at 128; the update pass at 85
// registers takes 0.18 ms less than at 64 and 0.1 ms less than at 128).
#ifndef DEM_PAIR_MIN_BLOCKS
#define DEM_PAIR_MIN_BLOCKS 3
#endif
#ifndef DEM_UPDATE_MIN_BLOCKS
#define DEM_UPDATE_MIN_BLOCKS 3
#endif

namespace demgb {

// --------------------------------------------------------------- contact records
// One record per (receiving particle, slot): the force and torque a contact's owner
// computed for the partner, or (part_sum) a particle's sums over its owned contacts
// with two words of bookkeeping for k_update.
struct alignas(32) RecF {
    float4 a, b;   // (F.xyz, info0), (T.xyz, info1)
};
struct alignas(64) RecD {
    double f[3], t[3];
    uint32_t info0, info1;
};
template <class T> struct RecOf;
template <> struct RecOf<float> { using type = RecF; };
template <> struct RecOf<double> { using type = RecD; };

__device__ __forceinline__ void put_rec(RecF* p, V3<float> f, V3<float> t, uint32_t i0, uint32_t i1) {
    p->a = make_float4(f.x, f.y, f.z, __uint_as_float(i0));
    p->b = make_float4(t.x, t.y, t.z, __uint_as_float(i1));
}
__device__ __forceinline__ void get_rec(const RecF* p, V3<float>& f, V3<float>& t, uint32_t& i0, uint32_t& i1) {
    const float4 a = __ldg(&p->a), b = __ldg(&p->b);
    f = mk(a.x, a.y, a.z);
    t = mk(b.x, b.y, b.z);
    i0 = __float_as_uint(a.w);
    i1 = __float_as_uint(b.w);
}
__device__ __forceinline__ void put_rec(RecD* p, V3<double> f, V3<double> t, uint32_t i0, uint32_t i1) {
    p->f[0] = f.x; p->f[1] = f.y; p->f[2] = f.z;
    p->t[0] = t.x; p->t[1] = t.y; p->t[2] = t.z;
    p->info0 = i0;
    p->info1 = i1;
}
__device__ __forceinline__ void get_rec(const RecD* p, V3<double>& f, V3<double>& t, uint32_t& i0, uint32_t& i1) {
    f = mk(p->f[0], p->f[1], p->f[2]);
    t = mk(p->t[0], p->t[1], p->t[2]);
    i0 = p->info0;
    i1 = p->info1;
}

template <class PR>
struct ListArgs {
    using T = typename PR::T;
    using R = typename RecOf<T>::type;
    const SceneDev* scenes;
    int nscenes;
    uint32_t n, cap;
    int maxc, stiffness;
    typename PR::State S0, S1;   // the two state sets; ctrl->cur names the current one
    CtrlDev* ctrl;
    const uint32_t* ncnt;        // owned list lengths
    const uint32_t* nl;          // owned entries (index | slot << DEM_NL_SHIFT), slot-major
    const float4* ref;           // positions at the last sort
    float thresh2;               // squared displacement that forces a sort
    int interval;                // sort at least every `interval` steps (0: never forced)
    const uint32_t* perm;
    const uint32_t* hin_cnt;     // springs read (owned pairs, then walls; count = pairs | walls << 16)
    const uint32_t* hin_pid;
    const T* hin_d;
    uint32_t* hout_cnt;          // springs written
    uint32_t* hout_pid;
    T* hout_d;
    uint32_t* inmask;            // received record slots of this step
    R* rec;                      // [DEM_LIST_OWNER_CAP][cap] records for the receiving particle, slot-major
    R* part;                     // [cap] sums over owned contacts
    StatusDev* st;
    double* dbgF;
    double* dbgT;
};

// ------------------------------------------------------------------ list build
// Candidates of particle q at a sort: every particle of the 27 cells around q's cell
// (Eq. 12; in list mode cells are numbered brick by brick) within r_i + r_j + skin (+ the FP32
// margin). With cells of edge >= 2 r_max + skin no pair that comes into contact before
// some particle has moved skin/2 is missed. The test is symmetric in i and j, so q lists
// j as owned exactly when j lists q as owner.
template <class PR>
__global__ void __launch_bounds__(256) k_nlist_split(uint32_t n, const SceneDev* scenes, int nscenes,
                                                     typename PR::State S0, typename PR::State S1, const CtrlDev* ctrl,
                                                     const uint32_t* __restrict__ skey, const uint32_t* __restrict__ cs,
                                                     const uint32_t* __restrict__ fin, uint32_t* __restrict__ ncnt,
                                                     uint32_t* __restrict__ nl, uint32_t* __restrict__ ocnt,
                                                     uint32_t* __restrict__ ol, size_t cap, float skin, StatusDev* st) {
    if (!ctrl->rebuild) return;
    const typename PR::State A = ctrl->cur ? S1 : S0;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const SceneDev& S = scenes[scene_of(scenes, nscenes, q)];
        const typename PR::Self me = PR::load(A, q);
        const float extra = skin + S.eps_f;
        int ix, iy, iz;
        cell_coords(S, skey[q] - S.c0, ix, iy, iz);
        uint32_t m = 0, o = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int cx = ix + dx, cy = iy + dy, cz = iz + dz;
                    if (cx < 0 || cy < 0 || cz < 0 || cx >= S.dims[0] || cy >= S.dims[1] || cz >= S.dims[2]) continue;
                    const uint32_t c = S.c0 + cell_index(S, (uint32_t)cx, (uint32_t)cy, (uint32_t)cz);
                    const uint32_t c1 = __ldg(&cs[c + 1]);
                    for (uint32_t jc = __ldg(&cs[c]); jc < c1; ++jc) {
                        const uint32_t j = fin[jc];   // the cell table holds (cell, id) positions
                        if (j == q || !PR::within(A, me, j, extra)) continue;
                        if (__ldg(&A.id[j]) > me.id) {
                            if (m < DEM_LIST_OWNED_CAP) nl[(size_t)m * cap + q] = j;
                            ++m;
                        } else {
                            if (o < DEM_LIST_OWNER_CAP) ol[(size_t)o * cap + q] = j;
                            ++o;
                        }
                    }
                }
        if (m > DEM_LIST_OWNED_CAP || o > DEM_LIST_OWNER_CAP) raise_status(st, ST_LIST, (int32_t)q);
        ncnt[q] = min(m, (uint32_t)DEM_LIST_OWNED_CAP);
        ocnt[q] = min(o, (uint32_t)DEM_LIST_OWNER_CAP);
    }
}

// Each owned entry (q -> j) gets the slot s at which j lists q as an owner; the contact's
// record for j goes to rec[j][s] and sets bit s of j's mask.
__global__ void __launch_bounds__(256) k_nlist_link(uint32_t n, const CtrlDev* ctrl, const uint32_t* __restrict__ ncnt,
                                                    uint32_t* __restrict__ nl, const uint32_t* __restrict__ ocnt,
                                                    const uint32_t* __restrict__ ol, size_t cap, StatusDev* st) {
    if (!ctrl->rebuild) return;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const uint32_t m = ncnt[q];
        for (uint32_t e = 0; e < m; ++e) {
            const uint32_t j = nl[(size_t)e * cap + q];
            const uint32_t oc = ocnt[j];
            uint32_t s = 0;
            while (s < oc && ol[(size_t)s * cap + j] != q) ++s;
            if (s == oc) {
                // j's owner list overflowed (already reported by k_nlist_split): the entry
                // keeps slot 0 of a list that is not used, since the step reports an error
                raise_status(st, ST_LIST, (int32_t)q);
                s = 0;
            }
            nl[(size_t)e * cap + q] = j | (s << DEM_NL_SHIFT);
        }
    }
}

// ------------------------------------------------------------------- force pass
// One thread per stored particle q. Phase 1 tests every owned list entry with the
// prefilter (FP32 on hi, or the FP64 contact test) and keeps the passing entries as a
// 64-bit mask; phase 2 runs the warp's lanes in lockstep over their masks: the exact
// contact decision, the law of the pair seen from q (the lower id), q's tangential
// spring (springs are stored once per pair, on the owner's side, keyed by partner id),
// and the partner's share written to the partner's reserved record slot.
// MODEL: 0 the practical law, 1 the simple law (Eq. 1), 2 the practical law with the
// scene's optional terms.
template <class PR, int MODEL, bool EVAL>
__global__ void __launch_bounds__(256, DEM_PAIR_MIN_BLOCKS) k_pair(ListArgs<PR> a) {
    using T = typename PR::T;
    constexpr bool PRACT = MODEL != 1;
    constexpr bool TERMS = MODEL == 2;
    extern __shared__ uint32_t smem[];
    const typename PR::State A = a.ctrl->cur ? a.S1 : a.S0;
    const bool pv = a.ctrl->perm_valid != 0;
    if (!EVAL && blockIdx.x == 0 && threadIdx.x == 0 && a.interval > 0 && a.ctrl->since + 1 >= a.interval)
        atomicOr(&a.ctrl->rebuild, 1);
    const uint32_t tid = threadIdx.x;
    const uint32_t bd = blockDim.x;
    const uint32_t maxc = (uint32_t)a.maxc;
    uint32_t* s_oid = smem;   // [maxc][bd] partner ids of the stored springs
    const uint32_t q = blockIdx.x * bd + tid;
    const size_t cap = a.cap;
    uint32_t c_pp = 0;
    float c_maxov = 0.f;
    const bool valid = q < a.n;
    const SceneDev& S = a.scenes[valid ? scene_of(a.scenes, a.nscenes, q) : 0];
    const bool live = valid && S.active;
    typename PR::Self me{};
    uint32_t src = 0, hraw = 0, np_old = 0, nnear = 0;
    uint64_t near_mask = 0;
    if (valid) {
        me = PR::load(A, q);
        src = pv ? __ldg(&a.perm[q]) : q;
        if (PRACT) {
            hraw = __ldg(&a.hin_cnt[src]);
            np_old = min(hraw & 0xFFFFu, maxc);
            // the stored springs are streamed from DRAM: start their loads now so they are
            // in L1 when phase 2 matches contacts against them
            for (uint32_t k = 0; k < np_old; ++k)
                for (int c = 0; c < 3; ++c) prefetch_l1(&a.hin_d[(c * (size_t)maxc + k) * cap + src]);
            for (uint32_t k = 0; k < np_old; ++k) s_oid[k * bd + tid] = __ldg(&a.hin_pid[k * cap + src]);
        }
    }
    if (live) {
        near_mask = PR::scan_list(A, me, S, a.nl, min(__ldg(&a.ncnt[q]), (uint32_t)DEM_LIST_OWNED_CAP), cap, q);
        nnear = __popcll(near_mask);
    }
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, nnear);
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
        if (!(live && k < nnear)) continue;
        const int e = __ffsll((long long)near_mask) - 1;
        near_mask &= near_mask - 1;
        const uint32_t ent = __ldg(&a.nl[(size_t)e * cap + q]);
        const uint32_t j = ent & DEM_NL_INDEX_MASK, slot = ent >> DEM_NL_SHIFT;
        V3<T> n;
        T delta;
        float rj;
        const typename PR::Partner o = PR::load_partner(A, j);
        if (!PR::exact_p(A, o, me, n, delta, rj)) continue;
        const uint32_t gid = o.id;
        V3<T> vj, wj;
        PR::partner_vw(o, vj, wj);
        const V3<T> v = me.v - vj;
        V3<T> Fj, Tj;
        if (PRACT) {
            const T rjT = (T)rj;
            const V3<T> rw = mk(sym_madd(ri, me.w.x, rjT, wj.x), sym_madd(ri, me.w.y, rjT, wj.y),
                                sym_madd(ri, me.w.z, rjT, wj.z));
            const T mj = PR::mass(S, rj);
            const T meff = law_div(mi * mj, mi + mj);
            const T Reff = law_div(ri * rjT, ri + rjT);
            const V3<T> dold = find_spring(s_oid, bd, tid, np_old, gid, a.hin_d, (size_t)maxc, cap, src);
            V3<T> Fc, Ftc, dnew, Mr;
            law_practical<TERMS>(L, n, delta, v, rw, Reff, meff, dold, Fc, Ftc, dnew, me.w - wj, Mr);
            F = F + Fc;
            const V3<T> G = cross(n, Ftc);   // Eq. 3: T_i = r_i n x F_t and T_j = r_j n x F_t
            Tq = Tq + G * ri;
            Fj = mk(-Fc.x, -Fc.y, -Fc.z);
            Tj = G * rjT;
            if (TERMS) {
                Tq = Tq + Mr;
                Tj = Tj - Mr;
            }
            if (nnew < maxc) {
                a.hout_pid[nnew * cap + q] = gid;
                a.hout_d[(0 * (size_t)maxc + nnew) * cap + q] = dnew.x;
                a.hout_d[(1 * (size_t)maxc + nnew) * cap + q] = dnew.y;
                a.hout_d[(2 * (size_t)maxc + nnew) * cap + q] = dnew.z;
            }
        } else {
            const V3<T> Fc = law_simple(L, n, delta, v);
            F = F + Fc;
            Fj = mk(-Fc.x, -Fc.y, -Fc.z);
            Tj = mk(T(0), T(0), T(0));
            if (EVAL && nnew < maxc) a.hout_pid[nnew * cap + q] = gid;
        }
        put_rec(&a.rec[(size_t)slot * cap + j], Fj, Tj, 0u, 0u);
        atomicOr(&a.inmask[j], 1u << slot);
        ++nnew;
        c_pp += 2;   // counted from both sides, as in the walk
        c_maxov = fmaxf(c_maxov, (float)delta);
    }
    if (valid && !live && PRACT && !EVAL) {
        // frozen scene: its springs are carried unchanged (k_update carries the walls')
        for (uint32_t k = 0; k < np_old; ++k) {
            a.hout_pid[k * cap + q] = s_oid[k * bd + tid];
            for (int c = 0; c < 3; ++c)
                a.hout_d[(c * (size_t)maxc + k) * cap + q] = a.hin_d[(c * (size_t)maxc + k) * cap + src];
        }
        nnew = np_old;
    }
    if (valid) {
        if (nnew > maxc) raise_status(a.st, ST_CAPACITY, (int32_t)q);
        nnew = min(nnew, maxc);
        if (PRACT || EVAL) a.hout_cnt[q] = (EVAL && !live) ? 0u : nnew;
        put_rec(&a.part[q], F, Tq, nnew, hraw);
    }
    const unsigned full = 0xffffffffu;
    const uint32_t s_pp = __reduce_add_sync(full, c_pp);
    const uint32_t s_ov = __reduce_max_sync(full, __float_as_uint(c_maxov));
    if ((tid & 31) == 0) {
        if (s_pp) atomicAdd(&a.st->live.ncontacts, s_pp);
        if (s_ov) atomicMax(&a.st->live.max_overlap_bits, s_ov);
    }
}

// Per particle q: the sums of its owned contacts (k_pair), then the records its owners
// wrote for it in slot order, walls (step 8), gravity, and the update of Sec. 4.2 step 1
// (or, in EVAL, the force and torque by id). Wall springs follow the owned pair springs
// in q's spring list; the count word is pairs | walls << 16.
template <class PR, int MODEL, bool EVAL>
__global__ void __launch_bounds__(256, DEM_UPDATE_MIN_BLOCKS) k_update(ListArgs<PR> a) {
    using T = typename PR::T;
    constexpr bool PRACT = MODEL != 1;
    constexpr bool TERMS = MODEL == 2;
    const int cur = a.ctrl->cur;
    const typename PR::State A = cur ? a.S1 : a.S0;
    const typename PR::State B = cur ? a.S0 : a.S1;
    const bool pv = a.ctrl->perm_valid != 0;
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cap = a.cap;
    const uint32_t maxc = (uint32_t)a.maxc;
    uint32_t c_wc = 0, c_clamp = 0, c_nnew = 0;
    float c_maxov = 0.f, c_disp2 = 0.f;
    if (q < a.n) {
        const SceneDev& S = a.scenes[scene_of(a.scenes, a.nscenes, q)];
        const typename PR::Self me = PR::load(A, q);
        V3<T> F, Tq;
        uint32_t npairs, hraw;
        get_rec(&a.part[q], F, Tq, npairs, hraw);
        const uint32_t mask = __ldg(&a.inmask[q]);
        if (mask) a.inmask[q] = 0u;
        for (uint32_t m = mask; m; m &= m - 1) {
            V3<T> f, t;
            uint32_t i0, i1;
            get_rec(&a.rec[(size_t)(__ffs(m) - 1) * cap + q], f, t, i0, i1);
            F = F + f;
            Tq = Tq + t;
        }
        // old wall springs: slots [np_old, np_old + nw_old) of the particle's old list
        const uint32_t np_old = PRACT ? min(hraw & 0xFFFFu, maxc) : 0u;
        const uint32_t nw_old = PRACT ? min(hraw >> 16, maxc - np_old) : 0u;
        const uint32_t src = (nw_old > 0 && pv) ? __ldg(&a.perm[q]) : q;
        if (!S.active) {
            // frozen scene: state and wall springs carried unchanged
            if (!EVAL) {
                PR::store(B, q, me);
                if (PRACT) {
                    for (uint32_t k = 0; k < nw_old; ++k) {
                        a.hout_pid[(npairs + k) * cap + q] = a.hin_pid[(np_old + k) * cap + src];
                        for (int c = 0; c < 3; ++c)
                            a.hout_d[(c * (size_t)maxc + npairs + k) * cap + q] =
                                a.hin_d[(c * (size_t)maxc + np_old + k) * cap + src];
                    }
                    if (nw_old) a.hout_cnt[q] = npairs | (nw_old << 16);
                }
            }
        } else {
            const Law<T> L = law_of(S, a.stiffness, T());
            const T mi = PR::mass(S, me.r);
            const T ri = (T)me.r;
            uint32_t nw = 0;
            for (int w = 0; w < S.nwalls; ++w) {
                const WallDev& W = S.walls[w];
                V3<T> n, cp;
                T delta;
                if (!PR::wall(W, me, S, n, delta, cp)) continue;
                const V3<T> v = me.v - PR::wall_vel(W, cp);
                const uint32_t gid = DEM_WALL_BASE + (uint32_t)w;
                if (PRACT) {
                    V3<T> dold = mk(T(0), T(0), T(0));
                    for (uint32_t k = 0; k < nw_old; ++k)
                        if (__ldg(&a.hin_pid[(np_old + k) * cap + src]) == gid) {
                            const size_t s0 = np_old + k;
                            dold = mk(__ldg(&a.hin_d[(0 * (size_t)maxc + s0) * cap + src]),
                                      __ldg(&a.hin_d[(1 * (size_t)maxc + s0) * cap + src]),
                                      __ldg(&a.hin_d[(2 * (size_t)maxc + s0) * cap + src]));
                            break;
                        }
                    V3<T> Fc, Ftc, dnew, Mr;
                    law_practical<TERMS>(L, n, delta, v, me.w * ri, ri, mi, dold, Fc, Ftc, dnew,
                                         me.w - PR::wall_omega(W), Mr);
                    F = F + Fc;
                    Tq = Tq + cross(n, Ftc) * ri;
                    if (TERMS) Tq = Tq + Mr;
                    const uint32_t slot = npairs + nw;
                    if (slot < maxc) {
                        a.hout_pid[slot * cap + q] = gid;
                        a.hout_d[(0 * (size_t)maxc + slot) * cap + q] = dnew.x;
                        a.hout_d[(1 * (size_t)maxc + slot) * cap + q] = dnew.y;
                        a.hout_d[(2 * (size_t)maxc + slot) * cap + q] = dnew.z;
                    }
                } else {
                    F = F + law_simple(L, n, delta, v);
                }
                ++nw;
                ++c_wc;
                c_maxov = fmaxf(c_maxov, (float)delta);
            }
            const uint32_t total = npairs + (uint32_t)__popc(mask) + nw;
            if (total > maxc) raise_status(a.st, ST_CAPACITY, (int32_t)q);
            c_nnew = total;
            if (PRACT && nw) a.hout_cnt[q] = npairs | (min(nw, maxc - npairs) << 16);
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
                // a particle that moved skin/2 (less the FP32 margin) since the last sort
                // makes this step end with a sort and new lists
                const float4 r0 = __ldg(&a.ref[q]);
                const float ex = pnew.x - r0.x, ey = pnew.y - r0.y, ez = pnew.z - r0.z;
                if (ex * ex + ey * ey + ez * ez > a.thresh2 || !finite) atomicOr(&a.ctrl->rebuild, 1);
            }
        }
    }
    // warp-aggregated counters (every lane reaches this point)
    const unsigned full = 0xffffffffu;
    const uint32_t s_wc = __reduce_add_sync(full, c_wc);
    const uint32_t s_cl = __reduce_add_sync(full, c_clamp);
    const uint32_t s_mx = __reduce_max_sync(full, c_nnew);
    const uint32_t s_ov = __reduce_max_sync(full, __float_as_uint(c_maxov));
    const uint32_t s_dp = __reduce_max_sync(full, __float_as_uint(c_disp2));
    if ((threadIdx.x & 31) == 0) {
        if (s_wc) atomicAdd(&a.st->live.nwallc, s_wc);
        if (s_cl) atomicAdd(&a.st->live.clamped, s_cl);
        if (s_mx) atomicMax(&a.st->live.max_nnew, s_mx);
        if (s_ov) atomicMax(&a.st->live.max_overlap_bits, s_ov);
        if (s_dp) atomicMax(&a.st->live.max_disp2_bits, s_dp);
    }
}

// ======================================================================= launchers
static inline uint32_t nblk(uint32_t n, uint32_t b) { return (n + b - 1) / b; }
static inline uint32_t sgrid(const Domain& d, uint32_t n) {
    return std::max(1u, std::min(nblk(n, 256), (uint32_t)std::max(d.sort_blocks, 1)));
}

#define DEM_LAUNCH_CHECK()                          \
    do {                                            \
        ++d.launches;                               \
        cudaError_t e_ = cudaGetLastError();        \
        if (e_ != cudaSuccess) return e_;           \
    } while (0)

size_t list_record_bytes(const Domain& d) { return d.precision == 0 ? sizeof(RecD) : sizeof(RecF); }

template <class PR>
static cudaError_t lists_impl(Domain& d, const typename PR::State& S0, const typename PR::State& S1) {
    k_nlist_split<PR><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.d_scenes, d.nscenes, S0, S1, d.ctrl, d.skey, d.cs,
                                                           d.fin, d.ncnt, d.nl, d.ocnt, d.ol, d.cap, d.skin_f, d.st);
    DEM_LAUNCH_CHECK();
    k_nlist_link<<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.ctrl, d.ncnt, d.nl, d.ocnt, d.ol, d.cap, d.st);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_lists(Domain& d) {
    if (d.n == 0) return cudaSuccess;
    if (d.precision == 0) return lists_impl<PF64>(d, d.S64[0], d.S64[1]);
    return lists_impl<PF32>(d, d.S32[0], d.S32[1]);
}

template <class PR>
static cudaError_t force_list_impl(Domain& d, const typename PR::State& S0, const typename PR::State& S1, bool eval,
                                   double* dbgF, double* dbgT) {
    using T = typename PR::T;
    using R = typename RecOf<T>::type;
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
    a.thresh2 = d.thresh2;
    a.interval = d.interval;
    a.perm = d.perm;
    const int hi = d.h_cur, ho = 1 - d.h_cur;
    a.hin_cnt = d.hcnt[hi];
    a.hin_pid = d.hpid[hi];
    a.hin_d = (const T*)d.hd[hi];
    a.hout_cnt = d.hcnt[ho];
    a.hout_pid = d.hpid[ho];
    a.hout_d = (T*)d.hd[ho];
    a.inmask = d.inmask;
    a.rec = (R*)d.rec;
    a.part = (R*)d.part_sum;
    a.st = d.st;
    a.dbgF = dbgF;
    a.dbgT = dbgT;
    const uint32_t b = (uint32_t)d.block;
    const size_t smem = (size_t)d.maxc * b * sizeof(uint32_t);
    const int model = d.model != 0 ? 1 : (d.terms != 0 ? 2 : 0);
    auto pair = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<nblk(d.n, b), b, smem, d.stream>>>(a);
        return cudaSuccess;
    };
    auto update = [&](auto kern) -> cudaError_t {
        kern<<<nblk(d.n, 256), 256, 0, d.stream>>>(a);
        return cudaSuccess;
    };
    cudaError_t e;
    if (model == 0) e = eval ? pair(k_pair<PR, 0, true>) : pair(k_pair<PR, 0, false>);
    else if (model == 2) e = eval ? pair(k_pair<PR, 2, true>) : pair(k_pair<PR, 2, false>);
    else e = eval ? pair(k_pair<PR, 1, true>) : pair(k_pair<PR, 1, false>);
    if (e != cudaSuccess) return e;
    DEM_LAUNCH_CHECK();
    if (model == 0) e = eval ? update(k_update<PR, 0, true>) : update(k_update<PR, 0, false>);
    else if (model == 2) e = eval ? update(k_update<PR, 2, true>) : update(k_update<PR, 2, false>);
    else e = eval ? update(k_update<PR, 1, true>) : update(k_update<PR, 1, false>);
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
