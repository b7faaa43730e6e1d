// List mode: the neighbour lists of a sort (Eq. 12's 27 cells, candidates within
// r_i + r_j + skin, in ascending partner id) and the walls each particle can reach before
// the next sort. The force pass that reads them is in dem_list.cu.
#include <algorithm>

#include <cuda_runtime.h>

#include "dem_domain.h"
#include "dem_policy.cuh"

namespace demgb {

// ------------------------------------------------------------------ list build
// Walls the particle can touch before the next sort: walls do not move (their velocity
// only enters the contact law), and a particle moves less than skin/2 between sorts, so
// every wall within r + skin/2 (+ the FP32 margin) of it now; bit w marks wall w.
// The test is a conservative FP32 distance (to a plane, from a cylinder's axis, from a
// half-plate's plane) with four times the FP32 position margin.
template <class PR>
__device__ __forceinline__ uint32_t reachable_walls(const typename PR::Self& me, const SceneDev& S) {
    const float4 x = PR::pos_f(me);
    const float eps = 4.f * S.eps_f;
    const float reach = me.r + 0.5f * S.skin_f + eps;
    uint32_t m = 0;
    for (int w = 0; w < S.nwalls; ++w) {
        const WallDev& W = S.walls[w];
        const float qx = x.x - W.pf[0], qy = x.y - W.pf[1], qz = x.z - W.pf[2];
        const float h = W.nf[0] * qx + W.nf[1] * qy + W.nf[2] * qz;
        bool near;
        if (W.kind == 1) {
            // distance from the axis (through p along n) against the radius
            const float rho2 = fmaxf(qx * qx + qy * qy + qz * qz - h * h, 0.f);
            const float lim = W.rad_hi - reach - eps;
            near = !(lim > 0.f && rho2 <= lim * lim);
        } else if (W.kind == 0) {
            near = h < reach;                 // signed distance into the domain
        } else {
            near = fabsf(h) < reach;          // either face of a half-plate, wherever its edge is
        }
        if (near) m |= 1u << w;
    }
    return m;
}

template <class PR>
__global__ void __launch_bounds__(256) k_wall_masks(uint32_t n, const SceneDev* scenes, int nscenes,
                                                    typename PR::State S0, typename PR::State S1, const CtrlDev* ctrl,
                                                    uint32_t* __restrict__ wmask) {
    const typename PR::State A = ctrl->cur ? S1 : S0;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        wmask[q] = reachable_walls<PR>(PR::load(A, q), scenes[scene_of(scenes, nscenes, q)]);
}

// Candidates of particle q at a sort: every particle of the 27 cells around q's cell
// (Eq. 12; list mode numbers the cells brick by brick, so each cell is looked up on its
// own) within r_i + r_j + skin (+ the FP32 margin), the skin of q's scene. With cells of
// edge >= 2 r_max + skin no pair that comes into contact before some particle has moved
// skin/2 is missed. A list is kept in ascending partner id, so the force pass sums a
// particle's contacts in that order whenever the list was built: results do not depend on
// when sorts happen (a batch sorts all its scenes together, and each scene still gets the
// bits of its own run). A list longer than DEM_LIST_CAP is reported (the step returns
// DEM_ERR_CAPACITY).
template <class PR>
__global__ void __launch_bounds__(256) k_nlist(uint32_t n, const SceneDev* scenes, int nscenes, typename PR::State S0,
                                               typename PR::State S1, const CtrlDev* ctrl,
                                               const uint32_t* __restrict__ skey, const uint32_t* __restrict__ cs,
                                               const uint32_t* __restrict__ fin, uint32_t* __restrict__ ncnt,
                                               uint32_t* __restrict__ nl, size_t cap, uint32_t* __restrict__ wmask,
                                               StatusDev* st) {
    if (ctrl->rebuild != 1) return;   // no sort this step (or a void step)
    const typename PR::State A = ctrl->cur ? S1 : S0;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const SceneDev& S = scenes[scene_of(scenes, nscenes, q)];
        const typename PR::Self me = PR::load(A, q);
        const float extra = S.skin_f + S.eps_f;
        int ix, iy, iz;
        cell_coords(S, skey[q] - S.c0, ix, iy, iz);
        uint32_t m = 0;
        // the list so far as (partner id << 32 | stored index), ascending: one 64-bit move per
        // insertion step (measured: the sort tail 6% shorter than with separate id and index
        // arrays)
        uint64_t lk[DEM_LIST_CAP];
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
                        if (m < DEM_LIST_CAP) {
                            const uint32_t idj = __ldg(&A.id[j]);
                            uint32_t k = m;
                            const uint64_t key = ((uint64_t)idj << 32) | j;
                            for (; k > 0 && lk[k - 1] > key; --k) lk[k] = lk[k - 1];
                            lk[k] = key;
                        }
                        ++m;
                    }
                }
        if (m > DEM_LIST_CAP) raise_status(st, ST_LIST, (int32_t)q);
        m = min(m, (uint32_t)DEM_LIST_CAP);
        for (uint32_t k = 0; k < m; ++k) nl[(size_t)k * cap + q] = (uint32_t)lk[k];
        ncnt[q] = m;
        wmask[q] = reachable_walls<PR>(me, S);
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

cudaError_t run_lists(Domain& d) {
    if (d.n == 0) return cudaSuccess;
    if (d.precision == 0)
        k_nlist<PF64><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.d_scenes, d.nscenes, d.S64[0], d.S64[1], d.ctrl, d.skey,
                                                          d.cs, d.fin, d.ncnt, d.nl, d.cap, d.wmask, d.st);
    else
        k_nlist<PF32><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.d_scenes, d.nscenes, d.S32[0], d.S32[1], d.ctrl, d.skey,
                                                          d.cs, d.fin, d.ncnt, d.nl, d.cap, d.wmask, d.st);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

cudaError_t run_wall_masks(Domain& d) {
    if (d.n == 0) return cudaSuccess;
    if (d.precision == 0)
        k_wall_masks<PF64><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.d_scenes, d.nscenes, d.S64[0], d.S64[1], d.ctrl,
                                                               d.wmask);
    else
        k_wall_masks<PF32><<<sgrid(d, d.n), 256, 0, d.stream>>>(d.n, d.d_scenes, d.nscenes, d.S32[0], d.S32[1], d.ctrl,
                                                               d.wmask);
    DEM_LAUNCH_CHECK();
    return cudaSuccess;
}

}  // namespace demgb
