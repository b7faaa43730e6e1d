// Slab decomposition of one scene into sub-domains along one axis, with a ghost (halo)
// layer one cell wide on each side of a slab, on one device: the device-side tables and
// the launchers of the exchange kernels (dem_halo.cu).
//
// A particle is owned by the slab whose range [zb[t], zb[t+1]) holds its coordinate
// along the axis, and is a ghost of every other slab t with zb[t] - G <= z < zb[t+1] + G
// (G = the cell edge h, larger than any contact distance 2 r_max). Every contact partner
// of an owned particle is then present in its slab, in the same cells of the same global
// grid, so the cell walk (Eq. 12) meets the same partners in the same (cell, id) order
// as in the undivided scene: the forces on owned particles are the same bits.
#pragma once
#include <cstdint>

#include "dem_domain.h"

#ifndef DEM_MAX_SLABS
#define DEM_MAX_SLABS 8   // as in dem.h
#endif

namespace demgb {

// One slab as the exchange sees it.
template <class St, class T>
struct SlabIO {
    St src;                         // state just computed by the force pass (index q)
    St dst;                         // free state set that receives the slab's new layout
    const uint32_t* hcnt_src;       // springs written by the force pass (index q)
    const uint32_t* hpid_src;
    const T* hd_src;
    uint32_t* hcnt_dst;             // springs of the new layout
    uint32_t* hpid_dst;
    T* hd_dst;
    uint32_t n;                     // particles in the source layout
    uint32_t p0;                    // first launch index of this slab
    uint32_t cap;                   // allocated particle capacity of the slab
    uint32_t pad;
};

struct HaloGeom {
    int32_t nslabs;
    int32_t axis;                   // 0, 1, 2
    double zb[DEM_MAX_SLABS + 1];   // slab boundaries, zb[0] = -inf, zb[nslabs] = +inf
    double G;                       // ghost width
    // the same tests as unsigned comparisons of order keys (order_key, set by set_keys):
    // owner = #{t >= 1 : key(z) >= kb[t]}; ghost of t when klo[t] <= key(z) < khi[t]
    uint64_t kb[DEM_MAX_SLABS + 1];   // key(zb[t])
    uint64_t klo[DEM_MAX_SLABS];      // key(zb[t] - G), the difference rounded as a double
    uint64_t khi[DEM_MAX_SLABS];      // key(zb[t + 1] + G)
};

// Order key of a double that is not NaN: a <= b exactly when order_key(a) <=
// order_key(b) (-0 is taken as +0), so the FP64 slab tests become integer comparisons.
__host__ __device__ inline uint64_t order_key(double d) {
#ifdef __CUDA_ARCH__
    uint64_t b = (uint64_t)__double_as_longlong(d);
#else
    uint64_t b;
    static_assert(sizeof(b) == sizeof(d), "64-bit double");
    __builtin_memcpy(&b, &d, sizeof b);
#endif
    if (b == 0x8000000000000000ull) b = 0;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

inline void set_keys(HaloGeom& g) {
    for (int t = 0; t <= g.nslabs; ++t) g.kb[t] = order_key(g.zb[t]);
    for (int t = 0; t < g.nslabs; ++t) {
        g.klo[t] = order_key(g.zb[t] - g.G);
        g.khi[t] = order_key(g.zb[t + 1] + g.G);
    }
}

// Counters of one exchange (device, zeroed before it).
struct HaloCounters {
    uint32_t fill[DEM_MAX_SLABS];   // particles written to each slab
    uint32_t owned[DEM_MAX_SLABS];  // of which owned
    uint32_t migrated;              // owned particles whose slab changed
    uint32_t overflow;              // records dropped because a slab was full (never with capacity n)
    uint32_t pad[2];
};

// Exchange after a force pass: every owned particle of every slab (owner_old[id] == slab)
// goes, with its springs, to the slab that owns its new position, and as a ghost (no
// springs) to every slab whose ghost layer holds it; owner_new[id] receives the new
// owner. One launch covers all slabs.
// `io` is a host array of nslabs SlabIO<StateF64, double> (FP64) or SlabIO<StateF32, float>,
// copied into the launch's parameters.
cudaError_t run_halo_route(int precision, const void* io, const HaloGeom& g,
                           uint32_t ntotal, uint32_t maxc, const uint8_t* owner_old, uint8_t* owner_new,
                           HaloCounters* hc, int sort_blocks, cudaStream_t stream);
// First distribution: n particles from host-layout device arrays (x, v, w: 3n doubles;
// r: n floats; particle k has id k) into the slabs' free sets, with no springs.
cudaError_t run_halo_import(int precision, const void* io, const HaloGeom& g, uint32_t n, const double* x,
                            const double* v, const double* w, const float* r, uint8_t* owner_new,
                            HaloCounters* hc, int sort_blocks, cudaStream_t stream);
// Step-control blocks of the slabs.
struct CtrlTable {
    CtrlDev* c[DEM_MAX_SLABS];
    int32_t n;
};
// Current-set indicator of every slab flipped (c[s]->cur ^= 1), one launch.
cudaError_t run_halo_flip(const CtrlTable& t, cudaStream_t stream);
// Owned particles of one slab's current set written to x, v, w at 3 * id (FP64).
cudaError_t run_halo_export(Domain& d, int slab, const uint8_t* owner, double* x, double* v, double* w);

}  // namespace demgb
