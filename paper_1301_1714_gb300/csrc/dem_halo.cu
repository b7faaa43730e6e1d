// Exchange kernels of the slab decomposition (declared in dem_halo.h): after each force
// pass, owned particles go with their tangential springs to the slab that owns their new
// position, and ghost copies (state only) go to every slab whose ghost layer holds them;
// then each slab sorts its new layout by cell (steps 2-4 of Sec. 4.2) as usual.
//
// Records are placed with block-aggregated atomics, so the pre-sort layout of a slab
// varies from run to run; the cell sort that follows gives the unique (cell, id) order
// of Eq. 11, and the springs travel at the same index as their particle, so the result
// does not.
#include <algorithm>
#include <cmath>

#include "dem_halo.h"

namespace demgb {
namespace {

// FP64 state: planes of doubles, radius, id.
struct H64 {
    using St = StateF64;
    using T = double;
    static __device__ __forceinline__ double coord(const St& s, uint32_t q, int axis) {
        return axis == 0 ? s.x[q] : (axis == 1 ? s.y[q] : s.z[q]);
    }
    static __device__ __forceinline__ uint32_t id(const St& s, uint32_t q) { return s.id[q]; }
    static __device__ __forceinline__ void copy(const St& a, uint32_t q, const St& b, uint32_t p) {
        b.x[p] = a.x[q]; b.y[p] = a.y[q]; b.z[p] = a.z[q];
        b.vx[p] = a.vx[q]; b.vy[p] = a.vy[q]; b.vz[p] = a.vz[q];
        b.wx[p] = a.wx[q]; b.wy[p] = a.wy[q]; b.wz[p] = a.wz[q];
        b.r[p] = a.r[q];
        b.id[p] = a.id[q];
    }
    // particle k of host-layout arrays (the same conversion as a single domain's import)
    static __device__ __forceinline__ void put(const St& b, uint32_t p, const double* x, const double* v,
                                               const double* w, const float* r, uint32_t k) {
        b.x[p] = x[3 * (size_t)k]; b.y[p] = x[3 * (size_t)k + 1]; b.z[p] = x[3 * (size_t)k + 2];
        b.vx[p] = v[3 * (size_t)k]; b.vy[p] = v[3 * (size_t)k + 1]; b.vz[p] = v[3 * (size_t)k + 2];
        b.wx[p] = w[3 * (size_t)k]; b.wy[p] = w[3 * (size_t)k + 1]; b.wz[p] = w[3 * (size_t)k + 2];
        b.r[p] = r[k];
        b.id[p] = k;
    }
    static __device__ __forceinline__ void get(const St& a, uint32_t q, double* x, double* v, double* w) {
        const size_t o = 3 * (size_t)a.id[q];
        if (x) { x[o] = a.x[q]; x[o + 1] = a.y[q]; x[o + 2] = a.z[q]; }
        if (v) { v[o] = a.vx[q]; v[o + 1] = a.vy[q]; v[o + 2] = a.vz[q]; }
        if (w) { w[o] = a.wx[q]; w[o + 1] = a.wy[q]; w[o + 2] = a.wz[q]; }
    }
};

// FP32 state: P0 = (hi, r), P1 = (lo, id bits), V, W; position = hi + lo exactly.
struct H32 {
    using St = StateF32;
    using T = float;
    static __device__ __forceinline__ double coord(const St& s, uint32_t q, int axis) {
        const float4 h = s.P0[q], l = s.P1[q];
        return axis == 0 ? (double)h.x + (double)l.x : (axis == 1 ? (double)h.y + (double)l.y : (double)h.z + (double)l.z);
    }
    static __device__ __forceinline__ uint32_t id(const St& s, uint32_t q) { return s.id[q]; }
    static __device__ __forceinline__ void copy(const St& a, uint32_t q, const St& b, uint32_t p) {
        b.P0[p] = a.P0[q]; b.P1[p] = a.P1[q]; b.V[p] = a.V[q]; b.W[p] = a.W[q];
        b.id[p] = a.id[q];
    }
    // double -> (hi, lo) with hi = fl32(x) and lo = fl32(x - hi), renormalised by TwoSum
    static __device__ __forceinline__ void split(double x, float& hi, float& lo) {
        const float h = (float)x;
        const float l = (float)(x - (double)h);
        two_sum(h, l, hi, lo);
    }
    static __device__ __forceinline__ void put(const St& b, uint32_t p, const double* x, const double* v,
                                               const double* w, const float* r, uint32_t k) {
        float h[3], l[3];
        for (int c = 0; c < 3; ++c) split(x[3 * (size_t)k + c], h[c], l[c]);
        b.P0[p] = make_float4(h[0], h[1], h[2], r[k]);
        b.P1[p] = make_float4(l[0], l[1], l[2], __uint_as_float(k));
        b.V[p] = make_float4((float)v[3 * (size_t)k], (float)v[3 * (size_t)k + 1], (float)v[3 * (size_t)k + 2], 0.f);
        b.W[p] = make_float4((float)w[3 * (size_t)k], (float)w[3 * (size_t)k + 1], (float)w[3 * (size_t)k + 2], 0.f);
        b.id[p] = k;
    }
    static __device__ __forceinline__ void get(const St& a, uint32_t q, double* x, double* v, double* w) {
        const size_t o = 3 * (size_t)a.id[q];
        if (x) {
            const float4 h = a.P0[q], l = a.P1[q];
            x[o] = (double)h.x + (double)l.x;
            x[o + 1] = (double)h.y + (double)l.y;
            x[o + 2] = (double)h.z + (double)l.z;
        }
        if (v) { const float4 c = a.V[q]; v[o] = c.x; v[o + 1] = c.y; v[o + 2] = c.z; }
        if (w) { const float4 c = a.W[q]; w[o] = c.x; w[o + 1] = c.y; w[o + 2] = c.z; }
    }
};

// Slab owning a coordinate of order key kz: the number of interior boundaries at or
// below it.
__device__ __forceinline__ int owner_slab(const HaloGeom& g, uint64_t kz) {
    int o = 0;
#pragma unroll
    for (int t = 1; t < DEM_MAX_SLABS; ++t)
        if (t < g.nslabs && kz >= g.kb[t]) ++o;
    return o;
}

// Destinations of a particle of coordinate key kz owned by slab o: bit o, plus bit t for
// every other slab whose range widened by G on both sides holds the coordinate.
__device__ __forceinline__ uint32_t destinations(const HaloGeom& g, uint64_t kz, int o) {
    uint32_t want = 1u << o;
#pragma unroll
    for (int t = 0; t < DEM_MAX_SLABS; ++t)
        if (t < g.nslabs && t != o && kz >= g.klo[t] && kz < g.khi[t]) want |= 1u << t;
    return want;
}

template <class HP>
struct RouteArgs {
    SlabIO<typename HP::St, typename HP::T> io[DEM_MAX_SLABS];   // by value: read from the parameter bank
    HaloGeom g;
    uint32_t ntotal, maxc;
    const uint8_t* owner_old;
    uint8_t* owner_new;
    HaloCounters* hc;
    // first distribution: launch index k is particle k of these host-layout arrays
    const double *x, *v, *w;
    const float* r;
};

constexpr int ROUTE_THREADS = 256;
constexpr int ROUTE_WARPS = ROUTE_THREADS / 32;
constexpr int ROUTE_ITEMS = 4;                        // launch indices per thread per block iteration
constexpr int ROUTE_CHUNK = ROUTE_THREADS * ROUTE_ITEMS;

// Source slab of launch index gi (slabs are laid end to end; empty ones are skipped).
template <class IO>
__device__ __forceinline__ int source_slab(const IO* io, int S, uint32_t gi) {
    int s = 0;
    while (s + 1 < S && gi >= io[s + 1].p0) ++s;
    return s;
}

// Springs of one particle, slot lists keyed by partner id (slot-major planes of stride
// cap), copied four slots at a time: the loads of a group are issued before its stores.
template <class T>
__device__ __forceinline__ void copy_springs(uint32_t c, uint32_t maxc, const uint32_t* __restrict__ ps,
                                             const T* __restrict__ ds, size_t cs, uint32_t q,
                                             uint32_t* __restrict__ pd, T* __restrict__ dd, size_t cd, uint32_t p) {
    for (uint32_t k0 = 0; k0 < c; k0 += 4) {
        uint32_t pid[4];
        T d0[4], d1[4], d2[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t k = k0 + u;
            if (k < c) {
                pid[u] = ps[k * cs + q];
                d0[u] = ds[k * cs + q];
                d1[u] = ds[(maxc + k) * cs + q];
                d2[u] = ds[(2 * (size_t)maxc + k) * cs + q];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t k = k0 + u;
            if (k < c) {
                pd[k * cd + p] = pid[u];
                dd[k * cd + p] = d0[u];
                dd[(maxc + k) * cd + p] = d1[u];
                dd[(2 * (size_t)maxc + k) * cd + p] = d2[u];
            }
        }
    }
}

// One launch over all slabs (IMPORT: over the n input particles). A block iteration
// covers 1,024 launch indices: the destinations of each particle, per-warp ballots and
// shared counters give each record its place within the block's share of every
// destination, one global atomic per (block iteration, destination) reserves that share,
// then the records are copied. Every thread of the block runs the same iterations, so
// the ballots and barriers see full warps.
template <class HP, bool IMPORT>
__global__ void __launch_bounds__(ROUTE_THREADS, 4) k_halo_route(const __grid_constant__ RouteArgs<HP> a) {
    using IO = SlabIO<typename HP::St, typename HP::T>;
    __shared__ uint32_t s_cnt[DEM_MAX_SLABS], s_own[DEM_MAX_SLABS], s_base[DEM_MAX_SLABS];
    __shared__ uint32_t s_woff[DEM_MAX_SLABS][ROUTE_ITEMS][ROUTE_WARPS];
    __shared__ uint32_t s_mig;
    const IO* s_io = a.io;   // the slab table: kernel parameters (constant bank), never aliased by stores
    const unsigned full = 0xffffffffu;
    const int S = a.g.nslabs;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t base = blockIdx.x * ROUTE_CHUNK; base < a.ntotal; base += gridDim.x * ROUTE_CHUNK) {
        if (threadIdx.x < DEM_MAX_SLABS) {
            s_cnt[threadIdx.x] = 0u;
            s_own[threadIdx.x] = 0u;
        }
        if (threadIdx.x == 0) s_mig = 0u;
        __syncthreads();
        // source position, id and coordinate of every item (loads issued together)
        int sv[ROUTE_ITEMS];
        uint32_t qv[ROUTE_ITEMS], idv[ROUTE_ITEMS];
        uint64_t zv[ROUTE_ITEMS];   // order keys of the coordinates
#pragma unroll
        for (int it = 0; it < ROUTE_ITEMS; ++it) {
            const uint32_t gi = base + it * ROUTE_THREADS + threadIdx.x;
            sv[it] = 0;
            qv[it] = gi;
            idv[it] = gi;
            zv[it] = 0;
            if (gi < a.ntotal) {
                if (IMPORT) {
                    zv[it] = order_key(a.x[3 * (size_t)gi + a.g.axis]);
                } else {
                    const int s = source_slab(s_io, S, gi);
                    const uint32_t q = gi - s_io[s].p0;
                    sv[it] = s;
                    qv[it] = q;
                    idv[it] = HP::id(s_io[s].src, q);
                    zv[it] = order_key(HP::coord(s_io[s].src, q, a.g.axis));
                }
            }
        }
        // destinations: bits 0-7 the slabs that receive the particle, bits 8-11 its owner
        // (15: none, a ghost being dropped or an index past the end)
        uint32_t info[ROUTE_ITEMS];
        uint32_t nmig = 0;
#pragma unroll
        for (int it = 0; it < ROUTE_ITEMS; ++it) {
            const uint32_t gi = base + it * ROUTE_THREADS + threadIdx.x;
            uint32_t want = 0, o = 15;
            // ghosts are dropped: their owner sends fresh copies
            const bool live = gi < a.ntotal && (IMPORT || a.owner_old[idv[it]] == (uint8_t)sv[it]);
            if (live) {
                o = (uint32_t)owner_slab(a.g, zv[it]);
                want = destinations(a.g, zv[it], (int)o);
                if (!IMPORT && (int)o != sv[it]) ++nmig;
            }
            info[it] = want | (o << 8);
        }
#pragma unroll
        for (int it = 0; it < ROUTE_ITEMS; ++it) {
            const uint32_t want = info[it] & 0xFFu, o = info[it] >> 8;
#pragma unroll
            for (int t = 0; t < DEM_MAX_SLABS; ++t) {
                if (t >= S) break;
                const uint32_t m = __ballot_sync(full, (want >> t) & 1u);
                const uint32_t mo = __ballot_sync(full, o == (uint32_t)t);
                if (lane == 0) {
                    s_woff[t][it][wid] = m ? atomicAdd(&s_cnt[t], (uint32_t)__popc(m)) : 0u;
                    if (mo) atomicAdd(&s_own[t], (uint32_t)__popc(mo));
                }
            }
        }
        if (!IMPORT) {
            nmig = __reduce_add_sync(full, nmig);
            if (lane == 0 && nmig) atomicAdd(&s_mig, nmig);
        }
        __syncthreads();
        if (threadIdx.x < (unsigned)S) {
            const int t = (int)threadIdx.x;
            s_base[t] = s_cnt[t] ? atomicAdd(&a.hc->fill[t], s_cnt[t]) : 0u;
            if (s_own[t]) atomicAdd(&a.hc->owned[t], s_own[t]);
        }
        if (threadIdx.x == 0 && s_mig) atomicAdd(&a.hc->migrated, s_mig);
        __syncthreads();
        // copies
#pragma unroll
        for (int it = 0; it < ROUTE_ITEMS; ++it) {
            const uint32_t gi = base + it * ROUTE_THREADS + threadIdx.x;
            const uint32_t want = info[it] & 0xFFu, o = info[it] >> 8;
            const int s = sv[it];
            const uint32_t q = qv[it];
#pragma unroll
            for (int t = 0; t < DEM_MAX_SLABS; ++t) {
                if (t >= S) break;
                const uint32_t m = __ballot_sync(full, (want >> t) & 1u);
                if ((want >> t) & 1u) {
                    const IO& D = s_io[t];
                    const uint32_t p = s_base[t] + s_woff[t][it][wid] + (uint32_t)__popc(m & lt);
                    if (p >= D.cap) {
                        atomicAdd(&a.hc->overflow, 1u);
                    } else if (IMPORT) {
                        HP::put(D.dst, p, a.x, a.v, a.w, a.r, gi);
                        D.hcnt_dst[p] = 0u;
                    } else {
                        const IO& src = s_io[s];
                        HP::copy(src.src, q, D.dst, p);
                        if (o == (uint32_t)t) {
                            // the owner's springs travel with it
                            const uint32_t c = min(src.hcnt_src[q], a.maxc);
                            D.hcnt_dst[p] = c;
                            copy_springs(c, a.maxc, src.hpid_src, src.hd_src, src.cap, q, D.hpid_dst, D.hd_dst, D.cap,
                                         p);
                        } else {
                            D.hcnt_dst[p] = 0u;   // a ghost's own forces are not used
                        }
                    }
                }
            }
            if (o < 15u) a.owner_new[idv[it]] = (uint8_t)o;
        }
        __syncthreads();   // the shared counters are reset by the next iteration
    }
}

__global__ void k_halo_flip(const CtrlTable t) {
    const int s = (int)threadIdx.x;
    if (s < t.n) t.c[s]->cur ^= 1;
}

template <class HP>
__global__ void k_halo_export(uint32_t n, typename HP::St S0, typename HP::St S1, const CtrlDev* ctrl,
                              const uint8_t* __restrict__ owner, uint8_t slab, double* x, double* v, double* w) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const typename HP::St A = ctrl->cur ? S1 : S0;
    if (owner[HP::id(A, q)] != slab) return;
    HP::get(A, q, x, v, w);
}

inline uint32_t route_grid(uint32_t n, int sort_blocks) {
    const uint32_t nb = (n + ROUTE_CHUNK - 1) / ROUTE_CHUNK;
    return std::max(1u, std::min(nb, (uint32_t)std::max(sort_blocks, 1)));
}

template <class HP, bool IMPORT>
cudaError_t launch_route(const RouteArgs<HP>& a, int sort_blocks, cudaStream_t stream) {
    k_halo_route<HP, IMPORT><<<route_grid(a.ntotal, sort_blocks), ROUTE_THREADS, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <class HP>
RouteArgs<HP> route_args(const void* io, int nslabs, const HaloGeom& g, uint32_t ntotal, uint32_t maxc,
                         const uint8_t* owner_old, uint8_t* owner_new, HaloCounters* hc) {
    RouteArgs<HP> a{};
    const auto* t = (const SlabIO<typename HP::St, typename HP::T>*)io;
    for (int k = 0; k < nslabs; ++k) a.io[k] = t[k];
    a.g = g;
    a.ntotal = ntotal;
    a.maxc = maxc;
    a.owner_old = owner_old;
    a.owner_new = owner_new;
    a.hc = hc;
    return a;
}

cudaError_t run_halo_route(int precision, const void* io, const HaloGeom& g, uint32_t ntotal, uint32_t maxc,
                           const uint8_t* owner_old, uint8_t* owner_new, HaloCounters* hc, int sort_blocks,
                           cudaStream_t stream) {
    if (ntotal == 0) return cudaSuccess;
    if (precision == 0)
        return launch_route<H64, false>(route_args<H64>(io, g.nslabs, g, ntotal, maxc, owner_old, owner_new, hc),
                                        sort_blocks, stream);
    return launch_route<H32, false>(route_args<H32>(io, g.nslabs, g, ntotal, maxc, owner_old, owner_new, hc),
                                    sort_blocks, stream);
}

cudaError_t run_halo_import(int precision, const void* io, const HaloGeom& g, uint32_t n, const double* x,
                            const double* v, const double* w, const float* r, uint8_t* owner_new, HaloCounters* hc,
                            int sort_blocks, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    if (precision == 0) {
        RouteArgs<H64> a = route_args<H64>(io, g.nslabs, g, n, 0u, nullptr, owner_new, hc);
        a.x = x; a.v = v; a.w = w; a.r = r;
        return launch_route<H64, true>(a, sort_blocks, stream);
    }
    RouteArgs<H32> a = route_args<H32>(io, g.nslabs, g, n, 0u, nullptr, owner_new, hc);
    a.x = x; a.v = v; a.w = w; a.r = r;
    return launch_route<H32, true>(a, sort_blocks, stream);
}

cudaError_t run_halo_flip(const CtrlTable& t, cudaStream_t stream) {
    k_halo_flip<<<1, 32, 0, stream>>>(t);
    return cudaGetLastError();
}

cudaError_t run_halo_export(Domain& d, int slab, const uint8_t* owner, double* x, double* v, double* w) {
    if (d.n == 0) return cudaSuccess;
    const uint32_t nb = (d.n + 255) / 256;
    if (d.precision == 0)
        k_halo_export<H64><<<nb, 256, 0, d.stream>>>(d.n, d.S64[0], d.S64[1], d.ctrl, owner, (uint8_t)slab, x, v, w);
    else
        k_halo_export<H32><<<nb, 256, 0, d.stream>>>(d.n, d.S32[0], d.S32[1], d.ctrl, owner, (uint8_t)slab, x, v, w);
    return cudaGetLastError();
}

}  // namespace demgb
