// dem_sort_cells_static: the cell hash and (cell, id) counting sort for callers that
// must not allocate device memory.
//
// Who needs this: a process that has already reserved all of the GPU's memory for its
// own pool (so a cudaMalloc from this library would fail or fragment that pool), and a
// loop that forbids allocation after start-up because cudaMalloc/cudaFree can block or
// synchronise the device at unpredictable moments. Such callers pass their own input and
// output buffers; the temporary counters and slot arrays this sort needs live in one
// fixed array of device memory that the library declares at file scope (about 6 MB, held
// on every GPU that loads the library until the process exits).
//
// The static array is shared by every call: calls whose work overlaps on the GPU (two
// streams, or two host threads) race on it and give wrong results. Each call clears the
// counters it relies on before use.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "dem.h"

namespace {

constexpr uint32_t SA_MAX_N = DEM_STATIC_SORT_MAX_N;
constexpr uint32_t SA_MAX_CELLS = DEM_STATIC_SORT_MAX_CELLS;
constexpr int SA_THREADS = 256;
constexpr int SA_ITEMS = 8;
constexpr uint32_t SA_TILE = SA_THREADS * SA_ITEMS;
constexpr uint32_t SA_MAX_PART = (SA_MAX_CELLS + 1 + SA_TILE - 1) / SA_TILE;

// offsets (in 32-bit words) of the pieces of the scratch array
constexpr size_t SA_OFF_CNT = 0;                                   // SA_MAX_CELLS + 1 counts
constexpr size_t SA_OFF_RANK = ((SA_MAX_CELLS + 1 + 63) / 64) * 64;  // SA_MAX_N ranks within a cell
constexpr size_t SA_OFF_TMP = SA_OFF_RANK + SA_MAX_N;              // SA_MAX_N cell-major slots
constexpr size_t SA_OFF_PART = SA_OFF_TMP + SA_MAX_N;              // SA_MAX_PART scan partials
constexpr size_t SA_WORDS = SA_OFF_PART + SA_MAX_PART;

static __device__ __align__(256) uint32_t g_sort_scratch[SA_WORDS];

// Device address of g_sort_scratch on each device (taken once per device).
std::mutex g_mu;
constexpr int SA_MAX_DEVICES = 64;
void* g_addr[SA_MAX_DEVICES] = {nullptr};

__device__ __forceinline__ uint32_t sa_axis(double xa, double o, double h, int64_t dim) {
    const double c = floor(__ddiv_rn(__dsub_rn(xa, o), h));
    if (!(c >= 0.0)) return 0;
    if (c >= (double)dim) return (uint32_t)(dim - 1);
    return (uint32_t)c;
}

__global__ void k_sa_hash(uint32_t n, const double* __restrict__ x, double ox, double oy, double oz, double h,
                          int64_t nx, int64_t ny, int64_t nz, uint32_t* __restrict__ cell_of, uint32_t* scratch) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t i = sa_axis(x[3 * (size_t)k], ox, h, nx);
    const uint32_t j = sa_axis(x[3 * (size_t)k + 1], oy, h, ny);
    const uint32_t l = sa_axis(x[3 * (size_t)k + 2], oz, h, nz);
    const uint32_t key = (l * (uint32_t)ny + j) * (uint32_t)nx + i;
    cell_of[k] = key;
    scratch[SA_OFF_RANK + k] = atomicAdd(&scratch[SA_OFF_CNT + key], 1u);
}

__global__ void __launch_bounds__(SA_THREADS) k_sa_reduce(uint32_t m, uint32_t* scratch) {
    __shared__ uint32_t ws[SA_THREADS / 32];
    const uint32_t base = blockIdx.x * SA_TILE;
    uint32_t s = 0;
    for (int i = 0; i < SA_ITEMS; ++i) {
        const uint32_t k = base + i * SA_THREADS + threadIdx.x;
        if (k < m) s += scratch[SA_OFF_CNT + k];
    }
    s = __reduce_add_sync(0xffffffffu, s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < SA_THREADS / 32; ++w) t += ws[w];
        scratch[SA_OFF_PART + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) k_sa_spine(uint32_t nb, uint32_t* scratch) {
    __shared__ uint32_t sh[1024];
    uint32_t* part = scratch + SA_OFF_PART;
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
    uint32_t run = sh[threadIdx.x] - s;
    for (uint32_t k = 0; k < per; ++k)
        if (b0 + k < nb) {
            const uint32_t v = part[b0 + k];
            part[b0 + k] = run;
            run += v;
        }
}

__global__ void __launch_bounds__(SA_THREADS) k_sa_down(uint32_t m, const uint32_t* scratch,
                                                        uint32_t* __restrict__ cell_start) {
    __shared__ uint32_t ws[SA_THREADS / 32];
    const uint32_t base = blockIdx.x * SA_TILE + threadIdx.x * SA_ITEMS;
    uint32_t v[SA_ITEMS];
    uint32_t s = 0;
    for (int i = 0; i < SA_ITEMS; ++i) {
        const uint32_t k = base + i;
        v[i] = k < m ? scratch[SA_OFF_CNT + k] : 0u;
        s += v[i];
    }
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = s;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= (uint32_t)off) inc += t;
    }
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < SA_THREADS / 32 ? ws[lane] : 0u;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= (uint32_t)off) w += t;
        }
        if (lane < SA_THREADS / 32) ws[lane] = w;
    }
    __syncthreads();
    uint32_t run = scratch[SA_OFF_PART + blockIdx.x] + (inc - s) + (wid > 0 ? ws[wid - 1] : 0u);
    for (int i = 0; i < SA_ITEMS; ++i) {
        const uint32_t k = base + i;
        if (k < m) cell_start[k] = run;
        run += v[i];
    }
}

__global__ void k_sa_scatter(uint32_t n, const uint32_t* __restrict__ cell_of, const uint32_t* __restrict__ cell_start,
                             uint32_t* scratch) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) scratch[SA_OFF_TMP + cell_start[cell_of[k]] + scratch[SA_OFF_RANK + k]] = k;
}

// place of particle p in its cell = number of cell-mates with a smaller id (each thread
// reads its whole cell, so the work grows with the square of the cells' occupancy)
__global__ void k_sa_order(uint32_t n, const uint32_t* __restrict__ cell_of, const uint32_t* __restrict__ cell_start,
                           const uint32_t* scratch, uint32_t* __restrict__ order) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t* tmp = scratch + SA_OFF_TMP;
    const uint32_t p = tmp[s];
    const uint32_t c = cell_of[p];
    const uint32_t lo = cell_start[c], hi = cell_start[c + 1];
    uint32_t r = 0;
    for (uint32_t k = lo; k < hi; ++k) r += tmp[k] < p ? 1u : 0u;
    order[lo + r] = p;
}

}  // namespace

extern "C" dem_status dem_sort_cells_static(int64_t n, const double* x, const double* origin, double cell,
                                            const int64_t* dims, uint32_t* cell_of, uint32_t* order,
                                            uint32_t* cell_start, void* cuda_stream) {
    if (n < 0 || !origin || !dims || !(cell > 0.0)) return DEM_ERR_INVALID_ARG;
    // each axis first (so that the product cannot overflow), then the product
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > (int64_t)SA_MAX_CELLS) return DEM_ERR_INVALID_ARG;
    const int64_t ncells = dims[0] * dims[1] * dims[2];
    if (n > (int64_t)SA_MAX_N || ncells > (int64_t)SA_MAX_CELLS) return DEM_ERR_INVALID_ARG;
    if (!cell_start || (n > 0 && (!x || !cell_of || !order))) return DEM_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SA_MAX_DEVICES) {
        cudaGetLastError();
        return DEM_ERR_CUDA;
    }
    uint32_t* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return DEM_ERR_CUDA;
            }
            g_addr[dev] = p;
        }
        scratch = (uint32_t*)g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const uint32_t nn = (uint32_t)n, m = (uint32_t)ncells + 1;
    // counts must start at zero: the array keeps whatever the previous call left
    if (cudaMemsetAsync(scratch + SA_OFF_CNT, 0, (size_t)m * sizeof(uint32_t), st) != cudaSuccess) {
        cudaGetLastError();
        return DEM_ERR_CUDA;
    }
    const uint32_t nb = (m + SA_TILE - 1) / SA_TILE;
    if (nn > 0)
        k_sa_hash<<<(nn + 255) / 256, 256, 0, st>>>(nn, x, origin[0], origin[1], origin[2], cell, dims[0], dims[1],
                                                    dims[2], cell_of, scratch);
    k_sa_reduce<<<nb, SA_THREADS, 0, st>>>(m, scratch);
    k_sa_spine<<<1, 1024, 0, st>>>(nb, scratch);
    k_sa_down<<<nb, SA_THREADS, 0, st>>>(m, scratch, cell_start);
    if (nn > 0) {
        k_sa_scatter<<<(nn + 255) / 256, 256, 0, st>>>(nn, cell_of, cell_start, scratch);
        k_sa_order<<<(nn + 255) / 256, 256, 0, st>>>(nn, cell_of, cell_start, scratch, order);
    }
    if (cudaGetLastError() != cudaSuccess) return DEM_ERR_CUDA;
    return DEM_OK;
}
