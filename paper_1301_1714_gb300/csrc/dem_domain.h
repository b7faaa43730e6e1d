// Host-side description of the device buffers of one packed particle domain (one or
// more scenes laid end to end), shared by the engine and the kernel launchers.
#pragma once
#include <cstdint>
#include <vector>

#include "dem_dev.cuh"

namespace demgb {

struct StateF64 {
    double *x, *y, *z, *vx, *vy, *vz, *wx, *wy, *wz;
    float* r;
    uint32_t* id;
};
struct StateF32 {
    float4 *P0, *P1, *V, *W;
    uint32_t* id;
};

struct Domain {
    // configuration
    int precision = 0;   // 0 FP64, 1 FP32 (compensated positions)
    int model = 0;       // 0 practical, 1 simple
    int stiffness = 0;   // 0 linear, 1 Hertz
    int maxc = 32;       // history slots per particle
    int block = 128;     // force kernel block size
    cudaStream_t stream = nullptr;

    // sizes
    uint32_t n = 0, cap = 0;       // particles, allocated capacity
    uint32_t ncells = 0;           // total cells over all scenes
    uint32_t cells_cap = 0;        // allocated cell-table capacity (entries, excluding the +1)
    int nscenes = 0;
    std::vector<SceneDev> h_scenes;
    SceneDev* d_scenes = nullptr;
    int scenes_cap = 0;

    // particle state: A = cell-sorted current state, B = next state (pre-sort order)
    StateF64 A64{}, B64{};
    StateF32 A32{}, B32{};

    // tangential history, double-buffered; h_cur is the buffer the next step reads
    uint32_t* hcnt[2] = {nullptr, nullptr};
    uint32_t* hpid[2] = {nullptr, nullptr};
    void* hd[2] = {nullptr, nullptr};
    int h_cur = 0;

    // counting sort by cell
    uint32_t *key = nullptr, *rank = nullptr, *tmp = nullptr, *perm = nullptr, *skey = nullptr;
    uint32_t *cnt = nullptr, *cs = nullptr, *part = nullptr;
    uint32_t part_cap = 0;

    // status
    StatusDev* st = nullptr;       // device: [0] live accumulators, [1] last completed force pass
    StatusDev* st_host = nullptr;  // pinned copy

    // diagnostics scratch
    double* diag_part = nullptr;
    uint32_t diag_part_cap = 0;
    double* diag_out = nullptr;

    int64_t launches = 0;
    int64_t sorts = 0;

    std::vector<void*> allocations;   // every cudaMalloc of this domain (freed together)
};

// -------- launchers (dem_kernels.cu); all enqueue on d.stream and count launches
cudaError_t run_import(Domain& d, const double* x, const double* v, const double* w, const float* r);
cudaError_t run_hash_initial(Domain& d);
cudaError_t run_rebuild(Domain& d);
cudaError_t run_force(Domain& d, bool eval, double* dbgF, double* dbgT);
cudaError_t run_export(Domain& d, double* x, double* v, double* w);
cudaError_t run_diag(Domain& d);   // fills d.diag_out[0..9] (device)

}  // namespace demgb
