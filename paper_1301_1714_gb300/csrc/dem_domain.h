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
    int sort_blocks = 0; // grid of the sort-phase kernels (a few blocks per SM)
    int terms = 0;       // union of the scenes' optional force terms (selects the kernel variant)
    int stiffness = 0;   // 0 linear, 1 Hertz
    int maxc = 32;       // history slots per particle
    int block = 128;     // force kernel block size
    int regrow = 0;      // 1: a contact-slot overflow voids the step (the handle grows its slots
                         // and runs the step again); 0: it is only reported
    cudaStream_t stream = nullptr;

    // sizes
    uint32_t n = 0, cap = 0;       // particles, allocated capacity
    uint32_t ncells = 0;           // total cells over all scenes
    uint32_t cells_cap = 0;        // allocated cell-table capacity (entries, excluding the +1)
    int nscenes = 0;
    std::vector<SceneDev> h_scenes;
    SceneDev* d_scenes = nullptr;
    int scenes_cap = 0;

    // particle state: two sets; ctrl->cur (on the device) names the current, cell-sorted
    // one, the other receives the next state
    StateF64 S64[2]{};
    StateF32 S32[2]{};
    CtrlDev* ctrl = nullptr;       // device
    CtrlDev* ctrl_host = nullptr;  // pinned copy

    // neighbour lists (list mode: resort_interval != 1): candidates within r_i + r_j + skin
    // of each particle at the last sort, slot-major nl[k*cap + q], counts ncnt[q]
    int list_mode = 0;
    int maxn = DEM_LIST_CAP;
    int interval = 1;              // sort at least every `interval` steps (0 = skin only)
    uint32_t* ncnt = nullptr;
    uint32_t* nl = nullptr;
    float4* ref = nullptr;         // positions at the last sort
    uint32_t* wmask = nullptr;     // walls each particle can reach before the next sort (bit w = wall w)
    uint32_t* canon = nullptr;     // (cell, id) position -> pre-sort position, at a sort
    uint32_t* fin = nullptr;       // (cell, id) position -> stored position (window order by contact count)

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

    std::vector<void*> allocations;   // every cudaMalloc of this domain (freed together)
};

// A CUDA graph of two captured timesteps and the kernel launches it holds.
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;        // kernels every replay launches
    int64_t body_launches = 0;   // kernels of one conditional sort body (list mode)
    cudaGraphExec_t sort_exec[2] = {nullptr, nullptr};   // phase timing: the sort tail per history parity
    int64_t sort_launches = 0;   // kernels every sort-tail replay launches
    cudaStream_t side = nullptr; // stream on which the conditional bodies are captured
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        for (auto& x : sort_exec) {
            if (x) cudaGraphExecDestroy(x);
            x = nullptr;
        }
        sort_launches = 0;
        launches = 0;
        body_launches = 0;
        if (side) cudaStreamDestroy(side);
        side = nullptr;
    }
};

// -------- launchers (dem_kernels.cu); all enqueue on d.stream and count launches
cudaError_t run_import(Domain& d, const double* x, const double* v, const double* w, const float* r);
// out[0]: 1 = a radius not finite and > 0, 2 = a non-finite x, v or w; out[1]: bits of r_max
cudaError_t run_check_input(Domain& d, uint32_t n, const double* x, const double* v, const double* w, const float* r,
                            uint32_t* out);
cudaError_t run_hash(Domain& d);      // cell key + in-cell rank of the next state (if sorting)
cudaError_t run_rebuild(Domain& d);   // scan, scatter, (cell, id) gather, lists (if sorting)
cudaError_t run_end_step(Domain& d);  // step bookkeeping (swap or keep, counters)
cudaError_t run_sort_cond(Domain& d, cudaGraphConditionalHandle h);  // graph condition = this step sorts
cudaError_t run_force(Domain& d, bool eval, double* dbgF, double* dbgT);
// list mode (dem_list.cu): the neighbour lists of a sort, and the force pass over them
cudaError_t run_lists(Domain& d);
cudaError_t run_wall_masks(Domain& d);   // the wall masks again (after the walls changed)
cudaError_t run_force_list(Domain& d, bool eval, double* dbgF, double* dbgT);
cudaError_t run_export(Domain& d, double* x, double* v, double* w);
cudaError_t run_diag(Domain& d);   // fills d.diag_out[0..9] (device)
// batches: springs into sorted order (into the free history buffer), new packed layout,
// import of one scene at an offset, export of one scene's range
cudaError_t run_hist_canon(Domain& d);
cudaError_t run_repack(Domain& od, Domain& d, const uint32_t* map, uint32_t n_new);
cudaError_t run_import_at(Domain& d, uint32_t p0, uint32_t np, const double* x, const double* v, const double* w,
                          const float* r);
cudaError_t run_export_range(Domain& d, uint32_t p0, uint32_t np, double* x, double* v, double* w);

}  // namespace demgb
