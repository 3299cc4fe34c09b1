// Host-side context of the library (shared by its translation units).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

// an NVTX range over a C-ABI call (seen by profilers; no cost without one attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

#include "dem.h"
#include "dem_internal.cuh"

using namespace cgdem;   // internal header: the library's own types

struct dem_ctx {
    cudaStream_t stream = nullptr;
    int device = 0;
    Dev dev{};
    int B = 0, Lmax = 0;
    int ncap = 0, ntiles = 0;
    int grid0 = 1, grid1 = 1;         // persistent grids of the step / evaluation kernels
    int step_bs = 0;                  // threads per block of the step kernel (64, 128, 256, 896; 0 automatic)
    int step_lanes = 1;               // lanes per particle of the step kernel (1, 2, 4 or 8; >1 at 128 threads)
    int grid_bs[3] = {1, 1, 1};       // persistent step grids for 64, 128 and 256 threads per block
    int grid_smw = 0;                 // persistent grid of SM-wide step blocks (0: not available)
    int grid_lanes[3] = {1, 1, 1};    // persistent step grids for 2, 4 and 8 lanes per particle
    bool list_staged = false;         // list build with the shared-memory window of cell-order positions
    int grid_build_staged = 1;
    int grid_rb = 1;                  // persistent grid of the per-slot rebuild kernels
    int grid_build = 1;               // one wave of the list build (occupancy-sized)
    unsigned ncodes = 0, nparts = 0;
    std::vector<InstC> ic;
    std::vector<HostInstLo> hl;
    std::vector<long long> count;     // host mirror of live counts
    HostInstLo* d_hl = nullptr;
    bool fresh = true;                // velocities at an integer step (next step primes)
    bool walls = false;               // some instance has axisymmetric walls (step kernel variant)
    bool count_stale = false;         // a coupling call changed the IDs handed out on the device
    bool have_state = false;
    long long steps = 0;
    unsigned status = 0;
    std::string err;
    // graphs
    int graph_steps = 0;
    int graph_mode = 0;               // 0: fused steps when the context fits, 1: a kernel per step, 2: fused
    bool graph_fused = false;         // the current graph runs its steps in fused cooperative launches
    int grid_fused = 0;               // co-resident blocks of the fused step kernel (0: unknown)
    cudaGraph_t rb_graph = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<cudaEvent_t> ev0, ev1;   // around each step kernel of the graph
    std::vector<double> nu;              // Poisson ratio per instance (for material updates)
    std::vector<double> rmax;            // largest radius per instance [m]
    struct Rollout {
        bool ready = false;
        long long nsteps = 0, K = 0;
        int ncp = 0;
        bool prime0 = false;
        std::vector<Snap> ck, seg;       // checkpoints (every K steps and the end), segment steps
        AdjBufs a{};
    } ro;
};
using Rollout = dem_ctx::Rollout;

namespace cgdem {
dem_status fail(dem_ctx* c, dem_status st, const std::string& msg);
dem_status check_status(dem_ctx* ctx);
dem_status refresh_count(dem_ctx* ctx);
dem_status launch_rebuild(dem_ctx* ctx, cudaStream_t st);
dem_status launch_eval(dem_ctx* ctx);
long long total_count(const dem_ctx* ctx);
void set_thread_error(const std::string& msg);
}  // namespace cgdem

#define CU(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return cgdem::fail(ctx, DEM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
