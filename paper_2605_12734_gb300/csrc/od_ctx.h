// od_ctx.h -- the context object behind od_ctx* (internal to libod).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "od.h"
#include "od_internal.h"
#include "od_plan.h"

constexpr uint64_t kDefaultSpinNs = 2000000000ull;

struct od_ctx {
    od_config cfg{};
    od::Plan plan;
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char *arena = nullptr;
    bool own_arena = false;
    ChareDev *d_ch = nullptr;
    TileDev *d_tiles = nullptr;
    ErrDev *d_err = nullptr;
    int32_t *d_queue = nullptr, *d_epoch = nullptr, *d_dep_ptr = nullptr, *d_dep_idx = nullptr,
            *d_order = nullptr;
    uint64_t *d_vmax = nullptr;       // largest value of the field (bits), in the arena's queue block
    bool ghosts_current = true;       // internal ghost layers of the current parity hold the
                                      // neighbours' faces (false after a fused step or an import)
    std::vector<ChareDev> h_ch;       // host copy (device pointers)
    double *d_stage = nullptr;        // lazily allocated host-transfer staging
    // od_read_async: the device-to-host copy of the staging buffer runs on
    // copy_stream after ev_gathered; ev_copied marks the staging buffer free
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_gathered = nullptr, ev_copied = nullptr;
    bool copy_pending = false;
    int path = OD_PATH_FUSED;
    int64_t steps = 0;
    int64_t launches = 0, api_calls = 0, graph_launches = 0;
    int persistent_grid = 0;
    int64_t stall_tile = -1;
    uint64_t spin_ns = kDefaultSpinNs;
    bool failed = false;
    bool tuned = false;       // execution shape chosen by the autotuner
    double tune_ms = 0;       // its measured time per step
    // per-chare path
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> ev;      // ev[2*c + slot]: chare c delivered its faces
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    // graph path
    cudaGraphExec_t g2 = nullptr, g1[2] = {nullptr, nullptr};
    // fused-graph path: kFusedGraphSteps fused steps from an even step, and
    // one step from each parity
    cudaGraphExec_t gf = nullptr, gf1[2] = {nullptr, nullptr};
    int64_t g2_kernels = 0, g1_kernels[2] = {0, 0};
    int64_t g2_calls = 0, g1_calls[2] = {0, 0};
};


namespace od {
// Record an error for od_last_error() (any translation unit).
od_status set_last_error(od_status s, const std::string &msg);
// Kernel arguments of a context's tile kernels (tables, ring shape, limits).
KArgs base_args(const od_ctx *c);
// Synchronise the context's stream and turn a device error record into a status.
od_status check_device_error(od_ctx *c);
// od_create; with sync = false it returns once the initialisation is queued
// on the context's stream (errors of the queued work surface at the next
// synchronising call), so a caller that keeps its own stream order -- the
// serving loop -- does not wait for the device.
od_status create_context(od_ctx **out, const od_config *cfg, bool sync);
}  // namespace od
