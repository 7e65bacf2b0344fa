// od_plan.h -- host-side decomposition and layout planner of libod.
// Pure C++: no CUDA calls, so it runs (and is tested) without a GPU.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "od.h"
#include "od_internal.h"

namespace od {

struct HostChare {
    int32_t cx, cy, cz;
    int64_t x0, y0, z0;
    int32_t bx, by, bz, pitch;
    int32_t rows, row0;             // plane layout (see ChareDev)
    int32_t nbr[6];
    int32_t foff[7];
    size_t offA[2];
    size_t offSend, offRecv[2];
    int32_t tile_begin, tile_end;   // tiles [begin,end) belong to this chare
    // the chare's tiles form a grid: per axis the tile starts (chare-local),
    // tile (a, b, e) = tile_begin + (e * tj.size() + b) * ti.size() + a
    std::vector<int32_t> ti, tj, tk;
};

struct Plan {
    int32_t stencil = 0;                      // OD_STENCIL_*; 2D runs as (nx, 1, ny)
    int64_t nx = 0, ny = 0, nz = 0;           // internal (3D) extents
    int64_t gnx = 0, gny = 0, gnz = 0;        // global grid (internal axes) this context is a shard of
    int64_t gx0 = 0, gy0 = 0, gz0 = 0;        // offset of this context's interior in it
    int32_t px = 0, py = 0, pz = 0;
    std::vector<int64_t> ex, ey, ez;          // block edges per axis
    std::vector<HostChare> ch;
    std::vector<TileDev> tiles;
    std::vector<int32_t> dep_ptr, dep_idx;    // CSR: tiles each tile reads
    std::vector<int32_t> order;               // persistent task order
    // execution shape
    int32_t threads = 256, cpt = 4, stages = 4, tile_y = 0, tile_z = 0, amode = 1;
    int32_t max_nj = 0, max_nk = 0;                // largest tile actually used
    int32_t stage_doubles = 0;                // per-stage smem slot
    int32_t smem_bytes = 0;                   // dynamic smem per CTA
    // arena layout (byte offsets from the arena base)
    size_t off_err = 0, off_queue = 0, off_epoch = 0, off_chares = 0, off_tiles = 0;
    size_t off_dep_ptr = 0, off_dep_idx = 0, off_order = 0;
    size_t arena_bytes = 0;
    // model
    int64_t cells = 0, face_internal = 0, face_dirichlet = 0;
    double bytes_per_step = 0.0;
};

// Build the full plan; returns OD_OK or OD_EINVAL with *err set.
od_status build_plan(const od_config *cfg, Plan *plan, std::string *err);
// The same, choosing the default CTA shape by the lanes its tiles use alone
// when fill_gpu is false (a batch of many jobs fills the GPU, so a job's own
// tile count does not count against a shape), as the serving loop does.
od_status build_plan(const od_config *cfg, Plan *plan, std::string *err, bool fill_gpu);

// Ring-slot size for a tile of `nj` rows in a chare of row pitch `pitch`
// (the rows plus the two y-halo rows), in doubles.
int32_t stage_doubles_for(int32_t nj, int32_t pitch);

// Fill plan->info.
void plan_info(const Plan &p, od_plan_info *out);

}  // namespace od
