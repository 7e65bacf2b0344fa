// od_kernels.h -- launch wrappers for libod's device kernels (host side).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "od_internal.h"

namespace od {

// Tile kernels exist for (threads, cells per thread) in {128}x{2,4,8},
// {256}x{1,2,4,8}, {512}x{1,2}, arithmetic modes 0..15 and both stencils
// (OD_STENCIL_3D7, OD_STENCIL_2D5) (od_tile.cuh).
bool tile_shape_supported(int threads, int cpt, int amode, int stencil);

// Raise the dynamic shared-memory limit of the tile kernels of one shape.
cudaError_t prepare_tile_kernels(int threads, int cpt, int amode, int smem_bytes, int stencil);

// One CTA per tile, tiles [a.tile_begin, a.tile_begin + grid), of stencil
// a.stencil (so for launch_persistent).  push = 1 also
// stores each new boundary value into the neighbour's ghost layer.
cudaError_t launch_tiles(const KArgs &a, int grid, int threads, int cpt, int amode, bool push, int smem_bytes,
                         cudaStream_t s);

// One fused step of several jobs (continuous batching): jobs[j] (device
// array) is job j's KArgs with its source parity, first[j] its first block
// (device array of njobs+1 prefix sums, first[njobs] = grid); geom (host)
// carries the launch's ring geometry and wait limit: stages, stage_doubles
// (at least every job's) and spin_ns.
cudaError_t launch_tiles_multi(const KArgs *jobs, const int32_t *first, int32_t njobs, const KArgs &geom, int grid,
                               int threads, int cpt, int amode, int smem_bytes, int stencil, cudaStream_t s);

// Several fused steps of several jobs in one persistent launch: jobs[j]
// (device array) carries job j's tables, its absolute first step (t0) and
// its steps in this launch (iters <= steps); first[] as for
// launch_tiles_multi; queue a zeroed device counter.
cudaError_t launch_persistent_multi(const KArgs *jobs, const int32_t *first, int32_t njobs, int32_t steps,
                                    int32_t *queue, const KArgs &geom, int grid, int threads, int cpt, int amode,
                                    int smem_bytes, int stencil, cudaStream_t s);

// Persistent ticket kernel over a.iters steps.
cudaError_t launch_persistent(const KArgs &a, int grid, int threads, int cpt, int amode, int smem_bytes,
                              cudaStream_t s);
cudaError_t persistent_occupancy(int threads, int cpt, int amode, int smem_bytes, int stencil,
                                 int *blocks_per_sm);
cudaError_t persistent_multi_occupancy(int threads, int cpt, int amode, int smem_bytes, int stencil,
                                       int *blocks_per_sm);

// The initial field of a shard at offset (gx0, gy0, gz0) of a global grid
// gnx x gny x gnz (the whole grid: offsets 0, global = local extents).
cudaError_t launch_init(const ChareDev *ch, int nch, int64_t gnx, int64_t gny, int64_t gnz, int64_t gx0,
                        int64_t gy0, int64_t gz0, uint64_t seed, int mode, int stencil, cudaStream_t s);
// Domain-face exchange of a shard (od_face_copy): dir 0 copies the boundary
// layer of parity p on face f into buf, dir 1 buf into the ghost layer.
cudaError_t launch_face_copy(const ChareDev *ch, int nch, int parity, int face, int dir, double *buf, int64_t nx,
                             int64_t ny, int64_t nz, cudaStream_t s);
cudaError_t launch_pack(const ChareDev *ch, int c, int parity, int elems, cudaStream_t s);
cudaError_t launch_unpack(const ChareDev *ch, int c, int parity, int slot, int elems, cudaStream_t s);
// out[i] = *addr[i] for n device addresses (od_read_cells).
cudaError_t launch_read_cells(const double *const *addr, int64_t n, double *out, cudaStream_t s);
cudaError_t launch_gather(const ChareDev *ch, int nch, int parity, int64_t nx, int64_t ny, double *g,
                          cudaStream_t s);
// Arithmetic self-test over device arrays (op: 0 div6, 1 add on the integer
// pipes; 2 division by 6, 3 add on the FP64 pipe).
cudaError_t launch_arith(int op, const double *a, const double *b, double *out, int64_t n, cudaStream_t s);
// Import (od_write): also raises *vmax (device word, may be null) to the
// bit pattern of the largest positive finite value written.
cudaError_t launch_scatter(const ChareDev *ch, int nch, int parity, int64_t nx, int64_t ny, int64_t nz,
                           const double *g, uint64_t *vmax, cudaStream_t s);
// Internal ghost layers of parity `parity` from the neighbours' boundaries.
cudaError_t launch_ghost_refresh(const ChareDev *ch, int nch, int parity, cudaStream_t s);

}  // namespace od
