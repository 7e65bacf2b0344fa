/*
 * od.h -- C ABI of libod: an overdecomposed FP64 Jacobi solver (3D 7-point,
 * and the paper's own 2D 5-point) on one GPU (sm_103a).
 *
 * The method (the paper's Sec. III "Managing Overdecomposition" and Sec. V
 * "jacobi2d"): the grid is cut into many more blocks ("chares") than there are
 * GPUs; every Jacobi iteration each chare packs its boundary faces, delivers
 * them to its neighbours (Sec. IV, intra-process transfer: device-to-device),
 * the neighbours unpack them into their ghost layers, and each chare updates
 * its block.  Iterations run a fixed count with no convergence check.  In this
 * library all chares share one GPU; four execution paths run the same
 * arithmetic:
 *
 *   OD_PATH_PER_CHARE   one stream per chare (pooled), pack kernel, one
 *                       cudaMemcpyAsync D2D per face into the neighbour's
 *                       receive slot, unpack kernel, compute kernel, events
 *                       between neighbours (the runtime-level flow of Sec. III
 *                       "non-blocking streams", transport of Sec. IV item 1);
 *   OD_PATH_FUSED       one kernel per iteration over every (chare, tile);
 *                       pack+deliver+unpack are fused into compute: each new
 *                       boundary value is stored straight into the neighbour's
 *                       ghost layer (its "mailbox"); the kernel boundary is the
 *                       step barrier (kernel fusion, Sec. I, prior work);
 *   OD_PATH_GRAPH       the per-chare flow for two iterations captured once as
 *                       a CUDA graph and replayed (CUDA Graphs, Sec. I);
 *   OD_PATH_PERSISTENT  one launch for all iterations: CTAs take (step, tile)
 *                       tickets from a device queue and wait (bounded) on the
 *                       per-tile step counters of the tiles they read;
 *   OD_PATH_FUSED_GRAPH the fused path's step loop -- eight fused step kernels,
 *                       parities alternating -- captured once as a CUDA graph
 *                       and replayed (one-step graphs cover odd remainders):
 *                       CUDA Graphs (Sec. I) applied on top of kernel fusion.
 *
 * Arithmetic (every path, bit-identical to an undecomposed sweep):
 *   u'[i,j,k] = (((((u[i-1]+u[i+1]) + u[j-1]) + u[j+1]) + u[k-1]) + u[k+1]) / 6.0
 * in IEEE binary64 round-to-nearest, no FMA contraction, on the nx*ny*nz
 * interior; a one-cell Dirichlet shell around it stays fixed.
 *
 * Initial field: the value of padded global cell L = gx + (nx+2)*(gy + (ny+2)*gz)
 * (gx in [0,nx+1], ...) is the (L+1)-th output of a SplitMix64 stream seeded
 * with `seed`, top 53 bits times 2^-53.  init_mode 0: interior 0, shell random;
 * init_mode 1: every cell random.
 *
 * Conventions for every function:
 *   - returns OD_OK or an error code; never aborts the process; the message of
 *     the last error on the calling thread is od_last_error();
 *   - device pointers are plain CUDA device addresses of the context's device;
 *     host pointers are ordinary (pageable or pinned) host memory, except for
 *     od_write_async / od_read_async, which take pinned memory only;
 *   - the caller owns every buffer it passes; the library owns everything it
 *     allocates and frees it in od_destroy;
 *   - work is enqueued on the context's stream; od_read, od_read_cells,
 *     od_sync and od_stats_get synchronise that stream (and the copy stream
 *     of a pending od_read_async) and report device-side errors (OD_ETIMEOUT
 *     for a bounded wait that ran out, OD_ECUDA for a CUDA error);
 *   - one context is used by one host thread at a time (calls on the same
 *     od_ctx must not overlap); different contexts, and every od_server_*
 *     call, may be used from any threads concurrently.
 */
#ifndef OD_H
#define OD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* every entry point is exported from libod.so (built with hidden default
 * visibility) */
#if defined(__GNUC__)
#define OD_API __attribute__((visibility("default")))
#else
#define OD_API
#endif

typedef enum {
    OD_OK = 0,
    OD_EINVAL = 1,    /* bad argument or decomposition */
    OD_ENOMEM = 2,    /* device or host allocation failed, or arena too small */
    OD_ECUDA = 3,     /* a CUDA call or kernel failed */
    OD_ETIMEOUT = 4,  /* a bounded device-side wait ran out (no hang) */
    OD_EBUDGET = 5,   /* serving: job larger than the HBM budget */
    OD_ESTATE = 6,    /* call not valid in the object's current state */
    OD_ENOTFOUND = 7  /* serving: unknown job id */
} od_status;

typedef enum {
    OD_PATH_PER_CHARE = 0,
    OD_PATH_FUSED = 1,
    OD_PATH_GRAPH = 2,
    OD_PATH_PERSISTENT = 3,
    OD_PATH_FUSED_GRAPH = 4
} od_path;

#define OD_INIT_ZERO_INTERIOR 0
#define OD_INIT_UNIFORM 1

/* Stencils: the 3D 7-point Jacobi, and the paper's own 2D 5-point Jacobi
 * (Sec. V "jacobi2d"): u'[i,j] = ((((u[i-1]+u[i+1]) + u[j-1]) + u[j+1]) / 4 on
 * an nx*ny grid (nz = 1, one block along z), with the same seeded field,
 * Dirichlet shell and paths; the padded 2D cell L = gx + (nx+2)*gy gets
 * SplitMix64 output L+1.  A 2D configuration splits x by px / cuts_x and y by
 * py / cuts_y; od_read / od_write move nx*ny doubles, x fastest.  The tile
 * shape fields apply with tile_y capping a tile's row segment (cells along
 * x) and tile_z its rows. */
#define OD_STENCIL_3D7 0
#define OD_STENCIL_2D5 1

/* Problem, decomposition and execution settings.  Fill with
 * od_config_default() first, then set fields. */
typedef struct od_config {
    int64_t nx, ny, nz;          /* interior cells per axis, each >= 1 */
    int32_t px, py, pz;          /* chares per axis for a balanced split: the
                                    first n mod p blocks get ceil(n/p) cells,
                                    the rest floor(n/p); ignored on an axis
                                    whose cut list is given */
    const int32_t *cuts_x;       /* optional explicit block edges per axis:   */
    const int32_t *cuts_y;       /* ncuts+1 strictly ascending values from 0 */
    const int32_t *cuts_z;       /* to n (host memory, read during the call) */
    int32_t ncuts_x, ncuts_y, ncuts_z; /* blocks on that axis when cuts given */
    uint64_t seed;               /* initial-field seed */
    int32_t init_mode;           /* OD_INIT_ZERO_INTERIOR or OD_INIT_UNIFORM */
    int32_t path;                /* od_path */
    int32_t autotune;            /* 1: od_create times candidate execution
                                    shapes (CTA shape x arithmetic mode, then
                                    ring depth x planes per tile) on this
                                    decomposition and keeps the fastest; the
                                    field is initialised after tuning, so
                                    results do not change.  The choice is
                                    cached in OD_TUNE_CACHE (default
                                    $HOME/.cache/libod/tune.txt, "off" = no
                                    cache).  Needs a second arena's worth of
                                    device memory while tuning (skipped if
                                    that is not available). */
    int32_t tile_y;              /* max rows per tile (0 = planner default) */
    int32_t tile_z;              /* planes per tile (0 = planner default) */
    int32_t threads;             /* threads per CTA: 128, 256 or 512 */
    int32_t cells_per_thread;    /* 1, 2, 4 or 8; supported pairs 128 x {2,4,8},
                                    256 x {1,2,4,8}, 512 x {1,2}.  Both 0: the
                                    planner picks among 128x4, 128x2, 256x4
                                    (and 256x8 for rows past 1024 cells) by
                                    the lanes its tiles use, the halo rows and
                                    the tile count, preferring 128x4 */
    int32_t stages;              /* TMA ring slots, 3..8 (0 = 4): planes k-1,
                                    k, k+1 resident, the rest in flight */
    int32_t arith;               /* where the update's operations run (the bits
                                    never change): 0 all on the FP64 pipe;
                                    1 division by 6 on the integer pipes;
                                    1+k (k = 1..5) also the first k adds in an
                                    integer window aligned per cell; 7 / 8:
                                    modes 2 and 3 mixed cell by cell (half / a
                                    quarter of the cells in mode 3); 9 / 10:
                                    the last one / two adds in that window and
                                    the division from their result; 11: 9 and
                                    10 mixed; 12: two FP64 adds, the other
                                    three adds and the division in one integer
                                    window anchored for the whole field at its
                                    largest value (see od_write); 13: one FP64
                                    add, four window adds; 14 / 15: 13 on every
                                    other / every fourth cell, 12 on the rest.
                                    2D: 12 one FP64 add and two window adds,
                                    13 none and three, 14 the two mixed, 15
                                    two FP64 adds and one window add.  -1 =
                                    library default (12) */
    int32_t order;               /* persistent path task order, bits: 1 = reversed
                                    on odd steps, 2 = chares in Morton (Z) order
                                    instead of x-fastest; 0..3 */
    int32_t stream_pool;         /* per-chare path: streams (0 = min(nchares,32)) */
    int32_t device;              /* CUDA device ordinal */
    void *stream;                /* cudaStream_t to enqueue on; NULL = the
                                    library creates a non-blocking stream */
    void *arena;                 /* optional caller-owned device memory for all
                                    chare state (size from od_plan); NULL = the
                                    library allocates with cudaMalloc */
    uint64_t arena_bytes;        /* size of `arena` in bytes */
    uint64_t spin_limit_ns;      /* device-side wait limit (0 = 2 000 000 000) */
    int32_t stencil;             /* OD_STENCIL_3D7 (default) or OD_STENCIL_2D5 */
    int32_t pe_threads;          /* per-chare path: host threads that submit the
                                    chares' work in parallel, each with its own
                                    slice of the stream pool (the paper's several
                                    PEs per GPU); 0 or 1 = the calling thread */
    /* A shard: this context holds the sub-box [gx0, gx0+nx) x [gy0, gy0+ny) x
     * [gz0, gz0+nz) of a global grid gnx x gny x gnz (gnx = 0: the context is
     * the whole grid).  The initial field, including every ghost layer, is the
     * global field's; faces inside the global grid are fed by od_face_copy
     * imports, faces on its boundary hold the Dirichlet shell.  2D: gnz = 1,
     * gz0 = 0. */
    int64_t gnx, gny, gnz;
    int64_t gx0, gy0, gz0;
} od_config;

/* Host-only summary of a configuration's decomposition and memory. */
typedef struct od_plan_info {
    int64_t nchares;
    int64_t ntiles;                /* compute tasks per iteration */
    int64_t cells;                 /* interior cells (updates per iteration) */
    int64_t face_cells_internal;   /* ghost cells fed by a neighbour, summed
                                      over chares (each shared face twice) */
    int64_t face_cells_dirichlet;  /* ghost cells on the domain shell */
    uint64_t arena_bytes;          /* device bytes od_create needs */
    double bytes_per_step;         /* algorithmic HBM bytes per iteration:
                                      16*cells + 16*face_internal + 8*face_dirichlet */
    int32_t tile_y, tile_z;        /* largest tile used: rows, planes */
    int32_t threads, cells_per_thread, stages, arith;
    int32_t smem_bytes;            /* dynamic shared memory per CTA */
} od_plan_info;

typedef struct od_stats {
    int64_t steps_done;            /* iterations completed so far */
    int64_t kernel_launches;       /* kernels this context launched in od_step */
    int64_t api_calls;             /* CUDA stream operations issued by od_step
                                      (launches, copies, event records/waits,
                                      graph launches) */
    int64_t graph_launches;
    int32_t path;
    int32_t persistent_grid;       /* CTAs of the last persistent launch */
    int32_t tuned;                 /* 1: the execution shape came from the autotuner */
    double tune_ms_per_step;       /* the autotuner's time per step for it */
    od_plan_info plan;
} od_stats;

typedef struct od_ctx od_ctx;

/* Fill *cfg with defaults (a 1-chare 64^3 problem, fused path). */
OD_API void od_config_default(od_config *cfg);

/* Decompose and size a configuration without touching a GPU.  Errors:
 * OD_EINVAL for an impossible decomposition (a block thinner than one cell,
 * cut lists not ascending, more than 2^31 tiles). */
OD_API od_status od_plan(const od_config *cfg, od_plan_info *out);

/* Chare boxes of a configuration, host-only: for chare c (x fastest:
 * c = cx + px*(cy + py*cz)) writes box[6c..6c+5] = x0,bx,y0,by,z0,bz and
 * nbr[6c..6c+5] = neighbour chare on the x-,x+,y-,y+,z-,z+ side or -1 on the
 * domain boundary.  For OD_STENCIL_2D5 the boxes are x0,bx,y0,by,0,1 and the
 * neighbours x-,x+,y-,y+,-1,-1 of the 2D grid.  `capacity` = chares the
 * arrays hold. */
OD_API od_status od_decompose(const od_config *cfg, int64_t *box, int32_t *nbr, int64_t capacity);

/* The persistent path's schedule, host-only: the tiles of a configuration
 * and, per tile, the tiles it waits for (CSR).  *ntiles and *ndeps are always
 * set; tiles[8t..8t+7] = chare, x0, nx, y0, ny, z0, nz, 0 (the tile's box in
 * the context's interior coordinates; a 2D grid appears as (nx, 1, ny)) is
 * written when tiles_cap >= *ntiles, and dep_ptr (ntiles+1 entries) and
 * dep_idx when, in addition, deps_cap >= *ndeps.  Tile b is in tile a's list
 * iff a 7-point update of a's cells reads b's cells or the other way round:
 * the boxes overlap, or touch across a face. */
OD_API od_status od_plan_tiles(const od_config *cfg, int64_t *tiles, int64_t tiles_cap, int32_t *dep_ptr,
                               int32_t *dep_idx, int64_t deps_cap, int64_t *ntiles, int64_t *ndeps);

/* Allocate device state on cfg->device, build the chare/tile tables, tune if
 * asked, and write the initial field (u^0) including every ghost layer.
 * Synchronous.  *out is NULL on error.
 * Defined by: the paper's Sec. III "Managing Overdecomposition" (many chares
 * of one application share one GPU; device memory and execution resources
 * are set up once, Sec. III "Using Kokkos in charm++ runtime") and Sec. IV
 * (the pre-filled location table: here the neighbour table built from the
 * decomposition). */
OD_API od_status od_create(od_ctx **out, const od_config *cfg);

/* Enqueue `iters` >= 0 Jacobi iterations on the context's stream with its
 * current path.  Asynchronous: returns once the work is enqueued.  No
 * allocation and no host synchronisation happen inside (the graph path
 * captures its graphs on the first call).
 * Defined by: Sec. V "jacobi2d" (Jacobi iterations with a halo exchange
 * between chares, a fixed count, no convergence check), each chare's
 * per-iteration work -- pack, intra-process delivery, unpack, compute --
 * from Sec. III "Managing Overdecomposition" and Sec. IV item 1
 * (intra-process transfers as device-to-device copies). */
OD_API od_status od_step(od_ctx *ctx, int32_t iters);

/* Select the execution path for later od_step calls (any path continues the
 * same iteration sequence).  The paths are the flows of Sec. III (per-chare
 * streams) and Sec. I (kernel fusion and CUDA graphs, prior work). */
OD_API od_status od_set_path(od_ctx *ctx, int32_t path);

/* Wait for all enqueued work; reports device-side errors.  (Sec. III "Using
 * Kokkos in charm++ runtime": the library never fences implicitly; this is
 * the one explicit wait besides the reads.) */
OD_API od_status od_sync(od_ctx *ctx);

/* Defined by: Sec. V "jacobi2d" (the field the iterations produce; the
 * paper gives no output format, so the interior is returned in the
 * undecomposed grid's order).
 * Copy the current field u^{steps_done} (interior only, x fastest,
 * nx*ny*nz doubles) to dst.  dst_is_device != 0: dst is device memory of the
 * context's device; otherwise host memory: pinned (page-locked) host memory
 * is written in place by the gather kernel over the host link, pageable
 * memory through a device staging buffer of nx*ny*nz doubles allocated on
 * the first such read or write and kept.  Synchronises the stream. */
OD_API od_status od_read(od_ctx *ctx, double *dst, int32_t dst_is_device);

/* Read n (0..2^24) cells of the current field into out (host), without
 * reading the whole grid: cells[i] is a global interior index, x fastest
 * (x + nx*(y + ny*z); 2D: x + nx*y).  Allocates two small device buffers for
 * the call; synchronises the stream.  OD_EINVAL for an index outside the
 * grid. */
OD_API od_status od_read_cells(od_ctx *ctx, const int64_t *cells, int64_t n, double *out);

/* Defined by: Sec. II "Charm++ and Overdecomposition" (chares migrate, so
 * their state must be exported and restored: od_read and this call) and
 * Sec. V "jacobi2d" (the iterated field); the layout is od_read's.
 * Replace the current field's interior with src (nx*ny*nz doubles, x fastest;
 * device memory, or host memory copied through the staging buffer) and
 * refresh every internal ghost layer; the
 * Dirichlet shell is kept.  Used to import a checkpoint or a user field.
 * Enqueued on the stream (host sources are copied before return).  The
 * context keeps the largest positive value its field has held (the initial
 * field's values lie in [0, 1)), raised here by the values written; the
 * anchored arithmetic modes place their integer window there, so a field
 * that later lies far below that value runs mostly in the IEEE form --
 * slower, with the same bits. */
OD_API od_status od_write(od_ctx *ctx, const double *src, int32_t src_is_device);

/* Asynchronous forms of od_write / od_read for pinned (page-locked) host
 * memory: the transfer is enqueued and the call returns at once; the caller
 * leaves the buffer alone until od_sync (or any call that synchronises the
 * context) returns.  Host data moves by the copy engine through the staging
 * buffer (allocated on first use, nx*ny*nz doubles), with the scatter /
 * gather kernel on the device side, so a transfer overlaps other contexts'
 * work and holds SMs only for the short kernel.  od_write_async enqueues the
 * copy and the scatter on the context's stream.  od_read_async enqueues the
 * gather on the context's stream and the device-to-host copy on a copy
 * stream of the context that waits for the gather: work enqueued on the
 * context's stream afterwards (an event that another context's stream waits
 * on, say) follows the gather but not the copy, which lets a caller run two
 * contexts as a pipeline, one job's copies under the other's iterations.
 * OD_EINVAL when the buffer is not pinned host memory. */
OD_API od_status od_write_async(od_ctx *ctx, const double *src);
OD_API od_status od_read_async(od_ctx *ctx, double *dst);

/* Face exchange of a shard (a context holding a sub-box of a global grid,
 * see od_config.gnx): the data of the paper's transports between chares of
 * different processes (Sec. IV).  dir 0 (export) copies the current field's
 * boundary layer on domain face `face` -- the interior cells next to it --
 * into buf; dir 1 (import) copies buf into the ghost layer on that face,
 * which the next iteration reads.  face: 0..5 = x-, x+, y-, y+, z-, z+ (2D:
 * 0..3 = x-, x+, y-, y+ of the 2D grid).  buf holds the whole face, dense:
 * x faces nz x ny doubles (y fastest), y faces nz x nx, z faces ny x nx (x
 * fastest); 2D x faces ny, y faces nx.  buf_is_device != 0: device memory of
 * the context's device, the copy is enqueued on the context's stream;
 * otherwise host memory, and the call synchronises.  od_write does not touch
 * the ghost layers of a shard's domain faces: import them after it. */
OD_API od_status od_face_copy(od_ctx *ctx, int32_t face, int32_t dir, double *buf, int32_t buf_is_device);

/* Counters and the plan; synchronises and reports device-side errors.  The
 * launch and API-call counts are the quantities Sec. III measures (kernel
 * launch cost per chare). */
OD_API od_status od_stats_get(od_ctx *ctx, od_stats *out);

/* Fault injection for tests: on the persistent path, tile `tile` never
 * publishes its step counter, so the tiles that wait on it run into the wait
 * limit and od_sync returns OD_ETIMEOUT.  -1 switches it off. */
OD_API od_status od_debug_stall_tile(od_ctx *ctx, int64_t tile);

/* Self-test of the exact integer-pipe arithmetic the kernels use (a
 * correctly rounded division by 6 and a correctly rounded addition, written
 * from the IEEE 754 binary64 definition).  op 0: out[i] = a[i] / 6.0;
 * op 1: out[i] = a[i] + b[i] (b unused for op 0); op 2 / 3: the same on the
 * FP64 pipe (device only); op 10+m (m = 0..6): the whole Jacobi update
 * (((((a0+a1)+a2)+a3)+a4)+a5)/6 of the six operands a[6i..6i+5] in
 * arithmetic mode m (see od_config.arith), b unused; op 17 / 18: the same
 * update in the tail form with one / two window adds (modes 9 and 10); op
 * 20+m (m = 0..4): the 2D update (((a0+a1)+a2)+a3)/4 of a[4i..4i+3] in mode m
 * (m = 4: three window adds); op 25 / 26: its tail form; op 30+f (f = 0..3)
 * / 40+f (f = 0..2): the 3D / 2D update in the anchored window with its
 * first f adds on the FP64 pipe, b[0] holding the anchor exponent E0 (an
 * integer, clamped to [4, 2030]); op 34+f / 44+f: the anchored form alone,
 * NaN where a cell leaves it.  od_arith_host runs the routines on the host
 * CPU over host arrays; od_arith_device runs them in a kernel over device
 * arrays of the current device and synchronises.  n >= 0 elements. */
OD_API od_status od_arith_host(int32_t op, const double *a, const double *b, double *out, int64_t n);
OD_API od_status od_arith_device(int32_t op, const double *a, const double *b, double *out, int64_t n);

/* ------------------------------------------------------------------ inter-process transport
 *
 * The paper's intra-node, inter-process path (Sec. IV, transport item 2):
 * every process allocates one device communication buffer and a pool of
 * interprocess events once (od_comm_create), and every peer maps them once
 * through their IPC handles (od_comm_handles in the owner, od_comm_open in
 * the peer), so no handle is opened per message.  A face of a shard then
 * moves by two device-to-device copies: the sender exports it into its own
 * buffer (od_face_copy, dir 0) and records an event (od_comm_record); after a
 * host control message with the buffer offset and the event index, the
 * receiver makes its stream wait on that event of the sender's endpoint
 * (od_comm_wait) and imports from the mapped buffer (od_face_copy, dir 1).
 * The endpoints work within one process too (no od_comm_open needed). */
typedef struct od_comm od_comm;

/* Bytes of an endpoint's handle block: a 16-byte header, the buffer's IPC
 * handle and one IPC handle per event (64 bytes each). */
#define OD_COMM_HANDLE_BYTES(nevents) (16u + 64u * (1u + (uint64_t)(nevents)))

/* A new endpoint on `device`: `bytes` (1..2^40) of device memory and
 * `nevents` (1..4096) interprocess events (timing disabled).  Owned by the
 * caller until od_comm_destroy. */
OD_API od_status od_comm_create(od_comm **out, int32_t device, uint64_t bytes, int32_t nevents);
/* Write the endpoint's handle block (OD_COMM_HANDLE_BYTES(nevents) bytes) for
 * the peers.  OD_ESTATE for an endpoint opened from a peer. */
OD_API od_status od_comm_handles(const od_comm *c, void *handles, uint64_t capacity);
/* Map a peer process's endpoint from its handle block (`size` bytes) into
 * this process on `device` (the same physical GPU or a peer of it).  The
 * handles of an endpoint of this same process cannot be opened (CUDA
 * refuses): use that endpoint directly. */
OD_API od_status od_comm_open(od_comm **out, int32_t device, const void *handles, uint64_t size);
/* The endpoint's buffer (device pointer, valid in this process), its size
 * and event count; any output may be NULL. */
OD_API od_status od_comm_buffer(const od_comm *c, double **buf, uint64_t *bytes, int32_t *nevents);
/* Record event `event` of the endpoint on `stream` (a cudaStream_t). */
OD_API od_status od_comm_record(od_comm *c, int32_t event, void *stream);
/* Make `stream` wait for the last recording of event `event` of the endpoint
 * that happened before this call (host order: the recorder's control
 * message must have arrived first). */
OD_API od_status od_comm_wait(od_comm *c, int32_t event, void *stream);
/* Free the buffer and events (or unmap a peer's); the caller must have
 * finished every stream that uses them. */
OD_API od_status od_comm_destroy(od_comm *c);

/* ------------------------------------------------------------------ launch overhead
 *
 * Microbenchmarks of what a kernel launch costs an overdecomposed application
 * (the paper's Sec. III measurements), the context for the per-chare path's
 * slowdown with ODF.  Each call runs on `device`, creates and frees its own
 * streams, events and buffers, returns after the GPU has finished, and bounds
 * every host wait (10 s per wait: OD_ETIMEOUT).  Arguments are checked before
 * any CUDA call (OD_EINVAL). */

/* One kernel at a time: an empty one-block kernel is launched and waited for,
 * `reps` times (1..1e6) after 10 untimed ones.  wait: 0 = cudaStreamSynchronize,
 * 1 = polling an event (cudaEventQuery), 2 = a host function enqueued behind
 * the kernel (cudaLaunchHostFunc) sets a flag the caller polls -- the
 * callback style of a task runtime.  *us = mean wall-clock microseconds per
 * launch-and-wait round trip. */
OD_API od_status od_bench_launch_latency(int32_t device, int32_t wait, int32_t reps, double *us);

/* Pre-enqueued release: `total_threads` (1..2^30) threads of a fixed-work
 * kernel are split into `nkernels` (1..1024) contiguous kernels, one
 * non-blocking stream each; every stream first waits on one host-mapped flag
 * (cuStreamWaitValue32, resolved from the driver at run time), and the host
 * releases all of them at once.  Thread g iterates the 32-bit LCG
 * x <- 1664525 x + 1013904223 `work` times (0..1e6, total_threads*work <= 2^40)
 * from x = g and stores x in out[g]; `out` is a device buffer of
 * total_threads uint32 owned by the caller, or NULL for a scratch buffer.
 * *us = time from the first stream passing the flag until the last kernel
 * finished (device events). */
OD_API od_status od_bench_release(int32_t device, int64_t total_threads, int32_t nkernels, int32_t work,
                                  uint32_t *out, double *us);

/* Launch rate: `host_threads` (1..64) host threads each drive `chares`
 * (1..64) chares; a chare owns a stream and fires an empty kernel of one
 * block per SM, then the next once its thread has seen (by polling an
 * event) that the previous one completed, `kernels` times (at most 1e7
 * kernels in all).  *per_s = kernels completed per second of wall time. */
OD_API od_status od_bench_launch_rate(int32_t device, int32_t host_threads, int32_t chares, int32_t kernels,
                                      double *per_s);

/* ------------------------------------------------------------------ serving
 *
 * A server admits independent solves as they arrive and keeps their state
 * resident in one device pool of hbm_budget_bytes.  By default (job_streams
 * > 0) each admitted job's whole run is one persistent launch on its own
 * stream and the jobs' kernels share the SMs; with job_streams = 0 it
 * advances every running job by batch_steps iterations per batched launch
 * (continuous batching: jobs that arrive while others run join the next
 * launch, finished jobs drop out).  Admission is first come, first served, while a slot is free
 * (max_active, 0 = no limit) and the pool has room for the job's arena.  A
 * worker thread inside the server drives the device; every call below is
 * thread-safe.  Each job's result is bit-identical to the same job solved
 * alone with od_create/od_step.  The paper's runtime schedules many chares of
 * one application per GPU (Sec. III); serving many applications on one GPU
 * has no counterpart in the paper. */
#define OD_JOB_QUEUED 0
#define OD_JOB_RUNNING 1
#define OD_JOB_DONE 2
#define OD_JOB_FAILED 3

typedef struct od_server od_server;

typedef struct od_server_config {
    uint64_t hbm_budget_bytes;   /* device memory for all resident jobs */
    int32_t max_active;          /* jobs resident at once (0 = no limit) */
    int32_t max_jobs_per_launch; /* batched mode: batch table size (0 = 256) */
    int32_t device;
    int32_t threads, cells_per_thread, stages; /* CTA shape for every job; threads and
                                    cells_per_thread both 0: the planner picks
                                    each job's shape (as od_config; batched mode
                                    runs one launch per shape in use); stages
                                    0 = 4 */
    int32_t arith;               /* as od_config.arith (-1 = 12) */
    void *pool;                  /* caller device memory of hbm_budget_bytes, 256-byte
                                    aligned, or NULL: the server allocates it once */
    int32_t batch_steps;         /* steps of every running job that one launch advances
                                    (0 = 8): a persistent launch per CTA shape takes
                                    (step, job, tile) tickets, so no step ends in a
                                    partial wave; jobs admitted meanwhile join the next
                                    launch.  1: one fused step per launch */
    int32_t job_streams;         /* 0: the batched launches above.  N in [1, 64]: each
                                    admitted job's whole run is one persistent launch
                                    (od_step on the job's context, path persistent) on
                                    the least-loaded of N streams, and the jobs' kernels
                                    share the SMs as the hardware schedules them;
                                    batch_steps is then unused.  od_server_config_default
                                    sets 16 */
} od_server_config;

typedef struct od_job_info {
    int32_t state;               /* OD_JOB_* */
    int32_t iters;
    int64_t cells;
    uint64_t arena_bytes;        /* the job's share of the budget */
    double t_submit, t_admit, t_done;  /* seconds since the server was created */
} od_job_info;

typedef struct od_server_stats_t {
    int64_t queued, running, done, failed;
    int64_t launches;            /* batched kernel launches */
    double updates_done;         /* cell updates of completed jobs */
    uint64_t pool_used, pool_peak;
    double seconds;              /* since the server was created */
    double admit_seconds;        /* spent creating job contexts (on the
                                    admission thread, beside the launches) */
    double busy_seconds;         /* device time of the completed batched
                                    launches (events around each kernel) */
} od_server_stats_t;

OD_API void od_server_config_default(od_server_config *cfg);
/* Allocate the pool (unless given), streams and launch tables; start the worker. */
OD_API od_status od_server_create(od_server **out, const od_server_config *cfg);
/* Queue a job: the decomposition and seed of *job (cut lists are copied;
 * path, tile shape, stream and arena fields are ignored) and its iteration
 * count.  OD_EBUDGET if the job alone exceeds the whole budget; OD_EINVAL for
 * a stencil other than OD_STENCIL_3D7 with batched launches (job_streams = 0:
 * a batched launch shares one kernel); per-job launches also take
 * OD_STENCIL_2D5 jobs. */
OD_API od_status od_server_submit(od_server *s, const od_config *job, int32_t iters, uint64_t *job_id);
/* Wait up to timeout_s seconds for the job to be done or failed; *state is
 * its state on return (OD_OK also on timeout). */
OD_API od_status od_server_wait(od_server *s, uint64_t job_id, double timeout_s, int32_t *state);
/* The serving loop's completion queue: *job_id = the next job that ended
 * (done or failed), in the order they ended, waiting up to timeout_s seconds
 * for one; *job_id = 0 when none ended in time (OD_OK either way).  Each job
 * is reported once, whether or not it was waited for; a client that releases
 * jobs as they end keeps the budget free for new arrivals. */
OD_API od_status od_server_next_completion(od_server *s, double timeout_s, uint64_t *job_id);
OD_API od_status od_server_job_info(od_server *s, uint64_t job_id, od_job_info *out);
/* Copy a done job's field (nx*ny*nz doubles, x fastest) to dst (device or host). */
OD_API od_status od_server_fetch(od_server *s, uint64_t job_id, double *dst, int32_t dst_is_device);
/* Short names of the serving loop: od_submit = od_server_submit, od_fetch =
 * od_server_fetch; od_poll sets *done = 1 once the job is done or failed (0
 * while it is queued or running) without waiting. */
OD_API od_status od_submit(od_server *s, const od_config *job, int32_t iters, uint64_t *job_id);
OD_API od_status od_poll(od_server *s, uint64_t job_id, int32_t *done);
OD_API od_status od_fetch(od_server *s, uint64_t job_id, double *dst, int32_t dst_is_device);
/* Forget a job that is done, failed or still queued, returning its memory to
 * the pool.  OD_ESTATE while it runs, and in the short window in which the
 * admission thread is creating its context (release it after it has run). */
OD_API od_status od_server_release(od_server *s, uint64_t job_id);
OD_API od_status od_server_stats(od_server *s, od_server_stats_t *out);
/* Stop the worker (after the launches in flight) and free everything. */
OD_API od_status od_server_destroy(od_server *s);

/* Jacobi iterations on a caller's field without allocating device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory where they call -- a framework that owns all
 * device memory through its own pool and forbids allocations it does not
 * track, or a latency-critical loop where cudaMalloc/cudaFree would
 * synchronise the device.  It calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * u_in, u_out: caller-owned device arrays of the current device, each the
 * padded field (nx+2)*(ny+2)*(nz+2) doubles, x fastest (cell (gx,gy,gz) at
 * gx + (nx+2)*(gy + (ny+2)*gz)); the one-cell shell is the fixed Dirichlet
 * boundary.  u_in is read only; on completion u_out holds the field after
 * `iters` >= 0 iterations (shell copied from u_in), bit-identical to the
 * undecomposed sweep and to od_step.  u_in and u_out must not overlap.
 * Work is enqueued on `stream` (a cudaStream_t, NULL = the legacy default
 * stream); the call returns without waiting.
 *
 * Scratch: the second buffer of the double buffer is a static device array of
 * OD_NOALLOC_MAX_PADDED_CELLS doubles (64 MiB) that every GPU which loads
 * this library holds until the process exits.  Larger grids are rejected with
 * OD_EINVAL.  Every call shares that array and it keeps the last call's
 * contents (each call first overwrites the part it uses), so calls whose work
 * overlaps on the GPU -- on different streams or from different host threads
 * -- race and must be serialised by the caller.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture.
 * Errors: OD_EINVAL (null, aliasing or out-of-range arguments, grid too
 * large), OD_ECUDA (a CUDA call failed); message in od_last_error(). */
#define OD_NOALLOC_MAX_PADDED_CELLS (8ll * 1024 * 1024)
OD_API od_status od_jacobi_noalloc(const double *u_in, double *u_out, int64_t nx, int64_t ny, int64_t nz,
                                   int32_t iters, void *stream);

/* Free everything the context owns (synchronises first).  NULL is allowed.
 * Defined by: Sec. III "Using Kokkos in charm++ runtime" (device state is
 * created once and released once, never inside the iterations). */
OD_API od_status od_destroy(od_ctx *ctx);

/* Message of the last failed call on this thread ("" if none). */
OD_API const char *od_last_error(void);

/* Library version string. */
OD_API const char *od_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OD_H */
