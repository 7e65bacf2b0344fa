// od_internal.h -- structures shared by the host planner and the CUDA kernels
// of libod (overdecomposed 3D 7-point FP64 Jacobi on one GPU).
//
// Memory layout of one chare (block) in HBM, per parity p in {0,1}:
//   A[p] : (bz+2) planes x (by+2) rows x pitch doubles, pitch = bx+2 rounded
//          up to 2 (every row starts 16-byte aligned).  Plane 0 / bz+1 are the
//          z-ghost planes, row 0 / by+1 of every plane the y-ghost rows,
//          column 0 / bx+1 of every row the x-ghost cells, columns [1,bx] the
//          cells; a last column may be padding.
//          Interior cell (i,j,k) is A[p][((k+1)*(by+2) + (j+1))*pitch + i+1].
// A tile of full rows plus its two y-halo rows is then one contiguous run
// that already holds the x-ghosts, fetched by a single 1D bulk copy (TMA),
// and in shared memory x-1 / x+1 are the neighbouring words for every cell.
// Edge and corner ghost cells of the padded box exist but are never read by
// a 7-point stencil.
//
// The 2D 5-point stencil runs on the internal grid (nx, 1, ny): a chare's 2D
// rows are its "planes", and a plane is a single row (rows = 1, no y-ghost
// rows), so A[p] is the chare's padded 2D block, (bz+2) rows x pitch:
// interior cell (i, k) is A[p][(k+1)*pitch + i+1].  In general a plane holds
// `rows` rows and interior row j sits at row j + row0 of it: rows = by+2,
// row0 = 1 in 3D; rows = 1, row0 = 0 in 2D.
//
// On the per-chare path a neighbour delivers a face into these ghost cells
// (pack, copy, unpack: the chare's mailbox).  The fused tile sweeps instead
// read a face straight from the neighbour's own array -- its boundary
// planes and rows by bulk copies into the tile's ring slots, its boundary
// column by plain loads -- so an internal ghost layer of a chare is only
// current after a per-chare step, od_create or od_write (the context tracks
// this and refreshes the ghosts before a per-chare step needs them).  Faces
// on the domain boundary hold the Dirichlet shell in both parities and are
// never written after initialisation.
#pragma once
#include <stdint.h>

#define OD_FACE_XLO 0
#define OD_FACE_XHI 1
#define OD_FACE_YLO 2
#define OD_FACE_YHI 3
#define OD_FACE_ZLO 4
#define OD_FACE_ZHI 5

#define OD_ERR_TMA_TIMEOUT 1    // a bulk-copy wait ran out
#define OD_ERR_DEP_TIMEOUT 2    // a dependency (step counter) wait ran out
#define OD_ERR_BAD_LAUNCH 3     // kernel saw an inconsistent launch shape

// One chare as the kernels see it (device table, one entry per chare).
struct ChareDev {
    int32_t bx, by, bz;     // interior extents
    int32_t pitch;          // row stride of A, doubles
    int32_t rows, row0;     // rows per plane; row of interior row 0 in a plane
    int32_t nbr[6];         // neighbour per face or -1 (Dirichlet)
    int32_t foff[7];        // face offsets inside send/recv buffers (doubles)
    int64_t x0, y0, z0;     // global interior offset of cell (0,0,0)
    double *A[2];
    double *send;           // per-chare path: packed new faces
    double *recv[2];        // per-chare path: faces from neighbours, 2 slots
};

// One compute task: columns [i0,i0+ni) x rows [j0,j0+nj) x planes
// [k0,k0+nk) of chare c (3D tiles take whole rows: i0 = 0, ni = bx).
struct TileDev {
    int32_t c, j0, nj, k0, nk;
    int32_t i0, ni;
    int32_t pad;
};

// Error record written by kernels (first error wins).
struct ErrDev {
    int32_t code;
    int32_t tile;
    int32_t step;
    int32_t pad[13];
};

// Arguments of the tile kernels (passed by value).
struct KArgs {
    const ChareDev *ch;
    const TileDev *tiles;
    ErrDev *err;
    int32_t *queue;          // persistent: ticket counter (zeroed per launch)
    int32_t *epoch;          // persistent: steps finished per tile in this launch
    const int32_t *dep_ptr;  // persistent: CSR of the tiles each tile reads
    const int32_t *dep_idx;
    const int32_t *order;    // persistent: tile of each queue position
    const uint64_t *vmax;    // bit pattern of the largest value the field holds (a positive
                             // double), from which the anchored arithmetic takes its window
    int32_t tile_begin;      // static launch: tile of blockIdx.x == 0
    int32_t ntiles;          // tiles per step
    int32_t parity;          // static launch: parity of the source buffer
    int32_t iters;           // persistent: steps in this launch
    int32_t t0;              // persistent: absolute step of the first one
    int32_t order_mode;      // persistent: 1 = reverse order on odd steps
    int32_t stages;          // TMA ring depth
    int32_t stage_doubles;   // doubles per ring slot
    int32_t stencil;         // OD_STENCIL_3D7 or OD_STENCIL_2D5
    uint32_t one;            // 1, passed at run time so that the arithmetic's adds written as
                             // multiply-adds by it stay on the FMA pipe (od_arith.cuh)
    int64_t stall_tile;      // fault injection (-1 = off)
    uint64_t spin_ns;        // bound on every device-side wait
};
