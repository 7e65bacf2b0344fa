// od_tile.cuh -- the tile sweep of libod (sm_103a), shared by the per-chare
// compute kernel, the fused step kernel and the persistent kernel.
//
// A 3D task is nj full rows x nk planes of one chare.  One elected thread
// issues, per z-plane, a 1D bulk copy (cp.async.bulk, the TMA's untiled form)
// of the tile's nj rows plus its two y-halo rows -- one contiguous run of the
// chare's padded array that already holds the x-ghosts -- into a ring slot
// whose mbarrier counts the transaction bytes.  The ring keeps planes k-1, k
// and k+1 resident while plane k is computed, with the other `stages` - 3
// slots in flight.  Every thread owns the same cells of every plane and reads
// all six neighbours from shared memory.  The new value is stored once to
// HBM, coalesced.  On the fused paths a tile reads the faces of its
// neighbour chares straight from their arrays (their boundary planes and
// rows by further bulk copies into the same ring slot, their boundary column
// by plain loads issued a plane ahead): delivery and unpack are fused into
// the load, pack needs nothing, and the cell loop has no face branches.  The
// 2D task (run_tile_2d) is a row segment over a run of rows, the same way,
// storing its boundary values into the neighbours' ghost cells.
//
// The arithmetic is the Jacobi update of the paper's stencil proxy (Sec. V,
// "jacobi2d"; 3D 7-point, or the paper's own 2D 5-point) with round-to-
// nearest binary64 adds and division and no contraction, which is what makes
// every path bit-identical to an undecomposed sweep.
//
// Every wait is bounded by KArgs::spin_ns (wall clock, %globaltimer): a wait
// that runs out records an error and the CTA leaves after draining its own
// copies in flight, so a lost copy or a stalled neighbour never hangs the GPU.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "od.h"
#include "od_arith.cuh"
#include "od_internal.h"

namespace od {
namespace tile {

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1D bulk copy global -> shared, completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int32_t ld_acquire(const int32_t *p) {
    int32_t v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int32_t *p, int32_t v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int32_t ld_relaxed(const int32_t *p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// orders this CTA's generic stores to shared memory before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (now_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void record_err(ErrDev *e, int code, int tile, int step) {
    if (atomicCAS(&e->code, 0, code) == 0) {
        e->tile = tile;
        e->step = step;
    }
}

// ---------------------------------------------------------------- update

// ---------------------------------------------------------------- tile sweep

// IEEE form of the update for the rare cells whose operands leave the
// integer routines' domain.  Kept out of line so the compiler cannot merge it
// with (or speculate it beside) the fast form in the hot loop.
static __device__ __noinline__ double update_slow(double W, double E, double S, double N, double D, double U) {
    // IEEE adds, the division by 6 on the integer pipes (exact for every
    // input): the FP64 pipe's division sequence made each such cell cost
    // more than twice as much on that pipe
    return jacobi_update_ieee<true>(W, E, S, N, D, U);
}

// Which thread refills a ring slot: lane 0 of a different warp each plane
// (1) or thread 0 always (0); a build may choose (-DOD_ROTATE_ISSUE=0).
#ifndef OD_ROTATE_ISSUE
#define OD_ROTATE_ISSUE 1
#endif

struct Ring {
    double *base;      // first slot
    uint64_t *bars;    // one mbarrier per slot
    uint32_t seq;      // planes issued by this CTA before the current tile
};

// The anchored arithmetic's parameters for one launch: the window anchor for
// cells with one or no FP64 add (e0), +1 for cells with two or three, and
// the run-time 1 of the multiply-adds.
struct Arith {
    uint32_t e0, one;
};

template <int AM>
__device__ __forceinline__ Arith arith_setup(const KArgs &a, const KArgs &g) {
    Arith r;
    r.one = g.one;  // from the kernel parameter g (a constant-bank operand, no register)
    r.e0 = AM >= 12 ? anchor_for(a.vmax ? *a.vmax : 0ull, 1) : 0u;
    return r;
}

// Where a 3D fused tile reads the faces of its neighbours (source parity),
// prepared once per tile by thread 0 in shared memory:
//   x-/x+: the neighbour's column next to the face, cell (row, plane) at
//          x? + (plane+1)*x?_plane + row*x?_pitch (padded coordinates)
//   y-/y+: the neighbour's row next to the face in padded plane q at
//          y? + q*y?_plane (same x extent, so the same pitch)
//   z-/z+: the neighbour's plane next to the face, the tile's rows (same x
//          and y extents, so the same layout)
// (null: a domain face, whose ghost layer holds the Dirichlet shell).
struct PullInfo {
    const double *xlo, *xhi, *ylo, *yhi, *zlo, *zhi;
    int32_t xlo_pitch, xlo_plane, xhi_pitch, xhi_plane, ylo_plane, yhi_plane;
};

constexpr int kSmemBars = 0;     // up to 8 mbarriers
constexpr int kSmemPush = 64;    // PullInfo
constexpr int kSmemRing = 256;   // first ring slot (matches the planner's header)
static_assert(sizeof(PullInfo) <= kSmemRing - kSmemPush, "pull info overflows the header");

// The 3D update of one cell in arithmetic mode AM (see od_config.arith);
// ok = false sends the cell to update_slow.  m is the cell's slot in its
// thread (a compile-time constant after unrolling), which the mixed modes
// use to alternate forms.
template <int AM>
__device__ __forceinline__ double update_cell(const double *sd, const double *sc, const double *su, int r, int pitch,
                                              int m, const Arith &ar, bool &ok) {
    const double W = sc[r - 1], E = sc[r + 1], S = sc[r - pitch], N = sc[r + pitch], D = sd[r], U = su[r];
    if constexpr (AM == 12) {
        return jacobi_update_anchored<2>(W, E, S, N, D, U, ar.e0 + 1u, ok, ar.one);
    } else if constexpr (AM == 13) {
        return jacobi_update_anchored<1>(W, E, S, N, D, U, ar.e0, ok, ar.one);
    } else if constexpr (AM == 14 || AM == 15) {
        // 14: one FP64 add on every other cell, 15: on every fourth cell
        if ((AM == 14 && (m & 1)) || (AM == 15 && (m & 3) == 0))
            return jacobi_update_anchored<1>(W, E, S, N, D, U, ar.e0, ok, ar.one);
        return jacobi_update_anchored<2>(W, E, S, N, D, U, ar.e0 + 1u, ok, ar.one);
    } else if constexpr (AM == 9 || AM == 10 || AM == 11) {
        // the tail form: the last one or two adds in the window, the division
        // from the window word; 11 mixes them cell by cell
        if ((AM == 11 && (m & 1)) || AM == 10) return jacobi_update_tail<2>(W, E, S, N, D, U, ok);
        return jacobi_update_tail<1>(W, E, S, N, D, U, ok);
    } else if constexpr ((AM == 7 || AM == 8)) {
        // 7: every other cell with two window adds, 8: one cell in four
        if ((AM == 7 && (m & 1)) || (AM == 8 && (m & 3) == 0))
            return jacobi_update_fast<3>(W, E, S, N, D, U, ok);
        return jacobi_update_fast<2>(W, E, S, N, D, U, ok);
    } else {
        return jacobi_update_fast<AM>(W, E, S, N, D, U, ok);
    }
}

// Sweep one tile from parity sp into parity sp^1.  Returns false (all
// threads agree) if a wait ran out, after thread 0 has waited, bounded, for
// the copies this tile still had in flight; the caller records the error
// (keeping the error record out of the sweep keeps the job's arguments out
// of its registers).
//
// FUSED = false (the per-chare path): the chare's own ghost layers are
// current (unpacked), and the tile reads them with its rows.  FUSED = true
// (the fused and persistent paths): every internal face is read from the
// neighbour's array in the source parity, which the neighbour finished in
// the previous step -- a z-ghost plane is copied from the neighbour's
// boundary plane, a y-ghost row from its boundary row (a second and third
// bulk copy beside the tile's own rows), and the x-ghost column of each
// computed plane is patched into the ring slot from the neighbour's boundary
// column by plain loads, issued one plane ahead.  Nothing is written outside
// the chare's own interior, so the cell loop has no face branches.
template <int NT, int CPT, bool FUSED, int AM>
__device__ __forceinline__ bool run_tile(const KArgs &a, int tile_id, int sp, Ring &ring, PullInfo *pi, int step,
                                         const Arith &ar, const KArgs &g) {
    const TileDev T = a.tiles[tile_id];
    const ChareDev &C = a.ch[T.c];
    const int bx = C.bx, by = C.by, bz = C.bz, pitch = C.pitch;
    const int plane = (by + 2) * pitch;
    const int dp = sp ^ 1;
    const int nj = T.nj, j0 = T.j0;
    // row j0 (the tile's lower y-halo row) of plane 0; plane p+1 holds interior plane p
    const double *__restrict__ src = C.A[sp] + (size_t)j0 * pitch;
    double *__restrict__ dst = C.A[dp] + (size_t)j0 * pitch;
    const uint32_t row_bytes = (uint32_t)pitch * 8u;
    const uint32_t run_bytes = (uint32_t)(nj + 2) * row_bytes;  // one plane's rows
    const int S = g.stages, SD = g.stage_doubles;
    const int kb = T.k0 - 1, ke = T.k0 + T.nk;  // planes kb..ke are loaded
    const int tid = threadIdx.x;
    const uint32_t seq0 = ring.seq;

    // Plane p lives in ring slot (seq0 + p - kb) % S; its mbarrier phase is
    // the slot's use count & 1.
    auto slot = [&](int p) -> uint32_t { return (seq0 + (uint32_t)(p - kb)) % (uint32_t)S; };
    auto phase = [&](int p) -> uint32_t { return ((seq0 + (uint32_t)(p - kb)) / (uint32_t)S) & 1u; };
    // (thread 0) the copies of plane p into slot s
    auto issue = [&](int p, uint32_t s) {
        uint64_t *bar = ring.bars + s;
        double *slot_p = ring.base + (size_t)s * SD;
        mbar_expect_tx(bar, run_bytes);
        if (FUSED && p < 0 && pi->zlo) {  // the z- neighbour's top plane
            bulk_g2s(slot_p, pi->zlo, run_bytes, bar);
        } else if (FUSED && p >= bz && pi->zhi) {  // the z+ neighbour's bottom plane
            bulk_g2s(slot_p, pi->zhi, run_bytes, bar);
        } else {
            // a computed plane's y-ghost rows come from the y neighbours (the
            // planes below and above the tile are read at its own cells only)
            const bool computed = p >= T.k0 && p < ke;
            const double *row0 = src + (size_t)(p + 1) * plane;
            int first = 0, last = nj + 1;  // rows of the run taken from this chare
            if (FUSED && computed && pi->ylo) {  // the run's first row is the y-ghost row
                bulk_g2s(slot_p, pi->ylo + (size_t)(p + 1) * pi->ylo_plane, row_bytes, bar);
                first = 1;
            }
            if (FUSED && computed && pi->yhi) {
                bulk_g2s(slot_p + (size_t)(nj + 1) * pitch, pi->yhi + (size_t)(p + 1) * pi->yhi_plane, row_bytes,
                         bar);
                last = nj;
            }
            bulk_g2s(slot_p + (size_t)first * pitch, row0 + (size_t)first * pitch,
                     (uint32_t)(last - first + 1) * row_bytes, bar);
        }
    };
    int issued_hi = kb - 1;  // highest plane issued so far (same value in every thread)
    // (a ring of S slots holds planes k-1, k, k+1 and S-3 planes in flight)
    auto drain = [&](int from) {
        if (tid == 0)
            for (int p = from; p <= issued_hi; ++p) mbar_wait_bounded(ring.bars + slot(p), phase(p), g.spin_ns);
        ring.seq = seq0 + (uint32_t)(issued_hi - kb + 1);
    };

    // thread 0 prepares the pull info (the six faces' table reads are
    // independent loads) and issues the first planes' copies at once; the
    // barrier after them publishes the info to the x-halo threads (measured:
    // spreading the faces over six threads with a barrier before the first
    // copies was 0.3 % slower)
    if (tid == 0) {
        if (FUSED) {
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                const int n = C.nbr[f];
                const ChareDev *N = n >= 0 ? &a.ch[n] : nullptr;
                if (f == OD_FACE_XLO) {  // its column bx_n
                    pi->xlo = N ? N->A[sp] + N->bx : nullptr;
                    pi->xlo_pitch = N ? N->pitch : 0;
                    pi->xlo_plane = N ? (N->by + 2) * N->pitch : 0;
                } else if (f == OD_FACE_XHI) {  // its column 1
                    pi->xhi = N ? N->A[sp] + 1 : nullptr;
                    pi->xhi_pitch = N ? N->pitch : 0;
                    pi->xhi_plane = N ? (N->by + 2) * N->pitch : 0;
                } else if (f == OD_FACE_YLO) {  // its row by_n, when the tile's first halo row is the ghost row
                    const bool on = N && j0 == 0;
                    pi->ylo = on ? N->A[sp] + (size_t)N->by * pitch : nullptr;
                    pi->ylo_plane = on ? (N->by + 2) * pitch : 0;
                } else if (f == OD_FACE_YHI) {  // its row 1
                    const bool on = N && j0 + nj == by;
                    pi->yhi = on ? N->A[sp] + pitch : nullptr;
                    pi->yhi_plane = on ? (N->by + 2) * pitch : 0;
                } else if (f == OD_FACE_ZLO) {  // its plane bz_n, the tile's rows
                    pi->zlo = N && kb < 0 ? N->A[sp] + (size_t)N->bz * plane + (size_t)j0 * pitch : nullptr;
                } else {  // its plane 1
                    pi->zhi = N && ke >= bz ? N->A[sp] + plane + (size_t)j0 * pitch : nullptr;
                }
            }
        }
        const int last = min(ke, kb + S - 1);
        for (int p = kb; p <= last; ++p) issue(p, slot(p));
    }
    if (FUSED) __syncthreads();  // the pull info
    issued_hi = min(ke, kb + S - 1);

    // this thread's cells: q = tid + m*NT in the tile plane, row-major, as
    // ring-slot offsets.  A slot past the end of the tile repeats the tile's
    // first cell (it stores the same value to the same place), so the cell
    // loop needs no validity branch.
    const int ncell = nj * bx;
    int rf[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        const int q0 = tid + m * NT;
        const int q = q0 < ncell ? q0 : 0;
        const int j = q / bx, i = q - j * bx;
        rf[m] = (j + 1) * pitch + i + 1;
    }

    // x-halo patches of a plane (fused only): item t < 2*nj is row t % nj of
    // face t / nj, handled by thread t (the first warps: spreading the items
    // over every warp measured slower, each warp then running the patch
    // code for a few lanes); ring-slot offset of its ghost cell and the
    // neighbour cell it copies
    constexpr int kWarps = NT / 32;
    const int npatch = FUSED ? 2 * nj : 0;
    const int pt = tid;
    auto patch_src = [&](int t, int p) -> const double * {
        const bool hi = t >= nj;
        const int j = hi ? t - nj : t;
        const double *base = hi ? pi->xhi : pi->xlo;
        if (!base) return nullptr;
        const int pl = hi ? pi->xhi_plane : pi->xlo_plane, pt = hi ? pi->xhi_pitch : pi->xlo_pitch;
        return base + (size_t)(p + 1) * pl + (size_t)(j0 + j + 1) * pt;
    };
    auto patch_dst = [&](int t) -> int {
        const bool hi = t >= nj;
        return ((hi ? t - nj : t) + 1) * pitch + (hi ? bx + 1 : 0);
    };

    // Planes k-1, k and k+1 must be resident while plane k is computed, so a
    // slot is refilled once the plane after next has been computed.
    bool fail = !mbar_wait_bounded(ring.bars + slot(kb), phase(kb), g.spin_ns);
    if (!fail) fail = !mbar_wait_bounded(ring.bars + slot(kb + 1), phase(kb + 1), g.spin_ns);
    if (FUSED && !fail) {  // the first computed plane's x halo
        double *sl = ring.base + (size_t)slot(kb + 1) * SD;
        for (int t = pt; t < npatch; t += NT) {
            const double *g = patch_src(t, kb + 1);
            if (g) sl[patch_dst(t)] = *g;
        }
    }
    if (__syncthreads_or(fail)) {
        drain(kb);
        return false;
    }

    // ring slots of planes k-1, k, k+1 and the phase of k+1, advanced by one
    // position per plane (no division by the run-time ring depth in the loop)
    uint32_t sl_m1 = slot(kb), sl_0 = slot(kb + 1), sl_p1 = slot(kb + 2), ph_p1 = phase(kb + 2);
    // this thread's x-halo item, as a source pointer advanced by one
    // neighbour plane per plane (measured 1.7 % faster than recomputing it)
    const double *xbase = FUSED && pt < npatch ? patch_src(pt, -1) : nullptr;
    const int xpl = FUSED ? (pt >= nj ? pi->xhi_plane : pi->xlo_plane) : 0;
    const int xdst = patch_dst(pt);
    for (int k = T.k0; k < ke; ++k) {
        // the next plane's x halo, loaded while this plane is computed
        const bool patch_next = FUSED && k + 1 < ke;
        double xv = 0.0;
        const double *xg = nullptr;
        if (patch_next && xbase) {
            xg = xbase + (size_t)(k + 2) * xpl;
            xv = *xg;
        }
        fail = !mbar_wait_bounded(ring.bars + sl_p1, ph_p1, g.spin_ns);
        if (!fail) {
            const double *sd = ring.base + (size_t)sl_m1 * SD;
            const double *sc = ring.base + (size_t)sl_0 * SD;
            double *su = ring.base + (size_t)sl_p1 * SD;
            double *dpl = dst + (size_t)(k + 1) * plane;
            uint32_t bad = 0;  // bit m: cell m left the integer routines' domain
#pragma unroll
            for (int m = 0; m < CPT; ++m) {
                const int r = rf[m];
                bool ok;
                const double v = update_cell<AM>(sd, sc, su, r, pitch, m, ar, ok);
                bad |= (ok ? 0u : 1u) << m;
                dpl[r] = v;
            }
            if (bad) {  // rare: recompute those cells with IEEE operations and store them again
#pragma unroll
                for (int m = 0; m < CPT; ++m) {
                    const int r = rf[m];
                    if (bad & (1u << m))
                        dpl[r] = update_slow(sc[r - 1], sc[r + 1], sc[r - pitch], sc[r + pitch], sd[r], su[r]);
                }
            }
            if (patch_next) {  // plane k+1's x halo (its slot is only read at interior cells above)
                if (xg) su[xdst] = xv;
                for (int t = pt + NT; t < npatch; t += NT) {  // tiles of more than NT/2 rows
                    const double *g = patch_src(t, k + 1);
                    if (g) su[patch_dst(t)] = *g;
                }
            }
        }
        if (__syncthreads_or(fail)) {
            drain(k + 1);
            return false;
        }
        // plane k-1 is no longer needed: refill its slot (after the barrier,
        // and after a proxy fence when the slot took generic stores of a
        // halo), from lane 0 of a different warp each plane
        if (k - 1 + S <= ke) {
            if (tid == (OD_ROTATE_ISSUE ? (k % kWarps) << 5 : 0)) {
                if (FUSED) fence_proxy_async_smem();
                issue(k - 1 + S, sl_m1);
            }
            issued_hi = k - 1 + S;
        }
        sl_m1 = sl_0;
        sl_0 = sl_p1;
        if (++sl_p1 == (uint32_t)S) {
            sl_p1 = 0;
            ph_p1 ^= 1u;
        }
    }
    ring.seq = seq0 + (uint32_t)(ke - kb + 1);
    if (FUSED && tid == 0) fence_proxy_async_smem();  // before the next tile's copies into these slots
    return true;
}

// IEEE form of the 2D update (out of line, as update_slow).
static __device__ __noinline__ double update2d_slow(double W, double E, double S, double N) {
    return jacobi2d_update_ieee<true>(W, E, S, N);  // the division by 4 as an exponent step where exact
}

// The 2D 5-point sweep (the paper's Jacobi2D, Sec. V) on the internal grid
// (nx, 1, ny): a chare's 2D rows are its planes, one row each, so A is the
// padded 2D block and plane k (interior row k) starts at (k+1)*pitch.  A tile
// is one row segment, columns [i0, i0+ni), over planes [k0, k0+nk).  Per
// plane one bulk copy brings columns i0 .. i0+ni+1 (the segment plus its
// x-halo, rounded up to an even count; i0 and pitch are even, so the copy
// starts 16-byte aligned) into a ring slot; slot offset r = i+1 holds column
// i0+i+1, i.e. the tile's cell i.
// The update reads W = slot[r-1], E = slot[r+1] of plane k, S = plane k-1,
// N = plane k+1 at r, summed in that order and divided by 4.
// The 2D update of one cell in arithmetic mode AM (m as in update_cell).
template <int AM>
__device__ __forceinline__ double update_cell_2d(double W, double E, double S, double N, int m, const Arith &ar,
                                                 bool &ok) {
    if constexpr (AM == 12) {
        return jacobi2d_update_anchored<1>(W, E, S, N, ar.e0, ok, ar.one);
    } else if constexpr (AM == 13) {
        return jacobi2d_update_anchored<0>(W, E, S, N, ar.e0, ok, ar.one);
    } else if constexpr (AM == 14) {  // no FP64 add on every other cell
        if (m & 1) return jacobi2d_update_anchored<0>(W, E, S, N, ar.e0, ok, ar.one);
        return jacobi2d_update_anchored<1>(W, E, S, N, ar.e0, ok, ar.one);
    } else if constexpr (AM == 15) {
        return jacobi2d_update_anchored<2>(W, E, S, N, ar.e0 + 1u, ok, ar.one);
    } else if constexpr (AM == 9 || AM == 10 || AM == 11) {
        if ((AM == 11 && (m & 1)) || AM == 10) return jacobi2d_update_tail<2>(W, E, S, N, ok);
        return jacobi2d_update_tail<1>(W, E, S, N, ok);
    } else if constexpr (AM == 7 || AM == 8) {
        if ((AM == 7 && (m & 1)) || (AM == 8 && (m & 3) == 0)) return jacobi2d_update_fast<3>(W, E, S, N, ok);
        return jacobi2d_update_fast<2>(W, E, S, N, ok);
    } else {
        return jacobi2d_update_fast<AM>(W, E, S, N, ok);
    }
}

// FUSED = true (the fused and persistent paths): the faces of neighbour
// chares are read from their arrays in the source parity, as in run_tile --
// a z-ghost row (the row above or below the chare) by the plane's bulk copy
// from the neighbour's boundary row, an x-ghost cell of a computed row by a
// plain load one row ahead -- and nothing is stored outside the chare.
template <int NT, int CPT, bool FUSED, int AM>
__device__ __forceinline__ bool run_tile_2d(const KArgs &a, int tile_id, int sp, Ring &ring, PullInfo *pi,
                                            int step, const Arith &ar, const KArgs &g) {
    const TileDev T = a.tiles[tile_id];
    const ChareDev &C = a.ch[T.c];
    const int bx = C.bx, bz = C.bz, pitch = C.pitch;
    const int plane = pitch;
    const int dp = sp ^ 1;
    const int i0 = T.i0, ni = T.ni;
    const double *__restrict__ src = C.A[sp] + i0;  // column i0 of the lower ghost row
    double *__restrict__ dst = C.A[dp] + i0;
    const uint32_t run_bytes = (uint32_t)((ni + 3) & ~1) * 8u;
    const int S = g.stages, SD = g.stage_doubles;
    const int kb = T.k0 - 1, ke = T.k0 + T.nk;
    const int tid = threadIdx.x;
    const uint32_t seq0 = ring.seq;

    auto slot = [&](int p) -> uint32_t { return (seq0 + (uint32_t)(p - kb)) % (uint32_t)S; };
    auto phase = [&](int p) -> uint32_t { return ((seq0 + (uint32_t)(p - kb)) / (uint32_t)S) & 1u; };
    auto issue = [&](int p, uint32_t s) {  // s = slot(p)
        uint64_t *bar = ring.bars + s;
        mbar_expect_tx(bar, run_bytes);
        const double *from = src + (size_t)(p + 1) * plane;
        if (FUSED && p < 0 && pi->zlo) from = pi->zlo;        // the z- neighbour's top row
        if (FUSED && p >= bz && pi->zhi) from = pi->zhi;      // the z+ neighbour's bottom row
        bulk_g2s(ring.base + (size_t)s * SD, from, run_bytes, bar);
    };
    int issued_hi = kb - 1;
    auto drain = [&](int from) {
        if (tid == 0)
            for (int p = from; p <= issued_hi; ++p) mbar_wait_bounded(ring.bars + slot(p), phase(p), g.spin_ns);
        ring.seq = seq0 + (uint32_t)(issued_hi - kb + 1);
    };

    if (FUSED && tid < 4) {  // the pull info, one face per thread (2D faces: x-, x+, z-, z+)
        const int f = tid < 2 ? tid : tid + 2, n = C.nbr[f];
        const ChareDev *N = n >= 0 ? &a.ch[n] : nullptr;
        if (f == OD_FACE_XLO) {  // its column bx_n, when the segment starts at the chare's edge
            pi->xlo = N && i0 == 0 ? N->A[sp] + N->bx : nullptr;
            pi->xlo_plane = N ? N->pitch : 0;
        } else if (f == OD_FACE_XHI) {  // its column 1
            pi->xhi = N && i0 + ni == bx ? N->A[sp] + 1 : nullptr;
            pi->xhi_plane = N ? N->pitch : 0;
        } else if (f == OD_FACE_ZLO) {  // its row bz_n (same x extent, same pitch)
            pi->zlo = N && kb < 0 ? N->A[sp] + (size_t)N->bz * plane + i0 : nullptr;
        } else {  // its row 1
            pi->zhi = N && ke >= bz ? N->A[sp] + plane + i0 : nullptr;
        }
    }
    if (FUSED) __syncthreads();  // the pull info
    if (tid == 0) {
        const int last = min(ke, kb + S - 1);
        for (int p = kb; p <= last; ++p) issue(p, slot(p));
    }
    issued_hi = min(ke, kb + S - 1);

    // this thread's cells q = tid + m*NT of the segment, as ring-slot offsets;
    // a slot past its end repeats cell 0 (same value, same place)
    int rf[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        const int q0 = tid + m * NT;
        rf[m] = (q0 < ni ? q0 : 0) + 1;
    }
    // x-halo patches (fused only): thread 0 the x- ghost (slot offset 0),
    // thread 1 the x+ ghost (offset ni + 1) of a computed row
    auto patch_src = [&](int p) -> const double * {
        if (!FUSED || tid > 1) return nullptr;
        const double *base = tid ? pi->xhi : pi->xlo;
        return base ? base + (size_t)(p + 1) * (tid ? pi->xhi_plane : pi->xlo_plane) : nullptr;
    };
    const int patch_dst = tid ? ni + 1 : 0;

    bool fail = !mbar_wait_bounded(ring.bars + slot(kb), phase(kb), g.spin_ns);
    if (!fail) fail = !mbar_wait_bounded(ring.bars + slot(kb + 1), phase(kb + 1), g.spin_ns);
    if (FUSED && !fail) {  // the first computed row's x halo
        const double *g = patch_src(kb + 1);
        if (g) ring.base[(size_t)slot(kb + 1) * SD + patch_dst] = *g;
    }
    if (__syncthreads_or(fail)) {
        drain(kb);
        return false;
    }

    uint32_t sl_m1 = slot(kb), sl_0 = slot(kb + 1), sl_p1 = slot(kb + 2), ph_p1 = phase(kb + 2);
    for (int k = T.k0; k < ke; ++k) {
        // the next row's x halo, loaded while this row is computed
        const double *xg = FUSED && k + 1 < ke ? patch_src(k + 1) : nullptr;
        const double xv = xg ? *xg : 0.0;
        fail = !mbar_wait_bounded(ring.bars + sl_p1, ph_p1, g.spin_ns);
        if (!fail) {
            const double *sd = ring.base + (size_t)sl_m1 * SD;
            const double *sc = ring.base + (size_t)sl_0 * SD;
            double *su = ring.base + (size_t)sl_p1 * SD;
            double *dpl = dst + (size_t)(k + 1) * plane;
            // no validity branch: a slot past the segment's end repeats its
            // cell 0, so it stores the same value to the same place
            uint32_t bad = 0;  // bit m: cell m left the integer routines' domain
#pragma unroll
            for (int m = 0; m < CPT; ++m) {
                const int r = rf[m];
                bool ok;
                dpl[r] = update_cell_2d<AM>(sc[r - 1], sc[r + 1], sd[r], su[r], m, ar, ok);
                bad |= (ok ? 0u : 1u) << m;
            }
            if (bad) {  // rare: recompute those cells with IEEE operations and store them again
#pragma unroll
                for (int m = 0; m < CPT; ++m) {
                    const int r = rf[m];
                    if (bad & (1u << m)) dpl[r] = update2d_slow(sc[r - 1], sc[r + 1], sd[r], su[r]);
                }
            }
            if (xg) su[patch_dst] = xv;  // row k+1's x halo (its slot is only read at the cells above)
        }
        if (__syncthreads_or(fail)) {
            drain(k + 1);
            return false;
        }
        if (k - 1 + S <= ke) {  // refilled from lane 0 of a different warp each plane
            if (tid == (OD_ROTATE_ISSUE ? (k % (NT / 32)) << 5 : 0)) {
                if (FUSED) fence_proxy_async_smem();  // after the halo's generic stores
                issue(k - 1 + S, sl_m1);
            }
            issued_hi = k - 1 + S;
        }
        sl_m1 = sl_0;
        sl_0 = sl_p1;
        if (++sl_p1 == (uint32_t)S) {
            sl_p1 = 0;
            ph_p1 ^= 1u;
        }
    }
    ring.seq = seq0 + (uint32_t)(ke - kb + 1);
    if (FUSED && tid == 0) fence_proxy_async_smem();  // before the next tile's copies into these slots
    return true;
}

// Stencil dispatch at compile time: ST = OD_STENCIL_3D7 or OD_STENCIL_2D5.
// FUSED: the fused and persistent paths' tile (halos read from the
// neighbours).  g carries the launch's ring geometry and wait limit
// (stages, stage_doubles, spin_ns): a kernel parameter, which the sweep
// reads from the constant bank instead of holding it in registers -- the
// tile's own arguments a may live in global memory (batched launches).
template <int NT, int CPT, bool FUSED, int AM, int ST>
__device__ __forceinline__ bool run_any_tile(const KArgs &a, int tile_id, int sp, Ring &ring, unsigned char *info,
                                             int step, const Arith &ar, const KArgs &g) {
    if constexpr (ST == OD_STENCIL_2D5)
        return run_tile_2d<NT, CPT, FUSED, AM>(a, tile_id, sp, ring, reinterpret_cast<PullInfo *>(info), step, ar,
                                               g);
    else
        return run_tile<NT, CPT, FUSED, AM>(a, tile_id, sp, ring, reinterpret_cast<PullInfo *>(info), step, ar, g);
}

template <int NT>
__device__ __forceinline__ Ring ring_setup(const KArgs &g, unsigned char *smem) {
    Ring r;
    r.bars = reinterpret_cast<uint64_t *>(smem + kSmemBars);
    r.base = reinterpret_cast<double *>(smem + kSmemRing);
    r.seq = 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < g.stages; ++s) mbar_init(r.bars + s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    return r;
}

// One CTA per tile (per-chare compute when !FUSED, fused step when FUSED).
// Resident threads per SM the register budget must allow (1280 = 51
// registers a thread): the FP64 pipe needs many warps to hide shared-memory
// and pipe latency.  A build may override it (-DOD_MIN_THREADS_PER_SM=...).
#ifndef OD_MIN_THREADS_PER_SM
#define OD_MIN_THREADS_PER_SM 1280
#endif
// The 2D sweep needs fewer registers and gains from more resident warps
// (measured: 1536 threads per SM, 38 registers, 2.9 % faster than 1280).
#ifndef OD_MIN_THREADS_PER_SM_2D
#define OD_MIN_THREADS_PER_SM_2D 1536
#endif
// The batched serving kernels read each job's arguments from global memory
// and keep more values live; at the 1280-thread budget they spill (72 bytes),
// at 1024 threads (64 registers) they do not, and run faster (measured with
// one 512^3 job in 4096 chares: 172 against 159 G updates/s in one launch).
#ifndef OD_MIN_THREADS_PER_SM_MULTI
#define OD_MIN_THREADS_PER_SM_MULTI 1024
#endif
constexpr int min_blocks(int nt, int st) {
    return (st == OD_STENCIL_2D5 ? OD_MIN_THREADS_PER_SM_2D : OD_MIN_THREADS_PER_SM) / nt;
}
constexpr int min_blocks_multi(int nt, int st) {
    return (st == OD_STENCIL_2D5 ? OD_MIN_THREADS_PER_SM_2D : OD_MIN_THREADS_PER_SM_MULTI) / nt;
}

template <int NT, int CPT, bool FUSED, int AM, int ST>
__global__ void __launch_bounds__(NT, min_blocks(NT, ST)) k_tiles(const KArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (blockDim.x != NT) {
        if (threadIdx.x == 0) record_err(a.err, OD_ERR_BAD_LAUNCH, -1, -1);
        return;
    }
    const Arith ar = arith_setup<AM>(a, a);
    Ring ring = ring_setup<NT>(a, smem);
    const int tile = a.tile_begin + (int)blockIdx.x;
    if (!run_any_tile<NT, CPT, FUSED, AM, ST>(a, tile, a.parity, ring, smem + kSmemPush, -1, ar, a) &&
        threadIdx.x == 0)
        record_err(a.err, OD_ERR_TMA_TIMEOUT, tile, -1);
}

// Continuous batching: one fused step of several independent jobs in one
// launch.  jobs[j] holds job j's tables and source parity; job j owns blocks
// [first[j], first[j+1]); every block runs one tile of its job.  All jobs
// share the launch's CTA shape and ring geometry (geom: stages,
// stage_doubles -- the largest slot of the launch's jobs -- and spin_ns).
template <int NT, int CPT, int AM, int ST>
__global__ void __launch_bounds__(NT, min_blocks_multi(NT, ST)) k_tiles_multi(const KArgs *jobs, const int32_t *first,
                                                                   int32_t njobs, const KArgs geom) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int32_t s_job;
    if (threadIdx.x == 0) {
        int lo = 0, hi = njobs - 1;  // last job whose first block <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= (int32_t)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_job = lo;
    }
    __syncthreads();
    const KArgs &a = jobs[s_job];
    if (blockDim.x != NT) {
        if (threadIdx.x == 0) record_err(a.err, OD_ERR_BAD_LAUNCH, -1, -1);
        return;
    }
    const Arith ar = arith_setup<AM>(a, geom);
    Ring ring = ring_setup<NT>(geom, smem);
    const int tile = (int)blockIdx.x - first[s_job];
    if (!run_any_tile<NT, CPT, true, AM, ST>(a, tile, a.parity, ring, smem + kSmemPush, -1, ar, geom) &&
        threadIdx.x == 0)
        record_err(a.err, OD_ERR_TMA_TIMEOUT, tile, -1);
}

// Wait, bounded, until every tile in `tile`'s dependency list has finished
// `need` steps; each thread watches its own share of the list, so the waits
// (and their load latencies) overlap.  Returns this thread's verdict (all
// threads must then agree through a barrier); a wait that runs out records
// the error.
__device__ __forceinline__ int wait_deps(const KArgs &a, int tile, int32_t need, int step) {
    int ok = 1;
    const int q1 = a.dep_ptr[tile + 1];
    for (int q = a.dep_ptr[tile] + (int)threadIdx.x; q < q1 && ok; q += (int)blockDim.x) {
        const int32_t *e = a.epoch + a.dep_idx[q];
        if (ld_acquire(e) >= need) continue;
        const uint64_t t0 = now_ns();
        while (ld_acquire(e) < need) {
            if (ld_relaxed(&a.err->code) != 0) { ok = 0; break; }
            if (now_ns() - t0 > a.spin_ns) {
                record_err(a.err, OD_ERR_DEP_TIMEOUT, tile, step);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
    }
    return ok;
}

// Persistent kernel: CTAs take tickets in step-major order; ticket
// r*ntiles + pos is step r of tile order[pos] (reversed on odd r when
// order_mode == 1).  Before running it, the CTA waits until every tile it
// reads (and itself) has finished step r-1.  A waited-on ticket is always
// smaller than the waiter's, and tickets are taken in order by running CTAs,
// so the wait graph has no cycle and needs no co-residency guarantee.
template <int NT, int CPT, int AM, int ST>
__global__ void __launch_bounds__(NT, min_blocks(NT, ST)) k_persistent(const KArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int32_t s_ticket;
    if (blockDim.x != NT) {
        if (threadIdx.x == 0) record_err(a.err, OD_ERR_BAD_LAUNCH, -1, -1);
        return;
    }
    const Arith ar = arith_setup<AM>(a, a);
    Ring ring = ring_setup<NT>(a, smem);
    const int64_t total = (int64_t)a.iters * a.ntiles;
    // A ticket is taken when the CTA is free to run it (measured: taking the
    // next one a tile ahead, to hide the atomic's latency, was 2.5 % slower --
    // the ticket is then bound to a CTA that is still busy while others idle).
    for (;;) {
        if (threadIdx.x == 0) {
            int32_t tk = atomicAdd(a.queue, 1);
            if (ld_relaxed(&a.err->code) != 0) tk = INT32_MAX;
            s_ticket = tk;
        }
        __syncthreads();
        const int32_t tk = s_ticket;
        if ((int64_t)tk >= total) break;
        const int r = tk / a.ntiles, pos = tk - r * a.ntiles;
        const int step = a.t0 + r;
        const int tile = (a.order_mode == 1 && (r & 1)) ? a.order[a.ntiles - 1 - pos] : a.order[pos];
        const int ok = wait_deps(a, tile, r, step);
        if (!__syncthreads_and(ok)) break;
        // data written by other CTAs (generic proxy) is next read by bulk
        // copies (async proxy)
        if (threadIdx.x == 0) fence_proxy_async();
        if (!run_any_tile<NT, CPT, true, AM, ST>(a, tile, step & 1, ring, smem + kSmemPush, step, ar, a)) {
            if (threadIdx.x == 0) record_err(a.err, OD_ERR_TMA_TIMEOUT, tile, step);
            break;
        }
        if (threadIdx.x == 0 && (int64_t)tile != a.stall_tile) {
            __threadfence();
            st_release(a.epoch + tile, r + 1);
        }
    }
}

// Continuous batching over several steps: the persistent form of
// k_tiles_multi.  jobs[j] holds job j's tables, the absolute step t0 at which
// it enters this launch and the steps it runs in it (iters <= S); job j owns
// the tile positions [first[j], first[j+1]) of the launch (first[njobs] =
// total).  Ticket r*total + pos is step t0+r of tile pos - first[j] of job j,
// and a ticket with r >= jobs[j].iters does nothing.  A tile publishes the
// absolute number of steps it has finished, in the job's own step counters
// (zero when the job was created, never reset), so before step t0+r a tile
// waits until every tile it reads has finished t0+r steps.  As in
// k_persistent, a waited-on ticket is always smaller than the waiter's, so
// the waits cannot form a cycle.  Every job of a launch shares its CTA
// shape and ring geometry (geom, as for k_tiles_multi); queue is the
// launch's ticket counter (zeroed before the launch).
template <int NT, int CPT, int AM, int ST>
__global__ void __launch_bounds__(NT, min_blocks_multi(NT, ST))
    k_persistent_multi(const KArgs *jobs, const int32_t *first, int32_t njobs, int32_t S, int32_t *queue,
                       const KArgs geom) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int32_t s_ticket, s_job;
    if (blockDim.x != NT) {
        if (threadIdx.x == 0) record_err(jobs[0].err, OD_ERR_BAD_LAUNCH, -1, -1);
        return;
    }
    Ring ring = ring_setup<NT>(geom, smem);
    const int32_t total = first[njobs];
    const int64_t tickets = (int64_t)S * total;
    // the job owning tile position pos: the last one whose first position <= pos
    auto job_of = [&](int32_t pos) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= pos) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    for (;;) {
        if (threadIdx.x == 0) {  // a ticket is taken when the CTA is free to run it (see k_persistent)
            const int32_t tk = atomicAdd(queue, 1);
            s_ticket = tk;
            if ((int64_t)tk < tickets) s_job = job_of(tk % total);
        }
        __syncthreads();
        const int32_t tk = s_ticket;
        if ((int64_t)tk >= tickets) break;
        const int job = s_job;
        const int r = tk / total, tile = tk - r * total - first[job];
        const KArgs &a = jobs[job];
        if (r >= a.iters) {  // this job runs fewer steps in the launch
            __syncthreads();   // every thread has read the ticket before thread 0 takes the next
            continue;
        }
        const int step = a.t0 + r;
        const Arith ar = arith_setup<AM>(a, geom);
        const int ok = wait_deps(a, tile, step, step);
        if (!__syncthreads_and(ok)) break;
        if (threadIdx.x == 0) fence_proxy_async();
        const bool swept = run_any_tile<NT, CPT, true, AM, ST>(a, tile, step & 1, ring, smem + kSmemPush, step, ar,
                                                                geom);
        if (threadIdx.x == 0) {
            // the ticket's job, tile and step, re-derived from shared memory
            // (the sweep then holds none of them in registers)
            const int32_t tk1 = *(volatile int32_t *)&s_ticket;
            const int job1 = *(volatile int32_t *)&s_job;
            const int32_t tot1 = first[njobs];
            const int r1 = tk1 / tot1, tile1 = tk1 - r1 * tot1 - first[job1];
            const KArgs &a1 = jobs[job1];
            const int step1 = a1.t0 + r1;
            if (!swept) {
                record_err(a1.err, OD_ERR_TMA_TIMEOUT, tile1, step1);
            } else {
                __threadfence();
                st_release(a1.epoch + tile1, step1 + 1);
            }
        }
        if (!swept) break;
    }
}

}  // namespace tile
}  // namespace od
