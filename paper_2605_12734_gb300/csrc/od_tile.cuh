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
// HBM, coalesced, and, on a chare boundary, once more straight into the
// neighbour's ghost layer (the fused paths' pack + delivery + unpack).  The
// 2D task (run_tile_2d) is a row segment over a run of rows, the same way.
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
    return jacobi_update_ieee<false>(W, E, S, N, D, U);
}

struct Ring {
    double *base;      // first slot
    uint64_t *bars;    // one mbarrier per slot
    uint32_t seq;      // planes issued by this CTA before the current tile
};

// Where a tile's boundary values go (the neighbours' ghost cells of the
// destination parity), prepared once per tile by thread 0 in shared memory.
// For a cell with ring-slot offset r in tile row j and plane k:
//   x-: xlo + (k+1)*xlo_plane + (j+1)*xlo_pitch    x+: same with xhi
//   y-: ylo + (k+1)*ylo_plane + r                  y+: same with yhi
//   z-: zlo + r (plane k == 0)                      z+: zhi + r (k == bz-1)
struct PushInfo {
    double *xlo, *xhi, *ylo, *yhi, *zlo, *zhi;
    int32_t xlo_pitch, xlo_plane, xhi_pitch, xhi_plane, ylo_plane, yhi_plane;
};

constexpr int kSmemBars = 0;     // up to 8 mbarriers
constexpr int kSmemPush = 64;    // PushInfo
constexpr int kSmemRing = 256;   // first ring slot (matches the planner's header)
static_assert(sizeof(PushInfo) <= kSmemRing - kSmemPush, "push info overflows the header");

// Per-cell word: bits 0-15 ring-slot offset r of the cell, 16-26 tile row j,
// 27 the slot holds a real cell (not a copy of cell 0 past the tile's end),
// 28/29/30/31 the cell lies on a face with an x-/x+/y-/y+ neighbour.
constexpr uint32_t kValid = 1u << 27;
constexpr uint32_t kXlo = 1u << 28, kXhi = 1u << 29, kYlo = 1u << 30, kYhi = 1u << 31;

// Sweep one tile from parity sp into parity sp^1.  Returns false (all
// threads agree) if a wait ran out; the error is recorded and thread 0 has
// waited, bounded, for the copies this tile still had in flight.
template <int NT, int CPT, bool PUSH, int AM>
__device__ __forceinline__ bool run_tile(const KArgs &a, int tile_id, int sp, Ring &ring, PushInfo *pi,
                                         int step) {
    const TileDev T = a.tiles[tile_id];
    const ChareDev &C = a.ch[T.c];
    const int bx = C.bx, by = C.by, bz = C.bz, pitch = C.pitch;
    const int plane = (by + 2) * pitch;
    const int dp = sp ^ 1;
    // row j0 (the tile's lower y-halo row) of plane 0; plane p+1 holds interior plane p
    const double *__restrict__ src = C.A[sp] + (size_t)T.j0 * pitch;
    double *__restrict__ dst = C.A[dp] + (size_t)T.j0 * pitch;
    const uint32_t run_bytes = (uint32_t)((T.nj + 2) * pitch) * 8u;  // one plane's rows
    const int S = a.stages, SD = a.stage_doubles;
    const int kb = T.k0 - 1, ke = T.k0 + T.nk;  // planes kb..ke are loaded
    const int tid = threadIdx.x;
    const uint32_t seq0 = ring.seq;

    // Plane p lives in ring slot (seq0 + p - kb) % S; its mbarrier phase is
    // the slot's use count & 1.
    auto slot = [&](int p) -> uint32_t { return (seq0 + (uint32_t)(p - kb)) % (uint32_t)S; };
    auto phase = [&](int p) -> uint32_t { return ((seq0 + (uint32_t)(p - kb)) / (uint32_t)S) & 1u; };
    auto issue = [&](int p, uint32_t s) {  // s = slot(p)
        uint64_t *bar = ring.bars + s;
        mbar_expect_tx(bar, run_bytes);
        bulk_g2s(ring.base + (size_t)s * SD, src + (size_t)(p + 1) * plane, run_bytes, bar);
    };
    int issued_hi = kb - 1;  // highest plane issued so far (same value in every thread)
    // (a ring of S slots holds planes k-1, k, k+1 and S-3 planes in flight)
    auto drain = [&](int from) {
        if (tid == 0)
            for (int p = from; p <= issued_hi; ++p) mbar_wait_bounded(ring.bars + slot(p), phase(p), a.spin_ns);
        ring.seq = seq0 + (uint32_t)(issued_hi - kb + 1);
    };

    if (tid == 0) {
        const int last = min(ke, kb + S - 1);
        for (int p = kb; p <= last; ++p) issue(p, slot(p));
        if (PUSH) {
            PushInfo q;
            q.xlo = q.xhi = q.ylo = q.yhi = q.zlo = q.zhi = nullptr;
            q.xlo_pitch = q.xlo_plane = q.xhi_pitch = q.xhi_plane = q.ylo_plane = q.yhi_plane = 0;
            if (C.nbr[OD_FACE_XLO] >= 0) {
                const ChareDev &N = a.ch[C.nbr[OD_FACE_XLO]];
                q.xlo_pitch = N.pitch;
                q.xlo_plane = (N.by + 2) * N.pitch;
                q.xlo = N.A[dp] + (size_t)T.j0 * N.pitch + (N.bx + 1);
            }
            if (C.nbr[OD_FACE_XHI] >= 0) {
                const ChareDev &N = a.ch[C.nbr[OD_FACE_XHI]];
                q.xhi_pitch = N.pitch;
                q.xhi_plane = (N.by + 2) * N.pitch;
                q.xhi = N.A[dp] + (size_t)T.j0 * N.pitch;
            }
            if (C.nbr[OD_FACE_YLO] >= 0) {  // cell row 0 -> its ghost row by_n+1
                const ChareDev &N = a.ch[C.nbr[OD_FACE_YLO]];
                q.ylo_plane = (N.by + 2) * pitch;
                q.ylo = N.A[dp] + (size_t)N.by * pitch;
            }
            if (C.nbr[OD_FACE_YHI] >= 0) {  // cell row by-1 -> its ghost row 0
                const ChareDev &N = a.ch[C.nbr[OD_FACE_YHI]];
                q.yhi_plane = (N.by + 2) * pitch;
                q.yhi = N.A[dp] - (ptrdiff_t)(by - T.j0) * pitch;
            }
            if (C.nbr[OD_FACE_ZLO] >= 0) {  // plane 0 -> its ghost plane bz_n+1
                const ChareDev &N = a.ch[C.nbr[OD_FACE_ZLO]];
                q.zlo = N.A[dp] + (size_t)(N.bz + 1) * plane + (size_t)T.j0 * pitch;
            }
            if (C.nbr[OD_FACE_ZHI] >= 0) q.zhi = a.ch[C.nbr[OD_FACE_ZHI]].A[dp] + (size_t)T.j0 * pitch;
            *pi = q;
        }
    }
    issued_hi = min(ke, kb + S - 1);

    // this thread's cells: q = tid + m*NT in the tile plane, row-major.  A slot
    // past the end of the tile repeats the tile's first cell (it stores the
    // same value to the same place, and pushes nothing), so the cell loop
    // needs no validity branch.
    const int ncell = T.nj * bx;
    uint32_t rf[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        const int q0 = tid + m * NT;
        const bool valid = q0 < ncell;
        const int q = valid ? q0 : 0;
        const int j = q / bx, i = q - j * bx, gj = T.j0 + j;
        uint32_t w = (uint32_t)((j + 1) * pitch + i + 1) | ((uint32_t)j << 16);
        if (valid) {
            w |= kValid;
            if (PUSH) {
                if (i == 0 && C.nbr[OD_FACE_XLO] >= 0) w |= kXlo;
                if (i == bx - 1 && C.nbr[OD_FACE_XHI] >= 0) w |= kXhi;
                if (gj == 0 && C.nbr[OD_FACE_YLO] >= 0) w |= kYlo;
                if (gj == by - 1 && C.nbr[OD_FACE_YHI] >= 0) w |= kYhi;
            }
        }
        rf[m] = w;
    }

    // Planes k-1, k and k+1 must be resident while plane k is computed (the
    // z-1 value is read from the ring, not kept in registers), so a slot is
    // refilled once the plane after next has been computed.
    bool fail = !mbar_wait_bounded(ring.bars + slot(kb), phase(kb), a.spin_ns);
    if (!fail) fail = !mbar_wait_bounded(ring.bars + slot(kb + 1), phase(kb + 1), a.spin_ns);
    if (__syncthreads_or(fail)) {
        if (tid == 0) record_err(a.err, OD_ERR_TMA_TIMEOUT, tile_id, step);
        drain(kb);
        return false;
    }

    // One plane: ZP = the plane is a chare z-face with a neighbour there, so
    // every cell is also stored into that neighbour's ghost plane (zp).
    auto compute_plane = [&](auto zp_tag, int k, double *zp, const double *sd, const double *sc,
                             const double *su) {
        constexpr bool ZP = decltype(zp_tag)::value;
        double *dpl = dst + (size_t)(k + 1) * plane;
        // no validity branch: a slot past the tile's end repeats the tile's
        // first cell, so it stores the same value to the same place
        auto store = [&](uint32_t w, int r, double v) {
            dpl[r] = v;
            if (PUSH) {
                const uint32_t xf = w & (kXlo | kXhi);
                if (xf) {  // a row's first and last lanes take one path together
                    const int j1 = (int)((w >> 16) & 0x7FFu) + 1;
                    const bool lo = (w & kXlo) != 0;
                    double *base = lo ? pi->xlo : pi->xhi;
                    const int pl = lo ? pi->xlo_plane : pi->xhi_plane, pt = lo ? pi->xlo_pitch : pi->xhi_pitch;
                    base[(size_t)(k + 1) * pl + (size_t)j1 * pt] = v;
                    if (xf == (kXlo | kXhi))  // bx == 1: the cell is on both x faces
                        pi->xhi[(size_t)(k + 1) * pi->xhi_plane + (size_t)j1 * pi->xhi_pitch] = v;
                }
                const uint32_t yf = w & (kYlo | kYhi);
                if (yf) {  // whole rows: the branch is uniform across a row's lanes
                    const bool lo = (w & kYlo) != 0;
                    double *base = lo ? pi->ylo : pi->yhi;
                    base[(size_t)(k + 1) * (lo ? pi->ylo_plane : pi->yhi_plane) + r] = v;
                    if (yf == (kYlo | kYhi))  // by == 1: the row is on both y faces
                        pi->yhi[(size_t)(k + 1) * pi->yhi_plane + r] = v;
                }
                if (ZP) zp[r] = v;
            }
        };
        uint32_t bad = 0;  // bit m: cell m left the integer routines' domain
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            const uint32_t w = rf[m];
            const int r = (int)(w & 0xFFFFu);
            bool ok;
            // modes 7 and 8 mix the per-cell placement to balance the FP64 and
            // integer pipes: 7 = every other cell with two window adds, 8 =
            // one cell in four (m is a compile-time constant after unrolling)
            // modes 9-11: the tail form (the last one or two adds in the window,
            // the division from the window word); 11 mixes them like 7
            [[maybe_unused]] constexpr int AMa = AM == 7 || AM == 8 ? 2 : AM;
            double v;
            if constexpr (AM == 9 || AM == 10 || AM == 11) {
                if ((AM == 11 && (m & 1)) || AM == 10)
                    v = jacobi_update_tail<2>(sc[r - 1], sc[r + 1], sc[r - pitch], sc[r + pitch], sd[r], su[r], ok);
                else
                    v = jacobi_update_tail<1>(sc[r - 1], sc[r + 1], sc[r - pitch], sc[r + pitch], sd[r], su[r], ok);
            } else if ((AM == 7 && (m & 1)) || (AM == 8 && (m & 3) == 0)) {
                v = jacobi_update_fast<3>(sc[r - 1], sc[r + 1], sc[r - pitch], sc[r + pitch], sd[r], su[r], ok);
            } else {
                v = jacobi_update_fast<AMa>(sc[r - 1], sc[r + 1], sc[r - pitch], sc[r + pitch], sd[r], su[r], ok);
            }
            bad |= (ok ? 0u : 1u) << m;
            store(w, r, v);
        }
        if (bad) {  // rare: recompute those cells with IEEE operations and store them again
#pragma unroll
            for (int m = 0; m < CPT; ++m) {
                const uint32_t w = rf[m];
                const int r = (int)(w & 0xFFFFu);
                if (bad & (1u << m))
                    store(w, r, update_slow(sc[r - 1], sc[r + 1], sc[r - pitch], sc[r + pitch], sd[r], su[r]));
            }
        }
    };

    // ring slots of planes k-1, k, k+1 and the phase of k+1, advanced by one
    // position per plane (no division by the run-time ring depth in the loop)
    uint32_t sl_m1 = slot(kb), sl_0 = slot(kb + 1), sl_p1 = slot(kb + 2), ph_p1 = phase(kb + 2);
    for (int k = T.k0; k < ke; ++k) {
        fail = !mbar_wait_bounded(ring.bars + sl_p1, ph_p1, a.spin_ns);
        if (!fail) {
            const double *sd = ring.base + (size_t)sl_m1 * SD;
            const double *sc = ring.base + (size_t)sl_0 * SD;
            const double *su = ring.base + (size_t)sl_p1 * SD;
            double *z0 = (PUSH && k == 0) ? pi->zlo : nullptr;
            double *z1 = (PUSH && k == bz - 1) ? pi->zhi : nullptr;
            if (z0) compute_plane(std::true_type(), k, z0, sd, sc, su);
            if (z1) compute_plane(std::true_type(), k, z1, sd, sc, su);  // bz == 1 with both: the plane twice
            if (!z0 && !z1) compute_plane(std::false_type(), k, nullptr, sd, sc, su);
        }
        if (__syncthreads_or(fail)) {
            if (tid == 0) record_err(a.err, OD_ERR_TMA_TIMEOUT, tile_id, step);
            drain(k + 1);
            return false;
        }
        // plane k-1 is no longer needed: refill its slot
        if (k - 1 + S <= ke) {
            if (tid == 0) issue(k - 1 + S, sl_m1);
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
    return true;
}

// IEEE form of the 2D update (out of line, as update_slow).
static __device__ __noinline__ double update2d_slow(double W, double E, double S, double N) {
    return jacobi2d_update_ieee<false>(W, E, S, N);
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
template <int NT, int CPT, bool PUSH, int AM>
__device__ __forceinline__ bool run_tile_2d(const KArgs &a, int tile_id, int sp, Ring &ring, PushInfo *pi,
                                            int step) {
    const TileDev T = a.tiles[tile_id];
    const ChareDev &C = a.ch[T.c];
    const int bx = C.bx, bz = C.bz, pitch = C.pitch;
    const int plane = pitch;
    const int dp = sp ^ 1;
    const double *__restrict__ src = C.A[sp] + T.i0;  // column i0 of the lower ghost row
    double *__restrict__ dst = C.A[dp] + T.i0;
    const uint32_t run_bytes = (uint32_t)((T.ni + 3) & ~1) * 8u;
    const int S = a.stages, SD = a.stage_doubles;
    const int kb = T.k0 - 1, ke = T.k0 + T.nk;
    const int tid = threadIdx.x;
    const uint32_t seq0 = ring.seq;

    auto slot = [&](int p) -> uint32_t { return (seq0 + (uint32_t)(p - kb)) % (uint32_t)S; };
    auto phase = [&](int p) -> uint32_t { return ((seq0 + (uint32_t)(p - kb)) / (uint32_t)S) & 1u; };
    auto issue = [&](int p, uint32_t s) {  // s = slot(p)
        uint64_t *bar = ring.bars + s;
        mbar_expect_tx(bar, run_bytes);
        bulk_g2s(ring.base + (size_t)s * SD, src + (size_t)(p + 1) * plane, run_bytes, bar);
    };
    int issued_hi = kb - 1;
    auto drain = [&](int from) {
        if (tid == 0)
            for (int p = from; p <= issued_hi; ++p) mbar_wait_bounded(ring.bars + slot(p), phase(p), a.spin_ns);
        ring.seq = seq0 + (uint32_t)(issued_hi - kb + 1);
    };

    if (tid == 0) {
        const int last = min(ke, kb + S - 1);
        for (int p = kb; p <= last; ++p) issue(p, slot(p));
        if (PUSH) {
            PushInfo q;
            q.xlo = q.xhi = q.ylo = q.yhi = q.zlo = q.zhi = nullptr;
            q.xlo_pitch = q.xlo_plane = q.xhi_pitch = q.xhi_plane = q.ylo_plane = q.yhi_plane = 0;
            if (C.nbr[OD_FACE_XLO] >= 0) {  // column 0 -> its ghost column bx_n+1
                const ChareDev &N = a.ch[C.nbr[OD_FACE_XLO]];
                q.xlo_plane = N.pitch;
                q.xlo = N.A[dp] + (N.bx + 1);
            }
            if (C.nbr[OD_FACE_XHI] >= 0) {  // column bx-1 -> its ghost column 0
                const ChareDev &N = a.ch[C.nbr[OD_FACE_XHI]];
                q.xhi_plane = N.pitch;
                q.xhi = N.A[dp];
            }
            if (C.nbr[OD_FACE_ZLO] >= 0) {  // row 0 -> its ghost row bz_n+1 (same bx, same pitch)
                const ChareDev &N = a.ch[C.nbr[OD_FACE_ZLO]];
                q.zlo = N.A[dp] + (size_t)(N.bz + 1) * plane + T.i0;
            }
            if (C.nbr[OD_FACE_ZHI] >= 0) q.zhi = a.ch[C.nbr[OD_FACE_ZHI]].A[dp] + T.i0;
            *pi = q;
        }
    }
    issued_hi = min(ke, kb + S - 1);

    // this thread's cells q = tid + m*NT of the segment; a slot past its end
    // repeats cell 0 (same value, same place, no flags)
    uint32_t rf[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        const int q0 = tid + m * NT;
        const bool valid = q0 < T.ni;
        const int q = valid ? q0 : 0;
        uint32_t w = (uint32_t)(q + 1);
        if (valid) {
            w |= kValid;
            if (PUSH) {
                if (T.i0 + q == 0 && C.nbr[OD_FACE_XLO] >= 0) w |= kXlo;
                if (T.i0 + q == bx - 1 && C.nbr[OD_FACE_XHI] >= 0) w |= kXhi;
            }
        }
        rf[m] = w;
    }

    bool fail = !mbar_wait_bounded(ring.bars + slot(kb), phase(kb), a.spin_ns);
    if (!fail) fail = !mbar_wait_bounded(ring.bars + slot(kb + 1), phase(kb + 1), a.spin_ns);
    if (__syncthreads_or(fail)) {
        if (tid == 0) record_err(a.err, OD_ERR_TMA_TIMEOUT, tile_id, step);
        drain(kb);
        return false;
    }

    auto compute_plane = [&](auto zp_tag, int k, double *zp, const double *sd, const double *sc,
                             const double *su) {
        constexpr bool ZP = decltype(zp_tag)::value;
        double *dpl = dst + (size_t)(k + 1) * plane;
        // no validity branch: a slot past the segment's end repeats its cell
        // 0, so it stores the same value to the same place
        auto store = [&](uint32_t w, int r, double v) {
            dpl[r] = v;
            if (PUSH) {
                if (w & kXlo) pi->xlo[(size_t)(k + 1) * pi->xlo_plane] = v;
                if (w & kXhi) pi->xhi[(size_t)(k + 1) * pi->xhi_plane] = v;
                if (ZP) zp[r] = v;
            }
        };
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            const uint32_t w = rf[m];
            const int r = (int)(w & 0xFFFFu);
            bool ok;
            [[maybe_unused]] constexpr int AMa = AM == 7 || AM == 8 ? 2 : AM;
            double v;
            if constexpr (AM == 9 || AM == 10 || AM == 11) {
                if ((AM == 11 && (m & 1)) || AM == 10)
                    v = jacobi2d_update_tail<2>(sc[r - 1], sc[r + 1], sd[r], su[r], ok);
                else
                    v = jacobi2d_update_tail<1>(sc[r - 1], sc[r + 1], sd[r], su[r], ok);
            } else if ((AM == 7 && (m & 1)) || (AM == 8 && (m & 3) == 0)) {
                v = jacobi2d_update_fast<3>(sc[r - 1], sc[r + 1], sd[r], su[r], ok);
            } else {
                v = jacobi2d_update_fast<AMa>(sc[r - 1], sc[r + 1], sd[r], su[r], ok);
            }
            if (!ok) v = update2d_slow(sc[r - 1], sc[r + 1], sd[r], su[r]);
            store(w, r, v);
        }
    };

    uint32_t sl_m1 = slot(kb), sl_0 = slot(kb + 1), sl_p1 = slot(kb + 2), ph_p1 = phase(kb + 2);
    for (int k = T.k0; k < ke; ++k) {
        fail = !mbar_wait_bounded(ring.bars + sl_p1, ph_p1, a.spin_ns);
        if (!fail) {
            const double *sd = ring.base + (size_t)sl_m1 * SD;
            const double *sc = ring.base + (size_t)sl_0 * SD;
            const double *su = ring.base + (size_t)sl_p1 * SD;
            double *z0 = (PUSH && k == 0) ? pi->zlo : nullptr;
            double *z1 = (PUSH && k == bz - 1) ? pi->zhi : nullptr;
            if (z0) compute_plane(std::true_type(), k, z0, sd, sc, su);
            if (z1) compute_plane(std::true_type(), k, z1, sd, sc, su);
            if (!z0 && !z1) compute_plane(std::false_type(), k, nullptr, sd, sc, su);
        }
        if (__syncthreads_or(fail)) {
            if (tid == 0) record_err(a.err, OD_ERR_TMA_TIMEOUT, tile_id, step);
            drain(k + 1);
            return false;
        }
        if (k - 1 + S <= ke) {
            if (tid == 0) issue(k - 1 + S, sl_m1);
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
    return true;
}

// Stencil dispatch at compile time: ST = OD_STENCIL_3D7 or OD_STENCIL_2D5.
template <int NT, int CPT, bool PUSH, int AM, int ST>
__device__ __forceinline__ bool run_any_tile(const KArgs &a, int tile_id, int sp, Ring &ring, PushInfo *pi,
                                             int step) {
    if constexpr (ST == OD_STENCIL_2D5) return run_tile_2d<NT, CPT, PUSH, AM>(a, tile_id, sp, ring, pi, step);
    else return run_tile<NT, CPT, PUSH, AM>(a, tile_id, sp, ring, pi, step);
}

template <int NT>
__device__ __forceinline__ Ring ring_setup(const KArgs &a, unsigned char *smem) {
    Ring r;
    r.bars = reinterpret_cast<uint64_t *>(smem + kSmemBars);
    r.base = reinterpret_cast<double *>(smem + kSmemRing);
    r.seq = 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) mbar_init(r.bars + s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    return r;
}

// One CTA per tile (per-chare compute when !PUSH, fused step when PUSH).
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
constexpr int min_blocks(int nt, int st) {
    return (st == OD_STENCIL_2D5 ? OD_MIN_THREADS_PER_SM_2D : OD_MIN_THREADS_PER_SM) / nt;
}

template <int NT, int CPT, bool PUSH, int AM, int ST>
__global__ void __launch_bounds__(NT, min_blocks(NT, ST)) k_tiles(const KArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (blockDim.x != NT) {
        if (threadIdx.x == 0) record_err(a.err, OD_ERR_BAD_LAUNCH, -1, -1);
        return;
    }
    Ring ring = ring_setup<NT>(a, smem);
    run_any_tile<NT, CPT, PUSH, AM, ST>(a, a.tile_begin + (int)blockIdx.x, a.parity, ring,
                                        reinterpret_cast<PushInfo *>(smem + kSmemPush), -1);
}

// Continuous batching: one fused step of several independent jobs in one
// launch.  jobs[j] holds job j's tables and source parity; job j owns blocks
// [first[j], first[j+1]); every block runs one tile of its job.  All jobs
// share the launch's CTA shape, ring depth and slot size.
template <int NT, int CPT, int AM, int ST>
__global__ void __launch_bounds__(NT, min_blocks(NT, ST)) k_tiles_multi(const KArgs *jobs, const int32_t *first,
                                                                   int32_t njobs) {
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
    Ring ring = ring_setup<NT>(a, smem);
    run_any_tile<NT, CPT, true, AM, ST>(a, (int)blockIdx.x - first[s_job], a.parity, ring,
                                        reinterpret_cast<PushInfo *>(smem + kSmemPush), -1);
}

// Persistent kernel: CTAs take tickets in step-major order; ticket
// r*ntiles + pos is step r of tile order[pos] (reversed on odd r when
// order_mode == 1).  Before running it, thread 0 waits until every tile it
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
    Ring ring = ring_setup<NT>(a, smem);
    const int64_t total = (int64_t)a.iters * a.ntiles;
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
        int ok = 1;
        if (threadIdx.x == 0) {
            const int q1 = a.dep_ptr[tile + 1];
            for (int q = a.dep_ptr[tile]; q < q1 && ok; ++q) {
                const int32_t *e = a.epoch + a.dep_idx[q];
                if (ld_acquire(e) >= r) continue;
                const uint64_t t0 = now_ns();
                while (ld_acquire(e) < r) {
                    if (ld_relaxed(&a.err->code) != 0) { ok = 0; break; }
                    if (now_ns() - t0 > a.spin_ns) {
                        record_err(a.err, OD_ERR_DEP_TIMEOUT, tile, step);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            // data written by other CTAs (generic proxy) is next read by bulk
            // copies (async proxy)
            fence_proxy_async();
        }
        if (!__syncthreads_and(ok)) break;
        if (!run_any_tile<NT, CPT, true, AM, ST>(a, tile, step & 1, ring,
                                                 reinterpret_cast<PushInfo *>(smem + kSmemPush), step))
            break;
        if (threadIdx.x == 0 && (int64_t)tile != a.stall_tile) {
            __threadfence();
            st_release(a.epoch + tile, r + 1);
        }
    }
}


}  // namespace tile
}  // namespace od
