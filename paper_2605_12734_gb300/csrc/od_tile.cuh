// od_tile.cuh -- the tile sweep of libod (sm_103a), shared by the per-chare
// compute kernel, the fused step kernel and the persistent kernel.
//
// A task is nj full rows x nk planes of one chare.  One elected thread issues,
// per z-plane, a 1D bulk copy (cp.async.bulk, the TMA's untiled form) of the
// tile's nj rows plus its two y-halo rows -- one contiguous run of the chare's
// padded array -- and two small copies of that plane's x-ghost spans into a
// ring slot whose mbarrier counts the transaction bytes; `stages` planes are
// in flight.  Every thread owns the same cells of every plane and keeps the
// z-1 value in registers, so a cell reads x-1, x+1, y-1, y+1, z+1 from shared
// memory.  The new value is stored once to HBM, coalesced, and, on a chare
// boundary, once more straight into the neighbour's ghost layer (the fused
// paths' pack + delivery + unpack).
//
// The arithmetic is the Jacobi update of the paper's stencil proxy (Sec. V,
// "jacobi2d", here 3D 7-point) with round-to-nearest binary64 adds and
// division and no contraction, which is what makes every path bit-identical
// to an undecomposed sweep.
//
// Every wait is bounded by KArgs::spin_ns (wall clock, %globaltimer): a wait
// that runs out records an error and the CTA leaves after draining its own
// copies in flight, so a lost copy or a stalled neighbour never hangs the GPU.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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

// The Jacobi update (((((W+E)+S)+N)+D)+U)/6 in binary64 round-to-nearest.
// AM selects where the operations run, never what they compute:
//   AM = 0  every add and the division on the FP64 pipe (__dadd_rn, __ddiv_rn)
//   AM = 1  adds on the FP64 pipe, division by 6 on the integer pipes
//   AM = 1+k, k = 1..5: additionally the first k adds on the integer pipes
// (od_arith.cuh; identical bits for every input).
template <int AM>
__device__ __forceinline__ double jacobi_update(double W, double E, double S, double N, double D, double U) {
    constexpr int NE = AM > 1 ? AM - 1 : 0;
    double s = NE >= 1 ? add(W, E) : __dadd_rn(W, E);
    s = NE >= 2 ? add(s, S) : __dadd_rn(s, S);
    s = NE >= 3 ? add(s, N) : __dadd_rn(s, N);
    s = NE >= 4 ? add(s, D) : __dadd_rn(s, D);
    s = NE >= 5 ? add(s, U) : __dadd_rn(s, U);
    return AM >= 1 ? div6(s) : __ddiv_rn(s, 6.0);
}

// ---------------------------------------------------------------- tile sweep

struct Ring {
    double *base;      // first slot
    uint64_t *bars;    // one mbarrier per slot
    uint32_t seq;      // planes issued by this CTA before the current tile
};

// Sweep one tile from parity sp into parity sp^1.  Returns false (all
// threads agree) if a wait ran out; the error is recorded and thread 0 has
// waited, bounded, for the copies this tile still had in flight.
template <int NT, int CPT, bool PUSH, int AM>
__device__ __forceinline__ bool run_tile(const KArgs &a, int tile_id, int sp, Ring &ring, int step) {
    const TileDev T = a.tiles[tile_id];
    const ChareDev &C = a.ch[T.c];
    const int bx = C.bx, by = C.by, bz = C.bz, pitch = C.pitch, xgp = C.xgp;
    const int plane = (by + 2) * pitch;
    const int dp = sp ^ 1;
    const double *__restrict__ src = C.A[sp];
    double *__restrict__ dst = C.A[dp];
    const double *xlo_src = C.XG[sp][0];
    const double *xhi_src = C.XG[sp][1];
    const int rows_d = (T.nj + 2) * pitch;            // doubles of one plane's rows
    const int xj0 = T.j0 & ~1;                        // 16-byte aligned start
    const int xcnt = ((T.j0 + T.nj + 1) & ~1) - xj0;  // even count covering [j0, j0+nj)
    const int xoff = T.j0 - xj0;
    const int S = a.stages, SD = a.stage_doubles;
    const int kb = T.k0 - 1, ke = T.k0 + T.nk;        // planes kb..ke are loaded
    const int tid = threadIdx.x;
    const uint32_t seq0 = ring.seq;

    // Plane p lives in ring slot (seq0 + p - kb) % S; its mbarrier phase is
    // the slot's use count & 1.
    auto slot = [&](int p) -> uint32_t { return (seq0 + (uint32_t)(p - kb)) % (uint32_t)S; };
    auto phase = [&](int p) -> uint32_t { return ((seq0 + (uint32_t)(p - kb)) / (uint32_t)S) & 1u; };
    auto issue = [&](int p) {
        const uint32_t s = slot(p);
        double *sb = ring.base + (size_t)s * SD;
        uint64_t *bar = ring.bars + s;
        const bool xg = (p >= 0 && p < bz);
        const uint32_t rb = (uint32_t)rows_d * 8u, xb = (uint32_t)xcnt * 8u;
        mbar_expect_tx(bar, rb + (xg ? 2u * xb : 0u));
        bulk_g2s(sb, src + (size_t)(p + 1) * plane + (size_t)T.j0 * pitch, rb, bar);
        if (xg) {
            bulk_g2s(sb + rows_d, xlo_src + (size_t)p * xgp + xj0, xb, bar);
            bulk_g2s(sb + rows_d + xcnt, xhi_src + (size_t)p * xgp + xj0, xb, bar);
        }
    };
    int issued_hi = kb - 1;  // highest plane issued so far (same value in every thread)
    auto drain = [&](int from) {
        if (tid == 0)
            for (int p = from; p <= issued_hi; ++p) mbar_wait_bounded(ring.bars + slot(p), phase(p), a.spin_ns);
        ring.seq = seq0 + (uint32_t)(issued_hi - kb + 1);
    };

    // cells of this thread: plane-local (j, i) for q = tid + m*NT
    const int ncell = T.nj * bx;
    int cj[CPT], ci[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        const int q = tid + m * NT;
        cj[m] = q / bx;
        ci[m] = q - cj[m] * bx;
    }

    // neighbour mailboxes (ghost layers of parity dp) for the fused paths
    double *nb_xlo = nullptr, *nb_xhi = nullptr, *nb_ylo = nullptr, *nb_yhi = nullptr;
    double *nb_zlo = nullptr, *nb_zhi = nullptr;
    int plane_ylo = 0, plane_yhi = 0;
    if (PUSH) {
        if (C.nbr[OD_FACE_XLO] >= 0) nb_xlo = a.ch[C.nbr[OD_FACE_XLO]].XG[dp][1] + T.j0;
        if (C.nbr[OD_FACE_XHI] >= 0) nb_xhi = a.ch[C.nbr[OD_FACE_XHI]].XG[dp][0] + T.j0;
        if (C.nbr[OD_FACE_YLO] >= 0) {
            const ChareDev &N = a.ch[C.nbr[OD_FACE_YLO]];
            plane_ylo = (N.by + 2) * pitch;
            nb_ylo = N.A[dp] + (size_t)(N.by + 1) * pitch;
        }
        if (C.nbr[OD_FACE_YHI] >= 0) {
            const ChareDev &N = a.ch[C.nbr[OD_FACE_YHI]];
            plane_yhi = (N.by + 2) * pitch;
            nb_yhi = N.A[dp];
        }
        if (C.nbr[OD_FACE_ZLO] >= 0) {
            const ChareDev &N = a.ch[C.nbr[OD_FACE_ZLO]];
            nb_zlo = N.A[dp] + (size_t)(N.bz + 1) * plane;
        }
        if (C.nbr[OD_FACE_ZHI] >= 0) nb_zhi = a.ch[C.nbr[OD_FACE_ZHI]].A[dp];
    }

    if (tid == 0) {
        const int last = min(ke, kb + S - 1);
        for (int p = kb; p <= last; ++p) issue(p);
    }
    issued_hi = min(ke, kb + S - 1);

    double down[CPT], cur[CPT];
    bool fail = !mbar_wait_bounded(ring.bars + slot(kb), phase(kb), a.spin_ns);
    if (!fail) {
        const double *sb = ring.base + (size_t)slot(kb) * SD;
#pragma unroll
        for (int m = 0; m < CPT; ++m)
            if (tid + m * NT < ncell) down[m] = sb[(cj[m] + 1) * pitch + ci[m]];
        fail = !mbar_wait_bounded(ring.bars + slot(kb + 1), phase(kb + 1), a.spin_ns);
    }
    if (!fail) {
        const double *sb = ring.base + (size_t)slot(kb + 1) * SD;
#pragma unroll
        for (int m = 0; m < CPT; ++m)
            if (tid + m * NT < ncell) cur[m] = sb[(cj[m] + 1) * pitch + ci[m]];
    }
    if (__syncthreads_or(fail)) {
        if (tid == 0) record_err(a.err, OD_ERR_TMA_TIMEOUT, tile_id, step);
        drain(kb);
        return false;
    }
    if (kb + S <= ke) {
        if (tid == 0) issue(kb + S);
        issued_hi = kb + S;
    }

    for (int k = T.k0; k < ke; ++k) {
        fail = !mbar_wait_bounded(ring.bars + slot(k + 1), phase(k + 1), a.spin_ns);
        if (!fail) {
            const double *sc = ring.base + (size_t)slot(k) * SD;
            const double *su = ring.base + (size_t)slot(k + 1) * SD;
            const double *xl = sc + rows_d + xoff;
            const double *xh = sc + rows_d + xcnt + xoff;
            double *dplane = dst + (size_t)(k + 1) * plane + (size_t)(T.j0 + 1) * pitch;
#pragma unroll
            for (int m = 0; m < CPT; ++m) {
                if (tid + m * NT < ncell) {
                    const int j = cj[m], i = ci[m];
                    const int r = (j + 1) * pitch + i;
                    const double up = su[r];
                    const double W = (i > 0) ? sc[r - 1] : xl[j];
                    const double E = (i < bx - 1) ? sc[r + 1] : xh[j];
                    const double v = jacobi_update<AM>(W, E, sc[r - pitch], sc[r + pitch], down[m], up);
                    dplane[(size_t)j * pitch + i] = v;
                    if (PUSH) {
                        const int gj = T.j0 + j;
                        if (i == 0 && nb_xlo) nb_xlo[(size_t)k * xgp + j] = v;
                        if (i == bx - 1 && nb_xhi) nb_xhi[(size_t)k * xgp + j] = v;
                        if (gj == 0 && nb_ylo) nb_ylo[(size_t)(k + 1) * plane_ylo + i] = v;
                        if (gj == by - 1 && nb_yhi) nb_yhi[(size_t)(k + 1) * plane_yhi + i] = v;
                        if (k == 0 && nb_zlo) nb_zlo[(size_t)(gj + 1) * pitch + i] = v;
                        if (k == bz - 1 && nb_zhi) nb_zhi[(size_t)(gj + 1) * pitch + i] = v;
                    }
                    down[m] = cur[m];
                    cur[m] = up;
                }
            }
        }
        if (__syncthreads_or(fail)) {
            if (tid == 0) record_err(a.err, OD_ERR_TMA_TIMEOUT, tile_id, step);
            drain(k + 1);
            return false;
        }
        if (k + S <= ke) {
            if (tid == 0) issue(k + S);
            issued_hi = k + S;
        }
    }
    ring.seq = seq0 + (uint32_t)(ke - kb + 1);
    return true;
}

template <int NT>
__device__ __forceinline__ Ring ring_setup(const KArgs &a, unsigned char *smem) {
    Ring r;
    r.bars = reinterpret_cast<uint64_t *>(smem);
    r.base = reinterpret_cast<double *>(smem + 128);
    r.seq = 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) mbar_init(r.bars + s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    return r;
}

// One CTA per tile (per-chare compute when !PUSH, fused step when PUSH).
template <int NT, int CPT, bool PUSH, int AM>
__global__ void __launch_bounds__(NT) k_tiles(const KArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (blockDim.x != NT) {
        if (threadIdx.x == 0) record_err(a.err, OD_ERR_BAD_LAUNCH, -1, -1);
        return;
    }
    Ring ring = ring_setup<NT>(a, smem);
    run_tile<NT, CPT, PUSH, AM>(a, a.tile_begin + (int)blockIdx.x, a.parity, ring, -1);
}

// Persistent kernel: CTAs take tickets in step-major order; ticket
// r*ntiles + pos is step r of tile order[pos] (reversed on odd r when
// order_mode == 1).  Before running it, thread 0 waits until every tile it
// reads (and itself) has finished step r-1.  A waited-on ticket is always
// smaller than the waiter's, and tickets are taken in order by running CTAs,
// so the wait graph has no cycle and needs no co-residency guarantee.
template <int NT, int CPT, int AM>
__global__ void __launch_bounds__(NT) k_persistent(const KArgs a) {
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
        if (!run_tile<NT, CPT, true, AM>(a, tile, step & 1, ring, step)) break;
        if (threadIdx.x == 0 && (int64_t)tile != a.stall_tile) {
            __threadfence();
            st_release(a.epoch + tile, r + 1);
        }
    }
}


}  // namespace tile
}  // namespace od
