// od_kernels.cu -- initialisation, per-chare pack/unpack, gather/scatter and
// arithmetic self-test kernels of libod (sm_103a), and the dispatch of the
// tile kernels (od_tile.cuh, instantiated per arithmetic mode in od_tiles.cu).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "od.h"
#include "od_arith.cuh"
#include "od_internal.h"
#include "od_kernels.h"

namespace od {

void *tile_kernel_am0(int threads, int cpt, int kind);
void *tile_kernel_am1(int threads, int cpt, int kind);
void *tile_kernel_am2(int threads, int cpt, int kind);
void *tile_kernel_am3(int threads, int cpt, int kind);
void *tile_kernel_am4(int threads, int cpt, int kind);
void *tile_kernel_am5(int threads, int cpt, int kind);
void *tile_kernel_am6(int threads, int cpt, int kind);
void *tile_kernel_am7(int threads, int cpt, int kind);
void *tile_kernel_am8(int threads, int cpt, int kind);
void *tile_kernel_am9(int threads, int cpt, int kind);
void *tile_kernel_am10(int threads, int cpt, int kind);
void *tile_kernel_am11(int threads, int cpt, int kind);
void *tile_kernel_am12(int threads, int cpt, int kind);
void *tile_kernel_am13(int threads, int cpt, int kind);
void *tile_kernel_am14(int threads, int cpt, int kind);
void *tile_kernel_am15(int threads, int cpt, int kind);
void *tile_kernel2d_am0(int threads, int cpt, int kind);
void *tile_kernel2d_am1(int threads, int cpt, int kind);
void *tile_kernel2d_am2(int threads, int cpt, int kind);
void *tile_kernel2d_am3(int threads, int cpt, int kind);
void *tile_kernel2d_am4(int threads, int cpt, int kind);
void *tile_kernel2d_am7(int threads, int cpt, int kind);
void *tile_kernel2d_am8(int threads, int cpt, int kind);
void *tile_kernel2d_am9(int threads, int cpt, int kind);
void *tile_kernel2d_am10(int threads, int cpt, int kind);
void *tile_kernel2d_am11(int threads, int cpt, int kind);
void *tile_kernel2d_am12(int threads, int cpt, int kind);
void *tile_kernel2d_am13(int threads, int cpt, int kind);
void *tile_kernel2d_am14(int threads, int cpt, int kind);
void *tile_kernel2d_am15(int threads, int cpt, int kind);

namespace {

void *tile_kernel(int stencil, int amode, int threads, int cpt, int kind) {
    if (stencil == OD_STENCIL_2D5) switch (amode) {
        // the 2D update has three adds, so modes 4..6 (three or more window
        // adds) are the same kernel
        case 0: return tile_kernel2d_am0(threads, cpt, kind);
        case 1: return tile_kernel2d_am1(threads, cpt, kind);
        case 2: return tile_kernel2d_am2(threads, cpt, kind);
        case 3: return tile_kernel2d_am3(threads, cpt, kind);
        case 4: case 5: case 6: return tile_kernel2d_am4(threads, cpt, kind);
        case 7: return tile_kernel2d_am7(threads, cpt, kind);
        case 8: return tile_kernel2d_am8(threads, cpt, kind);
        case 9: return tile_kernel2d_am9(threads, cpt, kind);
        case 10: return tile_kernel2d_am10(threads, cpt, kind);
        case 11: return tile_kernel2d_am11(threads, cpt, kind);
        case 12: return tile_kernel2d_am12(threads, cpt, kind);
        case 13: return tile_kernel2d_am13(threads, cpt, kind);
        case 14: return tile_kernel2d_am14(threads, cpt, kind);
        case 15: return tile_kernel2d_am15(threads, cpt, kind);
        default: return nullptr;
    }
    if (stencil != OD_STENCIL_3D7) return nullptr;
    switch (amode) {
        case 0: return tile_kernel_am0(threads, cpt, kind);
        case 1: return tile_kernel_am1(threads, cpt, kind);
        case 2: return tile_kernel_am2(threads, cpt, kind);
        case 3: return tile_kernel_am3(threads, cpt, kind);
        case 4: return tile_kernel_am4(threads, cpt, kind);
        case 5: return tile_kernel_am5(threads, cpt, kind);
        case 6: return tile_kernel_am6(threads, cpt, kind);
        case 7: return tile_kernel_am7(threads, cpt, kind);
        case 8: return tile_kernel_am8(threads, cpt, kind);
        case 9: return tile_kernel_am9(threads, cpt, kind);
        case 10: return tile_kernel_am10(threads, cpt, kind);
        case 11: return tile_kernel_am11(threads, cpt, kind);
        case 12: return tile_kernel_am12(threads, cpt, kind);
        case 13: return tile_kernel_am13(threads, cpt, kind);
        case 14: return tile_kernel_am14(threads, cpt, kind);
        case 15: return tile_kernel_am15(threads, cpt, kind);
        default: return nullptr;
    }
}

// ---------------------------------------------------------------- init / io

// SplitMix64 output number index+1 for `seed` (Steele, Lea & Flood 2014),
// top 53 bits scaled to [0,1).
__device__ __forceinline__ double field_uniform(uint64_t seed, uint64_t index) {
    uint64_t z = seed + (index + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
}

// Initial value of padded global cell (gx, gy, gz).
__device__ __forceinline__ double field_init(int64_t gx, int64_t gy, int64_t gz, int64_t nx, int64_t ny,
                                             int64_t nz, uint64_t seed, int mode) {
    const bool shell = gx == 0 || gy == 0 || gz == 0 || gx == nx + 1 || gy == ny + 1 || gz == nz + 1;
    if (!shell && mode == 0) return 0.0;
    return field_uniform(seed, (uint64_t)(gx + (nx + 2) * (gy + (ny + 2) * gz)));
}

// A2: the initial field in both parities, interior and every ghost cell
// (edge/corner ghosts and row padding, never read, get 0).  One warp per
// padded row.  A 2D chare's rows are single-row planes whose cells take the
// 2D padded index gx + (nx+2)*gz; (ox, oy, oz) is a shard's offset in the
// global grid nx x ny x nz.
__global__ void k_init(const ChareDev *ch, int nch, int64_t nx, int64_t ny, int64_t nz, int64_t ox, int64_t oy,
                       int64_t oz, uint64_t seed, int mode, int stencil) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int c = blockIdx.y; c < nch; c += gridDim.y) {
        const ChareDev &C = ch[c];
        const int nrow = C.rows * (C.bz + 2);
        for (int rr = blockIdx.x * nwarps + warp; rr < nrow; rr += gridDim.x * nwarps) {
            const int kp = rr / C.rows, rp = rr - kp * C.rows;
            const int jp = rp + 1 - C.row0;  // padded y index (a 2D chare's single row is row 1)
            const int ghosts_yz = (jp == 0 || jp == C.by + 1) + (kp == 0 || kp == C.bz + 1);
            const int64_t gy = C.y0 + jp + oy, gz = C.z0 + kp + oz;
            double *a0 = C.A[0] + (int64_t)rr * C.pitch, *a1 = C.A[1] + (int64_t)rr * C.pitch;
            for (int cp = lane; cp < C.pitch; cp += 32) {
                double v = 0.0;
                if (cp <= C.bx + 1 && ghosts_yz + (cp == 0 || cp == C.bx + 1) <= 1) {
                    const int64_t gx = C.x0 + cp + ox;
                    if (stencil == OD_STENCIL_2D5) {
                        const bool shell = gx == 0 || gz == 0 || gx == nx + 1 || gz == nz + 1;
                        if (shell || mode != 0) v = field_uniform(seed, (uint64_t)(gx + (nx + 2) * gz));
                    } else {
                        v = field_init(gx, gy, gz, nx, ny, nz, seed, mode);
                    }
                }
                a0[cp] = v;
                a1[cp] = v;
            }
        }
    }
}

// Offset in A of face element q of face f: `ghost` = false gives the
// chare's own boundary cell (pack), true the ghost cell facing it (unpack).
__device__ __forceinline__ int64_t face_offset(const ChareDev &C, int f, int q, bool ghost) {
    const int bx = C.bx, by = C.by, bz = C.bz, pitch = C.pitch, r0 = C.row0;
    const int64_t plane = (int64_t)C.rows * pitch;
    if (f < 2) {
        const int k = q / by, j = q - k * by;
        const int col = f == OD_FACE_XLO ? (ghost ? 0 : 1) : (ghost ? bx + 1 : bx);
        return (k + 1) * plane + (int64_t)(j + r0) * pitch + col;
    }
    if (f < 4) {  // (3D only: a 2D chare has no y faces)
        const int k = q / bx, i = q - k * bx;
        const int row = f == OD_FACE_YLO ? (ghost ? 0 : 1) : (ghost ? by + 1 : by);
        return (k + 1) * plane + (int64_t)row * pitch + i + 1;
    }
    const int j = q / bx, i = q - j * bx;
    const int pl = f == OD_FACE_ZLO ? (ghost ? 0 : 1) : (ghost ? bz + 1 : bz);
    return (int64_t)pl * plane + (int64_t)(j + r0) * pitch + i + 1;
}

// Per-chare path, A4: new boundary planes of parity p -> contiguous send
// buffer (faces with a neighbour only).
__global__ void k_pack(const ChareDev *ch, int c, int p) {
    const ChareDev &C = ch[c];
    const double *A = C.A[p];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < C.foff[6]; e += gridDim.x * blockDim.x) {
        int f = 0;
        while (e >= C.foff[f + 1]) ++f;
        if (C.nbr[f] < 0) continue;
        C.send[e] = A[face_offset(C, f, e - C.foff[f], false)];
    }
}

// Per-chare path, A6: receive slot -> ghost layers of parity p.
__global__ void k_unpack(const ChareDev *ch, int c, int p, int slot) {
    const ChareDev &C = ch[c];
    double *A = C.A[p];
    const double *R = C.recv[slot];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < C.foff[6]; e += gridDim.x * blockDim.x) {
        int f = 0;
        while (e >= C.foff[f + 1]) ++f;
        if (C.nbr[f] < 0) continue;
        A[face_offset(C, f, e - C.foff[f], true)] = R[e];
    }
}

// Internal ghost layers of parity p from the neighbours' boundary layers,
// every chare at once (face element q of face f is the neighbour's element
// q of the opposite face, as in pack / unpack).  Run before a per-chare step
// that follows fused 3D steps, which read the neighbours' faces directly and
// leave the ghost layers behind.
__global__ void k_ghost_refresh(const ChareDev *ch, int nch, int p) {
    for (int c = blockIdx.y; c < nch; c += gridDim.y) {
        const ChareDev &C = ch[c];
        double *A = C.A[p];
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < C.foff[6]; e += gridDim.x * blockDim.x) {
            int f = 0;
            while (e >= C.foff[f + 1]) ++f;
            if (C.nbr[f] < 0) continue;
            const ChareDev &N = ch[C.nbr[f]];
            const int q = e - C.foff[f];
            A[face_offset(C, f, q, true)] = N.A[p][face_offset(N, f ^ 1, q, false)];
        }
    }
}

// Domain-face exchange of a shard: the chares on domain face f (no neighbour
// there) copy, cell by cell, their boundary layer of parity p into buf
// (dir 0) or buf into their ghost layer (dir 1).  buf is the whole face,
// dense: x faces nz x ny (y fastest), y faces nz x nx, z faces ny x nx (x
// fastest).
__global__ void k_face_copy(const ChareDev *ch, int nch, int p, int f, int dir, double *buf, int64_t nx, int64_t ny,
                            int64_t nz) {
    for (int c = blockIdx.y; c < nch; c += gridDim.y) {
        const ChareDev &C = ch[c];
        const bool on_face = f == OD_FACE_XLO ? C.x0 == 0 : f == OD_FACE_XHI ? C.x0 + C.bx == nx
                           : f == OD_FACE_YLO ? C.y0 == 0 : f == OD_FACE_YHI ? C.y0 + C.by == ny
                           : f == OD_FACE_ZLO ? C.z0 == 0 : C.z0 + C.bz == nz;
        if (!on_face) continue;
        const int n = f < 2 ? C.by * C.bz : f < 4 ? C.bx * C.bz : C.bx * C.by;
        const int w = f < 2 ? C.by : C.bx;  // fastest extent of the chare's face
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
            const int a = q % w, b = q / w;
            int64_t g;  // position in buf
            if (f < 2) g = (C.z0 + b) * ny + C.y0 + a;
            else if (f < 4) g = (C.z0 + b) * nx + C.x0 + a;
            else g = (C.y0 + b) * nx + C.x0 + a;
            const int64_t o = face_offset(C, f, q, dir != 0);
            if (dir == 0) buf[g] = C.A[p][o];
            else C.A[p][o] = buf[g];
        }
    }
}

// Selected cells: out[i] = *addr[i] (addresses inside the chares' arrays).
__global__ void k_read_cells(const double *const *addr, int64_t n, double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = *addr[i];
}

// Rows a warp moves per pass of the gather and scatter: the loads of all of
// them are in flight before the first store, so a warp keeps several memory
// requests outstanding (one row at a time left both kernels latency-bound
// on 32-cell rows).
constexpr int kIoRows = 4;

// A11: interiors of parity p -> global x-fastest array.  Each warp moves
// kIoRows interior rows per pass (coalesced on both sides), one 32-bit
// division per row.
__global__ void k_gather(const ChareDev *ch, int nch, int p, int64_t nx, int64_t ny, double *g) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int c = blockIdx.y; c < nch; c += gridDim.y) {
        const ChareDev &C = ch[c];
        const int nrow = C.by * C.bz, bx = C.bx;
        const int64_t plane = (int64_t)C.rows * C.pitch;
        for (int r0 = (blockIdx.x * nwarps + warp) * kIoRows; r0 < nrow; r0 += gridDim.x * nwarps * kIoRows) {
            const double *src[kIoRows];
            double *dst[kIoRows];
#pragma unroll
            for (int u = 0; u < kIoRows; ++u) {
                const int rr = r0 + u < nrow ? r0 + u : r0;  // past the end: repeat the first row
                const int k = rr / C.by, j = rr - k * C.by;
                src[u] = C.A[p] + (k + 1) * plane + (int64_t)(j + C.row0) * C.pitch + 1;
                dst[u] = g + ((C.z0 + k) * ny + C.y0 + j) * nx + C.x0;
            }
            for (int i = lane; i < bx; i += 32) {
                double v[kIoRows];
#pragma unroll
                for (int u = 0; u < kIoRows; ++u) v[u] = src[u][i];
#pragma unroll
                for (int u = 0; u < kIoRows; ++u) dst[u][i] = v[u];  // a repeated row stores the same value
            }
        }
    }
}

// Import: global x-fastest interior -> interiors of parity p, the mirror of
// k_gather (kIoRows rows per warp pass).  Ghost layers are left alone: the
// fused and persistent sweeps read their neighbours' faces from the
// neighbours' arrays, and the per-chare flow refreshes its internal ghost
// layers before its next step (od_write marks them stale); Dirichlet and
// imported domain faces keep their values.
// The largest positive finite value written goes into *vmax (its bit
// pattern, atomic maximum: positive doubles order like their bit patterns),
// which anchors the exact arithmetic's window (od_arith.cuh); at most one
// atomic per warp.
__global__ void k_scatter(const ChareDev *ch, int nch, int p, int64_t nx, int64_t ny, int64_t nz,
                          const double *g, unsigned long long *vmax) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    unsigned long long vm = 0;
    for (int c = blockIdx.y; c < nch; c += gridDim.y) {
        const ChareDev &C = ch[c];
        const int nrow = C.by * C.bz, bx = C.bx;
        const int64_t plane = (int64_t)C.rows * C.pitch;
        for (int r0 = (blockIdx.x * nwarps + warp) * kIoRows; r0 < nrow; r0 += gridDim.x * nwarps * kIoRows) {
            const double *src[kIoRows];
            double *dst[kIoRows];
#pragma unroll
            for (int u = 0; u < kIoRows; ++u) {
                const int rr = r0 + u < nrow ? r0 + u : r0;  // past the end: repeat the first row
                const int k = rr / C.by, j = rr - k * C.by;
                dst[u] = C.A[p] + (k + 1) * plane + (int64_t)(j + C.row0) * C.pitch + 1;
                src[u] = g + ((C.z0 + k) * ny + C.y0 + j) * nx + C.x0;
            }
            for (int i = lane; i < bx; i += 32) {
                double v[kIoRows];
#pragma unroll
                for (int u = 0; u < kIoRows; ++u) v[u] = src[u][i];
#pragma unroll
                for (int u = 0; u < kIoRows; ++u) {
                    dst[u][i] = v[u];  // a repeated row stores the same value
                    const unsigned long long b = (unsigned long long)__double_as_longlong(v[u]);
                    if (b < 0x7FF0000000000000ull && b > vm) vm = b;  // positive and finite
                }
            }
        }
    }
    (void)nz;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xFFFFFFFFu, vm, o);
        vm = w > vm ? w : vm;
    }
    // the word only grows: a warp whose maximum is not above it skips the
    // atomic (a field within the initial bound [0, 1) then issues none)
    if (lane == 0 && vm != 0 && vmax && vm > *(volatile unsigned long long *)vmax) atomicMax(vmax, vm);
}

// Arithmetic self-test: op 0 div6, 1 add (integer pipes); 2 division by 6,
// 3 add (FP64 pipe); 10+m the whole Jacobi update in arithmetic mode m over
// six operands per element (a[6i .. 6i+5]).
__global__ void k_arith(int op, const double *a, const double *b, double *out, int64_t n) {
    // anchored ops: b[0] holds the anchor exponent (clamped as on the host)
    const uint32_t e0 =
        op >= 30 ? (uint32_t)fmin(fmax(b[0], (double)kAnchorMin), (double)kAnchorMax) : kAnchorMin;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double r;
        switch (op) {
            case 0: r = div6(a[i]); break;
            case 1: r = add(a[i], b[i]); break;
            case 2: r = __ddiv_rn(a[i], 6.0); break;
            case 3: r = __dadd_rn(a[i], b[i]); break;
            default:
                if (op >= 40) r = jacobi2d_update_anchored_mode(op - 40, a + 4 * i, e0);
                else if (op >= 30) r = jacobi_update_anchored_mode(op - 30, a + 6 * i, e0);
                else r = op < 20 ? jacobi_update_mode(op - 10, a + 6 * i) : jacobi2d_update_mode(op - 20, a + 4 * i);
                break;
        }
        out[i] = r;
    }
}

int io_grid_y(int nch) { return nch < 65535 ? nch : 65535; }

// blocks per chare so that small chare counts still fill the GPU
int io_grid_x(int nch) {
    int gx = 8192 / (nch > 0 ? nch : 1);
    return gx < 8 ? 8 : (gx > 4096 ? 4096 : gx);
}

}  // namespace

bool tile_shape_supported(int threads, int cpt, int amode, int stencil) {
    return tile_kernel(stencil, amode, threads, cpt, 0) != nullptr;
}

// The dynamic shared-memory cap is per kernel function and shared by every
// context in the process, so it is raised once to what the hardware allows
// (227 KB per CTA less the kernel's static shared memory) and never lowered:
// the launch's own size decides occupancy, the cap only permits it.
cudaError_t prepare_tile_kernels(int threads, int cpt, int amode, int smem_bytes, int stencil) {
    void *fns[5] = {tile_kernel(stencil, amode, threads, cpt, 0), tile_kernel(stencil, amode, threads, cpt, 1),
                    tile_kernel(stencil, amode, threads, cpt, 2), tile_kernel(stencil, amode, threads, cpt, 3),
                    tile_kernel(stencil, amode, threads, cpt, 4)};
    for (void *f : fns) {
        if (!f) return cudaErrorInvalidValue;
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
        const int cap = 232448 - (int)fa.sharedSizeBytes;
        if (smem_bytes > cap) return cudaErrorInvalidValue;
        if (fa.maxDynamicSharedSizeBytes < cap) {
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_tiles(const KArgs &a, int grid, int threads, int cpt, int amode, bool push, int smem_bytes,
                         cudaStream_t s) {
    void *f = tile_kernel(a.stencil, amode, threads, cpt, push ? 1 : 0);
    if (!f) return cudaErrorInvalidValue;
    if (grid <= 0) return cudaSuccess;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, (size_t)smem_bytes, s);
}

cudaError_t launch_persistent(const KArgs &a, int grid, int threads, int cpt, int amode, int smem_bytes,
                              cudaStream_t s) {
    void *f = tile_kernel(a.stencil, amode, threads, cpt, 2);
    if (!f) return cudaErrorInvalidValue;
    if (grid <= 0) return cudaSuccess;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, (size_t)smem_bytes, s);
}

cudaError_t launch_tiles_multi(const KArgs *jobs, const int32_t *first, int32_t njobs, const KArgs &geom, int grid,
                               int threads, int cpt, int amode, int smem_bytes, int stencil, cudaStream_t s) {
    void *f = tile_kernel(stencil, amode, threads, cpt, 3);
    if (!f) return cudaErrorInvalidValue;
    if (grid <= 0 || njobs <= 0) return cudaSuccess;
    void *args[] = {(void *)&jobs, (void *)&first, (void *)&njobs, (void *)&geom};
    return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, (size_t)smem_bytes, s);
}

cudaError_t launch_persistent_multi(const KArgs *jobs, const int32_t *first, int32_t njobs, int32_t steps,
                                    int32_t *queue, const KArgs &geom, int grid, int threads, int cpt, int amode,
                                    int smem_bytes, int stencil, cudaStream_t s) {
    void *f = tile_kernel(stencil, amode, threads, cpt, 4);
    if (!f) return cudaErrorInvalidValue;
    if (grid <= 0 || njobs <= 0 || steps <= 0) return cudaSuccess;
    void *args[] = {(void *)&jobs, (void *)&first, (void *)&njobs, (void *)&steps, (void *)&queue, (void *)&geom};
    return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, (size_t)smem_bytes, s);
}

cudaError_t persistent_multi_occupancy(int threads, int cpt, int amode, int smem_bytes, int stencil,
                                       int *blocks_per_sm) {
    void *f = tile_kernel(stencil, amode, threads, cpt, 4);
    if (!f) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, (size_t)smem_bytes);
}

cudaError_t persistent_occupancy(int threads, int cpt, int amode, int smem_bytes, int stencil,
                                 int *blocks_per_sm) {
    void *f = tile_kernel(stencil, amode, threads, cpt, 2);
    if (!f) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, (size_t)smem_bytes);
}

cudaError_t launch_init(const ChareDev *ch, int nch, int64_t gnx, int64_t gny, int64_t gnz, int64_t gx0,
                        int64_t gy0, int64_t gz0, uint64_t seed, int mode, int stencil, cudaStream_t s) {
    k_init<<<dim3(io_grid_x(nch), io_grid_y(nch)), 256, 0, s>>>(ch, nch, gnx, gny, gnz, gx0, gy0, gz0, seed, mode,
                                                                stencil);
    return cudaGetLastError();
}

cudaError_t launch_face_copy(const ChareDev *ch, int nch, int parity, int face, int dir, double *buf, int64_t nx,
                             int64_t ny, int64_t nz, cudaStream_t s) {
    k_face_copy<<<dim3(io_grid_x(nch), io_grid_y(nch)), 256, 0, s>>>(ch, nch, parity, face, dir, buf, nx, ny, nz);
    return cudaGetLastError();
}

cudaError_t launch_pack(const ChareDev *ch, int c, int parity, int elems, cudaStream_t s) {
    int grid = (elems + 255) / 256;
    if (grid < 1) grid = 1;
    if (grid > 1024) grid = 1024;
    k_pack<<<grid, 256, 0, s>>>(ch, c, parity);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const ChareDev *ch, int c, int parity, int slot, int elems, cudaStream_t s) {
    int grid = (elems + 255) / 256;
    if (grid < 1) grid = 1;
    if (grid > 1024) grid = 1024;
    k_unpack<<<grid, 256, 0, s>>>(ch, c, parity, slot);
    return cudaGetLastError();
}

cudaError_t launch_read_cells(const double *const *addr, int64_t n, double *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 1024);
    k_read_cells<<<grid, 256, 0, s>>>(addr, n, out);
    return cudaGetLastError();
}

cudaError_t launch_gather(const ChareDev *ch, int nch, int parity, int64_t nx, int64_t ny, double *g,
                          cudaStream_t s) {
    k_gather<<<dim3(io_grid_x(nch), io_grid_y(nch)), 256, 0, s>>>(ch, nch, parity, nx, ny, g);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const ChareDev *ch, int nch, int parity, int64_t nx, int64_t ny, int64_t nz,
                           const double *g, uint64_t *vmax, cudaStream_t s) {
    k_scatter<<<dim3(io_grid_x(nch), io_grid_y(nch)), 256, 0, s>>>(ch, nch, parity, nx, ny, nz, g,
                                                                    (unsigned long long *)vmax);
    return cudaGetLastError();
}

cudaError_t launch_ghost_refresh(const ChareDev *ch, int nch, int parity, cudaStream_t s) {
    k_ghost_refresh<<<dim3(8, io_grid_y(nch)), 256, 0, s>>>(ch, nch, parity);
    return cudaGetLastError();
}

}  // namespace od

namespace od {

cudaError_t launch_arith(int op, const double *a, const double *b, double *out, int64_t n, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_arith<<<(int)blocks, 256, 0, s>>>(op, a, b, out, n);
    return cudaGetLastError();
}

}  // namespace od
