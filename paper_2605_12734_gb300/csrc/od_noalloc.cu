// od_noalloc.cu -- od_jacobi_noalloc: Jacobi iterations on a caller's padded
// field without allocating any device memory.
//
// Some callers cannot allocate device memory where they call this library: a
// host framework that owns every byte of device memory through its own pool
// and forbids allocations it does not track, or a latency-critical loop in
// which cudaMalloc / cudaFree would synchronise the device.  This entry point
// serves them: the caller passes the input field and the output field, and the
// one piece of scratch the iteration needs -- the second buffer of the double
// buffer -- is a file-scope static device array of fixed size that the
// module holds on every GPU that loads this library, until the process exits.
//
// It is a variant of the fused step kernel (one chare covering the whole
// grid, the same update, so the same bits), over the caller's plain padded
// layout instead of the context arena.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "od.h"
#include "od_arith.cuh"

namespace od {
od_status set_last_error(od_status s, const std::string &msg);  // od_api.cu
}  // namespace od

namespace {

// 64 MiB of doubles: padded grids up to 8 Mi cells, e.g. 200^3 interior.
constexpr int64_t kScratchDoubles = OD_NOALLOC_MAX_PADDED_CELLS;
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
od_status set_error(od_status s, const std::string &m) { return od::set_last_error(s, m); }

// One step over the interior of a padded field (x fastest, row length nx+2):
// the same update as the fused tile kernel (arithmetic mode 2).  The padded
// grid holds at most OD_NOALLOC_MAX_PADDED_CELLS (2^23) cells, so every index
// fits 32 bits; threads run along x, blocks along y (grid y) and z (grid z),
// striding when a grid axis is shorter than the field's, so no index needs
// a division.
__global__ void k_noalloc_step(const double *__restrict__ src, double *__restrict__ dst, uint32_t nx, uint32_t ny,
                               uint32_t nz) {
    const uint32_t sx = nx + 2u, sxy = sx * (ny + 2u);
    for (uint32_t k = blockIdx.z; k < nz; k += gridDim.z)
        for (uint32_t j = blockIdx.y; j < ny; j += gridDim.y) {
            const uint32_t row = (k + 1u) * sxy + (j + 1u) * sx + 1u;
            for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
                const uint32_t c = row + i;
                dst[c] = od::jacobi_update<2>(src[c - 1u], src[c + 1u], src[c - sx], src[c + sx], src[c - sxy],
                                              src[c + sxy]);
            }
        }
}

// Device address of the static scratch array on the current device, looked
// up once per device (the symbol's name is only a host-side stand-in).
od_status scratch_for_current_device(double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(OD_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(OD_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return set_error(OD_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return OD_OK;
}

}  // namespace

extern "C" OD_API od_status od_jacobi_noalloc(const double *u_in, double *u_out, int64_t nx, int64_t ny,
                                                int64_t nz, int32_t iters, void *stream) {
    if (!u_in || !u_out) return set_error(OD_EINVAL, "od_jacobi_noalloc: null field pointer");
    if (nx < 1 || ny < 1 || nz < 1 || iters < 0)
        return set_error(OD_EINVAL, "od_jacobi_noalloc: extents must be >= 1 and iters >= 0");
    if (nx > kScratchDoubles || ny > kScratchDoubles || nz > kScratchDoubles ||
        (nx + 2) * (ny + 2) > kScratchDoubles || (nx + 2) * (ny + 2) * (nz + 2) > kScratchDoubles)
        return set_error(OD_EINVAL, "od_jacobi_noalloc: padded grid (nx+2)(ny+2)(nz+2) exceeds the static scratch "
                                    "of " + std::to_string(kScratchDoubles) + " cells");
    const int64_t npad = (nx + 2) * (ny + 2) * (nz + 2);
    const size_t bytes = (size_t)npad * sizeof(double);
    const uintptr_t a0 = (uintptr_t)u_in, b0 = (uintptr_t)u_out;
    if (a0 < b0 + bytes && b0 < a0 + bytes)
        return set_error(OD_EINVAL, "od_jacobi_noalloc: input and output fields overlap");
    double *scratch = nullptr;
    od_status s = scratch_for_current_device(&scratch);
    if (s != OD_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // Both buffers start as the input, so both hold the Dirichlet shell and
    // nothing of an earlier call survives in the scratch.
    cudaError_t e = cudaMemcpyAsync(u_out, u_in, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && iters > 1) e = cudaMemcpyAsync(scratch, u_in, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return set_error(OD_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    const int block = 128;
    const dim3 grid((unsigned)std::min<int64_t>((nx + block - 1) / block, 64), (unsigned)std::min<int64_t>(ny, 65535),
                    (unsigned)std::min<int64_t>(nz, 65535));
    // step t writes u_out when iters-1-t is even, so the last step lands there
    const double *src = u_in;
    for (int32_t t = 0; t < iters; ++t) {
        double *dst = ((iters - 1 - t) % 2 == 0) ? u_out : scratch;
        k_noalloc_step<<<grid, block, 0, st>>>(src, dst, (uint32_t)nx, (uint32_t)ny, (uint32_t)nz);
        e = cudaGetLastError();
        if (e != cudaSuccess) return set_error(OD_ECUDA, std::string("k_noalloc_step: ") + cudaGetErrorString(e));
        src = dst;
    }
    return OD_OK;
}
