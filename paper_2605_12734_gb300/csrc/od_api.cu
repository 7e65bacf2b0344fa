// od_api.cu -- the C ABI of libod (see include/od.h): context lifetime and
// the four execution paths.
//
// No call below allocates device memory or synchronises the host inside
// od_step: every buffer, stream and event is created in od_create (Sec. III
// "Using Kokkos": persistent views, preallocated scratch, no implicit fences,
// execution spaces created once), and every path only enqueues work.
#include <cuda_runtime.h>

#include <sys/stat.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "od.h"
#include "od_arith.cuh"
#include "od_internal.h"
#include "od_kernels.h"
#include "od_plan.h"
#include "od_ctx.h"

namespace {

thread_local std::string g_last_error;

od_status fail(od_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

od_status cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(OD_ECUDA, m);
}

#define OD_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace




namespace {

KArgs base_args_impl(const od_ctx *c) {
    KArgs a;
    memset(&a, 0, sizeof a);
    a.ch = c->d_ch;
    a.tiles = c->d_tiles;
    a.err = c->d_err;
    a.queue = c->d_queue;
    a.epoch = c->d_epoch;
    a.dep_ptr = c->d_dep_ptr;
    a.dep_idx = c->d_dep_idx;
    a.order = c->d_order;
    a.vmax = c->d_vmax;
    a.one = 1u;
    a.ntiles = (int32_t)c->plan.tiles.size();
    a.order_mode = c->cfg.order & 1;
    a.stages = c->plan.stages;
    a.stage_doubles = c->plan.stage_doubles;
    a.stall_tile = c->stall_tile;
    a.spin_ns = c->spin_ns;
    a.stencil = c->plan.stencil;
    return a;
}

// --- fused path: one kernel per step over all tiles
od_status enqueue_fused(od_ctx *c, int32_t iters) {
    const od::Plan &p = c->plan;
    for (int32_t s = 0; s < iters; ++s) {
        KArgs a = base_args_impl(c);
        a.tile_begin = 0;
        a.parity = (int32_t)(c->steps & 1);
        OD_CUDA(od::launch_tiles(a, (int)p.tiles.size(), p.threads, p.cpt, p.amode, true, p.smem_bytes, c->stream));
        c->steps++;
        c->launches++;
        c->api_calls++;
    }
    return OD_OK;
}

// --- persistent path: one launch for many steps
od_status enqueue_persistent(od_ctx *c, int32_t iters) {
    const od::Plan &p = c->plan;
    const int64_t nt = (int64_t)p.tiles.size();
    int bps = 0;
    OD_CUDA(od::persistent_occupancy(p.threads, p.cpt, p.amode, p.smem_bytes, p.stencil, &bps));
    if (bps < 1) return fail(OD_EINVAL, "persistent kernel does not fit on an SM with this tiling");
    int grid = (int)std::min<int64_t>(nt, (int64_t)bps * c->num_sms);
    c->persistent_grid = grid;
    // keep tickets inside int32
    int32_t chunk_max = (int32_t)std::max<int64_t>(1, (INT32_MAX - 65536) / nt);
    int32_t done = 0;
    while (done < iters) {
        int32_t n = std::min(iters - done, chunk_max);
        OD_CUDA(cudaMemsetAsync(c->d_queue, 0, sizeof(int32_t), c->stream));
        OD_CUDA(cudaMemsetAsync(c->d_epoch, 0, (size_t)nt * sizeof(int32_t), c->stream));
        KArgs a = base_args_impl(c);
        a.iters = n;
        a.t0 = (int32_t)(c->steps & 0x7fffffff);
        OD_CUDA(od::launch_persistent(a, grid, p.threads, p.cpt, p.amode, p.smem_bytes, c->stream));
        c->steps += n;
        c->launches++;
        c->api_calls += 3;
        done += n;
    }
    return OD_OK;
}

// --- per-chare path (also what the graph path captures)
// Step t, chare c on stream pool[c % P]:
//   phase A: compute (own tiles, no push) -> pack new faces -> one D2D copy per
//            face into the neighbour's receive slot t&1 -> record ev[c][t&1]
//   phase B: wait for each neighbour's ev[n][t&1] -> unpack into ghosts.
// Receive slots alternate by step, so a sender at step t+2 overwrites slot
// t&1 only after its own stream has waited (in phase B of step t+1) for the
// receiver's step t+1 delivery, which its stream issued after the receiver's
// step-t unpack.
// Phase A of chare ci at step t on stream st (see above).
cudaError_t per_chare_phase_a(od_ctx *c, int ci, int64_t t, cudaStream_t st, int64_t *kernels, int64_t *calls) {
    const od::Plan &p = c->plan;
    const int sp = (int)(t & 1), dp = sp ^ 1, slot = (int)(t & 1);
    const od::HostChare &h = p.ch[(size_t)ci];
    KArgs a = base_args_impl(c);
    a.tile_begin = h.tile_begin;
    a.parity = sp;
    cudaError_t e = od::launch_tiles(a, h.tile_end - h.tile_begin, p.threads, p.cpt, p.amode, false, p.smem_bytes, st);
    if (e == cudaSuccess) e = od::launch_pack(c->d_ch, ci, dp, h.foff[6], st);
    if (e != cudaSuccess) return e;
    (*kernels) += 2;
    (*calls) += 2;
    for (int f = 0; f < 6; ++f) {
        const int n = h.nbr[f];
        if (n < 0) continue;
        const int opp = f ^ 1;
        const ChareDev &dn = c->h_ch[(size_t)n];
        const ChareDev &me = c->h_ch[(size_t)ci];
        const size_t bytes = (size_t)(h.foff[f + 1] - h.foff[f]) * sizeof(double);
        if (bytes == 0) continue;
        e = cudaMemcpyAsync(dn.recv[slot] + dn.foff[opp], me.send + me.foff[f], bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        (*calls)++;
    }
    (*calls)++;
    return cudaEventRecord(c->ev[2 * (size_t)ci + slot], st);
}

// Phase B of chare ci at step t: wait for the neighbours' deliveries, unpack.
cudaError_t per_chare_phase_b(od_ctx *c, int ci, int64_t t, cudaStream_t st, int64_t *kernels, int64_t *calls) {
    const od::HostChare &h = c->plan.ch[(size_t)ci];
    const int dp = (int)(t & 1) ^ 1, slot = (int)(t & 1);
    bool any = false;
    for (int f = 0; f < 6; ++f) {
        const int n = h.nbr[f];
        if (n < 0) continue;
        any = true;
        const cudaError_t e = cudaStreamWaitEvent(st, c->ev[2 * (size_t)n + slot], 0);
        if (e != cudaSuccess) return e;
        (*calls)++;
    }
    if (!any) return cudaSuccess;
    (*kernels)++;
    (*calls)++;
    return od::launch_unpack(c->d_ch, ci, dp, slot, h.foff[6], st);
}

od_status enqueue_per_chare_steps(od_ctx *c, int64_t t_first, int32_t iters, int64_t *kernels,
                                  int64_t *calls) {
    const int P = (int)c->pool.size();
    const int nch = (int)c->plan.ch.size();
    OD_CUDA(cudaEventRecord(c->fork, c->stream));
    (*calls)++;
    for (int i = 0; i < P; ++i) {
        OD_CUDA(cudaStreamWaitEvent(c->pool[i], c->fork, 0));
        (*calls)++;
    }
    for (int32_t s = 0; s < iters; ++s) {
        const int64_t t = t_first + s;
        for (int ci = 0; ci < nch; ++ci) OD_CUDA(per_chare_phase_a(c, ci, t, c->pool[ci % P], kernels, calls));
        for (int ci = 0; ci < nch; ++ci) OD_CUDA(per_chare_phase_b(c, ci, t, c->pool[ci % P], kernels, calls));
    }
    for (int i = 0; i < P; ++i) {
        OD_CUDA(cudaEventRecord(c->join[i], c->pool[i]));
        OD_CUDA(cudaStreamWaitEvent(c->stream, c->join[i], 0));
        (*calls) += 2;
    }
    return OD_OK;
}

// A reusable barrier for the submitting host threads (spin, then yield).
class HostBarrier {
  public:
    explicit HostBarrier(int n) : n_(n) {}
    void wait() {
        const int64_t g = gen_.load(std::memory_order_acquire);
        if (count_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
            count_.store(0, std::memory_order_relaxed);
            gen_.store(g + 1, std::memory_order_release);
            return;
        }
        for (int spin = 0; gen_.load(std::memory_order_acquire) == g; ++spin)
            if (spin > 256) std::this_thread::yield();
    }

  private:
    const int n_;
    std::atomic<int> count_{0};
    std::atomic<int64_t> gen_{0};
};

// The per-chare path submitted by T host threads (the paper's several PEs
// per GPU, Sec. III): thread k owns a contiguous block of chares and its own
// slice of the stream pool.  Phase A of a step (every chare's records) must
// be issued before any phase-B wait on those events, so the threads meet at
// a barrier between the phases and after each step.
od_status enqueue_per_chare_mt(od_ctx *c, int32_t iters, int T) {
    const int P = (int)c->pool.size();
    const int nch = (int)c->plan.ch.size();
    T = std::max(1, std::min({T, P, nch}));
    OD_CUDA(cudaEventRecord(c->fork, c->stream));
    for (int i = 0; i < P; ++i) OD_CUDA(cudaStreamWaitEvent(c->pool[i], c->fork, 0));
    int64_t calls_all = 1 + P;
    HostBarrier bar(T);
    std::atomic<int> failed{0};
    std::vector<cudaError_t> err((size_t)T, cudaSuccess);
    std::vector<int64_t> kern((size_t)T, 0), calls((size_t)T, 0);
    const int64_t t_first = c->steps;
    auto work = [&](int k) {
        const int c0 = (int)((int64_t)nch * k / T), c1 = (int)((int64_t)nch * (k + 1) / T);
        const int s0 = P * k / T, ns = std::max(1, P * (k + 1) / T - s0);
        cudaError_t e = cudaSetDevice(c->device);
        for (int32_t s = 0; s < iters; ++s) {
            const int64_t t = t_first + s;
            for (int ci = c0; ci < c1 && e == cudaSuccess && !failed.load(); ++ci)
                e = per_chare_phase_a(c, ci, t, c->pool[s0 + (ci - c0) % ns], &kern[k], &calls[k]);
            if (e != cudaSuccess) failed.store(1);
            bar.wait();  // every record of this step is issued before any wait on it
            for (int ci = c0; ci < c1 && e == cudaSuccess && !failed.load(); ++ci)
                e = per_chare_phase_b(c, ci, t, c->pool[s0 + (ci - c0) % ns], &kern[k], &calls[k]);
            if (e != cudaSuccess) failed.store(1);
            bar.wait();
        }
        err[(size_t)k] = e;
    };
    std::vector<std::thread> th;
    for (int k = 1; k < T; ++k) th.emplace_back(work, k);
    work(0);
    for (auto &x : th) x.join();
    for (int k = 0; k < T; ++k)
        if (err[(size_t)k] != cudaSuccess) return cuda_fail(err[(size_t)k], "per-chare submission");
    for (int i = 0; i < P; ++i) {
        OD_CUDA(cudaEventRecord(c->join[i], c->pool[i]));
        OD_CUDA(cudaStreamWaitEvent(c->stream, c->join[i], 0));
    }
    calls_all += 2 * P;
    for (int k = 0; k < T; ++k) {
        c->launches += kern[(size_t)k];
        calls_all += calls[(size_t)k];
    }
    c->api_calls += calls_all;
    c->steps += iters;
    return OD_OK;
}

od_status enqueue_per_chare(od_ctx *c, int32_t iters) {
    if (c->cfg.pe_threads > 1) return enqueue_per_chare_mt(c, iters, c->cfg.pe_threads);
    int64_t k = 0, calls = 0;
    od_status s = enqueue_per_chare_steps(c, c->steps, iters, &k, &calls);
    c->launches += k;
    c->api_calls += calls;
    if (s == OD_OK) c->steps += iters;
    return s;
}

od_status capture(od_ctx *c, int64_t t_first, int32_t iters, cudaGraphExec_t *out, int64_t *kernels,
                  int64_t *calls) {
    cudaGraph_t g = nullptr;
    OD_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    od_status s = enqueue_per_chare_steps(c, t_first, iters, kernels, calls);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (s != OD_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return OD_OK;
}

od_status enqueue_graph(od_ctx *c, int32_t iters) {
    if (iters <= 0) return OD_OK;
    if (!c->g2) {
        // captured once: two steps from an even step, and one step from each parity
        od_status s = capture(c, 0, 2, &c->g2, &c->g2_kernels, &c->g2_calls);
        if (s == OD_OK) s = capture(c, 0, 1, &c->g1[0], &c->g1_kernels[0], &c->g1_calls[0]);
        if (s == OD_OK) s = capture(c, 1, 1, &c->g1[1], &c->g1_kernels[1], &c->g1_calls[1]);
        if (s != OD_OK) return s;
    }
    int32_t left = iters;
    if (c->steps & 1) {
        OD_CUDA(cudaGraphLaunch(c->g1[1], c->stream));
        c->launches += c->g1_kernels[1];
        c->graph_launches++;
        c->api_calls++;
        c->steps++;
        left--;
    }
    while (left >= 2) {
        OD_CUDA(cudaGraphLaunch(c->g2, c->stream));
        c->launches += c->g2_kernels;
        c->graph_launches++;
        c->api_calls++;
        c->steps += 2;
        left -= 2;
    }
    if (left == 1) {
        OD_CUDA(cudaGraphLaunch(c->g1[0], c->stream));
        c->launches += c->g1_kernels[0];
        c->graph_launches++;
        c->api_calls++;
        c->steps++;
    }
    return OD_OK;
}

// --- fused-graph path: the fused step loop captured as CUDA graphs.  A
// fused step's only state is the parity of its source buffer, so a graph of
// kFusedGraphSteps steps from an even step serves every even start and the
// two one-step graphs cover an odd start and an odd remainder.
constexpr int32_t kFusedGraphSteps = 8;

od_status capture_fused(od_ctx *c, int64_t t_first, int32_t iters, cudaGraphExec_t *out) {
    const od::Plan &p = c->plan;
    cudaGraph_t g = nullptr;
    OD_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int32_t s = 0; s < iters && e == cudaSuccess; ++s) {
        KArgs a = base_args_impl(c);
        a.tile_begin = 0;
        a.parity = (int32_t)((t_first + s) & 1);
        e = od::launch_tiles(a, (int)p.tiles.size(), p.threads, p.cpt, p.amode, true, p.smem_bytes, c->stream);
    }
    const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e != cudaSuccess ? e : e2, "capturing the fused step loop");
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return OD_OK;
}

od_status enqueue_fused_graph(od_ctx *c, int32_t iters) {
    if (iters <= 0) return OD_OK;
    if (!c->gf) {
        od_status s = capture_fused(c, 0, kFusedGraphSteps, &c->gf);
        if (s == OD_OK) s = capture_fused(c, 0, 1, &c->gf1[0]);
        if (s == OD_OK) s = capture_fused(c, 1, 1, &c->gf1[1]);
        if (s != OD_OK) return s;
    }
    auto replay = [&](cudaGraphExec_t g, int32_t steps) -> od_status {
        OD_CUDA(cudaGraphLaunch(g, c->stream));
        c->launches += steps;
        c->graph_launches++;
        c->api_calls++;
        c->steps += steps;
        return OD_OK;
    };
    int32_t left = iters;
    od_status s = OD_OK;
    if (c->steps & 1) {
        s = replay(c->gf1[1], 1);
        left--;
    }
    while (s == OD_OK && left >= kFusedGraphSteps) {
        s = replay(c->gf, kFusedGraphSteps);
        left -= kFusedGraphSteps;
    }
    while (s == OD_OK && left > 0) {
        s = replay(c->gf1[c->steps & 1], 1);
        left--;
    }
    return s;
}

od_status check_device_error_impl(od_ctx *c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && c->copy_pending) {
        e = cudaStreamSynchronize(c->copy_stream);
        c->copy_pending = false;
    }
    if (e != cudaSuccess) {
        c->failed = true;
        return cuda_fail(e, "cudaStreamSynchronize");
    }
    ErrDev h;
    e = cudaMemcpy(&h, c->d_err, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        c->failed = true;
        return cuda_fail(e, "cudaMemcpy(error record)");
    }
    if (h.code != 0) {
        c->failed = true;
        char buf[200];
        if (h.code == OD_ERR_TMA_TIMEOUT || h.code == OD_ERR_DEP_TIMEOUT) {
            snprintf(buf, sizeof buf, "device wait ran out (%s) at tile %d, step %d",
                     h.code == OD_ERR_TMA_TIMEOUT ? "bulk copy" : "neighbour step counter", h.tile, h.step);
            return fail(OD_ETIMEOUT, buf);
        }
        snprintf(buf, sizeof buf, "kernel reported error %d", h.code);
        return fail(OD_ECUDA, buf);
    }
    return OD_OK;
}

// A host pointer the device can address directly: pinned (page-locked)
// host memory is mapped into the device's address space (unified
// addressing), so the gather kernel writes it in place over the host link
// instead of staging through a device buffer (measured faster than the copy
// engine's 192 GB/s device-to-host plus a staging pass).  Null otherwise.
template <class T>
T *device_view(T *host) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    // devicePointer maps the allocation's start; keep the offset of `host`
    return reinterpret_cast<T *>(static_cast<char *>(a.devicePointer) +
                                 (reinterpret_cast<const char *>(host) - static_cast<const char *>(a.hostPointer)));
}

od_status ensure_stage(od_ctx *c) {
    if (c->copy_pending) {  // an asynchronous export may still be reading the staging buffer
        cudaError_t e = cudaStreamWaitEvent(c->stream, c->ev_copied, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    }
    if (c->d_stage) return OD_OK;
    size_t bytes = (size_t)c->plan.cells * sizeof(double);
    cudaError_t e = cudaMalloc(&c->d_stage, bytes);
    if (e != cudaSuccess) {
        c->d_stage = nullptr;
        cudaGetLastError();
        return fail(OD_ENOMEM, "cannot allocate the host-transfer staging buffer");
    }
    return OD_OK;
}

void release(od_ctx *c) {
    if (!c) return;
    if (c->g2) cudaGraphExecDestroy(c->g2);
    for (auto &g : c->g1)
        if (g) cudaGraphExecDestroy(g);
    if (c->gf) cudaGraphExecDestroy(c->gf);
    for (auto &g : c->gf1)
        if (g) cudaGraphExecDestroy(g);
    for (auto e : c->ev) cudaEventDestroy(e);
    for (auto e : c->join) cudaEventDestroy(e);
    if (c->fork) cudaEventDestroy(c->fork);
    for (auto s : c->pool) cudaStreamDestroy(s);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->ev_gathered) cudaEventDestroy(c->ev_gathered);
    if (c->ev_copied) cudaEventDestroy(c->ev_copied);
    if (c->d_stage) cudaFree(c->d_stage);
    if (c->own_arena && c->arena) cudaFree(c->arena);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // namespace

// ---------------------------------------------------------------- autotuner
//
// od_create with autotune = 1 times candidate execution shapes on the real
// decomposition before the context is built: each candidate is a temporary
// context (autotune off) laid out in one shared tuning buffer, initialised,
// stepped twice untimed and then timed with events.  Candidates (in two
// rounds, coordinate descent): CTA shape x arithmetic mode (2, 3 and the
// mixed 7, 8) with the default ring, then ring depth x planes per tile for
// the best of those.  Every
// candidate computes the same bits, so the choice only changes speed.  The
// winner is cached in a text file (OD_TUNE_CACHE, default
// $HOME/.cache/libod/tune.txt; "off" disables the cache) keyed by device,
// path, grid and block edges.
namespace {

struct TuneChoice {
    int threads = 0, cpt = 0, stages = 0, arith = -1, tile_z = 0;
    double ms = 0;
};

std::string tune_cache_path() {
    const char *e = getenv("OD_TUNE_CACHE");
    if (e && *e) return std::string(e);
    const char *h = getenv("HOME");
    return std::string(h && *h ? h : "/tmp") + "/.cache/libod/tune.txt";
}

std::string tune_key(const od_config *cfg, const od::Plan &p, int device) {
    cudaDeviceProp prop;
    std::string name = "unknown";
    int sms = 0;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) {
        name = prop.name;
        sms = prop.multiProcessorCount;
    }
    for (auto &ch : name)
        if (ch == ' ') ch = '_';
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the block edges
    auto mix = [&](int64_t v) {
        for (int b = 0; b < 8; ++b) {
            h ^= (uint64_t)((v >> (8 * b)) & 0xff);
            h *= 1099511628211ull;
        }
    };
    for (auto v : p.ex) mix(v);
    mix(-1);
    for (auto v : p.ey) mix(v);
    mix(-1);
    for (auto v : p.ez) mix(v);
    char buf[256];
    // "k2": the kernel generation (pulled 3D halos, anchored arithmetic); an
    // entry timed on another generation's kernels is not reused
    snprintf(buf, sizeof buf, "k2/%s/%d/path%d/st%d/%lldx%lldx%lld/%016llx", name.c_str(), sms, cfg->path,
             p.stencil, (long long)p.nx, (long long)p.ny, (long long)p.nz, (unsigned long long)h);
    return buf;
}

bool tune_cache_lookup(const std::string &key, TuneChoice *c) {
    std::string path = tune_cache_path();
    if (path == "off") return false;
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return false;
    char k[256];
    TuneChoice t;
    bool found = false;
    while (fscanf(f, "%255s %d %d %d %d %d %lf", k, &t.threads, &t.cpt, &t.stages, &t.arith, &t.tile_z, &t.ms) == 7)
        if (key == k) {
            *c = t;
            found = true;
        }
    fclose(f);
    return found;
}

void tune_cache_store(const std::string &key, const TuneChoice &c) {
    std::string path = tune_cache_path();
    if (path == "off") return;
    std::string dir = path.substr(0, path.find_last_of('/'));
    if (!dir.empty()) {  // create the directory chain
        for (size_t i = 1; i <= dir.size(); ++i)
            if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
    }
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %.17g\n", key.c_str(), c.threads, c.cpt, c.stages, c.arith, c.tile_z, c.ms);
    fclose(f);
}

od_status run_tuning(const od_config *cfg, TuneChoice *best) {
    od::Plan base;
    std::string err;
    od_status s = od::build_plan(cfg, &base, &err);
    if (s != OD_OK) return fail(s, err);
    const std::string key = tune_key(cfg, base, cfg->device);
    if (tune_cache_lookup(key, best)) return OD_OK;

    const int shapes[6][2] = {{128, 4}, {128, 8}, {256, 4}, {256, 8}, {128, 2}, {256, 2}};
    // arithmetic modes worth timing: the anchored forms and the best earlier
    // integer-window forms of each stencil
    const int ariths3[5] = {12, 14, 15, 13, 10};
    const int ariths2[5] = {12, 14, 13, 2, 15};
    const int *ariths = base.stencil == OD_STENCIL_2D5 ? ariths2 : ariths3;
    std::vector<TuneChoice> round1;
    for (auto &sh : shapes)
        for (int k = 0; k < 5; ++k) {
            const int am = ariths[k];
            TuneChoice c;
            c.threads = sh[0];
            c.cpt = sh[1];
            c.stages = 4;
            c.arith = am;
            c.tile_z = cfg->tile_z;
            round1.push_back(c);
        }
    auto make_cfg = [&](const TuneChoice &c, void *arena, uint64_t bytes, cudaStream_t st) {
        od_config t = *cfg;
        t.autotune = 0;
        t.threads = c.threads;
        t.cells_per_thread = c.cpt;
        t.stages = c.stages;
        t.arith = c.arith;
        t.tile_z = c.tile_z;
        t.arena = arena;
        t.arena_bytes = bytes;
        t.stream = st;
        if (t.path == OD_PATH_PER_CHARE || t.path == OD_PATH_GRAPH) t.path = OD_PATH_FUSED;
        t.stream_pool = 1;
        return t;
    };
    // the tuning buffer: the largest arena any candidate needs
    uint64_t need = 0;
    std::vector<TuneChoice> cands;
    auto consider = [&](std::vector<TuneChoice> &list) {
        std::vector<TuneChoice> ok;
        for (auto &c : list) {
            od_config t = make_cfg(c, nullptr, 0, nullptr);
            od::Plan p;
            std::string e2;
            if (od::build_plan(&t, &p, &e2) != OD_OK) continue;
            // with a caller arena the final context must fit in it
            if (cfg->arena && p.arena_bytes > cfg->arena_bytes) continue;
            need = std::max<uint64_t>(need, p.arena_bytes);
            ok.push_back(c);
        }
        list.swap(ok);
    };
    consider(round1);
    if (round1.empty()) return fail(OD_EINVAL, "autotune: no candidate fits this decomposition");
    // round-2 candidates may need more table space; size generously
    need = need + need / 8 + (1u << 20);
    void *buf = nullptr;
    bool own_buf = false;
    if (cfg->arena && cfg->arena_bytes >= need) {
        buf = cfg->arena;  // the caller's arena is free until the context is built
    } else {
        if (cudaMalloc(&buf, need) != cudaSuccess) {
            cudaGetLastError();
            return OD_OK;  // no room to tune: keep the defaults
        }
        own_buf = true;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_one = [&](TuneChoice &c) -> bool {
        od_config t = make_cfg(c, buf, need, st);
        od_ctx *tmp = nullptr;
        if (od_create(&tmp, &t) != OD_OK) return false;
        bool good = od_step(tmp, 2) == OD_OK;
        if (good) {
            const int n = 5;
            cudaEventRecord(e0, st);
            good = od_step(tmp, n) == OD_OK;
            cudaEventRecord(e1, st);
            good = good && od_sync(tmp) == OD_OK;
            float ms = 0;
            if (good && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) c.ms = ms / n;
            else good = false;
        }
        od_destroy(tmp);
        return good;
    };
    TuneChoice win;
    win.ms = 1e30;
    for (auto &c : round1)
        if (time_one(c) && c.ms < win.ms) win = c;
    if (win.ms < 1e30) {
        std::vector<TuneChoice> round2;
        const int stages_c[3] = {3, 5, 6};
        const int tz_c[3] = {16, 32, 64};
        for (int sg : stages_c) {
            TuneChoice c = win;
            c.stages = sg;
            round2.push_back(c);
        }
        for (int tz : tz_c) {
            TuneChoice c = win;
            c.tile_z = tz;
            round2.push_back(c);
        }
        std::vector<TuneChoice> fits;
        for (auto &c : round2) {
            od_config t = make_cfg(c, nullptr, 0, nullptr);
            od::Plan p;
            std::string e2;
            if (od::build_plan(&t, &p, &e2) == OD_OK && p.arena_bytes <= need &&
                (!cfg->arena || p.arena_bytes <= cfg->arena_bytes))
                fits.push_back(c);
        }
        for (auto &c : fits)
            if (time_one(c) && c.ms < win.ms) win = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (own_buf) cudaFree(buf);
    g_last_error.clear();
    if (win.ms >= 1e30) return OD_OK;  // nothing ran: keep the defaults
    *best = win;
    tune_cache_store(key, win);
    return OD_OK;
}

}  // namespace

namespace od {
od_status set_last_error(od_status s, const std::string &msg) { return fail(s, msg); }
KArgs base_args(const od_ctx *c) { return base_args_impl(c); }
od_status check_device_error(od_ctx *c) { return check_device_error_impl(c); }
}  // namespace od

extern "C" {

const char *od_last_error(void) { return g_last_error.c_str(); }

const char *od_version(void) { return "libod 0.1 (sm_103a)"; }

void od_config_default(od_config *cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->nx = cfg->ny = cfg->nz = 64;
    cfg->px = cfg->py = cfg->pz = 1;
    cfg->seed = 1;
    cfg->init_mode = OD_INIT_UNIFORM;
    cfg->path = OD_PATH_FUSED;
    cfg->arith = -1;
}

// The anchor exponent of the anchored self-test ops, passed as b[0] (a
// double holding an integer), clamped to the range the routines accept.
static uint32_t anchor_arg(double v) {
    if (!(v >= (double)od::kAnchorMin)) return od::kAnchorMin;
    if (v > (double)od::kAnchorMax) return od::kAnchorMax;
    return (uint32_t)v;
}

od_status od_arith_host(int32_t op, const double *a, const double *b, double *out, int64_t n) {
    const bool anch = (op >= 30 && op <= 37) || (op >= 40 && op <= 46 && op != 43);
    if (n < 0 || (n > 0 && (!a || !out || ((op == 1 || anch) && !b)))) return fail(OD_EINVAL, "bad arguments");
    if (op != 0 && op != 1 && !(op >= 10 && op <= 18) && !(op >= 20 && op <= 26) && !anch)
        return fail(OD_EINVAL,
                    "host op must be 0 (div6), 1 (add), 10..18 (3D update), 20..26 (2D update), 30..37 or "
                    "40..42, 44..46 (anchored updates)");
    const uint32_t e0 = anch && n > 0 ? anchor_arg(b[0]) : 0u;
    for (int64_t i = 0; i < n; ++i)
        out[i] = op == 0   ? od::div6(a[i])
                 : op == 1 ? od::add(a[i], b[i])
                 : op < 20 ? od::jacobi_update_mode(op - 10, a + 6 * i)
                 : op < 30 ? od::jacobi2d_update_mode(op - 20, a + 4 * i)
                 : op < 40 ? od::jacobi_update_anchored_mode(op - 30, a + 6 * i, e0)
                           : od::jacobi2d_update_anchored_mode(op - 40, a + 4 * i, e0);
    return OD_OK;
}

od_status od_arith_device(int32_t op, const double *a, const double *b, double *out, int64_t n) {
    const bool anch = (op >= 30 && op <= 37) || (op >= 40 && op <= 46 && op != 43);
    if (n < 0 || (n > 0 && (!a || !out || ((op == 1 || op == 3 || anch) && !b))))
        return fail(OD_EINVAL, "bad arguments");
    if (!((op >= 0 && op <= 3) || (op >= 10 && op <= 18) || (op >= 20 && op <= 26) || anch))
        return fail(OD_EINVAL, "op must be 0..3, 10..18, 20..26, 30..37, 40..42 or 44..46");
    if (n == 0) return OD_OK;
    OD_CUDA(od::launch_arith(op, a, b, out, n, 0));
    OD_CUDA(cudaStreamSynchronize(0));
    return OD_OK;
}

od_status od_plan(const od_config *cfg, od_plan_info *out) {
    if (!cfg || !out) return fail(OD_EINVAL, "null argument");
    od::Plan p;
    std::string err;
    od_status s = od::build_plan(cfg, &p, &err);
    if (s != OD_OK) return fail(s, err);
    od::plan_info(p, out);
    return OD_OK;
}

od_status od_plan_tiles(const od_config *cfg, int64_t *tiles, int64_t tiles_cap, int32_t *dep_ptr,
                        int32_t *dep_idx, int64_t deps_cap, int64_t *ntiles, int64_t *ndeps) {
    if (!cfg || !ntiles || !ndeps) return fail(OD_EINVAL, "null argument");
    od::Plan p;
    std::string err;
    od_status s = od::build_plan(cfg, &p, &err);
    if (s != OD_OK) return fail(s, err);
    *ntiles = (int64_t)p.tiles.size();
    *ndeps = (int64_t)p.dep_idx.size();
    if (tiles && tiles_cap >= *ntiles) {
        for (size_t t = 0; t < p.tiles.size(); ++t) {
            const TileDev &T = p.tiles[t];
            const od::HostChare &h = p.ch[(size_t)T.c];
            int64_t *o = tiles + 8 * t;
            o[0] = T.c;
            o[1] = h.x0 + T.i0; o[2] = T.ni;
            o[3] = h.y0 + T.j0; o[4] = T.nj;
            o[5] = h.z0 + T.k0; o[6] = T.nk;
            o[7] = 0;
        }
    }
    if (dep_ptr && dep_idx && tiles_cap >= *ntiles && deps_cap >= *ndeps) {
        std::copy(p.dep_ptr.begin(), p.dep_ptr.end(), dep_ptr);
        std::copy(p.dep_idx.begin(), p.dep_idx.end(), dep_idx);
    }
    return OD_OK;
}

od_status od_decompose(const od_config *cfg, int64_t *box, int32_t *nbr, int64_t capacity) {
    if (!cfg || !box || !nbr) return fail(OD_EINVAL, "null argument");
    od::Plan p;
    std::string err;
    od_status s = od::build_plan(cfg, &p, &err);
    if (s != OD_OK) return fail(s, err);
    if ((int64_t)p.ch.size() > capacity) return fail(OD_EINVAL, "capacity smaller than the chare count");
    for (size_t c = 0; c < p.ch.size(); ++c) {
        const od::HostChare &h = p.ch[c];
        int64_t *b = box + 6 * c;
        if (p.stencil == OD_STENCIL_2D5) {  // report the 2D grid, not its internal (nx, 1, ny) layout
            b[0] = h.x0; b[1] = h.bx; b[2] = h.z0; b[3] = h.bz; b[4] = 0; b[5] = 1;
            const int32_t f2[6] = {h.nbr[OD_FACE_XLO], h.nbr[OD_FACE_XHI], h.nbr[OD_FACE_ZLO], h.nbr[OD_FACE_ZHI], -1, -1};
            for (int f = 0; f < 6; ++f) nbr[6 * c + f] = f2[f];
            continue;
        }
        b[0] = h.x0; b[1] = h.bx; b[2] = h.y0; b[3] = h.by; b[4] = h.z0; b[5] = h.bz;
        for (int f = 0; f < 6; ++f) nbr[6 * c + f] = h.nbr[f];
    }
    return OD_OK;
}

}  // extern "C"

namespace od {
od_status create_context(od_ctx **out, const od_config *cfg_in, bool sync) {
    if (!out || !cfg_in) return fail(OD_EINVAL, "null argument");
    *out = nullptr;
    od_config tuned = *cfg_in;
    const od_config *cfg = &tuned;
    double tune_ms = 0;
    if (cfg_in->autotune) {
        DeviceGuard dg0(cfg_in->device);
        TuneChoice best;
        od_status ts = run_tuning(cfg_in, &best);
        if (ts != OD_OK) return ts;
        if (best.threads) {
            tuned.threads = best.threads;
            tuned.cells_per_thread = best.cpt;
            tuned.stages = best.stages;
            tuned.arith = best.arith;
            tuned.tile_z = best.tile_z;
            tune_ms = best.ms;
        }
        tuned.autotune = 0;
    }
    od_ctx *c = new od_ctx();
    c->cfg = *cfg;
    c->tuned = cfg_in->autotune != 0;
    c->tune_ms = tune_ms;
    c->cfg.cuts_x = c->cfg.cuts_y = c->cfg.cuts_z = nullptr;  // not kept past the call
    std::string err;
    od_status s = od::build_plan(cfg, &c->plan, &err);
    if (s != OD_OK) {
        release(c);
        return fail(s, err);
    }
    od::Plan &p = c->plan;
    c->device = cfg->device;
    c->path = cfg->path;
    c->spin_ns = cfg->spin_limit_ns ? cfg->spin_limit_ns : kDefaultSpinNs;
    DeviceGuard dg(c->device);
    if (!dg.ok) {
        release(c);
        return fail(OD_ECUDA, "cannot select the CUDA device");
    }
#define OD_TRY(call)                                      \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) {                          \
            od_status r_ = cuda_fail(e_, #call);          \
            release(c);                                   \
            return r_;                                    \
        }                                                 \
    } while (0)
    OD_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    if (!od::tile_shape_supported(p.threads, p.cpt, p.amode, p.stencil)) {
        release(c);
        return fail(OD_EINVAL, "unsupported threads / cells_per_thread");
    }
    if (cfg->stream) {
        c->stream = (cudaStream_t)cfg->stream;
    } else {
        OD_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    if (cfg->arena) {
        if (cfg->arena_bytes < p.arena_bytes || ((uintptr_t)cfg->arena & 255u)) {
            release(c);
            return fail(OD_ENOMEM, "caller arena too small or not 256-byte aligned (size it with od_plan)");
        }
        c->arena = (char *)cfg->arena;
    } else {
        cudaError_t e = cudaMalloc(&c->arena, p.arena_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->arena = nullptr;
            release(c);
            return fail(OD_ENOMEM, "cudaMalloc of the chare arena failed");
        }
        c->own_arena = true;
    }
    char *A = c->arena;
    c->d_err = (ErrDev *)(A + p.off_err);
    c->d_queue = (int32_t *)(A + p.off_queue);
    c->d_epoch = (int32_t *)(A + p.off_epoch);
    c->d_ch = (ChareDev *)(A + p.off_chares);
    c->d_tiles = (TileDev *)(A + p.off_tiles);
    c->d_dep_ptr = (int32_t *)(A + p.off_dep_ptr);
    c->d_dep_idx = (int32_t *)(A + p.off_dep_idx);
    c->d_order = (int32_t *)(A + p.off_order);
    c->d_vmax = (uint64_t *)(A + p.off_queue + 8);  // the queue block holds 64 bytes
    c->h_ch.resize(p.ch.size());
    for (size_t i = 0; i < p.ch.size(); ++i) {
        const od::HostChare &h = p.ch[i];
        ChareDev &d = c->h_ch[i];
        memset(&d, 0, sizeof d);
        d.bx = h.bx; d.by = h.by; d.bz = h.bz; d.pitch = h.pitch;
        d.rows = h.rows; d.row0 = h.row0;
        for (int f = 0; f < 6; ++f) d.nbr[f] = h.nbr[f];
        for (int f = 0; f < 7; ++f) d.foff[f] = h.foff[f];
        d.x0 = h.x0; d.y0 = h.y0; d.z0 = h.z0;
        for (int s2 = 0; s2 < 2; ++s2) {
            d.A[s2] = (double *)(A + h.offA[s2]);
            d.recv[s2] = (double *)(A + h.offRecv[s2]);
        }
        d.send = (double *)(A + h.offSend);
    }
    OD_TRY(cudaMemsetAsync(A, 0, p.off_chares, c->stream));  // error record, queue, epochs
    OD_TRY(cudaMemcpyAsync(c->d_ch, c->h_ch.data(), c->h_ch.size() * sizeof(ChareDev),
                           cudaMemcpyHostToDevice, c->stream));
    OD_TRY(cudaMemcpyAsync(c->d_tiles, p.tiles.data(), p.tiles.size() * sizeof(TileDev),
                           cudaMemcpyHostToDevice, c->stream));
    OD_TRY(cudaMemcpyAsync(c->d_dep_ptr, p.dep_ptr.data(), p.dep_ptr.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice, c->stream));
    if (!p.dep_idx.empty())
        OD_TRY(cudaMemcpyAsync(c->d_dep_idx, p.dep_idx.data(), p.dep_idx.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, c->stream));
    OD_TRY(cudaMemcpyAsync(c->d_order, p.order.data(), p.order.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice, c->stream));
    OD_TRY(od::prepare_tile_kernels(p.threads, p.cpt, p.amode, p.smem_bytes, p.stencil));
    // per-chare path resources
    int P = cfg->stream_pool > 0 ? cfg->stream_pool : 32;
    P = (int)std::min<int64_t>(P, (int64_t)p.ch.size());
    c->pool.resize((size_t)P, nullptr);
    c->join.resize((size_t)P, nullptr);
    for (int i = 0; i < P; ++i) {
        OD_TRY(cudaStreamCreateWithFlags(&c->pool[i], cudaStreamNonBlocking));
        OD_TRY(cudaEventCreateWithFlags(&c->join[i], cudaEventDisableTiming));
    }
    OD_TRY(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
    c->ev.resize(2 * p.ch.size(), nullptr);
    for (auto &e : c->ev) OD_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    OD_TRY(od::launch_init(c->d_ch, (int)p.ch.size(), p.gnx, p.gny, p.gnz, p.gx0, p.gy0, p.gz0, cfg->seed,
                           cfg->init_mode, p.stencil,
                           c->stream));
    // every initial value lies in [0, 1): the largest possible one anchors
    // the exact arithmetic's window (od_write raises it for imported fields)
    const uint64_t vmax0 = 0x3FEFFFFFFFFFFFFFull;
    OD_TRY(cudaMemcpyAsync(c->d_vmax, &vmax0, sizeof vmax0, cudaMemcpyHostToDevice, c->stream));
    if (sync) OD_TRY(cudaStreamSynchronize(c->stream));
    c->ghosts_current = true;
#undef OD_TRY
    *out = c;
    return OD_OK;
}
}  // namespace od

extern "C" {

od_status od_create(od_ctx **out, const od_config *cfg_in) { return od::create_context(out, cfg_in, true); }

od_status od_step(od_ctx *c, int32_t iters) {
    if (!c) return fail(OD_EINVAL, "null context");
    if (iters < 0) return fail(OD_EINVAL, "iters must be >= 0");
    if (c->failed) return fail(OD_ESTATE, "context failed earlier; destroy it");
    if (iters == 0) return OD_OK;
    DeviceGuard dg(c->device);
    switch (c->path) {
        case OD_PATH_FUSED:
        case OD_PATH_FUSED_GRAPH:
        case OD_PATH_PERSISTENT: {
            // the fused sweeps read the neighbours' faces and leave the
            // ghost layers behind
            od_status s = c->path == OD_PATH_FUSED         ? enqueue_fused(c, iters)
                          : c->path == OD_PATH_FUSED_GRAPH ? enqueue_fused_graph(c, iters)
                                                           : enqueue_persistent(c, iters);
            c->ghosts_current = false;
            return s;
        }
        case OD_PATH_PER_CHARE:
        case OD_PATH_GRAPH: {
            // the per-chare flow reads its own ghost layers: refresh them
            // once after fused steps (its own steps keep them current)
            if (!c->ghosts_current) {
                OD_CUDA(od::launch_ghost_refresh(c->d_ch, (int)c->plan.ch.size(), (int)(c->steps & 1), c->stream));
                c->launches++;
                c->api_calls++;
                c->ghosts_current = true;
            }
            return c->path == OD_PATH_PER_CHARE ? enqueue_per_chare(c, iters) : enqueue_graph(c, iters);
        }
        default: return fail(OD_EINVAL, "unknown path");
    }
}

od_status od_set_path(od_ctx *c, int32_t path) {
    if (!c) return fail(OD_EINVAL, "null context");
    if (path < OD_PATH_PER_CHARE || path > OD_PATH_FUSED_GRAPH) return fail(OD_EINVAL, "unknown path");
    c->path = path;
    return OD_OK;
}

od_status od_sync(od_ctx *c) {
    if (!c) return fail(OD_EINVAL, "null context");
    DeviceGuard dg(c->device);
    return check_device_error_impl(c);
}

od_status od_read_cells(od_ctx *c, const int64_t *cells, int64_t n, double *out) {
    if (!c || (n > 0 && (!cells || !out)) || n < 0 || n > (1 << 24))
        return fail(OD_EINVAL, "od_read_cells: null argument or n outside [0, 2^24]");
    if (n == 0) return OD_OK;
    DeviceGuard dg(c->device);
    od_status s = check_device_error_impl(c);
    if (s != OD_OK) return s;
    const od::Plan &p = c->plan;
    const int par = (int)(c->steps & 1);
    // global index -> (x, y, z) of the internal grid -> chare -> address
    std::vector<const double *> addr((size_t)n);
    for (int64_t q = 0; q < n; ++q) {
        const int64_t g = cells[q];
        if (g < 0 || g >= p.cells) return fail(OD_EINVAL, "od_read_cells: cell index outside the grid");
        const int64_t x = g % p.nx, yz = g / p.nx, y = yz % p.ny, z = yz / p.ny;
        const int cx = (int)(std::upper_bound(p.ex.begin(), p.ex.end(), x) - p.ex.begin()) - 1;
        const int cy = (int)(std::upper_bound(p.ey.begin(), p.ey.end(), y) - p.ey.begin()) - 1;
        const int cz = (int)(std::upper_bound(p.ez.begin(), p.ez.end(), z) - p.ez.begin()) - 1;
        const size_t ci = (size_t)cx + (size_t)p.px * ((size_t)cy + (size_t)p.py * (size_t)cz);
        const ChareDev &C = c->h_ch[ci];
        const int64_t i = x - C.x0, j = y - C.y0, k = z - C.z0;
        addr[(size_t)q] = C.A[par] + ((k + 1) * C.rows + j + C.row0) * (int64_t)C.pitch + i + 1;
    }
    void *d_addr = nullptr, *d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_addr, (size_t)n * sizeof(void *));
    if (e == cudaSuccess) e = cudaMalloc(&d_out, (size_t)n * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_addr, addr.data(), (size_t)n * sizeof(void *), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = od::launch_read_cells(static_cast<const double *const *>(d_addr), n, static_cast<double *>(d_out),
                                  c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, d_out, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (d_addr) cudaFree(d_addr);
    if (d_out) cudaFree(d_out);
    return e == cudaSuccess ? OD_OK : cuda_fail(e, "od_read_cells");
}

od_status od_read(od_ctx *c, double *dst, int32_t dst_is_device) {
    if (!c || !dst) return fail(OD_EINVAL, "null argument");
    DeviceGuard dg(c->device);
    od_status s = check_device_error_impl(c);
    if (s != OD_OK) return s;
    const od::Plan &p = c->plan;
    const int par = (int)(c->steps & 1);
    double *mapped = dst_is_device ? nullptr : device_view(dst);
    if (dst_is_device || mapped) {
        OD_CUDA(od::launch_gather(c->d_ch, (int)p.ch.size(), par, p.nx, p.ny, dst_is_device ? dst : mapped,
                                  c->stream));
    } else {
        s = ensure_stage(c);
        if (s != OD_OK) return s;
        OD_CUDA(od::launch_gather(c->d_ch, (int)p.ch.size(), par, p.nx, p.ny, c->d_stage, c->stream));
        OD_CUDA(cudaMemcpyAsync(dst, c->d_stage, (size_t)p.cells * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
    }
    OD_CUDA(cudaStreamSynchronize(c->stream));
    return OD_OK;
}

od_status od_write(od_ctx *c, const double *src, int32_t src_is_device) {
    if (!c || !src) return fail(OD_EINVAL, "null argument");
    if (c->failed) return fail(OD_ESTATE, "context failed earlier; destroy it");
    DeviceGuard dg(c->device);
    const od::Plan &p = c->plan;
    const int par = (int)(c->steps & 1);
    const double *g = src;
    // host sources go through the staging buffer even when pinned: the copy
    // engine moves them faster (measured 210 GB/s) than the scatter kernel's
    // own reads across the host link, which also fetch the ghost cells twice
    if (!src_is_device) {
        od_status s = ensure_stage(c);
        if (s != OD_OK) return s;
        OD_CUDA(cudaMemcpyAsync(c->d_stage, src, (size_t)p.cells * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream));
        g = c->d_stage;
    }
    OD_CUDA(od::launch_scatter(c->d_ch, (int)p.ch.size(), par, p.nx, p.ny, p.nz, g, c->d_vmax, c->stream));
    c->ghosts_current = false;  // the scatter writes interiors only
    if (!src_is_device) OD_CUDA(cudaStreamSynchronize(c->stream));
    return OD_OK;
}

od_status od_write_async(od_ctx *c, const double *src) {
    if (!c || !src) return fail(OD_EINVAL, "null argument");
    if (c->failed) return fail(OD_ESTATE, "context failed earlier; destroy it");
    DeviceGuard dg(c->device);
    if (!device_view(src)) return fail(OD_EINVAL, "od_write_async: src is not pinned host memory");
    od_status s = ensure_stage(c);
    if (s != OD_OK) return s;
    const od::Plan &p = c->plan;
    OD_CUDA(cudaMemcpyAsync(c->d_stage, src, (size_t)p.cells * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    OD_CUDA(od::launch_scatter(c->d_ch, (int)p.ch.size(), (int)(c->steps & 1), p.nx, p.ny, p.nz, c->d_stage,
                               c->d_vmax, c->stream));
    c->ghosts_current = false;  // interiors only
    return OD_OK;
}

od_status od_read_async(od_ctx *c, double *dst) {
    if (!c || !dst) return fail(OD_EINVAL, "null argument");
    if (c->failed) return fail(OD_ESTATE, "context failed earlier; destroy it");
    DeviceGuard dg(c->device);
    if (!device_view(dst)) return fail(OD_EINVAL, "od_read_async: dst is not pinned host memory");
    od_status s = ensure_stage(c);
    if (s != OD_OK) return s;
    if (!c->copy_stream) {
        OD_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        OD_CUDA(cudaEventCreateWithFlags(&c->ev_gathered, cudaEventDisableTiming));
        OD_CUDA(cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming));
    }
    const od::Plan &p = c->plan;
    OD_CUDA(od::launch_gather(c->d_ch, (int)p.ch.size(), (int)(c->steps & 1), p.nx, p.ny, c->d_stage, c->stream));
    OD_CUDA(cudaEventRecord(c->ev_gathered, c->stream));
    OD_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_gathered, 0));
    OD_CUDA(cudaMemcpyAsync(dst, c->d_stage, (size_t)p.cells * sizeof(double), cudaMemcpyDeviceToHost,
                            c->copy_stream));
    OD_CUDA(cudaEventRecord(c->ev_copied, c->copy_stream));
    c->copy_pending = true;
    return OD_OK;
}

od_status od_face_copy(od_ctx *c, int32_t face, int32_t dir, double *buf, int32_t buf_is_device) {
    if (!c || !buf || (dir != 0 && dir != 1)) return fail(OD_EINVAL, "od_face_copy: null argument or dir not 0/1");
    if (c->failed) return fail(OD_ESTATE, "context failed earlier; destroy it");
    const od::Plan &p = c->plan;
    int f = face;
    if (p.stencil == OD_STENCIL_2D5) {  // the 2D grid's y faces are the internal z faces
        if (face < 0 || face > 3) return fail(OD_EINVAL, "od_face_copy: a 2D face is 0..3");
        f = face < 2 ? face : face + 2;
    } else if (face < 0 || face > 5) {
        return fail(OD_EINVAL, "od_face_copy: face must be 0..5");
    }
    const int64_t n = f < 2 ? p.ny * p.nz : f < 4 ? p.nx * p.nz : p.nx * p.ny;
    DeviceGuard dg(c->device);
    const int par = (int)(c->steps & 1);
    const int nch = (int)p.ch.size();
    if (buf_is_device) {
        OD_CUDA(od::launch_face_copy(c->d_ch, nch, par, f, dir, buf, p.nx, p.ny, p.nz, c->stream));
        return OD_OK;
    }
    if (double *mapped = device_view(buf)) {  // pinned host memory: in place
        OD_CUDA(od::launch_face_copy(c->d_ch, nch, par, f, dir, mapped, p.nx, p.ny, p.nz, c->stream));
        OD_CUDA(cudaStreamSynchronize(c->stream));
        return OD_OK;
    }
    od_status s = ensure_stage(c);
    if (s != OD_OK) return s;
    if (dir == 1)
        OD_CUDA(cudaMemcpyAsync(c->d_stage, buf, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    OD_CUDA(od::launch_face_copy(c->d_ch, nch, par, f, dir, c->d_stage, p.nx, p.ny, p.nz, c->stream));
    if (dir == 0)
        OD_CUDA(cudaMemcpyAsync(buf, c->d_stage, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    OD_CUDA(cudaStreamSynchronize(c->stream));
    return OD_OK;
}

od_status od_stats_get(od_ctx *c, od_stats *out) {
    if (!c || !out) return fail(OD_EINVAL, "null argument");
    DeviceGuard dg(c->device);
    memset(out, 0, sizeof *out);
    od_status s = check_device_error_impl(c);
    out->steps_done = c->steps;
    out->kernel_launches = c->launches;
    out->api_calls = c->api_calls;
    out->graph_launches = c->graph_launches;
    out->path = c->path;
    out->persistent_grid = c->persistent_grid;
    out->tuned = c->tuned ? 1 : 0;
    out->tune_ms_per_step = c->tune_ms;
    od::plan_info(c->plan, &out->plan);
    return s;
}

od_status od_debug_stall_tile(od_ctx *c, int64_t tile) {
    if (!c) return fail(OD_EINVAL, "null context");
    if (tile < -1 || tile >= (int64_t)c->plan.tiles.size()) return fail(OD_EINVAL, "tile out of range");
    c->stall_tile = tile;
    return OD_OK;
}

od_status od_destroy(od_ctx *c) {
    if (!c) return OD_OK;
    {
        DeviceGuard dg(c->device);
        cudaStreamSynchronize(c->stream);
        release(c);
    }
    return OD_OK;
}

}  // extern "C"
