// od_launch.cu -- launch-overhead microbenchmarks of libod (sm_103a).
//
// The paper's measurements of what a kernel launch costs an overdecomposed
// application (Sec. III, "Managing Overdecomposition"): the round trip of one
// kernel fired and waited for; a fixed amount of work split over more and
// more kernels that are all enqueued up front, each behind a wait on one
// host-mapped flag (cuStreamWaitValue32), and released at once; and the
// rate at which host threads driving several chares each can keep firing
// kernels that fill the GPU.  They are the context for the per-chare path's
// slowdown with ODF; the solver itself does not use them.
//
// Every host wait here is bounded (kWaitLimit): the kernels are finite and
// the release flag is always written, so a limit can only be hit by a broken
// device, and then the call returns OD_ETIMEOUT instead of blocking.
#include <cuda.h>  // driver API types for cuStreamWaitValue32 (resolved at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "od.h"

namespace od {
od_status set_last_error(od_status s, const std::string &msg);
}

namespace {

using clk = std::chrono::steady_clock;
constexpr double kWaitLimit = 10.0;  // seconds

od_status fail(od_status s, const std::string &m) { return od::set_last_error(s, m); }
od_status cuda_fail(cudaError_t e, const char *what) {
    return fail(OD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

double seconds_since(clk::time_point t0) { return std::chrono::duration<double>(clk::now() - t0).count(); }

__global__ void k_empty() {}

// The fixed per-thread work of the release benchmark: `work` steps of the
// 32-bit linear congruential generator x <- 1664525 x + 1013904223
// (Numerical Recipes) from x = the thread's global index.
__global__ void k_work(uint32_t *out, int64_t first, int64_t n, int32_t work) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t x = (uint32_t)(first + i);
    for (int32_t t = 0; t < work; ++t) x = 1664525u * x + 1013904223u;
    out[first + i] = x;
}

// Poll an event until it completes or the limit passes.
cudaError_t wait_event(cudaEvent_t e, double limit_s, bool *timed_out) {
    const clk::time_point t0 = clk::now();
    *timed_out = false;
    for (;;) {
        const cudaError_t q = cudaEventQuery(e);
        if (q == cudaSuccess) return cudaSuccess;
        if (q != cudaErrorNotReady) return q;
        if (seconds_since(t0) > limit_s) {
            *timed_out = true;
            return cudaSuccess;
        }
        std::this_thread::yield();
    }
}

typedef CUresult (*WaitValue32Fn)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);

struct HostFlag {
    std::atomic<int> done{0};
};

void CUDART_CB set_host_flag(void *p) { static_cast<HostFlag *>(p)->done.store(1, std::memory_order_release); }

}  // namespace

extern "C" {

OD_API od_status od_bench_launch_latency(int32_t device, int32_t wait, int32_t reps, double *us) {
    if (!us || reps < 1 || reps > 1000000 || wait < 0 || wait > 2)
        return fail(OD_EINVAL, "od_bench_launch_latency: reps in [1, 1e6], wait in {0, 1, 2}, us non-null");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
        cudaStreamDestroy(s);
        return cuda_fail(e, "event");
    }
    od_status st = OD_OK;
    HostFlag flag;
    auto one = [&]() -> bool {
        k_empty<<<1, 32, 0, s>>>();
        if ((e = cudaGetLastError()) != cudaSuccess) return false;
        if (wait == 0) {
            e = cudaStreamSynchronize(s);
            return e == cudaSuccess;
        }
        if (wait == 1) {
            bool to = false;
            if ((e = cudaEventRecord(ev, s)) != cudaSuccess) return false;
            e = wait_event(ev, kWaitLimit, &to);
            if (to) st = OD_ETIMEOUT;
            return e == cudaSuccess && !to;
        }
        flag.done.store(0, std::memory_order_relaxed);
        if ((e = cudaLaunchHostFunc(s, set_host_flag, &flag)) != cudaSuccess) return false;
        const clk::time_point t0 = clk::now();
        while (!flag.done.load(std::memory_order_acquire)) {
            if (seconds_since(t0) > kWaitLimit) {
                st = OD_ETIMEOUT;
                return false;
            }
        }
        return true;
    };
    bool ok = true;
    for (int i = 0; i < 10 && ok; ++i) ok = one();  // warm-up
    const clk::time_point t0 = clk::now();
    for (int i = 0; i < reps && ok; ++i) ok = one();
    const double dt = seconds_since(t0);
    cudaStreamSynchronize(s);  // a timed-out host callback still holds `flag`
    cudaEventDestroy(ev);
    cudaStreamDestroy(s);
    if (!ok) return st != OD_OK ? fail(st, "launch latency: a wait ran out") : cuda_fail(e, "launch latency");
    *us = dt * 1e6 / reps;
    return OD_OK;
}

OD_API od_status od_bench_release(int32_t device, int64_t total_threads, int32_t nkernels, int32_t work,
                                  uint32_t *out, double *us) {
    if (!us || total_threads < 1 || total_threads > (int64_t)1 << 30 || nkernels < 1 || nkernels > 1024 ||
        work < 0 || work > 1000000 || total_threads * (int64_t)work > (int64_t)1 << 40)
        return fail(OD_EINVAL, "od_bench_release: total_threads in [1, 2^30], nkernels in [1, 1024], "
                               "work in [0, 1e6], total_threads*work <= 2^40, us non-null");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuStreamWaitValue32", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(OD_ECUDA, "cuStreamWaitValue32 is not available from the driver");
    WaitValue32Fn wait_value = reinterpret_cast<WaitValue32Fn>(fn);

    uint32_t *own = nullptr;
    if (!out) {
        if ((e = cudaMalloc(&own, (size_t)total_threads * sizeof(uint32_t))) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc");
        out = own;
    }
    volatile uint32_t *h_flag = nullptr;
    uint32_t *d_flag = nullptr;
    std::vector<cudaStream_t> st((size_t)nkernels, nullptr);
    std::vector<cudaEvent_t> done((size_t)nkernels, nullptr);
    cudaEvent_t start = nullptr;
    od_status status = OD_OK;
    std::string what;
    bool released = false;
    auto bail = [&](cudaError_t err, const char *w) {
        if (status == OD_OK) {
            status = OD_ECUDA;
            what = std::string(w) + ": " + cudaGetErrorString(err);
        }
    };

    if ((e = cudaHostAlloc((void **)&h_flag, sizeof(uint32_t), cudaHostAllocMapped)) != cudaSuccess) {
        bail(e, "cudaHostAlloc");
    } else {
        *h_flag = 0;
        if ((e = cudaHostGetDevicePointer((void **)&d_flag, (void *)h_flag, 0)) != cudaSuccess)
            bail(e, "cudaHostGetDevicePointer");
    }
    if (status == OD_OK && (e = cudaEventCreate(&start)) != cudaSuccess) bail(e, "event");
    for (int k = 0; k < nkernels && status == OD_OK; ++k) {
        if ((e = cudaStreamCreateWithFlags(&st[k], cudaStreamNonBlocking)) != cudaSuccess) bail(e, "stream");
        else if ((e = cudaEventCreate(&done[k])) != cudaSuccess) bail(e, "event");
    }
    // enqueue: every stream waits on the flag, then runs its share
    for (int k = 0; k < nkernels && status == OD_OK; ++k) {
        if (wait_value((CUstream)st[k], (CUdeviceptr)d_flag, 1u, CU_STREAM_WAIT_VALUE_GEQ) != CUDA_SUCCESS) {
            status = OD_ECUDA;
            what = "cuStreamWaitValue32 failed";
            break;
        }
        if (k == 0 && (e = cudaEventRecord(start, st[0])) != cudaSuccess) {
            bail(e, "cudaEventRecord");
            break;
        }
        const int64_t first = total_threads * k / nkernels, n = total_threads * (k + 1) / nkernels - first;
        if (n > 0) k_work<<<(unsigned)((n + 255) / 256), 256, 0, st[k]>>>(out, first, n, work);
        if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventRecord(done[k], st[k])) != cudaSuccess) {
            bail(e, "enqueue");
            break;
        }
    }
    // release (always, so no stream is left waiting), then wait, bounded
    if (h_flag) {
        *h_flag = 1;
        released = true;
    }
    double worst = 0;
    for (int k = 0; k < nkernels && released; ++k) {
        if (!st[k]) continue;
        bool to = false;
        e = cudaStreamQuery(st[k]);
        const clk::time_point t0 = clk::now();
        while (e == cudaErrorNotReady && seconds_since(t0) < kWaitLimit) {
            std::this_thread::yield();
            e = cudaStreamQuery(st[k]);
        }
        if (e == cudaErrorNotReady) to = true;
        if (to) {
            if (status == OD_OK) {
                status = OD_ETIMEOUT;
                what = "release benchmark: a stream did not finish";
            }
        } else if (e != cudaSuccess) {
            bail(e, "stream");
        } else if (status == OD_OK) {
            float ms = 0;
            if ((e = cudaEventElapsedTime(&ms, start, done[k])) != cudaSuccess) bail(e, "elapsed");
            else if (ms > worst) worst = ms;
        }
    }
    if (status != OD_ETIMEOUT) {
        for (auto &x : done)
            if (x) cudaEventDestroy(x);
        for (auto &x : st)
            if (x) cudaStreamDestroy(x);
        if (start) cudaEventDestroy(start);
        if (own) cudaFree(own);
        if (h_flag) cudaFreeHost((void *)h_flag);
    }  // after a time-out the GPU may still use them: leak rather than free under it
    if (status != OD_OK) return fail(status, what);
    *us = worst * 1e3;
    return OD_OK;
}

OD_API od_status od_bench_launch_rate(int32_t device, int32_t host_threads, int32_t chares, int32_t kernels,
                                      double *per_s) {
    if (!per_s || host_threads < 1 || host_threads > 64 || chares < 1 || chares > 64 || kernels < 1 ||
        (int64_t)host_threads * chares * kernels > 10000000)
        return fail(OD_EINVAL, "od_bench_launch_rate: host_threads and chares in [1, 64], kernels >= 1, "
                               "at most 1e7 kernels in all, per_s non-null");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceGetAttribute");
    std::atomic<int> bad{0};
    std::atomic<int> timed_out{0};
    // each host thread is a scheduler over its chares: it fires a chare's next
    // kernel as soon as it sees (by polling) that the previous one completed
    auto worker = [&](std::vector<cudaStream_t> *ss, std::vector<cudaEvent_t> *es) {
        if (cudaSetDevice(device) != cudaSuccess) {
            bad = 1;
            return;
        }
        std::vector<int> fired((size_t)chares, 0), busy((size_t)chares, 0);
        int left = chares;
        const clk::time_point t0 = clk::now();
        while (left > 0 && !bad) {
            for (int c = 0; c < chares; ++c) {
                if (busy[c]) {
                    const cudaError_t q = cudaEventQuery((*es)[c]);
                    if (q == cudaErrorNotReady) continue;
                    if (q != cudaSuccess) {
                        bad = 1;
                        break;
                    }
                    busy[c] = 0;
                    if (fired[c] == kernels) --left;
                }
                if (!busy[c] && fired[c] < kernels) {
                    k_empty<<<sms, 32, 0, (*ss)[c]>>>();
                    if (cudaGetLastError() != cudaSuccess || cudaEventRecord((*es)[c], (*ss)[c]) != cudaSuccess) {
                        bad = 1;
                        break;
                    }
                    ++fired[c];
                    busy[c] = 1;
                }
            }
            if (seconds_since(t0) > 6 * kWaitLimit) {
                timed_out = 1;
                break;
            }
        }
    };
    std::vector<std::vector<cudaStream_t>> ss((size_t)host_threads, std::vector<cudaStream_t>((size_t)chares));
    std::vector<std::vector<cudaEvent_t>> es((size_t)host_threads, std::vector<cudaEvent_t>((size_t)chares));
    od_status status = OD_OK;
    for (auto &v : ss)
        for (auto &x : v)
            if (status == OD_OK && cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess)
                status = OD_ECUDA;
    for (auto &v : es)
        for (auto &x : v)
            if (status == OD_OK && cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess)
                status = OD_ECUDA;
    double dt = 0;
    if (status == OD_OK) {
        k_empty<<<sms, 32, 0, ss[0][0]>>>();  // warm-up
        cudaStreamSynchronize(ss[0][0]);
        std::vector<std::thread> th;
        const clk::time_point t0 = clk::now();
        for (int t = 0; t < host_threads; ++t) th.emplace_back(worker, &ss[t], &es[t]);
        for (auto &x : th) x.join();
        dt = seconds_since(t0);
    }
    for (auto &v : ss)
        for (auto &x : v)
            if (x) {
                cudaStreamSynchronize(x);
                cudaStreamDestroy(x);
            }
    for (auto &v : es)
        for (auto &x : v)
            if (x) cudaEventDestroy(x);
    if (status != OD_OK || bad) return fail(OD_ECUDA, "launch rate: a CUDA call failed");
    if (timed_out) return fail(OD_ETIMEOUT, "launch rate: the kernels did not complete in time");
    *per_s = (double)host_threads * chares * kernels / dt;
    return OD_OK;
}

}  // extern "C"
