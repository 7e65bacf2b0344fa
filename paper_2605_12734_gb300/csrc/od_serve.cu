// od_serve.cu -- serving loop: independent overdecomposed solves submitted as
// they arrive, admitted under an HBM budget, kept resident on the device and
// advanced together (continuous batching).
//
// One worker thread owns the device side.  Each pass it
//   1. admits queued jobs in arrival order while a slot is free and the
//      budget pool (one device allocation, first-fit) has room for the job's
//      arena -- a job larger than the whole budget is refused at submit;
//   2. launches batch_steps fused steps of every running job in one
//      persistent launch per CTA shape (k_persistent_multi: CTAs take (step,
//      job, tile) tickets and wait, bounded, on the per-tile step counters of
//      the tiles they read, each job at its own step and parity), or, with
//      batch_steps = 1, one fused step (k_tiles_multi: each block one tile of
//      one job); jobs that arrive while others run join the very next launch
//      and a finished job simply drops out of the next one;
//   3. watches the events of launches in flight (at most two ahead) and marks
//      a job done when the launch holding its last step has completed.
// With job_streams = N > 0 the worker instead launches each admitted job's
// whole run as its own persistent kernel (k_persistent, the job's arguments
// in the kernel's parameters) on one of N streams, and the hardware runs the
// jobs' kernels side by side: a job's CTAs start as others' leave, so a small
// job fills the SMs a large one leaves idle.  A job is done when the event
// after its kernel has completed.
// A job's result stays on the device until the client fetches and releases
// it.  Jobs never share memory, so each result is bit-identical to the same
// job solved alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "od.h"
#include "od_ctx.h"
#include "od_internal.h"
#include "od_kernels.h"
#include "od_plan.h"

namespace {

using Clock = std::chrono::steady_clock;

od_status fail(od_status s, const std::string &m) { return od::set_last_error(s, m); }

// First-fit allocator over one device allocation (offsets, 256-byte units).
class Pool {
public:
    void reset(size_t size) {
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

private:
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

struct Job {
    uint64_t id = 0;
    od_config cfg{};
    std::vector<int32_t> cuts[3];
    int32_t iters = 0;
    int64_t steps_enq = 0;      // steps enqueued on the device
    int state = OD_JOB_QUEUED;
    bool admitting = false;     // out of the queue, its context being created (lock released)
    double t_submit = 0, t_admit = 0, t_done = 0;
    size_t off = 0, bytes = 0;
    od_ctx *ctx = nullptr;
    int64_t done_batch = -1;    // launch index holding the job's last step
    int64_t cells = 0;
    int32_t threads = 0, cpt = 0;  // the job's CTA shape (from its plan)
    std::string err;
    // stream mode: the job's stream, the events around its kernel once it is
    // launched and the pinned slot its error record is copied into after it
    int stream = -1, err_slot = -1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

struct Batch {
    int64_t index;
    cudaEvent_t ev0, ev;  // before the kernel, after it (timed: the device's busy time)
};

}  // namespace

struct od_server {
    od_server_config cfg{};
    int device = 0;
    char *pool_base = nullptr;
    bool own_pool = false;
    Pool pool;
    cudaStream_t compute = nullptr, admit = nullptr;
    KArgs *d_jobs[2] = {nullptr, nullptr};
    int32_t *d_first[2] = {nullptr, nullptr};
    int32_t max_jobs = 0;
    int threads = 128, cpt = 4, stages = 4, arith = 2, smem_cap = 0;
    int batch_steps = 8, num_sms = 0;
    int32_t *d_queue = nullptr;  // ticket counters: [in-flight slot][shape group]
    // stream mode (job_streams > 0): one persistent launch per job
    std::vector<cudaStream_t> job_streams;
    std::vector<int> stream_jobs;   // unfinished jobs assigned to each stream
    ErrDev *h_err = nullptr;        // pinned error records, one slot per launched job
    std::vector<int> free_err;      // free slots of h_err
    cudaEvent_t base_ev = nullptr;  // device time origin of the jobs' kernels
    std::vector<std::pair<double, double>> kernel_spans;  // [start, end] seconds after base_ev
    std::vector<Job *> launched;    // running jobs whose kernel is in flight
    std::deque<uint64_t> completions;  // jobs that ended (done or failed), in the order they ended
    std::vector<cudaEvent_t> free_events;
    std::deque<Batch> inflight;
    int64_t next_batch = 0;
    std::thread worker, admitter;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_admit;
    std::deque<Job *> queue;
    std::vector<Job *> running;
    std::unordered_map<uint64_t, Job *> jobs;
    uint64_t next_id = 1;
    bool stop = false;
    Clock::time_point t0;
    // statistics
    int64_t launches = 0, done = 0, failed = 0;
    double updates_done = 0;
    double admit_seconds = 0;  // spent creating job contexts (admission thread)
    double busy_seconds = 0;   // device time of the retired batched launches
    std::string worker_error;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// CTA shapes the planner picks from; with per-job shapes a step runs at most
// one batched launch for each.
constexpr int kShapes = 4;

// A job ended (done or failed): queue it for od_server_next_completion (lock held).
void completed(od_server *s, Job *j) { s->completions.push_back(j->id); }
constexpr int kErrSlots = 1024;  // stream mode: jobs whose kernels are in flight at once
constexpr int32_t kAutoShapes[kShapes][2] = {{128, 4}, {128, 2}, {256, 4}, {256, 8}};

od_config job_config(od_server *s, Job *j) {
    od_config c = j->cfg;
    for (int a = 0; a < 3; ++a) {
        const int32_t *p = j->cuts[a].empty() ? nullptr : j->cuts[a].data();
        if (a == 0) c.cuts_x = p;
        if (a == 1) c.cuts_y = p;
        if (a == 2) c.cuts_z = p;
    }
    c.path = s->job_streams.empty() ? OD_PATH_FUSED : OD_PATH_PERSISTENT;
    c.autotune = 0;
    c.threads = s->threads ? s->threads : j->threads;
    c.cells_per_thread = s->threads ? s->cpt : j->cpt;
    c.stages = s->stages;
    c.arith = s->arith;
    c.stream_pool = 1;
    c.device = s->device;
    // stream mode: the job's own stream, so its initialisation and its run
    // queue behind no other job's kernel
    c.stream = j->stream >= 0 ? s->job_streams[(size_t)j->stream] : s->admit;
    return c;
}

// Admit queued jobs (called with the lock held; drops it around od_create).
// Returns whether any job left the queue.
bool admit(od_server *s, std::unique_lock<std::mutex> &lk) {
    bool progress = false;
    while (!s->queue.empty() && (s->cfg.max_active <= 0 || (int)s->running.size() < s->cfg.max_active) &&
           (int)s->running.size() < s->max_jobs) {
        Job *j = s->queue.front();
        size_t off = 0;
        if (!s->pool.alloc(j->bytes, &off)) return progress;  // wait for memory
        s->queue.pop_front();
        j->admitting = true;
        j->off = off;
        if (!s->job_streams.empty()) {  // stream mode: the stream with the fewest unfinished jobs
            j->stream = (int)(std::min_element(s->stream_jobs.begin(), s->stream_jobs.end()) - s->stream_jobs.begin());
            s->stream_jobs[(size_t)j->stream]++;
        }
        od_config c = job_config(s, j);
        c.arena = s->pool_base + off;
        c.arena_bytes = j->bytes;
        lk.unlock();
        const double t_create = s->now();
        od_ctx *ctx = nullptr;
        // stream mode: queue the job's initialisation on its stream and
        // return (its kernel follows on the same stream); batched mode: wait,
        // the batched launches run on another stream
        od_status st = od::create_context(&ctx, &c, s->job_streams.empty());
        std::string msg = st == OD_OK ? "" : od_last_error();
        lk.lock();
        j->admitting = false;
        s->admit_seconds += s->now() - t_create;
        progress = true;
        bool known_shape = false;  // one of the shapes a step launches for (at most kShapes groups)
        for (int g = 0; st == OD_OK && g < kShapes; ++g)
            known_shape |= s->threads ? (ctx->plan.threads == s->threads && ctx->plan.cpt == s->cpt)
                                      : (ctx->plan.threads == kAutoShapes[g][0] && ctx->plan.cpt == kAutoShapes[g][1]);
        // (per-job launches use each job's own plan: shape and shared memory are its own)
        const bool batched = s->job_streams.empty();
        if (st != OD_OK || (batched && (!known_shape || ctx->plan.stage_doubles * s->stages * 8 + 256 > s->smem_cap))) {
            if (j->stream >= 0) s->stream_jobs[(size_t)j->stream]--;
            // work queued by the creation (stream mode) may still write the arena
            if (!s->job_streams.empty()) cudaStreamSynchronize((cudaStream_t)c.stream);
            if (ctx) od_destroy(ctx);
            s->pool.release(j->off, j->bytes);
            j->state = OD_JOB_FAILED;
            completed(s, j);
            j->err = st != OD_OK ? msg
                     : !known_shape ? "the planner chose a CTA shape the server does not launch"
                                    : "tile needs more shared memory than the server's launch shape";
            s->failed++;
            s->cv_done.notify_all();
            continue;
        }
        j->ctx = ctx;
        j->t_admit = s->now();
        if (j->iters == 0) {  // nothing to run: done at admission
            if (j->stream >= 0) s->stream_jobs[(size_t)j->stream]--;
            j->state = OD_JOB_DONE;
            j->t_done = j->t_admit;
            completed(s, j);
            s->done++;
            s->cv_done.notify_all();
            continue;
        }
        j->state = OD_JOB_RUNNING;
        s->running.push_back(j);
        s->cv_work.notify_all();
    }
    return progress;
}

// Retire launches that completed (lock held).
void retire(od_server *s) {
    while (!s->inflight.empty() && cudaEventQuery(s->inflight.front().ev) == cudaSuccess) {
        const Batch b = s->inflight.front();
        s->inflight.pop_front();
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b.ev0, b.ev) == cudaSuccess) s->busy_seconds += ms * 1e-3;
        s->free_events.push_back(b.ev0);
        s->free_events.push_back(b.ev);
        const double t = s->now();
        for (auto &kv : s->jobs) {
            Job *j = kv.second;
            if (j->state == OD_JOB_RUNNING && j->done_batch == b.index) {
                j->state = OD_JOB_DONE;
                j->t_done = t;
                completed(s, j);
                j->ctx->steps = j->iters;
                s->done++;
                s->updates_done += (double)j->cells * j->iters;
            }
        }
        s->cv_done.notify_all();
    }
    cudaGetLastError();  // cudaErrorNotReady is not an error here
}

cudaEvent_t take_event(od_server *s) {
    cudaEvent_t ev;
    if (s->free_events.empty()) {
        cudaEventCreate(&ev);
    } else {
        ev = s->free_events.back();
        s->free_events.pop_back();
    }
    return ev;
}

// One fused step of every running job that still has steps (lock held):
// one batched launch per CTA shape among them (one shape unless the server
// lets the planner pick a shape per job).  The jobs of shape group g occupy
// hk[jo[g] .. jo[g+1]) and their first-block prefix hf[jo[g] + g ..].
bool launch_batch(od_server *s, std::vector<KArgs> &hk, std::vector<int32_t> &hf) {
    hk.clear();
    hf.clear();
    std::vector<Job *> in;
    int32_t shapes[kShapes][2];
    int ngroups = 0;
    std::vector<int32_t> jo, grid, max_sd;
    for (int g = 0; g < kShapes; ++g) {
        int32_t nt = 0, ct = 0, tiles = 0, sd = 0;
        const size_t first = in.size();
        for (Job *j : s->running) {
            if (j->done_batch >= 0 || j->steps_enq >= j->iters) continue;
            const od::Plan &p = j->ctx->plan;
            bool seen = false;  // shape already taken by an earlier group
            for (int h = 0; h < ngroups; ++h) seen |= shapes[h][0] == p.threads && shapes[h][1] == p.cpt;
            if (seen) continue;
            if (in.size() == first) {
                nt = p.threads;
                ct = p.cpt;
            } else if (p.threads != nt || p.cpt != ct) {
                continue;
            }
            KArgs a = od::base_args(j->ctx);
            a.tile_begin = 0;
            a.parity = (int32_t)(j->steps_enq & 1);
            a.stages = s->stages;
            a.t0 = (int32_t)j->steps_enq;  // persistent batches: absolute first step, steps in the batch
            a.iters = (int32_t)std::min<int64_t>(s->batch_steps, j->iters - j->steps_enq);
            if (in.size() == first) jo.push_back((int32_t)first);
            hk.push_back(a);
            hf.push_back(tiles);
            tiles += (int32_t)p.tiles.size();
            sd = std::max(sd, p.stage_doubles);
            in.push_back(j);
        }
        if (in.size() == first) break;
        hf.push_back(tiles);
        shapes[ngroups][0] = nt;
        shapes[ngroups][1] = ct;
        grid.push_back(tiles);
        max_sd.push_back(sd);
        ++ngroups;
    }
    if (in.empty()) return false;
    jo.push_back((int32_t)in.size());
    const int slot = (int)(s->next_batch & 1);
    cudaMemcpyAsync(s->d_jobs[slot], hk.data(), hk.size() * sizeof(KArgs), cudaMemcpyHostToDevice, s->compute);
    cudaMemcpyAsync(s->d_first[slot], hf.data(), hf.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s->compute);
    cudaEvent_t ev0 = take_event(s);
    cudaEventRecord(ev0, s->compute);
    int32_t steps = 1;  // steps of the batch: the most any of its jobs runs
    for (const KArgs &a : hk) steps = std::max(steps, a.iters);
    for (int g = 0; g < ngroups; ++g) {
        const int smem = 256 + s->stages * max_sd[(size_t)g] * 8;
        const KArgs *dj = s->d_jobs[slot] + jo[(size_t)g];
        const int32_t *df = s->d_first[slot] + jo[(size_t)g] + g;
        const int32_t nj = jo[(size_t)g + 1] - jo[(size_t)g];
        KArgs geom;  // the launch's ring geometry: every job's slots fit the largest
        memset(&geom, 0, sizeof geom);
        geom.stages = s->stages;
        geom.stage_doubles = max_sd[(size_t)g];
        geom.spin_ns = hk[(size_t)jo[(size_t)g]].spin_ns;
        geom.one = 1;  // the arithmetic's opaque constant
        cudaError_t e;
        if (s->batch_steps > 1) {
            int bps = 0;
            e = od::persistent_multi_occupancy(shapes[g][0], shapes[g][1], s->arith, smem, OD_STENCIL_3D7, &bps);
            int32_t *q = s->d_queue + slot * kShapes + g;
            if (e == cudaSuccess && bps < 1) e = cudaErrorInvalidConfiguration;
            if (e == cudaSuccess) e = cudaMemsetAsync(q, 0, sizeof(int32_t), s->compute);
            if (e == cudaSuccess)
                e = od::launch_persistent_multi(dj, df, nj, steps, q, geom,
                                                std::min(grid[(size_t)g], bps * s->num_sms), shapes[g][0],
                                                shapes[g][1], s->arith, smem, OD_STENCIL_3D7, s->compute);
        } else {
            e = od::launch_tiles_multi(dj, df, nj, geom, grid[(size_t)g], shapes[g][0], shapes[g][1], s->arith, smem,
                                       OD_STENCIL_3D7, s->compute);
        }
        if (e != cudaSuccess) {
            s->free_events.push_back(ev0);
            s->worker_error = std::string("batched launch: ") + cudaGetErrorString(e);
            return false;
        }
        s->launches++;
    }
    const int64_t idx = s->next_batch++;
    for (size_t k = 0; k < in.size(); ++k) {
        Job *j = in[k];
        j->steps_enq += s->batch_steps > 1 ? hk[k].iters : 1;
        if (j->steps_enq == j->iters) j->done_batch = idx;
    }
    cudaEvent_t ev = take_event(s);
    cudaEventRecord(ev, s->compute);
    s->inflight.push_back({idx, ev0, ev});
    return true;
}

// Stream mode (lock held): launch every running job that has no kernel yet,
// its whole run as one persistent kernel on its own stream, between two
// events.  Returns whether anything was launched.
bool launch_jobs(od_server *s) {
    bool any = false;
    for (Job *j : s->running) {
        if (j->ev1) continue;
        if (s->free_err.empty()) break;  // every error slot is in flight: launch later
        j->err_slot = s->free_err.back();
        s->free_err.pop_back();
        j->ev0 = take_event(s);
        j->ev1 = take_event(s);
        cudaEventRecord(j->ev0, j->ctx->stream);
        od_status st = od_step(j->ctx, j->iters);
        // the job's error record follows its kernel into pinned memory, so
        // completion is read without a synchronising call
        if (st == OD_OK && cudaMemcpyAsync(s->h_err + j->err_slot, j->ctx->d_err, sizeof(ErrDev),
                                           cudaMemcpyDeviceToHost, j->ctx->stream) != cudaSuccess)
            st = od::set_last_error(OD_ECUDA, "error record copy");
        if (st != OD_OK) s->h_err[j->err_slot].code = -1;  // no copy queued: retired as failed
        cudaEventRecord(j->ev1, j->ctx->stream);
        s->launched.push_back(j);  // retired (done or failed) once ev1 has completed
        if (st != OD_OK) {
            s->worker_error = std::string("job launch: ") + od_last_error();
            return any;
        }
        s->launches++;
        any = true;
    }
    return any;
}

// Stream mode (lock held): mark done every job whose kernel has completed,
// keeping its kernel's device interval for the busy time.
void retire_jobs(od_server *s) {
    bool any = false;
    const double t = s->now();
    for (size_t k = 0; k < s->launched.size();) {
        Job *j = s->launched[k];
        const cudaError_t q = cudaEventQuery(j->ev1);
        if (q == cudaErrorNotReady) {
            ++k;
            continue;
        }
        float a = 0.f, b = 0.f;
        if (q == cudaSuccess && cudaEventElapsedTime(&a, s->base_ev, j->ev0) == cudaSuccess &&
            cudaEventElapsedTime(&b, s->base_ev, j->ev1) == cudaSuccess)
            s->kernel_spans.emplace_back(a * 1e-3, b * 1e-3);
        s->free_events.push_back(j->ev0);
        s->free_events.push_back(j->ev1);
        j->ev0 = j->ev1 = nullptr;
        s->launched[k] = s->launched.back();
        s->launched.pop_back();
        const int32_t code = q == cudaSuccess ? s->h_err[j->err_slot].code : -1;
        s->free_err.push_back(j->err_slot);
        j->err_slot = -1;
        s->stream_jobs[(size_t)j->stream]--;
        if (code == 0) {
            j->state = OD_JOB_DONE;
            j->t_done = t;
            s->done++;
            s->updates_done += (double)j->cells * j->iters;
        } else {
            j->state = OD_JOB_FAILED;
            j->err = q != cudaSuccess ? cudaGetErrorString(q) : "the job's kernel reported an error (timeout)";
            s->failed++;
        }
        completed(s, j);
        any = true;
    }
    if (any) s->cv_done.notify_all();
}

// Stream mode: the device's busy time, the union of the jobs' kernel
// intervals (lock held).
double busy_union(od_server *s) {
    std::vector<std::pair<double, double>> v = s->kernel_spans;
    std::sort(v.begin(), v.end());
    double sum = 0, a = 0, b = -1;
    for (const auto &iv : v) {
        if (iv.first > b) {
            if (b > a) sum += b - a;
            a = iv.first;
            b = iv.second;
        } else {
            b = std::max(b, iv.second);
        }
    }
    if (b > a) sum += b - a;
    return sum;
}

// Admission thread: creates the contexts of queued jobs (tables, initial
// field) while the worker keeps the GPU busy with the running ones.
void admitter_main(od_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        if (admit(s, lk)) continue;
        s->cv_admit.wait_for(lk, std::chrono::milliseconds(2));
    }
}

void worker_main(od_server *s) {
    cudaSetDevice(s->device);
    std::vector<KArgs> hk;
    std::vector<int32_t> hf;
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        if (!s->job_streams.empty()) {  // stream mode: poll the jobs' kernels
            retire_jobs(s);
            const size_t before = s->running.size();
            s->running.erase(std::remove_if(s->running.begin(), s->running.end(),
                                            [](Job *j) { return j->state != OD_JOB_RUNNING; }),
                             s->running.end());
            if (s->running.size() != before) s->cv_admit.notify_all();
            if (s->worker_error.empty() && launch_jobs(s)) continue;
            // a short wait: a kernel's completion is only seen by polling
            s->cv_work.wait_for(lk, std::chrono::microseconds(s->launched.empty() ? 2000 : 100));
            continue;
        }
        retire(s);
        // drop finished jobs from the running set (their memory stays until release)
        const size_t before = s->running.size();
        s->running.erase(std::remove_if(s->running.begin(), s->running.end(),
                                        [](Job *j) { return j->state != OD_JOB_RUNNING; }),
                         s->running.end());
        if (s->running.size() != before) s->cv_admit.notify_all();  // an active slot is free
        bool launched = false;
        if (s->inflight.size() < 2 && s->worker_error.empty()) launched = launch_batch(s, hk, hf);
        if (launched) continue;
        if (!s->inflight.empty()) {
            // wait for the oldest launch outside the lock
            cudaEvent_t ev = s->inflight.front().ev;
            lk.unlock();
            cudaEventSynchronize(ev);
            lk.lock();
            continue;
        }
        s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
    }
}

Job *find(od_server *s, uint64_t id) {
    auto it = s->jobs.find(id);
    return it == s->jobs.end() ? nullptr : it->second;
}

}  // namespace

extern "C" {

void od_server_config_default(od_server_config *c) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->hbm_budget_bytes = 1ull << 30;
    c->max_active = 0;
    c->max_jobs_per_launch = 256;
    c->arith = -1;
    c->job_streams = 16;
}

od_status od_server_create(od_server **out, const od_server_config *cfg) {
    if (!out || !cfg) return fail(OD_EINVAL, "null argument");
    *out = nullptr;
    if (cfg->hbm_budget_bytes < (1u << 20)) return fail(OD_EINVAL, "budget below 1 MiB");
    od_server *s = new od_server();
    s->cfg = *cfg;
    s->device = cfg->device;
    // both 0: per-job shapes chosen by the planner; one given: the other defaults
    const bool auto_shape = cfg->threads == 0 && cfg->cells_per_thread == 0;
    s->threads = auto_shape ? 0 : cfg->threads ? cfg->threads : 128;
    s->cpt = auto_shape ? 0 : cfg->cells_per_thread ? cfg->cells_per_thread : 4;
    s->stages = cfg->stages ? cfg->stages : 4;
    s->arith = cfg->arith >= 0 ? cfg->arith : 12;
    s->max_jobs = cfg->max_jobs_per_launch > 0 ? cfg->max_jobs_per_launch : 256;
    s->batch_steps = cfg->batch_steps > 0 ? cfg->batch_steps : 8;
    if (cfg->batch_steps < 0 || cfg->batch_steps > 4096) {
        delete s;
        return fail(OD_EINVAL, "batch_steps must be in [0, 4096]");
    }
    if (cfg->job_streams < 0 || cfg->job_streams > 64) {
        delete s;
        return fail(OD_EINVAL, "job_streams must be in [0, 64]");
    }
    s->t0 = Clock::now();
    auto bail = [&](od_status st, const std::string &m) {
        od_server_destroy(s);
        return fail(st, m);
    };
    if (cudaSetDevice(s->device) != cudaSuccess) return bail(OD_ECUDA, "cannot select the CUDA device");
    for (int g = 0; g < kShapes; ++g) {
        const int nt = s->threads ? s->threads : kAutoShapes[g][0], ct = s->threads ? s->cpt : kAutoShapes[g][1];
        if (!od::tile_shape_supported(nt, ct, s->arith, OD_STENCIL_3D7)) return bail(OD_EINVAL, "unsupported tile shape");
        if (s->threads) break;  // one fixed shape
    }
    if (cfg->pool) {
        if ((uintptr_t)cfg->pool & 255u) return bail(OD_EINVAL, "pool must be 256-byte aligned");
        s->pool_base = (char *)cfg->pool;
    } else {
        if (cudaMalloc(&s->pool_base, cfg->hbm_budget_bytes) != cudaSuccess) {
            cudaGetLastError();
            s->pool_base = nullptr;
            return bail(OD_ENOMEM, "cannot allocate the HBM budget pool");
        }
        s->own_pool = true;
    }
    s->pool.reset(cfg->hbm_budget_bytes);
    if (cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->admit, cudaStreamNonBlocking) != cudaSuccess)
        return bail(OD_ECUDA, "cannot create streams");
    for (int k = 0; k < cfg->job_streams; ++k) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return bail(OD_ECUDA, "cannot create the job streams");
        s->job_streams.push_back(st);
        s->stream_jobs.push_back(0);
    }
    if (!s->job_streams.empty()) {
        if (cudaHostAlloc(&s->h_err, kErrSlots * sizeof(ErrDev), cudaHostAllocDefault) != cudaSuccess) {
            s->h_err = nullptr;
            return bail(OD_ENOMEM, "cannot allocate the pinned error records");
        }
        for (int k = kErrSlots - 1; k >= 0; --k) s->free_err.push_back(k);
        if (cudaEventCreate(&s->base_ev) != cudaSuccess || cudaEventRecord(s->base_ev, s->compute) != cudaSuccess ||
            cudaEventSynchronize(s->base_ev) != cudaSuccess)
            return bail(OD_ECUDA, "cannot record the time origin");
    }
    for (int k = 0; k < 2; ++k)
        if (cudaMalloc(&s->d_jobs[k], (size_t)s->max_jobs * sizeof(KArgs)) != cudaSuccess ||
            cudaMalloc(&s->d_first[k], (size_t)(s->max_jobs + kShapes) * sizeof(int32_t)) != cudaSuccess)
            return bail(OD_ENOMEM, "cannot allocate launch tables");
    if (cudaMalloc(&s->d_queue, 2 * kShapes * sizeof(int32_t)) != cudaSuccess)
        return bail(OD_ENOMEM, "cannot allocate ticket counters");
    if (cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
        return bail(OD_ECUDA, "cannot query the SM count");
    s->smem_cap = 200 * 1024;
    for (int g = 0; g < kShapes; ++g) {
        if (s->threads && g > 0) break;  // one fixed shape
        const int nt = s->threads ? s->threads : kAutoShapes[g][0], ct = s->threads ? s->cpt : kAutoShapes[g][1];
        if (od::prepare_tile_kernels(nt, ct, s->arith, s->smem_cap, OD_STENCIL_3D7) != cudaSuccess)
            return bail(OD_ECUDA, "cannot configure the tile kernels");
    }
    s->worker = std::thread(worker_main, s);
    s->admitter = std::thread(admitter_main, s);
    *out = s;
    return OD_OK;
}

od_status od_server_submit(od_server *s, const od_config *job, int32_t iters, uint64_t *job_id) {
    if (!s || !job || !job_id || iters < 0) return fail(OD_EINVAL, "bad arguments");
    // one batched launch shares one kernel, the 3D 7-point one
    // a batched launch shares one kernel, the 3D 7-point one; per-job launches
    // run each job's own kernel, so they also take the 2D 5-point stencil
    if (job->stencil != OD_STENCIL_3D7 && (s->job_streams.empty() || job->stencil != OD_STENCIL_2D5))
        return fail(OD_EINVAL, "batched serving runs 3D 7-point jobs only (job_streams > 0 also runs 2D 5-point)");
    Job *j = new Job();
    j->cfg = *job;
    const int32_t *cp[3] = {job->cuts_x, job->cuts_y, job->cuts_z};
    const int32_t nc[3] = {job->ncuts_x, job->ncuts_y, job->ncuts_z};
    for (int a = 0; a < 3; ++a)
        if (cp[a] && nc[a] > 0) j->cuts[a].assign(cp[a], cp[a] + nc[a] + 1);
    j->iters = iters;
    od::Plan plan;
    std::string err;
    od_config c = job_config(s, j);
    // per-job shapes: chosen by the lanes the job's tiles use -- the batch
    // fills the GPU, so a small job's own tile count does not count against
    // a shape (measured with 24 jobs of 160^3 in 27 chares batched: 128 x 4
    // 127, 128 x 2 110 G updates/s)
    od_status st = od::build_plan(&c, &plan, &err, false);
    if (st != OD_OK) {
        delete j;
        return fail(st, err);
    }
    j->threads = plan.threads;
    j->cpt = plan.cpt;
    j->bytes = plan.arena_bytes;
    j->cells = plan.cells;
    if (j->bytes > s->pool.size()) {
        delete j;
        return fail(OD_EBUDGET, "job needs more device memory than the whole budget");
    }
    std::lock_guard<std::mutex> lk(s->mu);
    j->id = s->next_id++;
    j->t_submit = s->now();
    s->jobs[j->id] = j;
    s->queue.push_back(j);
    *job_id = j->id;
    s->cv_admit.notify_all();
    return OD_OK;
}

od_status od_server_wait(od_server *s, uint64_t id, double timeout_s, int32_t *state) {
    if (!s) return fail(OD_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = Clock::now() + std::chrono::duration<double>(timeout_s < 0 ? 0 : timeout_s);
    for (;;) {
        Job *j = find(s, id);  // looked up again after every wake: another thread may release it
        if (!j) return fail(OD_ENOTFOUND, "unknown job");
        if ((j->state != OD_JOB_QUEUED && j->state != OD_JOB_RUNNING) ||
            s->cv_done.wait_until(lk, until) == std::cv_status::timeout) {
            j = find(s, id);
            if (!j) return fail(OD_ENOTFOUND, "unknown job");
            if (state) *state = j->state;
            return OD_OK;
        }
    }
}

od_status od_server_next_completion(od_server *s, double timeout_s, uint64_t *job_id) {
    if (!s || !job_id) return fail(OD_EINVAL, "null argument");
    *job_id = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = Clock::now() + std::chrono::duration<double>(timeout_s < 0 ? 0 : timeout_s);
    while (s->completions.empty())
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout) break;
    if (!s->completions.empty()) {
        *job_id = s->completions.front();
        s->completions.pop_front();
    }
    return OD_OK;
}

od_status od_submit(od_server *s, const od_config *job, int32_t iters, uint64_t *job_id) {
    return od_server_submit(s, job, iters, job_id);
}

od_status od_poll(od_server *s, uint64_t id, int32_t *done) {
    if (!s || !done) return fail(OD_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    Job *j = find(s, id);
    if (!j) return fail(OD_ENOTFOUND, "unknown job");
    *done = j->state == OD_JOB_DONE || j->state == OD_JOB_FAILED;
    return OD_OK;
}

od_status od_fetch(od_server *s, uint64_t id, double *dst, int32_t dst_is_device) {
    return od_server_fetch(s, id, dst, dst_is_device);
}

od_status od_server_job_info(od_server *s, uint64_t id, od_job_info *out) {
    if (!s || !out) return fail(OD_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    Job *j = find(s, id);
    if (!j) return fail(OD_ENOTFOUND, "unknown job");
    memset(out, 0, sizeof *out);
    out->state = j->state;
    out->iters = j->iters;
    out->cells = j->cells;
    out->arena_bytes = j->bytes;
    out->t_submit = j->t_submit;
    out->t_admit = j->t_admit;
    out->t_done = j->t_done;
    return OD_OK;
}

od_status od_server_fetch(od_server *s, uint64_t id, double *dst, int32_t dst_is_device) {
    if (!s || !dst) return fail(OD_EINVAL, "null argument");
    od_ctx *ctx = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        Job *j = find(s, id);
        if (!j) return fail(OD_ENOTFOUND, "unknown job");
        if (j->state != OD_JOB_DONE) return fail(OD_ESTATE, "job not done");
        ctx = j->ctx;
    }
    return ctx ? od_read(ctx, dst, dst_is_device) : fail(OD_ESTATE, "job has no state");
}

od_status od_server_release(od_server *s, uint64_t id) {
    if (!s) return fail(OD_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    Job *j = find(s, id);
    if (!j) return fail(OD_ENOTFOUND, "unknown job");
    if (j->state == OD_JOB_RUNNING) return fail(OD_ESTATE, "job still running");
    if (j->admitting) return fail(OD_ESTATE, "job is being admitted; release it once it has run");
    if (j->state == OD_JOB_QUEUED) {
        auto it = std::find(s->queue.begin(), s->queue.end(), j);
        if (it != s->queue.end()) s->queue.erase(it);
    }
    od_ctx *ctx = j->ctx;
    const bool had_memory = ctx != nullptr;
    s->jobs.erase(id);
    lk.unlock();
    if (ctx) od_destroy(ctx);
    lk.lock();
    if (had_memory) s->pool.release(j->off, j->bytes);
    delete j;
    s->cv_admit.notify_all();  // memory is free for queued jobs
    return OD_OK;
}

od_status od_server_stats(od_server *s, od_server_stats_t *out) {
    if (!s || !out) return fail(OD_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof *out);
    out->queued = (int64_t)s->queue.size();
    out->running = (int64_t)s->running.size();
    out->done = s->done;
    out->failed = s->failed;
    out->launches = s->launches;
    out->updates_done = s->updates_done;
    out->pool_used = s->pool.used();
    out->pool_peak = s->pool.peak();
    out->seconds = s->now();
    out->admit_seconds = s->admit_seconds;
    out->busy_seconds = s->job_streams.empty() ? s->busy_seconds : busy_union(s);
    if (!s->worker_error.empty()) return fail(OD_ECUDA, s->worker_error);
    return OD_OK;
}

od_status od_server_destroy(od_server *s) {
    if (!s) return OD_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
        s->cv_admit.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    if (s->admitter.joinable()) s->admitter.join();
    cudaSetDevice(s->device);
    if (s->compute) cudaStreamSynchronize(s->compute);
    for (cudaStream_t st : s->job_streams) cudaStreamSynchronize(st);
    for (auto &kv : s->jobs) {
        if (kv.second->ctx) od_destroy(kv.second->ctx);
        if (kv.second->ev0) cudaEventDestroy(kv.second->ev0);
        if (kv.second->ev1) cudaEventDestroy(kv.second->ev1);
        delete kv.second;
    }
    for (auto &b : s->inflight) {
        cudaEventDestroy(b.ev0);
        cudaEventDestroy(b.ev);
    }
    for (auto e : s->free_events) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        if (s->d_jobs[k]) cudaFree(s->d_jobs[k]);
        if (s->d_first[k]) cudaFree(s->d_first[k]);
    }
    if (s->d_queue) cudaFree(s->d_queue);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->admit) cudaStreamDestroy(s->admit);
    for (cudaStream_t st : s->job_streams) cudaStreamDestroy(st);
    if (s->base_ev) cudaEventDestroy(s->base_ev);
    if (s->h_err) cudaFreeHost(s->h_err);
    if (s->own_pool && s->pool_base) cudaFree(s->pool_base);
    delete s;
    return OD_OK;
}

}  // extern "C"
