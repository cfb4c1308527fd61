// Serving form of the library: a continuous-batching request loop.
//
// Requests (a configuration, a host point cloud and a sphere for φ^0) are
// queued by slr_server_submit. Worker threads drive the device:
//  - setup (setup_threads of them): each admits a queued request while an
//    active slot and enough of the HBM budget are free (policy 0: the oldest;
//    policy 1: the least estimated set-up time less its waiting time, so that
//    small requests pass large ones without starving them),
//    creates the job's context on its own stream, copies the cloud, builds
//    the exact distance grid and φ^0, and hands the job to the iteration
//    thread. Several set-ups run at once, so a large request's distance grid
//    does not hold back the admission of the requests queued behind it;
//  - iterate: round-robin over the running jobs, enqueues a few iterations
//    of each job's captured iteration graph on a stream of the greatest
//    priority (so that set-ups running beside them take only the SMs that
//    iterations leave idle), then an
//    asynchronous 16-byte status copy and an event; a job whose event has
//    completed and whose device stop flag is set is retired. New jobs join
//    the next round, so requests that arrive while others run overlap with
//    them on the GPU.
// A finished job's context (and its memory) stays with the server until the
// client releases it; its budget share is returned then.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "slr_internal.cuh"

struct slr_server;

namespace {

enum JobState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Job {
    uint64_t ticket = 0;
    slr_config cfg;
    std::vector<double> xyz;
    int64_t npts = 0;
    double sphere[4] = {0, 0, 0, 0};
    size_t bytes = 0;
    double setup_est_ms = 0.0;  // estimated set-up time (the exact distance grid dominates it)
    bool holds_budget = false;  // admitted and its share not yet returned
    slr_ctx* ctx = nullptr;
    std::atomic<int> state{kQueued};
    std::string error;
    // iteration thread bookkeeping
    bool started = false;
    bool outstanding = false;
    cudaEvent_t ev = nullptr;
    int* status = nullptr;  // pinned: n, stop, converged, error
    cudaStream_t run_stream = nullptr;    // iterations, greatest priority
    cudaStream_t setup_stream = nullptr;  // the context's own stream, restored when the job finishes
    std::chrono::steady_clock::time_point t_submit, t_start, t_ready, t_done;
};

// device bytes a job will hold: two φ buffers, d, argmin, band lists and
// candidate cells (bounded by the grid), the cloud and the distance scratch
size_t job_bytes(const slr_config& c, int64_t npts) {
    long long N = c.n[0] * c.n[1] * (c.dim == 3 ? c.n[2] : 1);
    size_t ts = c.precision == 32 ? 4 : 8;
    size_t grid = (size_t)N * (3 * ts + 4) + (size_t)N / 2 * 4;
    size_t cloud = (size_t)npts * (8 * c.dim + 4 + 16) + (size_t)(1u << 21) * 4 + (16u << 20);
    return grid + cloud;
}

// estimated set-up time of a job in ms: the exact distance grid takes about
// 4 ns per node on GB300 (65 ms at 256^3 with 1M points), the cloud's index
// a few ns per point
double setup_estimate_ms(const slr_config& c, int64_t npts) {
    const double N = (double)c.n[0] * (double)c.n[1] * (double)(c.dim == 3 ? c.n[2] : 1);
    return 4e-6 * N + 2e-5 * (double)npts;
}

}  // namespace

struct slr_server {
    size_t budget = 0;
    size_t used = 0;
    int max_active = 16;
    int device = 0;
    int rounds_per_check = 4;
    int policy = 0;  // admission order: 0 first come, 1 least estimated set-up less waiting time
    slr_allocator al{};
    bool have_al = false;
    std::mutex mu;
    std::condition_variable cv;       // wakes the setup thread (queue / budget changes)
    std::condition_variable cv_iter;  // wakes the iteration thread (new running jobs)
    std::deque<std::shared_ptr<Job>> queue;
    std::vector<std::shared_ptr<Job>> running;  // owned by the iteration thread after handoff
    std::vector<std::shared_ptr<Job>> incoming;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_ticket = 1;
    int active = 0;  // admitted and not yet released
    bool stop = false;
    std::vector<std::thread> setup_threads;
    std::thread iter_thread;
    std::string err;

    void setup_loop();
    void iter_loop();
    // the queued job to admit now (index into queue), or -1 (caller holds mu)
    long pick() const;
};

long slr_server::pick() const {
    if (queue.empty() || active >= max_active) return -1;
    auto fits = [&](const Job& j) { return used + j.bytes <= budget || active == 0; };
    if (policy == 0) return fits(*queue.front()) ? 0 : -1;
    // estimate less waiting time = estimate + submit time - now: the order by
    // estimate + submit time, which does not change while the jobs wait
    long best = -1;
    double best_key = 0.0;
    for (size_t i = 0; i < queue.size(); ++i) {
        const Job& j = *queue[i];
        if (!fits(j)) continue;
        const double key =
            j.setup_est_ms + std::chrono::duration<double, std::milli>(j.t_submit.time_since_epoch()).count();
        if (best < 0 || key < best_key) {
            best = (long)i;
            best_key = key;
        }
    }
    return best;
}

void slr_server::setup_loop() {
    cudaSetDevice(device);
    for (;;) {
        std::shared_ptr<Job> j;
        {
            std::unique_lock<std::mutex> lk(mu);
            long at = -1;
            cv.wait(lk, [&] {
                if (stop) return true;
                at = pick();
                return at >= 0;
            });
            if (stop) return;
            j = queue[(size_t)at];
            queue.erase(queue.begin() + at);
            used += j->bytes;
            ++active;
            j->holds_budget = true;
        }
        j->t_start = std::chrono::steady_clock::now();
        slr_ctx* c = nullptr;
        slr_status s = slr_create(&j->cfg, have_al ? &al : nullptr, nullptr, &c);
        if (s == SLR_OK) s = slr_load_cloud(c, j->xyz.data(), j->npts);
        if (s == SLR_OK) s = slr_build_distance(c);
        if (s == SLR_OK) s = slr_init_u(c, 0, j->sphere, nullptr);
        if (s != SLR_OK) {
            j->error = c ? slr_last_error(c) : slr_last_error(nullptr);
            if (c) slr_destroy(c);
            std::lock_guard<std::mutex> lk(mu);
            j->t_done = std::chrono::steady_clock::now();
            j->t_ready = j->t_done;
            j->state = kFailed;
            used -= j->bytes;
            --active;
            j->holds_budget = false;
            cv.notify_all();
            continue;
        }
        std::vector<double>().swap(j->xyz);  // the host copy is no longer needed
        j->ctx = c;
        j->t_ready = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lk(mu);
            j->state = kRunning;
            incoming.push_back(j);
        }
        cv_iter.notify_all();
    }
}

namespace {

// enqueue `rounds` iterations of the job's captured iteration graph and an
// asynchronous status copy; returns false on a CUDA error
bool enqueue_rounds(Job* j, int rounds) {
    slr_ctx* c = j->ctx;
    if (!j->started) {
        if (slr::evolve_prepare(c) != SLR_OK) return false;
        j->started = true;
    }
    for (int r = 0; r < rounds; ++r)
        if (slr::evolve_launch(c) != SLR_OK) return false;
    if (cudaMemcpyAsync(j->status, &c->ds->n, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return false;
    if (cudaEventRecord(j->ev, c->stream) != cudaSuccess) return false;
    j->outstanding = true;
    return true;
}

}  // namespace

void slr_server::iter_loop() {
    cudaSetDevice(device);
    std::vector<std::shared_ptr<Job>> run;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (run.empty()) cv_iter.wait(lk, [&] { return stop || !incoming.empty(); });
            if (stop) break;
            for (auto& j : incoming) run.push_back(j);
            incoming.clear();
        }
        bool progressed = false;
        for (size_t i = 0; i < run.size();) {
            Job* j = run[i].get();
            bool failed = false, done = false;
            if (!j->ev) {
                int least = 0, greatest = 0;
                cudaDeviceGetStreamPriorityRange(&least, &greatest);
                if (cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess ||
                    cudaMallocHost((void**)&j->status, 4 * sizeof(int)) != cudaSuccess ||
                    cudaStreamCreateWithPriority(&j->run_stream, cudaStreamNonBlocking, greatest) != cudaSuccess) {
                    cudaGetLastError();
                    failed = true;
                } else {
                    // the set-up is complete (slr_init_u returned); later work goes to the run stream
                    j->setup_stream = j->ctx->stream;
                    j->ctx->stream = j->run_stream;
                }
            }
            if (!failed && j->outstanding) {
                cudaError_t q = cudaEventQuery(j->ev);
                if (q == cudaSuccess) {
                    j->outstanding = false;
                    progressed = true;
                    if (j->status[3]) {
                        j->error = "a device-side check failed (band-list offsets)";
                        failed = true;
                    } else if (j->status[1]) {
                        done = true;
                    }
                } else if (q != cudaErrorNotReady) {
                    cudaGetLastError();
                    j->error = cudaGetErrorString(q);
                    failed = true;
                }
            }
            if (!failed && !done && !j->outstanding) {
                if (!enqueue_rounds(j, rounds_per_check)) {
                    j->error = slr_last_error(j->ctx);
                    failed = true;
                }
                progressed = true;
            }
            if (failed || done) {
                j->t_done = std::chrono::steady_clock::now();
                if (j->run_stream) {
                    cudaStreamSynchronize(j->run_stream);
                    j->ctx->stream = j->setup_stream;  // the client reads results on the context's own stream
                    cudaStreamDestroy(j->run_stream);
                    j->run_stream = nullptr;
                }
                if (j->ev) cudaEventDestroy(j->ev);
                j->ev = nullptr;
                if (j->status) cudaFreeHost(j->status);
                j->status = nullptr;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    j->state = failed ? kFailed : kDone;
                }
                run.erase(run.begin() + i);
                continue;
            }
            ++i;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    for (auto& j : run) {
        if (j->ctx) cudaStreamSynchronize(j->ctx->stream);
        if (j->run_stream) {
            j->ctx->stream = j->setup_stream;
            cudaStreamDestroy(j->run_stream);
        }
        if (j->ev) cudaEventDestroy(j->ev);
        if (j->status) cudaFreeHost(j->status);
    }
}

extern "C" {

slr_status slr_server_create(size_t hbm_budget, int max_active, int setup_threads, const slr_allocator* alloc,
                             slr_server** out) {
    if (!out || max_active < 1 || setup_threads < 1 || setup_threads > 64) return SLR_E_INVALID;
    slr_server* s = new slr_server();
    s->budget = hbm_budget;
    s->max_active = max_active;
    if (alloc && alloc->alloc && alloc->free) {
        s->al = *alloc;
        s->have_al = true;
    }
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return SLR_E_CUDA;
    }
    for (int i = 0; i < setup_threads; ++i) s->setup_threads.emplace_back([s] { s->setup_loop(); });
    s->iter_thread = std::thread([s] { s->iter_loop(); });
    *out = s;
    return SLR_OK;
}

slr_status slr_server_set_policy(slr_server* s, int policy) {
    if (!s || policy < 0 || policy > 1) return SLR_E_INVALID;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->policy = policy;
    }
    s->cv.notify_all();
    return SLR_OK;
}

slr_status slr_server_submit(slr_server* s, const slr_config* cfg, const double* xyz, int64_t n_points,
                             const double sphere[4], uint64_t* ticket) {
    if (!s || !cfg || !xyz || n_points < 1 || !sphere || !ticket) return SLR_E_INVALID;
    auto j = std::make_shared<Job>();
    j->cfg = *cfg;
    j->npts = n_points;
    j->xyz.assign(xyz, xyz + (size_t)n_points * cfg->dim);
    for (int a = 0; a < 4; ++a) j->sphere[a] = sphere[a];
    j->bytes = job_bytes(*cfg, n_points);
    j->setup_est_ms = setup_estimate_ms(*cfg, n_points);
    j->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        j->ticket = s->next_ticket++;
        s->jobs[j->ticket] = j;
        s->queue.push_back(j);
    }
    s->cv.notify_all();
    *ticket = j->ticket;
    return SLR_OK;
}

slr_status slr_server_poll(slr_server* s, uint64_t ticket, int* state, slr_ctx** result, double* latency_ms) {
    if (!s || !state) return SLR_E_INVALID;
    std::shared_ptr<Job> j;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return SLR_E_INVALID;
        j = it->second;
    }
    int st = j->state.load();
    *state = st;
    if (result) *result = st == kDone ? j->ctx : nullptr;
    if (latency_ms)
        *latency_ms = (st == kDone || st == kFailed)
                          ? std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count()
                          : -1.0;
    if (st == kFailed) {
        s->err = j->error;
        return SLR_E_CUDA;
    }
    return SLR_OK;
}

slr_status slr_server_timing(slr_server* s, uint64_t ticket, double* queue_ms, double* setup_ms, double* iterate_ms) {
    if (!s) return SLR_E_INVALID;
    std::shared_ptr<Job> j;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return SLR_E_INVALID;
        j = it->second;
    }
    const int st = j->state.load();
    if (st != kDone && st != kFailed) return SLR_E_STATE;
    using ms = std::chrono::duration<double, std::milli>;
    if (queue_ms) *queue_ms = ms(j->t_start - j->t_submit).count();
    if (setup_ms) *setup_ms = ms(j->t_ready - j->t_start).count();
    if (iterate_ms) *iterate_ms = ms(j->t_done - j->t_ready).count();
    return SLR_OK;
}

slr_status slr_server_release(slr_server* s, uint64_t ticket) {
    if (!s) return SLR_E_INVALID;
    std::shared_ptr<Job> j;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return SLR_E_INVALID;
        j = it->second;
        int st = j->state.load();
        if (st != kDone && st != kFailed) return SLR_E_STATE;
        s->jobs.erase(it);
    }
    if (j->ctx) slr_destroy(j->ctx);
    j->ctx = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (j->holds_budget) {
            s->used -= j->bytes;
            --s->active;
            j->holds_budget = false;
        }
    }
    s->cv.notify_all();
    return SLR_OK;
}

const char* slr_server_last_error(const slr_server* s) { return s ? s->err.c_str() : ""; }

void slr_server_destroy(slr_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    s->cv_iter.notify_all();
    for (auto& t : s->setup_threads)
        if (t.joinable()) t.join();
    if (s->iter_thread.joinable()) s->iter_thread.join();
    for (auto& kv : s->jobs)
        if (kv.second->ctx) slr_destroy(kv.second->ctx);
    delete s;
}

}  // extern "C"
