// Serving: continuous batching of MD jobs on one GPU.
//
// A worker thread owns all device work.  Submitted jobs wait in a FIFO; a
// job is admitted as soon as its device footprint fits in the HBM budget
// next to the jobs already resident.  Each admitted job keeps its state in
// device memory on its own stream.  Its creation (seeding, relaxation) and
// then slices of steps are enqueued asynchronously; the worker polls each
// job's slices and keeps two of them queued on its stream (the next is
// enqueued as soon as the older one is done), so a job's stream stays busy
// while the worker serves the other jobs or admits a new one, and the jobs'
// kernels overlap on the device.  A slice's error words are copied to pinned
// host memory behind it, so reaping a slice never synchronises a stream.
// Per-step latencies come from events on the job's stream.  Finished jobs
// are retired and waiting ones admitted.  A
// retired job's device memory is released only when the server is idle or
// when a waiting job needs the room: freeing device memory waits for the
// whole device, which would drain every other job's queued work and leave
// the GPU idle until the worker refills it.  A job's trajectory does not
// depend on the other jobs: each runs the same deterministic kernels as it
// would alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"

using pasta::Engine;
using pasta::fail;

namespace {

using Clock = std::chrono::steady_clock;

// A slice of a job's work enqueued on its stream: relaxation iterations or
// steps, with events around every step (latencies), the job's error words
// copied into pinned memory behind it, and a completion event.
struct Slice {
    bool steps = false;
    int64_t n = 0;
    std::vector<cudaEvent_t> ev;     // n + 1 used (steps only)
    cudaEvent_t done = nullptr;
    int* err = nullptr;              // pinned: the engine's error words after the slice
};

constexpr int kInFlight = 2;         // slices queued per job: its stream never runs dry
                                     // while the worker serves the other jobs

struct Job {
    int64_t id;
    md_job job;
    size_t bytes;
    Clock::time_point t_submit, t_admit;
    Engine* eng = nullptr;
    int64_t done_steps = 0;          // steps of completed slices
    int64_t queued_steps = 0;        // steps enqueued so far
    std::vector<double> lat_ms;
    Slice sl[kInFlight];
    int head = 0, count = 0;         // in-flight slices: sl[head], sl[(head + 1) % kInFlight], ...
    int64_t relax_left = 0;          // relaxation iterations not yet enqueued
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

double pct(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const size_t k = (size_t)std::min<double>(v.size() - 1, std::max(0.0, q * (v.size() - 1) + 0.5));
    return v[k];
}

}  // namespace

struct md_server {
    size_t budget;
    md_params prm;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> pending;
    std::vector<Job*> active;
    std::vector<std::pair<Engine*, size_t>> retired;   // engines whose memory is still held
    std::deque<md_result> done;
    int64_t next_id = 0, submitted = 0, finished = 0;
    size_t used = 0;
    bool stop = false;
    std::thread worker;
    int64_t slice_steps = 20;

    void run();
    void admit();
    void retire(Job* j, int status);
    void release_retired();
};

void md_server::release_retired() {
    size_t freed = 0;
    for (auto& e : retired) {
        delete e.first;
        freed += e.second;
    }
    retired.clear();
    if (freed) {
        std::lock_guard<std::mutex> lk(mu);
        used -= freed;
    }
}

void md_server::retire(Job* j, int status) {
    md_result r{};
    r.id = j->id;
    r.status = status;
    r.N = j->job.N;
    r.steps = j->done_steps;
    if (j->eng && status == MD_OK) {
        md_energy_t e{};
        int rc = j->eng->energy(0, &e);
        if (rc) r.status = rc;
        r.energy = e;
    }
    const auto now = Clock::now();
    r.wait_ms = ms_between(j->t_submit, j->t_admit);
    r.run_ms = ms_between(j->t_admit, now);
    r.step_p50_ms = pct(j->lat_ms, 0.50);
    r.step_p99_ms = pct(j->lat_ms, 0.99);
    if (j->eng && j->count > 0) cudaStreamSynchronize(j->eng->stream());   // (a failed job's queued slices)
    for (Slice& q : j->sl) {
        for (cudaEvent_t e : q.ev) cudaEventDestroy(e);
        if (q.done) cudaEventDestroy(q.done);
        if (q.err) cudaFreeHost(q.err);
    }
    // an admitted job's bytes stay in `used` until its engine is released;
    // a job larger than the budget was never admitted (no engine, no bytes)
    if (j->eng) retired.emplace_back(j->eng, j->bytes);
    {
        std::lock_guard<std::mutex> lk(mu);
        done.push_back(r);
        finished += 1;
    }
    cv.notify_all();
    delete j;
}

void md_server::admit() {
    for (;;) {
        Job* j = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (pending.empty()) return;
            Job* f = pending.front();
            if (f->bytes > budget) {
                pending.pop_front();
                j = f;
                j->t_admit = Clock::now();
            } else if (used + f->bytes <= budget) {
                pending.pop_front();
                used += f->bytes;
                j = f;
            } else if (retired.empty()) {
                return;   // FIFO: wait for running jobs to finish
            }
        }
        if (!j) {         // the memory of finished jobs makes the room
            release_retired();
            continue;
        }
        if (j->bytes > budget) {
            retire(j, MD_ENOMEM);
            continue;
        }
        j->t_admit = Clock::now();
        // Stream priority by job size: a small job's short kernels are
        // scheduled ahead of the large jobs' long force passes as SMs free up,
        // which bounds its step latency without slowing the large jobs much.
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);   // lo: least urgent, hi: most urgent
        int prio = lo;
        if (j->job.N < 20000) prio = hi;
        else if (j->job.N < 100000) prio = (lo + hi) / 2;
        Engine* e = new Engine(prio);
        int rc = e->add_system(j->job.N, j->job.Yp, j->job.rho, j->job.T, j->job.seed, prm);
        if (!rc) rc = e->build_tables();
        if (!rc) rc = e->initialise_async(false);   // relaxation follows in slices
        j->relax_left = e->relax_iters();
        j->eng = e;
        if (rc) {
            retire(j, rc);
            continue;
        }
        bool ok = true;
        for (Slice& q : j->sl) {
            q.ev.resize(slice_steps + 1);
            for (auto& ev : q.ev) ok = ok && cudaEventCreate(&ev) == cudaSuccess;
            ok = ok && cudaEventCreateWithFlags(&q.done, cudaEventDisableTiming) == cudaSuccess;
            ok = ok && cudaHostAlloc((void**)&q.err, sizeof(int) * (e->sys.size() + 1), cudaHostAllocDefault) ==
                           cudaSuccess;
        }
        if (!ok) {
            retire(j, MD_ECUDA);
            continue;
        }
        active.push_back(j);
    }
}

void md_server::run() {
    cudaSetDevice(device);
    for (;;) {
        if (active.empty() && !retired.empty()) release_retired();   // the device is idle
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] { return stop || !pending.empty() || !active.empty(); });
            if (stop && active.empty()) break;
        }
        admit();
        bool progressed = false;
        std::vector<Job*> keep;
        for (Job* j : active) {
            // reap the completed slices, oldest first
            int rc = MD_OK;
            while (j->count > 0) {
                Slice& q = j->sl[j->head];
                const cudaError_t e = cudaEventQuery(q.done);
                if (e == cudaErrorNotReady) break;
                progressed = true;
                rc = e == cudaSuccess ? j->eng->status_of(q.err) : MD_ECUDA;
                if (rc != MD_OK) break;
                if (q.steps) {
                    for (int64_t k = 0; k < q.n; ++k) {
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, q.ev[k], q.ev[k + 1]);
                        j->lat_ms.push_back(ms);
                    }
                    j->done_steps += q.n;
                }
                j->head = (j->head + 1) % kInFlight;
                j->count -= 1;
            }
            if (rc != MD_OK) {
                retire(j, rc);
                continue;
            }
            // keep kInFlight slices queued: relaxation first, then steps
            while (j->count < kInFlight && !stop && (j->relax_left > 0 || j->queued_steps < j->job.steps)) {
                Slice& q = j->sl[(j->head + j->count) % kInFlight];
                if (j->relax_left > 0) {
                    q.steps = false;
                    q.n = std::min(slice_steps, j->relax_left);
                    rc = j->eng->relax_async(q.n);
                    j->relax_left -= q.n;
                } else {
                    q.steps = true;
                    q.n = std::min(slice_steps, j->job.steps - j->queued_steps);
                    std::vector<double> xi(1, j->job.xi_dot);
                    rc = j->eng->step_async(q.n, &xi, q.ev.data());
                    j->queued_steps += q.n;
                }
                if (rc == MD_OK) rc = j->eng->enqueue_status(q.err);
                if (rc == MD_OK && cudaEventRecord(q.done, j->eng->stream()) != cudaSuccess) rc = MD_ECUDA;
                if (rc != MD_OK) break;
                j->count += 1;
                progressed = true;
            }
            if (rc != MD_OK) {
                retire(j, rc);
                continue;
            }
            if (j->count == 0) {       // all of its work has completed (or the server stops)
                const int64_t left = j->job.steps - j->done_steps;
                retire(j, stop && left > 0 ? MD_ETIMEOUT : MD_OK);
                continue;
            }
            keep.push_back(j);
        }
        active.swap(keep);
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    release_retired();
}

extern "C" {

int md_server_create(size_t hbm_budget_bytes, const md_params* p, md_server** out) {
    if (!out) return fail(MD_EINVAL, "out is null");
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(MD_ENODEV, "no CUDA device available");
    }
    if (hbm_budget_bytes == 0) return fail(MD_EINVAL, "budget must be > 0");
    md_server* sv = new md_server();
    sv->budget = hbm_budget_bytes;
    if (p) sv->prm = *p;
    else md_params_default(&sv->prm);
    cudaGetDevice(&sv->device);
    sv->worker = std::thread([sv] { sv->run(); });
    *out = sv;
    return MD_OK;
}

int md_server_submit(md_server* sv, const md_job* job, int64_t* id) {
    if (!sv || !job) return fail(MD_EINVAL, "null argument");
    if (job->N < 2 || job->steps < 0 || !(job->rho > 0) || !(job->Yp >= 0 && job->Yp <= 1) || !(job->T >= 0))
        return fail(MD_EINVAL, "invalid job");
    Job* j = new Job();
    j->job = *job;
    j->bytes = Engine::estimate_bytes(job->N, job->Yp, job->rho, sv->prm);
    j->t_submit = Clock::now();
    int64_t jid;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        jid = j->id = sv->next_id++;
        sv->pending.push_back(j);
        sv->submitted += 1;
    }
    sv->cv.notify_all();     // (the worker may finish and free j from here on)
    if (id) *id = jid;
    return MD_OK;
}

int md_server_poll(md_server* sv, md_result* out) {
    if (!sv || !out) return fail(MD_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->done.empty()) return MD_EAGAIN;
    *out = sv->done.front();
    sv->done.pop_front();
    return MD_OK;
}

int md_server_drain(md_server* sv, double timeout_s) {
    if (!sv) return fail(MD_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(sv->mu);
    const bool ok = sv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                    [&] { return sv->finished == sv->submitted; });
    return ok ? MD_OK : fail(MD_ETIMEOUT, "jobs still running after the timeout");
}

int md_server_destroy(md_server* sv) {
    if (!sv) return MD_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        for (Job* j : sv->pending) delete j;
        sv->pending.clear();
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    delete sv;
    return MD_OK;
}

}  // extern "C"
