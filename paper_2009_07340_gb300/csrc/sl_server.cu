// sl_server.cu -- a serving loop for drift-diffusion solves that arrive over
// time (host runtime around the solver; no kernels of its own).
//
// Requests (an sl_instance plus a step count) are queued on submission.  A
// scheduler thread runs rounds:
//   1. admission: queued requests are admitted in arrival order while their
//      device footprint (state, face buffer, Wiener scratch, moment
//      partials, node tables) fits in the memory budget next to the running
//      ones; a request larger than the whole budget is rejected;
//      (backfilling: a request that does not fit yet does not block later,
//      smaller ones); at most `heavy_slots` heavy requests run at once, so
//      that heavy work is served nearly in order instead of being shared
//      among many requests that would then all finish late;
//   2. a running request whose previous slice has completed (CUDA event)
//      gets its next slice on its stream, so requests' kernels overlap on the
//      GPU and a slow request never holds back the others.  Requests are
//      light or heavy by their estimated work per step; light ones run on
//      high-priority streams (the CTA scheduler serves them first when SMs
//      free up), heavy ones on low-priority streams with one step per slice;
//   3. a request that has taken all its steps computes its moments, releases
//      its memory and records its latency (completion minus submission);
//      new arrivals are admitted between slices (continuous batching).
// Creating a request's solver and completing it (moments, release) can wait
// on the GPU, so they run on a small worker pool; the scheduler thread only
// admits, polls events and launches slices, none of which blocks.
// Each request is an independent solver context, so its result is the same
// as that of the request run alone (bitwise in SL_FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "sl_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    long long ticket = 0;
    sl_instance spec;
    int steps = 0, done_steps = 0;
    double dt = 0.0;  // resolved time step
    int state = 0;  // 0 queued, 1 running, 2 done, < 0 error code
    size_t footprint = 0;
    double work = 0.0;  // estimated arithmetic per step
    bool heavy = false;
    sl_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;  // the request's own stream
    cudaEvent_t ev = nullptr;  // completion of the slice in flight
    int inflight = 0;          // steps of the slice in flight
    Clock::time_point t_submit, t_done;
    std::vector<double> mean, m2;
    long long esu = 0;
};

size_t footprint_of(const sl_instance &s, int slice, int precision)
{
    const int dim = s.mesh.dim;
    const long long E = (long long)s.mesh.K[0] * (dim == 2 ? s.mesh.K[1] : 1);
    const long long n = dim == 2 ? (long long)s.N * s.N : s.N;
    const long long V = E * n;
    const size_t elem = 8;  // FP64 or FP32 pair
    size_t b = size_t(s.M) * V * elem;                                  // state
    if (dim == 2) b += size_t(s.M) * E * 4 * s.N * elem;                // face buffer
    b += size_t(std::max(slice, 1)) * s.M * dim * sizeof(double);       // Wiener scratch
    b += size_t((s.M + 63) / 64) * V * 2 * sizeof(double);             // moment partials
    b += size_t(V) * (dim + 4) * sizeof(double) + size_t(2 * E * s.N) * 2 * sizeof(double);  // tables
    (void)precision;
    return b + (1u << 20);
}

// Arithmetic per step: E M N^2 in 1D (reduced remap), E M n^3 in 2D (dense
// per-element solves, n = N^2).
double work_of(const sl_instance &s)
{
    const double E = double(s.mesh.K[0]) * (s.mesh.dim == 2 ? s.mesh.K[1] : 1);
    const double n = s.mesh.dim == 2 ? double(s.N) * s.N : s.N;
    return E * s.M * (s.mesh.dim == 2 ? n * n * n : n * n);
}

constexpr double kHeavyWork = 2e9;  // about a millisecond of GPU time per step

}  // namespace

struct sl_server {
    sl_server_config cfg;
    int prio_light = 0, prio_heavy = 0;  // stream priorities
    std::mutex mu;
    std::condition_variable cv;
    std::deque<long long> queue;
    std::map<long long, Request> req;
    std::vector<long long> running;
    int heavy_running = 0;  // heavy requests admitted and not yet finished
    size_t used = 0, peak = 0;
    long long next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::vector<double> latencies;
    long long esu_done = 0, submitted = 0, completed = 0, rejected = 0, failed = 0;
    Clock::time_point t_first, t_last;
    bool any = false;
    int device = 0;
    // worker pool for solver creation and completion
    std::vector<std::thread> pool;
    std::deque<std::function<void()>> tasks;
    std::condition_variable task_cv;
    std::vector<long long> ready;  // created solvers waiting to join the running set
    int outstanding = 0;           // tasks queued or running
};

namespace {

void finish(sl_server *s, Request &r, int rc)
{
    if (r.ctx) {
        if (rc == SL_OK) {
            const size_t V = size_t(r.ctx->m.E) * r.ctx->m.n;
            r.mean.resize(V);
            r.m2.resize(V);
            rc = sl_moments(r.ctx, r.mean.data(), r.m2.data());
        }
        sl_free(r.ctx);
        r.ctx = nullptr;
    }
    if (r.ev) {
        cudaEventDestroy(r.ev);
        r.ev = nullptr;
    }
    if (r.st) {
        cudaStreamDestroy(r.st);  // pending frees on it still complete
        r.st = nullptr;
    }
    r.t_done = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    s->used -= r.footprint;
    if (r.heavy) s->heavy_running--;
    if (rc == SL_OK) {
        r.state = 2;
        s->completed++;
        s->esu_done += r.esu;
        s->latencies.push_back(std::chrono::duration<double>(r.t_done - r.t_submit).count());
        s->t_last = r.t_done;
    } else {
        r.state = rc;
        s->failed++;
    }
}

void post(sl_server *s, std::function<void()> f)
{
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->tasks.push_back(std::move(f));
        s->outstanding++;
    }
    s->task_cv.notify_one();
}

void pool_worker(sl_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::function<void()> f;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->task_cv.wait(lk, [&] { return s->stop || !s->tasks.empty(); });
            if (s->tasks.empty()) return;
            f = std::move(s->tasks.front());
            s->tasks.pop_front();
        }
        f();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->outstanding--;
        }
        s->cv.notify_one();
    }
}

// Creates the request's stream and solver (on a pool thread).
void create_request(sl_server *s, Request *r)
{
    int rc = SL_OK;
    if (cudaStreamCreateWithPriority(&r->st, cudaStreamNonBlocking, r->heavy ? s->prio_heavy : s->prio_light) !=
        cudaSuccess) {
        cudaGetLastError();
        r->st = nullptr;
        rc = SL_ERR_CUDA;
    }
    if (rc == SL_OK) {
        sl_options o = {};
        o.seed = r->spec.seed;
        o.precision = s->cfg.precision;
        o.device = -1;
        o.stream = r->st;
        rc = sl_init(&r->ctx, &r->spec.mesh, r->spec.N, r->spec.M, &r->spec.drift, &r->spec.diffusion, &r->spec.phi0,
                     &o);
        if (rc != SL_OK) r->ctx = nullptr;
    }
    if (rc == SL_OK && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) rc = SL_ERR_CUDA;
    if (rc != SL_OK) {
        finish(s, *r, rc);
        return;
    }
    r->dt = r->spec.dt_rule == 0 ? r->spec.dt : r->spec.dt * (r->spec.dt_rule == 1 ? r->ctx->dtmax : r->ctx->dtedge);
    r->esu = (long long)r->ctx->m.E * r->spec.M * r->steps;
    std::lock_guard<std::mutex> lk(s->mu);
    r->state = 1;
    s->ready.push_back(r->ticket);
}

void scheduler(sl_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<long long> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->queue.empty() || !s->running.empty() || !s->ready.empty() ||
                                        s->outstanding > 0; });
            if (s->stop) return;  // sl_server_free drains and releases
            // admission in arrival order with backfilling
            for (auto it = s->queue.begin(); it != s->queue.end();) {
                Request &r = s->req[*it];
                if (r.footprint > s->cfg.budget_bytes) {
                    r.state = SL_ERR_OOM;
                    s->rejected++;
                    it = s->queue.erase(it);
                    continue;
                }
                if (s->used + r.footprint > s->cfg.budget_bytes ||
                    (r.heavy && s->cfg.heavy_slots > 0 && s->heavy_running >= s->cfg.heavy_slots)) {
                    ++it;
                    continue;
                }
                s->used += r.footprint;
                if (r.heavy) s->heavy_running++;
                s->peak = std::max(s->peak, s->used);
                admit.push_back(r.ticket);
                it = s->queue.erase(it);
            }
        }
        // admission: solvers are created on the pool
        for (long long t : admit) {
            Request *r;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                r = &s->req[t];
            }
            post(s, [s, r] { create_request(s, r); });
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (long long t : s->ready) s->running.push_back(t);
            s->ready.clear();
        }
        // slices: every running request whose previous slice has completed
        std::vector<Request *> run;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (long long t : s->running) run.push_back(&s->req[t]);
        }
        bool progressed = !admit.empty();
        std::vector<long long> still;
        for (Request *r : run) {
            int rc = SL_OK;
            if (r->inflight) {
                const cudaError_t q = cudaEventQuery(r->ev);
                if (q == cudaErrorNotReady) {
                    still.push_back(r->ticket);
                    continue;
                }
                if (q != cudaSuccess) rc = SL_ERR_CUDA;
                r->done_steps += r->inflight;
                r->inflight = 0;
                progressed = true;
            }
            if (rc == SL_OK && r->done_steps < r->steps) {
                const int n = std::min(r->heavy ? 1 : s->cfg.slice_steps, r->steps - r->done_steps);
                rc = sl_step(r->ctx, r->dt, n);
                if (rc == SL_OK && cudaEventRecord(r->ev, r->st) != cudaSuccess)
                    rc = SL_ERR_CUDA;
                if (rc == SL_OK) {
                    r->inflight = n;
                    progressed = true;
                    still.push_back(r->ticket);
                    continue;
                }
            }
            post(s, [s, r, rc] { finish(s, *r, rc); });
            progressed = true;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->running.swap(still);
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
}

}  // namespace

extern "C" {

int sl_server_create(sl_server **out, const sl_server_config *cfg)
{
    if (!out || !cfg || cfg->slice_steps < 1 || cfg->budget_bytes == 0 || cfg->heavy_slots < 0)
        return SL_ERR_ARG;
    if (cfg->precision != SL_FP64 && cfg->precision != SL_MIXED && cfg->precision != SL_FP32) return SL_ERR_ARG;
    *out = nullptr;
    sl_server *s = new (std::nothrow) sl_server;
    if (!s) return SL_ERR_OOM;
    s->cfg = *cfg;
    if (cfg->device >= 0 && cudaSetDevice(cfg->device) != cudaSuccess) {
        delete s;
        return SL_ERR_CUDA;
    }
    cudaGetDevice(&s->device);
    int prio_least = 0, prio_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    s->prio_light = prio_greatest;
    s->prio_heavy = prio_least;
    s->worker = std::thread(scheduler, s);
    for (int i = 0; i < 4; ++i) s->pool.emplace_back(pool_worker, s);
    *out = s;
    return SL_OK;
}

int sl_server_submit(sl_server *s, const sl_instance *spec, int steps, long long *ticket)
{
    if (!s || !spec || steps < 1 || !(spec->dt > 0.0) || spec->dt_rule < 0 || spec->dt_rule > 2 ||
        (spec->dt_rule > 0 && spec->dt > 1.0))
        return SL_ERR_ARG;
    Request r;
    r.spec = *spec;
    r.steps = steps;
    r.footprint = footprint_of(*spec, s->cfg.slice_steps, s->cfg.precision);
    r.work = work_of(*spec);
    r.heavy = r.work > kHeavyWork;
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r.ticket = s->next_ticket++;
        if (!s->any) {
            s->t_first = r.t_submit;
            s->any = true;
        }
        s->submitted++;
        s->queue.push_back(r.ticket);
        if (ticket) *ticket = r.ticket;
        s->req.emplace(r.ticket, std::move(r));
    }
    s->cv.notify_one();
    return SL_OK;
}

int sl_server_poll(sl_server *s, long long ticket, int *state, double *mean, double *m2, double *latency_s)
{
    if (!s || !state) return SL_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->req.find(ticket);
    if (it == s->req.end()) return SL_ERR_ARG;
    const Request &r = it->second;
    *state = r.state;
    if (r.state == 2) {
        if (mean) std::memcpy(mean, r.mean.data(), r.mean.size() * sizeof(double));
        if (m2) std::memcpy(m2, r.m2.data(), r.m2.size() * sizeof(double));
        if (latency_s) *latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
    }
    return SL_OK;
}

int sl_server_wait_idle(sl_server *s, double timeout_s)
{
    if (!s) return SL_ERR_ARG;
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->queue.empty() && s->running.empty() && s->ready.empty() && s->outstanding == 0) return SL_OK;
        }
        if (Clock::now() > deadline) return SL_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
}

int sl_server_stats_get(sl_server *s, sl_server_stats *out)
{
    if (!s || !out) return SL_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->failed = s->failed;
    out->running = (long long)(s->running.size() + s->ready.size()) + s->outstanding;
    out->queued = (long long)s->queue.size();
    out->esu_completed = s->esu_done;
    out->memory_in_use = (long long)s->used;
    out->memory_peak = (long long)s->peak;
    std::vector<double> l = s->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            const double pos = q * double(l.size() - 1);
            const size_t i = size_t(pos);
            const double f = pos - double(i);
            return i + 1 < l.size() ? l[i] * (1.0 - f) + l[i + 1] * f : l[i];
        };
        out->p50_s = pct(0.50);
        out->p99_s = pct(0.99);
        double sum = 0.0;
        for (double v : l) sum += v;
        out->mean_s = sum / double(l.size());
        const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
        out->span_s = span;
        out->esu_per_s = span > 0.0 ? double(s->esu_done) / span : 0.0;
    }
    return SL_OK;
}

void sl_server_free(sl_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();
        s->tasks.clear();  // queued creations and completions are dropped
    }
    s->cv.notify_all();
    s->task_cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (std::thread &t : s->pool) t.join();  // a task already running finishes
    // slices in flight complete; the requests they belong to are abandoned
    for (auto &kv : s->req) {
        if (kv.second.st) cudaStreamSynchronize(kv.second.st);
        if (kv.second.ctx) sl_free(kv.second.ctx);
        if (kv.second.ev) cudaEventDestroy(kv.second.ev);
        if (kv.second.st) cudaStreamDestroy(kv.second.st);
    }
    delete s;
}

}  // extern "C"
