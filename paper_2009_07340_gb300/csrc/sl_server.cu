// sl_server.cu -- a serving loop for drift-diffusion solves that arrive over
// time (host runtime around the solver; no kernels of its own).
//
// Requests (an sl_instance plus a step count) are queued on submission and
// go through these phases:
//   1. admission (scheduler thread): queued requests are admitted in arrival
//      order while their device footprint (state, face buffer, Wiener
//      scratch, moment partials, node tables) fits in the memory budget next
//      to the running ones; a request larger than the whole budget is
//      rejected.  Backfilling: a request that does not fit yet does not block
//      later, smaller ones.  At most `heavy_slots` heavy requests run at once,
//      so that heavy work is served nearly in order instead of being shared
//      among many requests that would then all finish late, and at most
//      `max_active` requests are admitted and unfinished at once;
//   2. creation (worker thread): the request's stream and solver (sl_init);
//   3. steps.  Requests are light or heavy by their estimated work per step.
//      A light request runs on a high-priority stream (the CTA scheduler
//      serves it first when SMs free up) in slices of `slice_steps` steps
//      launched by the scheduler thread; each slice ends with a host callback
//      that hands the request back to the scheduler, which sleeps until a
//      callback, an arrival, a created solver or a completion wakes it (no
//      polling).  A heavy request runs on a low-priority stream and is driven
//      from creation to completion by one heavy worker thread, one step at a
//      time, its 2D kernels split into launches of bounded length with at
//      most two queued (sl_options.launch_chunk): CUDA multiplexes streams
//      onto a few in-order hardware queues, and a long or deeply queued heavy
//      stream would block every light stream sharing its queue;
//   4. completion (worker thread): moments, release of the solver, latency.
// New arrivals are admitted while others run (continuous batching).
// Creation and completion wait on the GPU, so they run on worker threads;
// light and heavy requests have separate workers, so that no thread that
// light requests depend on ever waits on heavy work.  The budget is reserved
// in the library's memory pool when the server is created, so requests'
// allocations never take new memory from the driver.
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
    sl_server *owner = nullptr;
    sl_instance spec;
    int steps = 0, done_steps = 0;
    double dt = 0.0;  // resolved time step
    int state = 0;  // 0 queued, 1 running, 2 done, < 0 error code
    size_t footprint = 0;
    double work = 0.0;  // estimated arithmetic per step
    bool heavy = false;
    sl_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;  // the request's own stream
    int inflight = 0;           // steps of the slice in flight
    // submitted, admitted, creation started, solver created, last slice seen
    // complete, completion started, moments copied, done
    Clock::time_point t_submit, t_admit, t_create, t_ready, t_ran, t_finish, t_moments, t_done;
    Clock::time_point t_launch;  // launch of the slice in flight
    double slice_max = 0.0;      // longest slice turnaround (launch to completion seen)
    std::vector<double> mean, m2;
    long long esu = 0;
    // Copies of the caller's nodal tables (phi0, drift and diffusion nodes and
    // interfaces): the solver is created later, on a worker thread.
    std::vector<double> tables[5];
};

// Keeps copies of the request's nodal tables and points its spec at them.
void own_tables(Request &r)
{
    sl_instance &s = r.spec;
    const int dim = s.mesh.dim, N = s.N;
    const long long K0 = s.mesh.K[0], K1 = dim == 2 ? s.mesh.K[1] : 1;
    const long long V = K0 * K1 * (dim == 2 ? (long long)N * N : N);
    const long long nif = dim == 1 ? K0 + 1 : K1 * (K0 + 1) * N + (K1 + 1) * K0 * N;
    auto keep = [](const double *&p, long long n, std::vector<double> &v) {
        if (!p) return;
        v.assign(p, p + n);
        p = v.data();
    };
    if (s.phi0.kind == SL_PHI_NODAL) keep(s.phi0.nodal, V, r.tables[0]);
    if (s.drift.kind == SL_U_NODAL) {
        keep(s.drift.nodal, dim * V, r.tables[1]);
        keep(s.drift.face, nif, r.tables[2]);
    }
    if (s.diffusion.kind == SL_D_NODAL) {
        keep(s.diffusion.nodal, V, r.tables[3]);
        keep(s.diffusion.face, nif, r.tables[4]);
    }
}

size_t footprint_of(const sl_instance &s, int slice)
{
    const int dim = s.mesh.dim;
    const long long E = (long long)s.mesh.K[0] * (dim == 2 ? s.mesh.K[1] : 1);
    const long long n = dim == 2 ? (long long)s.N * s.N : s.N;
    const long long V = E * n;
    const size_t elem = 8;  // FP64 or FP32 pair
    size_t b = size_t(s.M) * V * elem;                                  // state
    if (dim == 2) b += size_t(s.M) * E * 4 * s.N * elem;                // face buffer
    if (dim == 2) b += size_t(s.M) * V * elem + size_t(s.M) * E * 9;    // interpolant between phases, flags, slot list
    b += size_t(std::max(slice, 1)) * s.M * dim * sizeof(double);       // Wiener scratch
    b += size_t((s.M + 63) / 64) * V * 2 * sizeof(double);             // moment partials
    b += size_t(V) * (dim + 4) * sizeof(double) + size_t(2 * E * s.N) * 2 * sizeof(double);  // tables
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

constexpr double kHeavyWork = 2e9;    // about a millisecond of GPU time per step
constexpr double kLaunchWork = 2e10;  // arithmetic per heavy 2D launch: a few milliseconds
constexpr int kLightWorkers = 8;

// Element-sample groups per launch for a heavy request (2D: n^3 per group).
long long launch_chunk_of(const sl_instance &s)
{
    if (s.mesh.dim != 2) return 0;
    const double n = double(s.N) * s.N;
    return std::max<long long>(4096, (long long)(kLaunchWork / (n * n * n)));
}

}  // namespace

struct sl_server {
    sl_server_config cfg;
    int prio_light = 0, prio_heavy = 0;  // stream priorities
    int device = 0;
    std::mutex mu;               // guards everything below
    std::condition_variable cv;  // wakes the scheduler
    bool wake = false;           // something for the scheduler to do
    bool admit_changed = false;  // an arrival or a release: run admission
    std::deque<long long> queue;  // submitted, not admitted
    std::map<long long, Request> req;
    std::vector<long long> ready;   // light solvers created, first slice not launched
    std::vector<long long> landed;  // light slices completed (host callbacks)
    long long active = 0;           // admitted and not finished
    int heavy_running = 0;          // heavy requests among them
    size_t used = 0, peak = 0;
    long long next_ticket = 1;
    bool stop = false;
    std::vector<double> latencies;
    long long esu_done = 0, submitted = 0, completed = 0, rejected = 0, failed = 0;
    Clock::time_point t_first, t_last;
    bool any = false;
    // workers for creation, heavy requests and completion: lane 0 light, lane 1 heavy
    std::vector<std::thread> pool;
    std::deque<std::function<void()>> tasks[2];
    std::condition_variable task_cv[2];
    int outstanding = 0;  // tasks queued or running
    std::thread scheduler;
    // scheduler accounting
    long long slices = 0;
    double busy_s = 0.0, launch_s = 0.0, launch_max_s = 0.0;
};

namespace {

void wake_scheduler(sl_server *s, bool admit)  // caller holds s->mu
{
    s->wake = true;
    if (admit) s->admit_changed = true;
    s->cv.notify_one();
}

// Completion: moments to the host, release, bookkeeping (a worker thread).
void finish(sl_server *s, Request &r, int rc)
{
    r.t_finish = Clock::now();
    if (r.ctx) {
        if (rc == SL_OK) {
            const size_t V = size_t(r.ctx->m.E) * r.ctx->m.n;
            r.mean.resize(V);
            r.m2.resize(V);
            rc = sl_moments(r.ctx, r.mean.data(), r.m2.data());
        }
        r.t_moments = Clock::now();
        sl_free(r.ctx);
        r.ctx = nullptr;
    } else {
        r.t_moments = r.t_finish;
    }
    if (r.st) {
        cudaStreamDestroy(r.st);  // pending frees on it still complete
        r.st = nullptr;
    }
    r.t_done = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    s->used -= r.footprint;
    s->active--;
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
    wake_scheduler(s, true);
}

void post(sl_server *s, bool heavy, std::function<void()> f)
{
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->tasks[heavy].push_back(std::move(f));
        s->outstanding++;
    }
    s->task_cv[heavy].notify_one();
}

void pool_worker(sl_server *s, int lane)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::function<void()> f;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->task_cv[lane].wait(lk, [&] { return s->stop || !s->tasks[lane].empty(); });
            if (s->tasks[lane].empty()) return;
            f = std::move(s->tasks[lane].front());
            s->tasks[lane].pop_front();
        }
        f();
        std::lock_guard<std::mutex> lk(s->mu);
        s->outstanding--;
    }
}

// Creation: the request's stream and solver (a worker thread).  A light
// request then joins the scheduler's ready list; a heavy one returns to
// run_heavy.
void create_request(sl_server *s, Request *r)
{
    r->t_create = Clock::now();
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
        o.bc_weight = r->spec.bc_weight;
        o.device = -1;
        o.stream = r->st;
        o.launch_chunk = r->heavy ? launch_chunk_of(r->spec) : 0;
        rc = sl_init(&r->ctx, &r->spec.mesh, r->spec.N, r->spec.M, &r->spec.drift, &r->spec.diffusion, &r->spec.phi0,
                     &o);
        if (rc != SL_OK) r->ctx = nullptr;
    }
    r->t_ready = Clock::now();
    if (rc != SL_OK) {
        r->t_ran = r->t_ready;
        finish(s, *r, rc);
        return;
    }
    r->dt = r->spec.dt_rule == 0 ? r->spec.dt : r->spec.dt * (r->spec.dt_rule == 1 ? r->ctx->dtmax : r->ctx->dtedge);
    r->esu = (long long)r->ctx->m.E * r->spec.M * r->steps;
    std::lock_guard<std::mutex> lk(s->mu);
    r->state = 1;
    if (r->heavy) return;
    s->ready.push_back(r->ticket);
    wake_scheduler(s, false);
}

// A heavy request from creation to completion (a heavy worker thread): one
// step at a time, waiting on a blocking-sync event between steps.
void run_heavy(sl_server *s, Request *r)
{
    create_request(s, r);
    if (!r->ctx) return;  // creation failed and completed the request
    int rc = SL_OK;
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        rc = SL_ERR_CUDA;
    }
    while (rc == SL_OK && r->done_steps < r->steps) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->stop) break;
        }
        r->t_launch = Clock::now();
        rc = sl_step(r->ctx, r->dt, 1);
        if (rc == SL_OK && (cudaEventRecord(ev, r->st) != cudaSuccess || cudaEventSynchronize(ev) != cudaSuccess)) {
            cudaGetLastError();
            rc = SL_ERR_CUDA;
        }
        r->t_ran = Clock::now();
        r->slice_max = std::max(r->slice_max, std::chrono::duration<double>(r->t_ran - r->t_launch).count());
        if (rc == SL_OK) r->done_steps++;
    }
    if (ev) cudaEventDestroy(ev);
    if (r->done_steps == r->steps || rc != SL_OK) finish(s, *r, rc);  // else stopping: sl_server_free releases it
}

// Host callback at the end of a light slice: hands the request back to the
// scheduler.  Runs on a CUDA runtime thread and makes no CUDA call.
void CUDART_CB slice_landed(void *p)
{
    Request *r = static_cast<Request *>(p);
    sl_server *s = r->owner;
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    r->t_ran = now;
    s->landed.push_back(r->ticket);
    wake_scheduler(s, false);
}

// Launches a light request's next slice, or hands it to completion (scheduler).
void next_slice(sl_server *s, Request *r)
{
    int rc = SL_OK;
    if (r->done_steps < r->steps) {
        const int n = std::min(s->cfg.slice_steps, r->steps - r->done_steps);
        r->t_launch = Clock::now();
        rc = sl_step(r->ctx, r->dt, n);
        if (rc == SL_OK && cudaLaunchHostFunc(r->st, slice_landed, r) != cudaSuccess) {
            cudaGetLastError();
            rc = SL_ERR_CUDA;
        }
        const double took = std::chrono::duration<double>(Clock::now() - r->t_launch).count();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->slices++;
            s->launch_s += took;
            s->launch_max_s = std::max(s->launch_max_s, took);
        }
        if (rc == SL_OK) {
            r->inflight = n;
            return;
        }
        r->t_ran = Clock::now();
    }
    post(s, false, [s, r, rc] { finish(s, *r, rc); });
}

void scheduler(sl_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<Request *> admit, start, landed;
        Clock::time_point t_busy;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || s->wake; });
            if (s->stop) return;  // sl_server_free drains and releases
            s->wake = false;
            t_busy = Clock::now();
            if (s->admit_changed) {
                s->admit_changed = false;
                // admission in arrival order with backfilling
                for (auto it = s->queue.begin(); it != s->queue.end();) {
                    if (s->cfg.max_active > 0 && s->active >= s->cfg.max_active) break;
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
                    s->peak = std::max(s->peak, s->used);
                    s->active++;
                    if (r.heavy) s->heavy_running++;
                    r.t_admit = Clock::now();
                    admit.push_back(&r);
                    it = s->queue.erase(it);
                }
            }
            for (long long t : s->ready) start.push_back(&s->req[t]);
            s->ready.clear();
            for (long long t : s->landed) landed.push_back(&s->req[t]);
            s->landed.clear();
        }
        for (Request *r : admit) {
            if (r->heavy) post(s, true, [s, r] { run_heavy(s, r); });
            else post(s, false, [s, r] { create_request(s, r); });
        }
        for (Request *r : start) next_slice(s, r);
        for (Request *r : landed) {
            r->done_steps += r->inflight;
            r->inflight = 0;
            r->slice_max = std::max(r->slice_max, std::chrono::duration<double>(r->t_ran - r->t_launch).count());
            next_slice(s, r);
        }
        const double busy = std::chrono::duration<double>(Clock::now() - t_busy).count();
        std::lock_guard<std::mutex> lk(s->mu);
        s->busy_s += busy;
    }
}

}  // namespace

extern "C" {

int sl_server_create(sl_server **out, const sl_server_config *cfg)
{
    if (!out || !cfg || cfg->slice_steps < 1 || cfg->budget_bytes == 0 || cfg->heavy_slots < 0 || cfg->max_active < 0)
        return SL_ERR_ARG;
    if (cfg->precision != SL_FP64 && cfg->precision != SL_MIXED && cfg->precision != SL_FP32) return SL_ERR_ARG;
    *out = nullptr;
    if (cfg->device >= 0 && cudaSetDevice(cfg->device) != cudaSuccess) {
        cudaGetLastError();
        return SL_ERR_CUDA;
    }
    if (sl::ensure_loaded() != cudaSuccess) {  // no module load while requests run
        cudaGetLastError();
        return SL_ERR_CUDA;
    }
    int device = 0;
    cudaGetDevice(&device);
    {
        // reserve the budget: allocate it from the pool once and free it; the
        // pool keeps the memory mapped for the requests
        cudaStream_t st = nullptr;
        void *p = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&p, cfg->budget_bytes, sl::device_pool(device), st);
        if (e == cudaSuccess) e = cudaFreeAsync(p, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (st) cudaStreamDestroy(st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? SL_ERR_OOM : SL_ERR_CUDA;
        }
    }
    sl_server *s = new (std::nothrow) sl_server;
    if (!s) return SL_ERR_OOM;
    s->cfg = *cfg;
    s->device = device;
    int prio_least = 0, prio_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    s->prio_light = prio_greatest;
    s->prio_heavy = prio_least;
    s->scheduler = std::thread(scheduler, s);
    const int heavy_workers = cfg->heavy_slots > 0 ? cfg->heavy_slots : 2;
    for (int i = 0; i < kLightWorkers + heavy_workers; ++i)
        s->pool.emplace_back(pool_worker, s, int(i >= kLightWorkers));
    *out = s;
    return SL_OK;
}

int sl_server_submit(sl_server *s, const sl_instance *spec, int steps, long long *ticket)
{
    if (!s || !spec || steps < 1 || !(spec->dt > 0.0) || spec->dt_rule < 0 || spec->dt_rule > 2 ||
        (spec->dt_rule > 0 && spec->dt > 1.0))
        return SL_ERR_ARG;
    if (!spec->mesh.periodic[0] || (spec->mesh.dim == 2 && !spec->mesh.periodic[1]))
        return SL_ERR_UNSUPPORTED;  // requests carry no boundary values: periodic meshes only
    if ((spec->mesh.dim != 1 && spec->mesh.dim != 2) || spec->N < 2 || spec->N > sl::kMaxN ||
        spec->mesh.K[0] < 1 || (spec->mesh.dim == 2 && spec->mesh.K[1] < 1))
        return SL_ERR_ARG;  // (sizes of the nodal tables copied below)
    Request r;
    r.owner = s;
    r.spec = *spec;
    r.steps = steps;
    r.footprint = footprint_of(*spec, s->cfg.slice_steps);
    r.work = work_of(*spec);
    r.heavy = r.work > kHeavyWork;
    r.t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    r.ticket = s->next_ticket++;
    if (!s->any) {
        s->t_first = r.t_submit;
        s->any = true;
    }
    s->submitted++;
    s->queue.push_back(r.ticket);
    if (ticket) *ticket = r.ticket;
    own_tables(s->req.emplace(r.ticket, std::move(r)).first->second);
    wake_scheduler(s, true);
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

int sl_server_timing(sl_server *s, long long ticket, double *out)
{
    if (!s || !out) return SL_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->req.find(ticket);
    if (it == s->req.end()) return SL_ERR_ARG;
    const Request &r = it->second;
    if (r.state != 2) return SL_ERR_STATE;
    auto sec = [](Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); };
    out[0] = sec(r.t_submit, r.t_admit);
    out[1] = sec(r.t_admit, r.t_create);
    out[2] = sec(r.t_create, r.t_ready);
    out[3] = sec(r.t_ready, r.t_ran);
    out[4] = sec(r.t_ran, r.t_finish);
    out[5] = sec(r.t_finish, r.t_moments);
    out[6] = sec(r.t_moments, r.t_done);
    out[7] = sec(r.t_submit, r.t_done);
    out[8] = r.slice_max;
    return SL_OK;
}

int sl_server_wait_idle(sl_server *s, double timeout_s)
{
    if (!s) return SL_ERR_ARG;
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->queue.empty() && s->active == 0 && s->outstanding == 0) return SL_OK;
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
    out->running = s->active;
    out->queued = (long long)s->queue.size();
    out->esu_completed = s->esu_done;
    out->memory_in_use = (long long)s->used;
    out->memory_peak = (long long)s->peak;
    out->slices = s->slices;
    out->sched_busy_s = s->busy_s;
    out->launch_s = s->launch_s;
    out->launch_max_s = s->launch_max_s;
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
        s->tasks[0].clear();  // queued creations, heavy runs and completions are dropped
        s->tasks[1].clear();
    }
    s->cv.notify_all();
    s->task_cv[0].notify_all();
    s->task_cv[1].notify_all();
    if (s->scheduler.joinable()) s->scheduler.join();
    for (std::thread &t : s->pool) t.join();  // a task already running finishes
    // slices in flight (and their host callbacks) complete; their requests are abandoned
    for (auto &kv : s->req) {
        if (kv.second.st) cudaStreamSynchronize(kv.second.st);
        if (kv.second.ctx) sl_free(kv.second.ctx);
        if (kv.second.st) cudaStreamDestroy(kv.second.st);
    }
    if (cudaMemPool_t pool = sl::device_pool(s->device)) cudaMemPoolTrimTo(pool, 0);  // give back what is unused
    delete s;
}

}  // extern "C"
