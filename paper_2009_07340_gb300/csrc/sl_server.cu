// sl_server.cu -- a serving loop for drift-diffusion solves that arrive over
// time (host runtime around the solver; no kernels of its own).
//
// Requests (an sl_instance plus a step count) are queued on submission.  A
// scheduler thread runs rounds:
//   1. admission: queued requests are admitted in arrival order while their
//      device footprint (state, face buffer, Wiener scratch, moment
//      partials, node tables) fits in the memory budget next to the running
//      ones; a request larger than the whole budget is rejected;
//   2. every running request advances by up to `slice_steps` steps on one of
//      `streams` CUDA streams, so the requests' kernels overlap on the GPU;
//   3. after the streams drain, finished requests compute their moments,
//      release their memory and record their latency (completion minus
//      submission); new arrivals join at the next round (continuous batching).
// Each request is an independent solver context, so its result is the same
// as that of the request run alone (bitwise in SL_FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
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
    int state = 0;  // 0 queued, 1 running, 2 done, < 0 error code
    size_t footprint = 0;
    sl_ctx *ctx = nullptr;
    int stream = 0;
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

}  // namespace

struct sl_server {
    sl_server_config cfg;
    std::vector<cudaStream_t> streams;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<long long> queue;
    std::map<long long, Request> req;
    std::vector<long long> running;
    size_t used = 0, peak = 0;
    long long next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::vector<double> latencies;
    long long esu_done = 0, submitted = 0, completed = 0, rejected = 0, failed = 0;
    Clock::time_point t_first, t_last;
    bool any = false;
    int device = 0;
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
    r.t_done = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    s->used -= r.footprint;
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

void scheduler(sl_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<long long> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->queue.empty() || !s->running.empty(); });
            if (s->stop && s->running.empty()) return;
            while (!s->queue.empty()) {
                Request &r = s->req[s->queue.front()];
                if (r.footprint > s->cfg.budget_bytes) {
                    r.state = SL_ERR_OOM;
                    s->rejected++;
                    s->queue.pop_front();
                    continue;
                }
                if (s->used + r.footprint > s->cfg.budget_bytes) break;
                s->used += r.footprint;
                s->peak = std::max(s->peak, s->used);
                admit.push_back(r.ticket);
                s->queue.pop_front();
            }
        }
        // admission: contexts are created outside the lock
        for (long long t : admit) {
            Request *r;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                r = &s->req[t];
            }
            sl_options o = {};
            o.seed = r->spec.seed;
            o.precision = s->cfg.precision;
            o.device = -1;
            r->stream = int(t % (long long)s->streams.size());
            o.stream = s->streams[r->stream];
            const int rc = sl_init(&r->ctx, &r->spec.mesh, r->spec.N, r->spec.M, &r->spec.drift, &r->spec.diffusion,
                                   &r->spec.phi0, &o);
            if (rc != SL_OK) {
                r->ctx = nullptr;
                finish(s, *r, rc);
                continue;
            }
            r->esu = (long long)r->ctx->m.E * r->spec.M * r->steps;
            std::lock_guard<std::mutex> lk(s->mu);
            r->state = 1;
            s->running.push_back(t);
        }
        // one round: a slice of steps for every running request
        std::vector<Request *> run;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (long long t : s->running) run.push_back(&s->req[t]);
        }
        std::vector<int> rcs(run.size(), SL_OK);
        for (size_t i = 0; i < run.size(); ++i) {
            Request *r = run[i];
            const int n = std::min(s->cfg.slice_steps, r->steps - r->done_steps);
            if (n > 0) rcs[i] = sl_step(r->ctx, r->spec.dt, n);
            if (rcs[i] == SL_OK) r->done_steps += n;
        }
        for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
        std::vector<long long> still;
        for (size_t i = 0; i < run.size(); ++i) {
            Request *r = run[i];
            if (rcs[i] != SL_OK || r->done_steps >= r->steps)
                finish(s, *r, rcs[i]);
            else
                still.push_back(r->ticket);
        }
        std::lock_guard<std::mutex> lk(s->mu);
        s->running.swap(still);
    }
}

}  // namespace

extern "C" {

int sl_server_create(sl_server **out, const sl_server_config *cfg)
{
    if (!out || !cfg || cfg->slice_steps < 1 || cfg->streams < 1 || cfg->streams > 64 || cfg->budget_bytes == 0)
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
    for (int i = 0; i < cfg->streams; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return SL_ERR_CUDA;
        }
        s->streams.push_back(st);
    }
    s->worker = std::thread(scheduler, s);
    *out = s;
    return SL_OK;
}

int sl_server_submit(sl_server *s, const sl_instance *spec, int steps, long long *ticket)
{
    if (!s || !spec || steps < 1 || !(spec->dt > 0.0)) return SL_ERR_ARG;
    Request r;
    r.spec = *spec;
    r.steps = steps;
    r.footprint = footprint_of(*spec, s->cfg.slice_steps, s->cfg.precision);
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
            if (s->queue.empty() && s->running.empty()) return SL_OK;
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
    out->running = (long long)s->running.size();
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
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->req)
        if (kv.second.ctx) sl_free(kv.second.ctx);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"
