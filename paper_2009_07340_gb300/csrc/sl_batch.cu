// sl_batch.cu -- many independent solves of uneven size advanced together:
// one CUDA graph per call replays the whole multi-instance step.
//
// Instances are grouped into classes by (dimension, order N).  A call of
// sl_batch_step(b, steps) enqueues, in a graph captured once per `steps`:
//   1. one Wiener-increment kernel over every instance (device-side step
//      counters, so the replayed graph draws the next increments);
//   2. per 1D class, one persistent kernel: CTAs pull (instance, sample slot)
//      work items from an atomic counter and run all `steps` steps of an item
//      resident on chip (instances of any K <= 256, M, dt and fields mix);
//      1D instances with K > 256 get their own cluster launch;
//   3. per 2D class, two launches per step over the element-sample groups of
//      all instances of the class;
//   4. one kernel advancing the step counters.
// Steps 2 and 3 of different classes are independent (disjoint instances):
// they are spread over `lanes` streams forked from and joined back to the
// batch stream, so in the captured graph they are parallel branches and a
// small class can run beside a large one instead of after it.
// sl_batch_tune times, on the real instances, the persistent grid of each 1D
// class and then the number of branches (1, 2 or 4), restoring every
// instance's state afterwards.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <vector>

#include "sl_internal.cuh"

namespace {

struct Class1D {
    int N = 0;
    std::vector<int> ids;
    int grid = 0;       // persistent CTAs
    int max_grid = 0;   // occupancy limit
    size_t smem = 0;
    int *d_counter = nullptr;
};

struct Class2D {
    int N = 0;
    std::vector<int> ids;
    long long total = 0;
    long long groups = 0;        // element-sample groups of the class
    unsigned *d_slots = nullptr;  // [2 groups + 2]: the class's slot marks, list and list control
};

struct GraphSet {
    cudaGraphExec_t exec = nullptr;
    std::vector<void *> buffers;  // device argument tables referenced by the graph
};

}  // namespace

struct sl_batch {
    std::vector<sl_ctx *> inst;
    std::vector<double> dt;
    int precision = SL_FP64;
    cudaStream_t st = nullptr;
    std::vector<Class1D> c1;
    std::vector<Class2D> c2;
    std::vector<int> solo;  // 1D instances with K > 256 (cluster launches)
    long long *d_steps = nullptr;
    sl::WienerJob *d_jobs = nullptr;
    long long *d_jprefix = nullptr;
    int cap_steps = 0;
    std::map<int, GraphSet> graphs;
    int poisoned = 0;
    int nsm = 0;
    bool own_stream = false;  // graphs cannot be captured on the legacy default stream
    static constexpr int kMaxLanes = 4;
    int lanes = 1;                              // parallel branches of a step (sl_batch_tune)
    cudaStream_t lane_st[kMaxLanes] = {};       // branch streams (lane 0 is the batch stream itself)
    cudaEvent_t fork_ev = nullptr, join_ev[kMaxLanes] = {};
};

namespace {

int fail(sl_batch *b)
{
    cudaGetLastError();  // do not leave the error for unrelated later calls
    b->poisoned = 1;
    return SL_ERR_CUDA;
}

void drop_graphs(sl_batch *b)
{
    for (auto &g : b->graphs) {
        if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
        for (void *p : g.second.buffers) cudaFree(p);
    }
    b->graphs.clear();
}

// Wiener scratch of every instance for `steps` steps per call.
int ensure_capacity(sl_batch *b, int steps)
{
    if (steps <= b->cap_steps) return SL_OK;
    drop_graphs(b);
    for (sl_ctx *c : b->inst) {
        sl::ctx_free(c, c->dW);
        c->dW = nullptr;
        c->dW_cap = 0;
        if (sl::ctx_alloc(c, reinterpret_cast<void **>(&c->dW), size_t(steps) * c->M * c->m.dim * sizeof(double)) !=
            cudaSuccess) {
            cudaGetLastError();
            return SL_ERR_OOM;
        }
        c->dW_cap = steps;
    }
    b->cap_steps = steps;
    if (cudaStreamSynchronize(b->st) != cudaSuccess) return SL_ERR_CUDA;  // new buffers ready before use by the graph
    std::vector<sl::WienerJob> jobs(b->inst.size());
    for (size_t i = 0; i < b->inst.size(); ++i) {
        const sl_ctx *c = b->inst[i];
        jobs[i] = {c->seed, c->sample0, c->M, c->m.dim, std::sqrt(b->dt[i]), c->dW};
    }
    if (cudaMemcpy(b->d_jobs, jobs.data(), jobs.size() * sizeof(sl::WienerJob), cudaMemcpyHostToDevice) != cudaSuccess)
        return SL_ERR_CUDA;
    return SL_OK;
}

sl::Step1DArgs args1d(const sl_ctx *c, double dt, int steps)
{
    sl::Step1DArgs a;
    a.K = c->m.K[0];
    a.M = c->M;
    a.S = c->S;
    a.C = c->C;
    a.T = c->T;
    a.nsteps = steps;
    a.dt = dt;
    a.h = c->m.h[0];
    a.inv_w2 = c->inv_w2;
    a.periodic = 1;  // batches hold periodic, single-field instances only
    a.ncomp = 1;
    a.ghost = nullptr;
    a.xi = c->xi;
    a.nodeU = c->nodeU;
    a.nodeB = c->nodeB;
    a.nodeDiv = c->nodeDiv;
    a.faceU = c->faceU;
    a.faceB = c->faceB;
    a.dW = c->dW;
    a.Q = c->Q;
    a.err = c->err;
    return a;
}

sl::Step2DArgs args2d(const sl_ctx *c, double dt, int steps)
{
    sl::Step2DArgs a;
    a.Kx = c->m.K[0];
    a.Ky = c->m.K[1];
    a.M = c->M;
    a.nsteps = steps;
    a.dt = dt;
    a.hx = c->m.h[0];
    a.hy = c->m.h[1];
    a.s4x = 4.0 / c->m.h[0];
    a.s4y = 4.0 / c->m.h[1];
    a.xi = c->xi;
    a.tab = c->tab2d;
    a.fb = c->fb2d;
    a.nodeU = c->nodeU;
    a.nodeB = c->nodeB;
    a.nodeDiv = c->nodeDiv;
    a.faceU = c->faceU;
    a.faceB = c->faceB;
    a.dW = c->dW;
    a.Q = c->Q;
    a.faces = c->faces2d;
    a.alpha = c->alpha2d;
    a.coef = c->coef2d;  // formed for this dt at sl_batch_create
    a.err = c->err;
    a.w = c->bc_weight;
    a.periodic = 1;  // batches hold periodic instances only
    a.ghost = nullptr;
    a.ghost_w = 0;
    a.faceUhi = a.faceBhi = nullptr;
    a.chunk = 0;  // the batched launch covers all instances' groups
    a.g0 = a.g1 = 0;
    a.throttle = nullptr;
    return a;
}

template <typename T>
T *upload(const std::vector<T> &v, std::vector<void *> &keep)
{
    T *d = nullptr;
    if (cudaMalloc(&d, std::max<size_t>(1, v.size()) * sizeof(T)) != cudaSuccess) return nullptr;
    if (!v.empty() && cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    keep.push_back(d);
    return d;
}

cudaError_t launch_1d_class(const sl_batch *b, const Class1D &k, const sl::Batch1DLaunch &l, cudaStream_t st)
{
    if (b->precision == SL_FP64) return sl::launch_step1d_batch_fp64(l, k.N, st);
    if (b->precision == SL_MIXED) return sl::launch_step1d_batch_mixed(l, k.N, st);
    return sl::launch_step1d_batch_fp32(l, k.N, st);
}

size_t smem_1d(int precision, int N, int S, int T)
{
    if (precision == SL_FP64) return sl::step1d_smem_bytes_fp64(N, S, T);
    if (precision == SL_MIXED) return sl::step1d_smem_bytes_mixed(N, S, T);
    return sl::step1d_smem_bytes_fp32(N, S, T);
}

// Device argument tables of one multi-instance step of `steps` steps
// (allocated and uploaded before any capture; owned through `keep`).
struct StepTables {
    long long *jprefix = nullptr;
    long long jtotal = 0;
    std::vector<sl::Batch1DLaunch> l1;
    std::vector<sl::Batch2DLaunch> l2;
};

int prepare_step(sl_batch *b, int steps, StepTables &t, std::vector<void *> &keep)
{
    const int n = int(b->inst.size());
    std::vector<long long> jprefix(n + 1, 0);
    for (int i = 0; i < n; ++i) jprefix[i + 1] = jprefix[i] + (long long)steps * b->inst[i]->M;
    t.jprefix = upload(jprefix, keep);
    t.jtotal = jprefix[n];
    if (!t.jprefix) return SL_ERR_OOM;
    for (const Class1D &k : b->c1) {
        std::vector<sl::Step1DArgs> args;
        std::vector<int> prefix(1, 0);
        for (int id : k.ids) {
            args.push_back(args1d(b->inst[id], b->dt[id], steps));
            prefix.push_back(prefix.back() + (b->inst[id]->M + b->inst[id]->S - 1) / b->inst[id]->S);
        }
        sl::Batch1DLaunch l;
        l.args = upload(args, keep);
        l.prefix = upload(prefix, keep);
        if (!l.args || !l.prefix) return SL_ERR_OOM;
        l.ninst = int(k.ids.size());
        l.counter = k.d_counter;
        l.grid = k.grid;
        l.smem = k.smem;
        t.l1.push_back(l);
    }
    for (const Class2D &k : b->c2) {
        std::vector<sl::Step2DArgs> args;
        std::vector<long long> prefix(1, 0);
        for (int id : k.ids) {
            args.push_back(args2d(b->inst[id], b->dt[id], steps));
            args.back().slot_mark = k.d_slots;  // the class's groups share one slot list
            args.back().slot_list = k.d_slots + k.groups;
            args.back().slot_ctl = k.d_slots + 2 * k.groups;
            prefix.push_back(prefix.back() + (long long)b->inst[id]->m.E * b->inst[id]->M);
        }
        sl::Batch2DLaunch l;
        l.args = upload(args, keep);
        l.prefix = upload(prefix, keep);
        if (!l.args || !l.prefix) return SL_ERR_OOM;
        l.ninst = int(k.ids.size());
        l.total_groups = prefix.back();
        l.nsteps = steps;
        l.f64_factor = b->precision == SL_MIXED;
        t.l2.push_back(l);
    }
    return SL_OK;
}

// Enqueues the step on b->st: kernel launches, events and stream waits only,
// so it can be captured into a graph.  The classes' launches go to b->lanes
// branch streams forked from b->st after the Wiener kernel and joined back
// before the counters advance; each class goes to the branch with the least
// estimated work so far, in decreasing order of work.
int enqueue_step(sl_batch *b, int steps, const StepTables &t)
{
    const int n = int(b->inst.size());
    if (sl::launch_wiener_batch(b->d_jobs, t.jprefix, n, steps, b->d_steps, t.jtotal, b->st) != cudaSuccess)
        return SL_ERR_CUDA;
    const int L = std::max(1, std::min(b->lanes, sl_batch::kMaxLanes));
    b->lane_st[0] = b->st;
    if (L > 1) {
        if (cudaEventRecord(b->fork_ev, b->st) != cudaSuccess) return SL_ERR_CUDA;
        for (int l = 1; l < L; ++l)
            if (cudaStreamWaitEvent(b->lane_st[l], b->fork_ev, 0) != cudaSuccess) return SL_ERR_CUDA;
    }
    // work items: (estimated element-sample-node work, kind, index)
    struct Item {
        double work;
        int kind, idx;
    };
    std::vector<Item> items;
    auto work_of = [&](int id) {
        const sl_ctx *c = b->inst[id];
        const double nn = double(c->m.n);
        return double(c->m.E) * c->M * (c->m.dim == 1 ? nn * nn : nn * nn * nn);
    };
    for (size_t i = 0; i < b->c1.size(); ++i) {
        double w = 0.0;
        for (int id : b->c1[i].ids) w += work_of(id);
        items.push_back({w, 1, int(i)});
    }
    for (int id : b->solo) items.push_back({work_of(id), 0, id});
    for (size_t i = 0; i < b->c2.size(); ++i) {
        double w = 0.0;
        for (int id : b->c2[i].ids) w += work_of(id);
        items.push_back({w, 2, int(i)});
    }
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.work > y.work; });
    double load[sl_batch::kMaxLanes] = {};
    for (const Item &it : items) {
        int l = 0;
        for (int k = 1; k < L; ++k)
            if (load[k] < load[l]) l = k;
        load[l] += it.work;
        cudaStream_t st = b->lane_st[l];
        cudaError_t e = cudaSuccess;
        if (it.kind == 1) {
            e = launch_1d_class(b, b->c1[it.idx], t.l1[it.idx], st);
        } else if (it.kind == 0) {
            const int id = it.idx;
            const sl::Step1DArgs a = args1d(b->inst[id], b->dt[id], steps);
            if (b->precision == SL_FP64) e = sl::launch_step1d_fp64(a, b->inst[id]->m.N, st);
            else if (b->precision == SL_MIXED) e = sl::launch_step1d_mixed(a, b->inst[id]->m.N, st);
            else e = sl::launch_step1d_fp32(a, b->inst[id]->m.N, st);
        } else {
            e = b->precision == SL_FP64 ? sl::launch_step2d_batch_fp64(t.l2[it.idx], b->c2[it.idx].N, st)
                                        : sl::launch_step2d_batch_fp32(t.l2[it.idx], b->c2[it.idx].N, st);
            if (e == cudaErrorNotSupported) return SL_ERR_UNSUPPORTED;
        }
        if (e != cudaSuccess) return SL_ERR_CUDA;
    }
    for (int l = 1; l < L; ++l)
        if (cudaEventRecord(b->join_ev[l], b->lane_st[l]) != cudaSuccess ||
            cudaStreamWaitEvent(b->st, b->join_ev[l], 0) != cudaSuccess)
            return SL_ERR_CUDA;
    if (sl::launch_advance_counters(b->d_steps, n, steps, b->st) != cudaSuccess) return SL_ERR_CUDA;
    return SL_OK;
}

}  // namespace

extern "C" {

void sl_batch_free(sl_batch *b)
{
    if (!b) return;
    drop_graphs(b);
    for (sl_ctx *c : b->inst) sl_free(c);
    for (Class1D &k : b->c1) cudaFree(k.d_counter);
    for (Class2D &k : b->c2) cudaFree(k.d_slots);
    for (int l = 1; l < sl_batch::kMaxLanes; ++l) {
        if (b->lane_st[l]) cudaStreamDestroy(b->lane_st[l]);
        if (b->join_ev[l]) cudaEventDestroy(b->join_ev[l]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    cudaFree(b->d_steps);
    cudaFree(b->d_jobs);
    cudaFree(b->d_jprefix);
    if (b->own_stream) cudaStreamDestroy(b->st);
    delete b;
}

int sl_batch_create(sl_batch **out, int count, const sl_instance *specs, const sl_options *opt)
{
    if (!out || count < 1 || !specs) return SL_ERR_ARG;
    *out = nullptr;
    sl_batch *b = new (std::nothrow) sl_batch;
    if (!b) return SL_ERR_OOM;
    sl_options o = opt ? *opt : sl_options{};
    if (!opt) o.device = -1;
    b->precision = o.precision;
    if (o.device >= 0 && cudaSetDevice(o.device) != cudaSuccess) {
        delete b;
        return SL_ERR_CUDA;
    }
    b->st = static_cast<cudaStream_t>(o.stream);
    if (!b->st) {
        if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return SL_ERR_CUDA;
        }
        b->own_stream = true;
        o.stream = b->st;
    }
    for (int i = 0; i < count; ++i) {
        const sl_instance &s = specs[i];
        if (!(s.dt > 0.0) || !std::isfinite(s.dt) || s.dt_rule < 0 || s.dt_rule > 2 || (s.dt_rule > 0 && s.dt > 1.0)) {
            sl_batch_free(b);
            return SL_ERR_ARG;
        }
        if (!s.mesh.periodic[0] || (opt && opt->components > 1)) {  // these run alone (sl_init)
            sl_batch_free(b);
            return SL_ERR_UNSUPPORTED;
        }
        sl_options oi = o;
        oi.seed = s.seed;
        oi.sample0 = 0;
        if (s.bc_weight != 0.0) oi.bc_weight = s.bc_weight;
        sl_ctx *c = nullptr;
        const int rc = sl_init(&c, &s.mesh, s.N, s.M, &s.drift, &s.diffusion, &s.phi0, &oi);
        if (rc != SL_OK) {
            sl_batch_free(b);
            return rc;
        }
        const double dt = s.dt_rule == 0 ? s.dt : s.dt * (s.dt_rule == 1 ? c->dtmax : c->dtedge);
        if (o.strict_dt && dt > c->dtmax * (1.0 + 1e-12)) {
            sl_free(c);
            sl_batch_free(b);
            return SL_ERR_DT;
        }
        if (sl::ensure_coef2d(c, dt) != cudaSuccess) {
            sl_free(c);
            sl_batch_free(b);
            return SL_ERR_CUDA;
        }
        b->inst.push_back(c);
        b->dt.push_back(dt);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    std::map<int, int> idx1, idx2;
    for (int i = 0; i < count; ++i) {
        const sl_ctx *c = b->inst[i];
        if (c->m.dim == 1 && c->C > 1) {
            b->solo.push_back(i);
        } else if (c->m.dim == 1) {
            if (!idx1.count(c->m.N)) {
                idx1[c->m.N] = int(b->c1.size());
                b->c1.emplace_back();
                b->c1.back().N = c->m.N;
            }
            b->c1[idx1[c->m.N]].ids.push_back(i);
        } else {
            if (!idx2.count(c->m.N)) {
                idx2[c->m.N] = int(b->c2.size());
                b->c2.emplace_back();
                b->c2.back().N = c->m.N;
            }
            b->c2[idx2[c->m.N]].ids.push_back(i);
        }
    }
    for (Class1D &k : b->c1) {
        for (int id : k.ids) k.smem = std::max(k.smem, smem_1d(b->precision, k.N, b->inst[id]->S, b->inst[id]->T));
        if (cudaMalloc(&k.d_counter, sizeof(int)) != cudaSuccess) {
            sl_batch_free(b);
            return SL_ERR_OOM;
        }
        k.max_grid = 2 * b->nsm;  // refined by sl_batch_tune
        k.grid = b->nsm;
    }
    for (Class2D &k : b->c2) {
        for (int id : k.ids) k.groups += (long long)b->inst[id]->m.E * b->inst[id]->M;
        const size_t bytes = (2 * size_t(k.groups) + 2) * sizeof(unsigned);
        if (cudaMalloc(&k.d_slots, bytes) != cudaSuccess || cudaMemset(k.d_slots, 0, bytes) != cudaSuccess) {
            sl_batch_free(b);
            return SL_ERR_OOM;
        }
    }
    if (cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess) {
        sl_batch_free(b);
        return SL_ERR_CUDA;
    }
    for (int l = 1; l < sl_batch::kMaxLanes; ++l)
        if (cudaStreamCreateWithFlags(&b->lane_st[l], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join_ev[l], cudaEventDisableTiming) != cudaSuccess) {
            sl_batch_free(b);
            return SL_ERR_CUDA;
        }
    if (cudaMalloc(&b->d_steps, count * sizeof(long long)) != cudaSuccess ||
        cudaMemset(b->d_steps, 0, count * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&b->d_jobs, count * sizeof(sl::WienerJob)) != cudaSuccess) {
        sl_batch_free(b);
        return SL_ERR_OOM;
    }
    *out = b;
    return SL_OK;
}

int sl_batch_step(sl_batch *b, int steps)
{
    sl::TraceRange trace("sl_batch_step");
    if (!b || steps < 0) return SL_ERR_ARG;
    if (b->poisoned) return SL_ERR_STATE;
    if (steps == 0) return SL_OK;
    int rc = ensure_capacity(b, steps);
    if (rc != SL_OK) return rc;
    auto it = b->graphs.find(steps);
    if (it == b->graphs.end()) {
        GraphSet gs;
        StepTables tables;
        rc = prepare_step(b, steps, tables, gs.buffers);
        if (rc != SL_OK) {
            for (void *p : gs.buffers) cudaFree(p);
            return rc;
        }
        // the kernels' one-time attribute setup happens outside the capture
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeRelaxed) != cudaSuccess) return fail(b);
        rc = enqueue_step(b, steps, tables);
        const cudaError_t ec = cudaStreamEndCapture(b->st, &g);
        if (rc != SL_OK || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            for (void *p : gs.buffers) cudaFree(p);
            cudaGetLastError();
            return rc != SL_OK ? rc : fail(b);
        }
        const cudaError_t ei = cudaGraphInstantiate(&gs.exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            for (void *p : gs.buffers) cudaFree(p);
            return fail(b);
        }
        it = b->graphs.emplace(steps, std::move(gs)).first;
    }
    if (cudaGraphLaunch(it->second.exec, b->st) != cudaSuccess) return fail(b);
    for (sl_ctx *c : b->inst) c->step += steps;
    return SL_OK;
}

int sl_batch_tune(sl_batch *b, int probe_steps, double *best_ms)
{
    if (!b || probe_steps < 1) return SL_ERR_ARG;
    if (b->poisoned) return SL_ERR_STATE;
    int rc = ensure_capacity(b, std::max(probe_steps, b->cap_steps));
    if (rc != SL_OK) return rc;
    // save every instance's state and counters
    std::vector<void *> saved(b->inst.size(), nullptr);
    for (size_t i = 0; i < b->inst.size(); ++i) {
        const sl_ctx *c = b->inst[i];
        const size_t bytes = size_t(c->M) * c->m.E * c->m.n * c->state_elem;
        if (cudaMalloc(&saved[i], bytes) != cudaSuccess ||
            cudaMemcpyAsync(saved[i], c->Q, bytes, cudaMemcpyDeviceToDevice, b->st) != cudaSuccess) {
            for (void *p : saved) cudaFree(p);
            cudaGetLastError();
            return SL_ERR_OOM;
        }
    }
    std::vector<long long> steps_host(b->inst.size());
    cudaMemcpy(steps_host.data(), b->d_steps, steps_host.size() * sizeof(long long), cudaMemcpyDeviceToHost);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double total_best = 0.0;
    for (Class1D &k : b->c1) {
        int per_sm = 0;
        auto kernel_probe_grid = [&](int grid) -> float {
            k.grid = grid;
            std::vector<void *> keep;
            // enqueue this class alone: hide the other classes of b meanwhile
            std::vector<Class1D> c1_all;
            c1_all.swap(b->c1);
            std::vector<Class2D> c2_all;
            c2_all.swap(b->c2);
            std::vector<int> solo_all;
            solo_all.swap(b->solo);
            b->c1.push_back(k);
            StepTables tables;
            int r = prepare_step(b, probe_steps, tables, keep);
            cudaEventRecord(e0, b->st);
            if (r == SL_OK) r = enqueue_step(b, probe_steps, tables);
            cudaEventRecord(e1, b->st);
            cudaEventSynchronize(e1);
            b->c1.swap(c1_all);
            b->c2.swap(c2_all);
            b->solo.swap(solo_all);
            for (void *p : keep) cudaFree(p);
            float ms = -1.f;
            if (r == SL_OK) cudaEventElapsedTime(&ms, e0, e1);
            return r == SL_OK ? ms : -1.f;
        };
        // occupancy bound of the persistent kernel: at most 4 CTAs per SM
        // (256 threads each), fewer when shared memory is the limit
        per_sm = std::max(1, std::min(4, int((227 * 1024) / std::max<size_t>(k.smem + 1024, 1))));
        k.max_grid = per_sm * b->nsm;
        int best = b->nsm;
        float best_t = 1e30f;
        for (int m = 1; m <= per_sm; ++m) {
            const float t = kernel_probe_grid(m * b->nsm);
            if (t > 0.f && t < best_t) {
                best_t = t;
                best = m * b->nsm;
            }
        }
        k.grid = best;
        total_best += best_t;
    }
    // the number of parallel branches, timed on whole steps
    {
        int best_l = 1;
        float best_t = 1e30f;
        for (int L : {1, 2, 4}) {
            b->lanes = L;
            std::vector<void *> keep;
            StepTables tables;
            int r = prepare_step(b, probe_steps, tables, keep);
            cudaEventRecord(e0, b->st);
            if (r == SL_OK) r = enqueue_step(b, probe_steps, tables);
            cudaEventRecord(e1, b->st);
            cudaEventSynchronize(e1);
            for (void *p : keep) cudaFree(p);
            float ms = -1.f;
            if (r == SL_OK) cudaEventElapsedTime(&ms, e0, e1);
            if (ms > 0.f && ms < best_t) {
                best_t = ms;
                best_l = L;
            }
        }
        b->lanes = best_l;
        total_best = best_t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // restore states and counters; graphs captured before tuning are stale
    for (size_t i = 0; i < b->inst.size(); ++i) {
        const sl_ctx *c = b->inst[i];
        const size_t bytes = size_t(c->M) * c->m.E * c->m.n * c->state_elem;
        cudaMemcpyAsync(c->Q, saved[i], bytes, cudaMemcpyDeviceToDevice, b->st);
    }
    cudaMemcpyAsync(b->d_steps, steps_host.data(), steps_host.size() * sizeof(long long), cudaMemcpyHostToDevice,
                    b->st);
    const cudaError_t e = cudaStreamSynchronize(b->st);
    for (void *p : saved) cudaFree(p);
    drop_graphs(b);
    if (best_ms) *best_ms = total_best;
    return e == cudaSuccess ? SL_OK : fail(b);
}

int sl_batch_grid(const sl_batch *b, int cls, int *N, int *grid, int *instances)
{
    if (!b || cls < 0 || cls >= int(b->c1.size())) return SL_ERR_ARG;
    if (N) *N = b->c1[cls].N;
    if (grid) *grid = b->c1[cls].grid;
    if (instances) *instances = int(b->c1[cls].ids.size());
    return SL_OK;
}

int sl_batch_lanes(const sl_batch *b, int *lanes)
{
    if (!b || !lanes) return SL_ERR_ARG;
    *lanes = b->lanes;
    return SL_OK;
}

int sl_batch_moments(sl_batch *b, int i, double *mean, double *m2)
{
    if (!b || i < 0 || i >= int(b->inst.size())) return SL_ERR_ARG;
    if (b->poisoned) return SL_ERR_STATE;
    return sl_moments(b->inst[i], mean, m2);
}

int sl_batch_samples(sl_batch *b, int i, int s0, int count, double *out)
{
    if (!b || i < 0 || i >= int(b->inst.size())) return SL_ERR_ARG;
    if (b->poisoned) return SL_ERR_STATE;
    return sl_get_samples(b->inst[i], s0, count, out);
}

}  // extern "C"
