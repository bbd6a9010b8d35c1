// sl_api.cu -- the C ABI declared in include/sl.h: argument checking, device
// memory ownership, launch geometry and the step loop.  All arithmetic of the
// method runs in the kernels of sl_step1d*.cu, sl_step2d.cu and sl_setup.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "sl_internal.cuh"


namespace {

constexpr size_t kWienerScratchBytes = size_t(64) << 20;

int fail_cuda(sl_ctx *c)
{
    cudaGetLastError();  // do not leave the error for unrelated later calls
    if (c) c->poisoned = 1;
    return SL_ERR_CUDA;
}

bool valid_kind(int dim, int what, const sl_field *f)
{
    if (!f) return false;
    const int k = f->kind;
    if (what == 0)
        return k == SL_U_CONST || (dim == 1 && k == SL_U_SIN) || (dim == 2 && k == SL_U_ROTATION) ||
               (k == SL_U_NODAL && f->nodal != nullptr);
    if (what == 1)
        return k == SL_D_CONST || k == SL_D_COS || (dim == 2 && k == SL_D_SINSIN) ||
               (k == SL_D_NODAL && f->nodal != nullptr);
    if (k == SL_PHI_NODAL) return f->nodal != nullptr;
    if (k == SL_PHI_FOURIER) return dim == 1 && f->p[2] >= 0 && f->p[2] <= 18;
    return k == SL_PHI_GAUSS || (dim == 1 && k == SL_PHI_SINE) || (dim == 2 && k == SL_PHI_SINSIN);
}

// Entries of the interface table of a nodal field (1D K+1; 2D vertical
// K1 (K0+1) N then horizontal (K1+1) K0 N).
long long n_iface(int dim, int K0, int K1, int N)
{
    return dim == 1 ? K0 + 1 : (long long)K1 * (K0 + 1) * N + (long long)(K1 + 1) * K0 * N;
}

// D >= 0 (NaN refused): analytic kinds by their parameters, nodal ones at
// every node and every interface-table entry that is read (on a periodic
// mesh the last interface of each line is not).
bool diffusion_ok(const sl_field *f, int dim, int K0, int K1, int N, bool periodic)
{
    if (f->kind != SL_D_NODAL) return f->p[0] >= 0.0 && (f->kind == SL_D_CONST || std::fabs(f->p[1]) <= 1.0);
    const long long V = (long long)K0 * K1 * (dim == 2 ? N * N : N);
    for (long long v = 0; v < V; ++v)
        if (!(f->nodal[v] >= 0.0)) return false;
    if (!f->face) return true;
    const long long nif = n_iface(dim, K0, K1, N), nvert = dim == 1 ? K0 + 1 : (long long)K1 * (K0 + 1) * N;
    for (long long i = 0; i < nif; ++i) {
        bool last;
        if (dim == 1) last = i == K0;
        else if (i < nvert) last = (i / N) % (K0 + 1) == K0;
        else last = (i - nvert) / ((long long)K0 * N) == K1;
        if (periodic && last) continue;
        if (!(f->face[i] >= 0.0)) return false;
    }
    return true;
}

sl::FieldDev to_dev(const sl_field *f)
{
    sl::FieldDev d = {};
    d.kind = f->kind;
    std::memcpy(d.p, f->p, sizeof(d.p));
    return d;
}

template <typename T>
cudaError_t dalloc(const sl_ctx *c, T **p, size_t count)
{
    return sl::ctx_alloc(c, reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
}

// Device copies of a nodal drift's or diffusion's tables for the setup
// kernels (nvals node values, nif interface entries), stream-ordered on the
// context's stream; unstage_nodal frees them after those kernels.
cudaError_t stage_nodal(const sl_ctx *c, const sl_field *f, long long nvals, long long nif, sl::FieldDev &d)
{
    if (f->kind != SL_U_NODAL && f->kind != SL_D_NODAL) return cudaSuccess;
    double *a = nullptr, *b = nullptr;
    cudaError_t e = dalloc(c, &a, size_t(nvals));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(a, f->nodal, size_t(nvals) * sizeof(double), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess && f->face) {
        e = dalloc(c, &b, size_t(nif));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b, f->face, size_t(nif) * sizeof(double), cudaMemcpyHostToDevice, c->st);
    }
    d.nodal = a;
    d.face = b;
    return e;
}

void unstage_nodal(const sl_ctx *c, sl::FieldDev &d)
{
    sl::ctx_free(c, const_cast<double *>(d.nodal));
    sl::ctx_free(c, const_cast<double *>(d.face));
    d.nodal = d.face = nullptr;
}

// Node and face coefficients of the current drift and diffusion (the setup
// kernels), nodal tables staged for the duration.
cudaError_t set_coefficients(sl_ctx *c, const sl_field *drift, const sl_field *diffusion, const sl_field *phi0,
                             const double *phi0_nodal_dev, bool write_state, bool device_tables = false)
{
    const sl::Mesh &m = c->m;
    const long long V = (long long)m.E * m.n, nif = n_iface(m.dim, m.K[0], m.K[1], m.N);
    sl::FieldDev du = to_dev(drift), dD = to_dev(diffusion);
    cudaError_t e = cudaSuccess;
    if (device_tables) {  // the caller's device tables, read in place by the kernels below
        du.nodal = drift->nodal;
        du.face = drift->face;
        dD.nodal = diffusion->nodal;
        dD.face = diffusion->face;
        dD.err = c->err;
    } else {
        e = stage_nodal(c, drift, m.dim * V, nif, du);
        if (e == cudaSuccess) e = stage_nodal(c, diffusion, V, nif, dD);
    }
    ++c->fields_version;  // the 2D advance coefficients are formed again at the next step
    if (e == cudaSuccess)
        e = sl::launch_init_fields(m, du, dD, to_dev(phi0), phi0_nodal_dev, c->xi, c->nodeU, c->nodeB, c->nodeDiv,
                                   c->faceU, c->faceB, write_state ? c->Q : nullptr, c->M * c->ncomp,
                                   c->precision == SL_FP64, c->st);  // [M][ncomp] fields of E n values
    if (e == cudaSuccess && m.dim == 2) e = sl::launch_init_faces_hi(m, du, dD, c->faceUhi, c->faceBhi, c->st);
    if (!device_tables) {
        unstage_nodal(c, du);
        unstage_nodal(c, dD);
    }
    return e;
}

// Chebyshev-Gauss nodes (host copy for the time-step guards only).
double host_min_gap(int N)
{
    double g = 1.0;
    for (int i = 0; i + 1 < N; ++i) {
        const double a = 0.5 * (1.0 - std::cos((i + 0.5) * M_PI / N));
        const double b = 0.5 * (1.0 - std::cos((i + 1.5) * M_PI / N));
        g = std::min(g, b - a);
    }
    return g;
}

double host_edge_gap(int N) { return 0.5 * (1.0 - std::cos(0.5 * M_PI / N)); }

// Largest dt with |u|max dt + sqrt(2 Dmax dt) <= dx in direction d (Eq. 1d_timestep).
double step_bound(double umax, double bmax, double dx)
{
    if (umax == 0.0) return bmax > 0.0 ? dx * dx / (bmax * bmax) : INFINITY;
    const double s = (-bmax + std::sqrt(bmax * bmax + 4.0 * umax * dx)) / (2.0 * umax);
    return s * s;
}

}  // namespace

namespace sl {

namespace {
std::mutex g_load_mu;
unsigned long long g_loaded = 0;  // bit d: device d's kernels are prepared and its pool exists
cudaMemPool_t g_pool[64] = {};
}  // namespace

cudaMemPool_t device_pool(int device)
{
    return device >= 0 && device < 64 ? g_pool[device] : nullptr;
}

cudaError_t ensure_loaded()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    const unsigned long long bit = 1ull << dev;
    std::lock_guard<std::mutex> lk(g_load_mu);
    if (g_loaded & bit) return cudaSuccess;
    e = preload_setup();
    if (e == cudaSuccess) e = preload_step1d_fp64();
    if (e == cudaSuccess) e = preload_step1d_mixed();
    if (e == cudaSuccess) e = preload_step1d_fp32();
    if (e == cudaSuccess) e = preload_step2d_fp64();
    if (e == cudaSuccess) e = preload_step2d_fp32();
    if (e == cudaSuccess) e = preload_step2d_c2();
    if (e == cudaSuccess && !g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&g_pool[dev], &props);
        if (e == cudaSuccess) {
            unsigned long long keep = ~0ull;  // no release at synchronisation points
            e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        if (e == cudaSuccess) {
            // A block freed on one stream but not yet reached there is never
            // handed to another stream: that reuse would make the allocating
            // stream wait for the freeing one (a light solver created while a
            // heavy one's queue is long).  Blocks whose free has executed are
            // still reused across streams.
            int no = 0;
            e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolReuseAllowInternalDependencies, &no);
        }
    }
    if (e == cudaSuccess) g_loaded |= bit;
    return e;
}

}  // namespace sl

namespace {

// The time-step bounds (Eq. 1d_timestep with the node gap, and with the edge
// distance) from the current node coefficients (host copy; synchronises the
// context's stream).
int refresh_bounds(sl_ctx *c)
{
    const sl::Mesh &m = c->m;
    const int dim = m.dim, N = m.N;
    const long long V = (long long)m.E * m.n;
    std::vector<double> hu(size_t(dim) * V), hb(V);
    cudaError_t e = cudaMemcpyAsync(hu.data(), c->nodeU, hu.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hb.data(), c->nodeB, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return SL_ERR_CUDA;
    double best = INFINITY, best_edge = INFINITY;
    const double gap = host_min_gap(N), edge = host_edge_gap(N);
    double bmax = 0.0;
    for (double b : hb) bmax = std::max(bmax, b);
    for (int d = 0; d < dim; ++d) {
        double umax = 0.0;
        for (long long v = 0; v < V; ++v) umax = std::max(umax, std::fabs(hu[size_t(d) * V + v]));
        best = std::min(best, step_bound(umax, bmax, gap * m.h[d]));
        best_edge = std::min(best_edge, step_bound(umax, bmax, edge * m.h[d]));
    }
    c->dtmax = best;
    c->dtedge = best_edge;
    return SL_OK;
}

}  // namespace

namespace sl {
// The 2D advance coefficients for step size dt, formed on the context's
// stream when the step size or the fields changed since the last time.
cudaError_t ensure_coef2d(sl_ctx *c, double dt)
{
    if (c->m.dim != 2 || (c->coef2d_dt == dt && c->coef2d_version == c->fields_version)) return cudaSuccess;
    const cudaError_t e = launch_coef2d(c->nodeU, c->nodeB, c->nodeDiv, (long long)c->m.E * c->m.n, dt,
                                        4.0 / c->m.h[0], 4.0 / c->m.h[1], c->precision == SL_FP64, c->coef2d, c->st);
    if (e == cudaSuccess) {
        c->coef2d_dt = dt;
        c->coef2d_version = c->fields_version;
    }
    return e;
}
}  // namespace sl

extern "C" {

int sl_preload(int device)
{
    if (device >= 0 && cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SL_ERR_CUDA;
    }
    if (sl::ensure_loaded() != cudaSuccess) {
        cudaGetLastError();
        return SL_ERR_CUDA;
    }
    return SL_OK;
}

const char *sl_strerror(int code)
{
    switch (code) {
    case SL_OK: return "ok";
    case SL_ERR_ARG: return "invalid argument";
    case SL_ERR_DT: return "time step above the particle-gap bound";
    case SL_ERR_OOM: return "device allocation failed";
    case SL_ERR_CUDA: return "CUDA error";
    case SL_ERR_SINGULAR: return "non-finite remap (coincident advected particles)";
    case SL_ERR_TIMEOUT: return "bounded device wait expired";
    case SL_ERR_STATE: return "context poisoned by an earlier error";
    case SL_ERR_UNSUPPORTED: return "not supported";
    default: return "unknown error";
    }
}

void sl_free(sl_ctx *c)
{
    if (!c) return;
    for (auto &ev : c->events) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    for (cudaEvent_t ev : c->throttle.ev)
        if (ev) cudaEventDestroy(ev);
    sl::ctx_free(c, c->ghost);
    sl::ctx_free(c, c->faceUhi);
    sl::ctx_free(c, c->faceBhi);
    sl::ctx_free(c, c->xi);
    sl::ctx_free(c, c->nodeU);
    sl::ctx_free(c, c->nodeB);
    sl::ctx_free(c, c->nodeDiv);
    sl::ctx_free(c, c->faceU);
    sl::ctx_free(c, c->faceB);
    sl::ctx_free(c, c->Q);
    sl::ctx_free(c, c->dW);
    sl::ctx_free(c, c->psum);
    sl::ctx_free(c, c->psq);
    sl::ctx_free(c, c->mean_tmp);
    sl::ctx_free(c, c->m2_tmp);
    sl::ctx_free(c, c->err);
    sl::ctx_free(c, c->faces2d);
    sl::ctx_free(c, c->tab2d);
    sl::ctx_free(c, c->alpha2d);
    sl::ctx_free(c, c->coef2d);
    sl::ctx_free(c, c->fb2d);
    sl::ctx_free(c, c->fbcount2d);
    sl::ctx_free(c, c->slots2d);
    delete c;
}

int sl_init(sl_ctx **out, const sl_mesh *mesh, int N, int M, const sl_field *drift, const sl_field *diffusion,
            const sl_field *phi0, const sl_options *opt)
{
    sl::TraceRange trace("sl_init");
    if (!out) return SL_ERR_ARG;
    *out = nullptr;
    if (!mesh || (mesh->dim != 1 && mesh->dim != 2)) return SL_ERR_ARG;
    const int dim = mesh->dim;
    if (N < 2 || N > sl::kMaxN || M < 1) return SL_ERR_ARG;
    for (int d = 0; d < dim; ++d) {
        if (mesh->K[d] < 1 || !(mesh->hi[d] > mesh->lo[d]) || !std::isfinite(mesh->hi[d] - mesh->lo[d]))
            return SL_ERR_ARG;
        if (dim == 2 && !mesh->periodic[d] != !mesh->periodic[0]) return SL_ERR_UNSUPPORTED;  // all or none
    }
    if (!valid_kind(dim, 0, drift) || !valid_kind(dim, 1, diffusion) || !valid_kind(dim, 2, phi0))
        return SL_ERR_ARG;
    if (!diffusion_ok(diffusion, dim, mesh->K[0], dim == 2 ? mesh->K[1] : 1, N, mesh->periodic[0] != 0))
        return SL_ERR_ARG;
    const int precision = opt ? opt->precision : SL_FP64;
    if (precision != SL_FP64 && precision != SL_MIXED && precision != SL_FP32) return SL_ERR_ARG;
    if (dim == 1 && mesh->K[0] > sl::kMaxThreads1D * sl::kMaxCluster1D) return SL_ERR_UNSUPPORTED;
    if (dim == 2 && N > (precision == SL_FP64 ? 11 : 12)) return SL_ERR_UNSUPPORTED;
    if (opt && (opt->sample0 < 0 || opt->sample0 + M > (1ll << 32))) return SL_ERR_ARG;
    const double bc_w = opt && opt->bc_weight > 0.0 ? opt->bc_weight : 1.0;
    if (opt && std::isnan(opt->bc_weight)) return SL_ERR_ARG;
    if (dim == 2 && std::isinf(bc_w)) return SL_ERR_UNSUPPORTED;  // hard constraints: 1D only
    if (opt && opt->reseed_every < 0) return SL_ERR_ARG;
    const int ncomp = opt && opt->components > 1 ? opt->components : 1;
    if (opt && (opt->components < 0 || opt->components > 2)) return SL_ERR_UNSUPPORTED;
    if (ncomp > 1 && (!mesh->periodic[0] || (dim == 1 && precision == SL_MIXED) || (dim == 2 && N > 8)))
        return SL_ERR_UNSUPPORTED;  // two fields: periodic; 1D FP64 / FP32; 2D N <= 8 (any precision)

    if (opt && opt->device >= 0 && cudaSetDevice(opt->device) != cudaSuccess) return SL_ERR_CUDA;
    if (sl::ensure_loaded() != cudaSuccess) {
        cudaGetLastError();
        return SL_ERR_CUDA;
    }
    sl_ctx *c = new (std::nothrow) sl_ctx;
    if (!c) return SL_ERR_OOM;
    cudaGetDevice(&c->device);
    c->precision = precision;
    c->seed = opt ? opt->seed : 0ull;
    c->sample0 = opt ? opt->sample0 : 0ll;
    c->strict_dt = opt ? opt->strict_dt : 0;
    c->launch_chunk = opt && opt->launch_chunk > 0 ? opt->launch_chunk : 0;
    c->bc_weight = bc_w;
    c->periodic = mesh->periodic[0] ? 1 : 0;
    c->ghost_w = dim == 1 ? 2 : 2 * (mesh->K[0] + mesh->K[1]) * N;
    c->reseed_every = opt ? opt->reseed_every : 0;
    c->ncomp = ncomp;
    c->inv_w2 = std::isinf(bc_w) ? 0.0 : 1.0 / (bc_w * bc_w);
    if (c->launch_chunk > 0)
        for (cudaEvent_t &ev : c->throttle.ev)
            if (cudaEventCreateWithFlags(&ev, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                sl_free(c);
                return SL_ERR_CUDA;
            }
    c->st = opt ? static_cast<cudaStream_t>(opt->stream) : nullptr;
    c->M = M;
    sl::Mesh &m = c->m;
    m.dim = dim;
    m.N = N;
    m.n = dim == 2 ? N * N : N;
    m.K[0] = mesh->K[0];
    m.K[1] = dim == 2 ? mesh->K[1] : 1;
    m.E = m.K[0] * m.K[1];
    for (int d = 0; d < 2; ++d) {
        m.lo[d] = d < dim ? mesh->lo[d] : 0.0;
        m.hi[d] = d < dim ? mesh->hi[d] : 1.0;
        m.h[d] = (m.hi[d] - m.lo[d]) / m.K[d];
    }
    m.periodic = c->periodic;
    const long long V = (long long)m.E * m.n;
    c->state_elem = precision == SL_FP64 ? sizeof(double) : sizeof(float2);  // FP32 modes: hi + lo pair
    c->vals = (long long)ncomp * V;
    const int nf = dim == 1 ? m.E + 1 : 2 * m.E * N;  // 1D: interfaces 0..K
    c->mom_chunk = 64;
    const int nc = (M + c->mom_chunk - 1) / c->mom_chunk;
    bool ok = dalloc(c, &c->xi, N) == cudaSuccess && dalloc(c, &c->nodeU, size_t(dim) * V) == cudaSuccess &&
              dalloc(c, &c->nodeB, V) == cudaSuccess && dalloc(c, &c->nodeDiv, V) == cudaSuccess &&
              dalloc(c, &c->faceU, nf) == cudaSuccess && dalloc(c, &c->faceB, nf) == cudaSuccess &&
              sl::ctx_alloc(c, &c->Q, size_t(M) * ncomp * V * c->state_elem) == cudaSuccess &&
              dalloc(c, &c->psum, size_t(nc) * ncomp * V) == cudaSuccess &&
              dalloc(c, &c->psq, size_t(nc) * ncomp * V) == cudaSuccess &&
              dalloc(c, &c->mean_tmp, ncomp * V) == cudaSuccess && dalloc(c, &c->m2_tmp, ncomp * V) == cudaSuccess &&
              dalloc(c, &c->err, 1) == cudaSuccess &&
              (dim == 1 || (dalloc(c, &c->faceUhi, size_t(m.K[0] + m.K[1]) * N) == cudaSuccess &&
                            dalloc(c, &c->faceBhi, size_t(m.K[0] + m.K[1]) * N) == cudaSuccess));
    if (ok && dim == 2)
        ok = sl::ctx_alloc(c, &c->faces2d, size_t(M) * ncomp * m.E * 4 * N * c->state_elem) == cudaSuccess &&
             dalloc(c, &c->tab2d, size_t(N) * N + 5 * N) == cudaSuccess &&
             sl::ctx_alloc(c, &c->alpha2d, size_t(M) * ncomp * V * (precision == SL_FP64 ? 8 : 4)) == cudaSuccess &&
             sl::ctx_alloc(c, &c->coef2d, size_t(5) * V * (precision == SL_FP64 ? 8 : 4)) == cudaSuccess &&
             sl::ctx_alloc(c, reinterpret_cast<void **>(&c->fb2d), size_t(M) * m.E) == cudaSuccess &&
             sl::ctx_alloc(c, reinterpret_cast<void **>(&c->fbcount2d), 2 * sizeof(unsigned long long)) ==
                 cudaSuccess &&
             cudaMemsetAsync(c->fbcount2d, 0, 2 * sizeof(unsigned long long), c->st) == cudaSuccess &&
             sl::ctx_alloc(c, reinterpret_cast<void **>(&c->slots2d), (2 * size_t(M) * m.E + 2) * sizeof(unsigned)) ==
                 cudaSuccess &&
             cudaMemsetAsync(c->slots2d, 0, (2 * size_t(M) * m.E + 2) * sizeof(unsigned), c->st) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        sl_free(c);
        return SL_ERR_OOM;
    }
    double *nodal_dev = nullptr;
    if (phi0->kind == SL_PHI_NODAL) {
        if (sl::ctx_alloc(c, reinterpret_cast<void **>(&nodal_dev), V * sizeof(double)) != cudaSuccess ||
            cudaMemcpyAsync(nodal_dev, phi0->nodal, V * sizeof(double), cudaMemcpyHostToDevice, c->st) != cudaSuccess) {
            sl::ctx_free(c, nodal_dev);
            sl_free(c);
            return SL_ERR_OOM;
        }
    }
    cudaError_t e = cudaMemsetAsync(c->err, 0, sizeof(int), c->st);
    if (e == cudaSuccess) e = set_coefficients(c, drift, diffusion, phi0, nodal_dev, true);  // every sample phi0
    sl::ctx_free(c, nodal_dev);
    if (e != cudaSuccess || refresh_bounds(c) != SL_OK) {
        cudaGetLastError();
        sl_free(c);
        return SL_ERR_CUDA;
    }
    if (dim == 2) {  // the order's node tables, from the device's own nodes
        std::vector<double> xh(N), tab(size_t(N) * N + 5 * N);
        if (cudaMemcpyAsync(xh.data(), c->xi, N * sizeof(double), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
            cudaStreamSynchronize(c->st) != cudaSuccess) {
            cudaGetLastError();
            sl_free(c);
            return SL_ERR_CUDA;
        }
        sl::node_tables2d(N, xh.data(), tab.data());
        if (cudaMemcpyAsync(c->tab2d, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, c->st) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->st) != cudaSuccess) {
            cudaGetLastError();
            sl_free(c);
            return SL_ERR_CUDA;
        }
    }

    if (dim == 1) {
        const int K = m.K[0];
        if (K <= sl::kMaxThreads1D) {
            c->C = 1;
            c->T = K;
            c->S = std::max(1, std::min(sl::kMaxThreads1D / K, M));
        } else {
            c->C = (K + sl::kMaxThreads1D - 1) / sl::kMaxThreads1D;
            c->T = (K + c->C - 1) / c->C;
            c->S = 1;
        }
    }
    *out = c;
    return SL_OK;
}

// Bounds after sl_set_fields_device are recomputed on first use (this
// synchronises the context's stream); the context object itself is not const.
static int current_bounds(const sl_ctx *cc)
{
    sl_ctx *c = const_cast<sl_ctx *>(cc);
    if (!c->bounds_stale) return SL_OK;
    if (c->poisoned) return SL_ERR_STATE;
    if (refresh_bounds(c) != SL_OK) return fail_cuda(c);
    c->bounds_stale = 0;
    return SL_OK;
}

int sl_dt_max(const sl_ctx *c, double *dt)
{
    if (!c || !dt) return SL_ERR_ARG;
    const int rc = current_bounds(c);
    if (rc != SL_OK) return rc;
    *dt = c->dtmax;
    return SL_OK;
}

int sl_dt_edge(const sl_ctx *c, double *dt)
{
    if (!c || !dt) return SL_ERR_ARG;
    const int rc = current_bounds(c);
    if (rc != SL_OK) return rc;
    *dt = c->dtedge;
    return SL_OK;
}

int sl_step_count(const sl_ctx *c, long long *n)
{
    if (!c || !n) return SL_ERR_ARG;
    *n = c->step;
    return SL_OK;
}

int sl_fallback_count(sl_ctx *c, long long *phase1, long long *phase2)
{
    if (!c) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    unsigned long long h[2] = {0, 0};
    if (c->fbcount2d && (cudaMemcpyAsync(h, c->fbcount2d, sizeof(h), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
                         cudaStreamSynchronize(c->st) != cudaSuccess))
        return fail_cuda(c);
    if (phase1) *phase1 = (long long)h[0];
    if (phase2) *phase2 = (long long)h[1];
    return SL_OK;
}

int sl_set_step_count(sl_ctx *c, long long n)
{
    if (!c || n < 0) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    c->step = n;
    return SL_OK;
}

int sl_set_fields(sl_ctx *c, const sl_field *drift, const sl_field *diffusion)
{
    sl::TraceRange trace("sl_set_fields");
    if (!c) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    const int dim = c->m.dim;
    if (!valid_kind(dim, 0, drift) || !valid_kind(dim, 1, diffusion)) return SL_ERR_ARG;
    if (!diffusion_ok(diffusion, dim, c->m.K[0], c->m.K[1], c->m.N, c->periodic != 0)) return SL_ERR_ARG;
    sl_field none;
    std::memset(&none, 0, sizeof(none));
    none.kind = SL_PHI_GAUSS;  // no state is written
    const cudaError_t e = set_coefficients(c, drift, diffusion, &none, nullptr, false);
    if (e != cudaSuccess || refresh_bounds(c) != SL_OK) return fail_cuda(c);
    c->bounds_stale = 0;
    return SL_OK;
}

int sl_set_fields_device(sl_ctx *c, const sl_field *drift, const sl_field *diffusion)
{
    sl::TraceRange trace("sl_set_fields_device");
    if (!c) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    const int dim = c->m.dim;
    if (!valid_kind(dim, 0, drift) || !valid_kind(dim, 1, diffusion)) return SL_ERR_ARG;
    // analytic parameters are checked here, nodal values on the device
    if (diffusion->kind != SL_D_NODAL && !diffusion_ok(diffusion, dim, c->m.K[0], c->m.K[1], c->m.N, c->periodic != 0))
        return SL_ERR_ARG;
    sl_field none;
    std::memset(&none, 0, sizeof(none));
    none.kind = SL_PHI_GAUSS;  // no state is written
    if (set_coefficients(c, drift, diffusion, &none, nullptr, false, true) != cudaSuccess) return fail_cuda(c);
    c->bounds_stale = 1;
    return SL_OK;
}

int sl_step(sl_ctx *c, double dt, int steps)
{
    sl::TraceRange trace("sl_step");
    if (!c) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    if (!(dt > 0.0) || !std::isfinite(dt) || steps < 0) return SL_ERR_ARG;
    if (c->strict_dt && c->bounds_stale) {
        if (refresh_bounds(c) != SL_OK) return fail_cuda(c);
        c->bounds_stale = 0;
    }
    if (c->strict_dt && dt > c->dtmax * (1.0 + 1e-12)) return SL_ERR_DT;
    if (steps == 0) return SL_OK;
    if (!c->periodic && (c->step < c->ghost_base || c->step + steps > c->ghost_base + c->ghost_count))
        return SL_ERR_ARG;  // Dirichlet: boundary values must cover every step (sl_set_boundary)
    const sl::Mesh &m = c->m;
    const int dim = m.dim;
    const size_t per_step = size_t(c->M) * dim * sizeof(double);
    const int chunk = int(std::max<size_t>(1, std::min<size_t>(size_t(steps), kWienerScratchBytes / per_step)));
    if (chunk > c->dW_cap) {
        sl::ctx_free(c, c->dW);
        c->dW = nullptr;
        c->dW_cap = 0;
        if (sl::ctx_alloc(c, reinterpret_cast<void **>(&c->dW), chunk * per_step) != cudaSuccess) {
            cudaGetLastError();
            return SL_ERR_OOM;
        }
        c->dW_cap = chunk;
    }
    const double sqrt_dt = std::sqrt(dt);
    for (int done = 0; done < steps;) {
        int n = std::min(chunk, steps - done);
        if (c->reseed_every > 0)  // stop at the next reseed point
            n = int(std::min<long long>(n, c->reseed_every - c->step % c->reseed_every));
        cudaError_t e = sl::launch_wiener(c->seed, c->step, c->sample0, n, c->M, dim, sqrt_dt, c->dW, c->st);
        if (e != cudaSuccess) return fail_cuda(c);
        std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
        if (c->profiling) {
            if (cudaEventCreate(&ev.first) != cudaSuccess || cudaEventCreate(&ev.second) != cudaSuccess ||
                cudaEventRecord(ev.first, c->st) != cudaSuccess)
                return fail_cuda(c);
            c->events.push_back(ev);
        }
        if (dim == 1) {
            sl::Step1DArgs a;
            a.K = m.K[0];
            a.M = c->M;
            a.S = c->S;
            a.C = c->C;
            a.T = c->T;
            a.nsteps = n;
            a.dt = dt;
            a.h = m.h[0];
            a.inv_w2 = c->inv_w2;
            a.periodic = c->periodic;
            a.ncomp = c->ncomp;
            a.ghost = c->periodic ? nullptr : c->ghost + c->ghost_w * (c->step - c->ghost_base);
            a.xi = c->xi;
            a.nodeU = c->nodeU;
            a.nodeB = c->nodeB;
            a.nodeDiv = c->nodeDiv;
            a.faceU = c->faceU;
            a.faceB = c->faceB;
            a.dW = c->dW;
            a.Q = c->Q;
            a.err = c->err;
            if (c->precision == SL_FP64)
                e = sl::launch_step1d_fp64(a, m.N, c->st);
            else if (c->precision == SL_MIXED)
                e = sl::launch_step1d_mixed(a, m.N, c->st);
            else
                e = sl::launch_step1d_fp32(a, m.N, c->st);
        } else {
            sl::Step2DArgs a;
            a.Kx = m.K[0];
            a.Ky = m.K[1];
            a.M = c->M;
            a.nsteps = n;
            a.dt = dt;
            a.hx = m.h[0];
            a.hy = m.h[1];
            a.s4x = 4.0 / m.h[0];
            a.s4y = 4.0 / m.h[1];
            a.xi = c->xi;
            a.tab = c->tab2d;
            a.fb = c->fb2d;
            a.fbcount = c->fbcount2d;
            a.f64_factor = c->precision == SL_MIXED;
            a.slot_mark = c->slots2d;
            a.slot_list = c->slots2d + size_t(c->M) * m.E;
            a.slot_ctl = c->slots2d + 2 * size_t(c->M) * m.E;
            a.nodeU = c->nodeU;
            a.nodeB = c->nodeB;
            a.nodeDiv = c->nodeDiv;
            a.faceU = c->faceU;
            a.faceB = c->faceB;
            a.dW = c->dW;
            a.Q = c->Q;
            a.faces = c->faces2d;
            a.alpha = c->alpha2d;
            a.coef = c->coef2d;
            if (sl::ensure_coef2d(c, dt) != cudaSuccess) return fail_cuda(c);
            a.err = c->err;
            a.chunk = c->launch_chunk;
            a.g0 = a.g1 = 0;
            a.w = c->bc_weight;
            a.periodic = c->periodic;
            a.ghost = c->periodic ? nullptr : c->ghost + c->ghost_w * (c->step - c->ghost_base);
            a.ghost_w = c->ghost_w;
            a.faceUhi = c->faceUhi;
            a.faceBhi = c->faceBhi;
            a.throttle = c->launch_chunk > 0 ? &c->throttle : nullptr;
            if (c->ncomp > 1)
                e = sl::launch_step2d_c2(a, m.N, c->precision == SL_FP64, c->st);
            else
                e = c->precision == SL_FP64 ? sl::launch_step2d_fp64(a, m.N, c->st) : sl::launch_step2d_fp32(a, m.N, c->st);
        }
        if (e == cudaErrorNotSupported) return SL_ERR_UNSUPPORTED;
        if (e != cudaSuccess) return fail_cuda(c);
        if (c->profiling && cudaEventRecord(ev.second, c->st) != cudaSuccess) return fail_cuda(c);
        c->step += n;
        done += n;
        if (c->reseed_every > 0 && c->step % c->reseed_every == 0) {
            const int rc = sl_reseed(c);
            if (rc != SL_OK) return rc;
        }
    }
    return SL_OK;
}

int sl_reseed(sl_ctx *c)
{
    sl::TraceRange trace("sl_reseed");
    if (!c) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    const long long V = c->vals;  // values per sample (components x nodes)
    const int dbl = c->precision == SL_FP64;
    if (sl::launch_moments(c->Q, dbl, c->M, V, c->mom_chunk, c->psum, c->psq, c->mean_tmp, nullptr, c->st) !=
            cudaSuccess ||
        sl::launch_reseed(c->Q, dbl, c->M, V, c->mean_tmp, c->st) != cudaSuccess)
        return fail_cuda(c);
    return SL_OK;
}

int sl_set_boundary(sl_ctx *c, int nsteps, const double *values)
{
    if (!c || nsteps < 0 || (nsteps > 0 && !values)) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    if (c->periodic) return SL_ERR_ARG;
    if (nsteps > c->ghost_cap) {
        sl::ctx_free(c, c->ghost);
        c->ghost = nullptr;
        c->ghost_cap = 0;
        if (sl::ctx_alloc(c, reinterpret_cast<void **>(&c->ghost), size_t(nsteps) * c->ghost_w * sizeof(double)) !=
            cudaSuccess) {
            cudaGetLastError();
            return SL_ERR_OOM;
        }
        c->ghost_cap = nsteps;
    }
    if (nsteps > 0 &&
        (cudaMemcpyAsync(c->ghost, values, size_t(nsteps) * c->ghost_w * sizeof(double), cudaMemcpyHostToDevice, c->st) !=
             cudaSuccess ||
         cudaStreamSynchronize(c->st) != cudaSuccess))
        return fail_cuda(c);
    c->ghost_base = c->step;
    c->ghost_count = nsteps;
    return SL_OK;
}

static int check_device_error(sl_ctx *c)
{
    int h = 0;
    if (cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess)
        return fail_cuda(c);
    if (h & 4) {  // a negative D in tables read in place (sl_set_fields_device); the cause
        c->poisoned = 1;  // of any non-finite remap that followed, so reported first
        return SL_ERR_ARG;
    }
    if (h & 1) {
        c->poisoned = 1;
        return SL_ERR_SINGULAR;
    }
    if (h & 2) {
        c->poisoned = 1;
        return SL_ERR_TIMEOUT;
    }
    return SL_OK;
}

int sl_moments_device(sl_ctx *c, double *d_mean, double *d_m2)
{
    sl::TraceRange trace("sl_moments");
    if (!c || !d_mean) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    const long long V = c->vals;  // values per sample (components x nodes)
    if (sl::launch_moments(c->Q, c->precision == SL_FP64, c->M, V, c->mom_chunk, c->psum, c->psq, d_mean, d_m2,
                           c->st) != cudaSuccess)
        return fail_cuda(c);
    return SL_OK;
}

int sl_moments_partial(sl_ctx *c, double *d_psum, double *d_psq)
{
    sl::TraceRange trace("sl_moments_partial");
    if (!c || !d_psum || !d_psq) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    if (sl::launch_moment_partials(c->Q, c->precision == SL_FP64, c->M, c->vals, c->mom_chunk, d_psum, d_psq,
                                   c->st) != cudaSuccess)
        return fail_cuda(c);
    return SL_OK;
}

int sl_moment_chunk(void) { return 64; }

int sl_moments_combine(const double *d_psum, const double *d_psq, int nchunks, long long V, long long M_total,
                       double *d_mean, double *d_m2, void *stream)
{
    sl::TraceRange trace("sl_moments_combine");
    if (!d_psum || !d_psq || !d_mean || nchunks < 1 || V < 1 || M_total < 1) return SL_ERR_ARG;
    if (sl::ensure_loaded() != cudaSuccess) return SL_ERR_CUDA;
    return sl::launch_moments_combine(d_psum, d_psq, nchunks, V, M_total, d_mean, d_m2,
                                      static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? SL_OK
               : SL_ERR_CUDA;
}

int sl_pdf_device(sl_ctx *c, int nbins, double lo, double hi, unsigned int *d_counts)
{
    if (!c || !d_counts || nbins < 1 || nbins > 4096 || !std::isfinite(lo) || !std::isfinite(hi) || !(hi > lo))
        return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    const long long V = c->vals;  // values per sample (components x nodes)
    if (sl::launch_pdf(c->Q, c->precision == SL_FP64, c->M, V, nbins, lo, hi, d_counts, c->st) != cudaSuccess)
        return fail_cuda(c);
    return SL_OK;
}

int sl_pdf(sl_ctx *c, int nbins, double lo, double hi, unsigned int *counts)
{
    if (!c || !counts || nbins < 1 || nbins > 4096) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    const size_t bytes = size_t(c->vals) * nbins * sizeof(unsigned int);
    unsigned int *d = nullptr;
    if (sl::ctx_alloc(c, reinterpret_cast<void **>(&d), bytes) != cudaSuccess) {
        cudaGetLastError();
        return SL_ERR_OOM;
    }
    int rc = sl_pdf_device(c, nbins, lo, hi, d);
    if (rc == SL_OK && (cudaMemcpyAsync(counts, d, bytes, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
                        cudaStreamSynchronize(c->st) != cudaSuccess))
        rc = fail_cuda(c);
    sl::ctx_free(c, d);
    return rc;
}

int sl_moments(sl_ctx *c, double *mean, double *m2)
{
    if (!c || !mean) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    const long long V = c->vals;  // values per sample (components x nodes)
    int rc = sl_moments_device(c, c->mean_tmp, m2 ? c->m2_tmp : nullptr);
    if (rc != SL_OK) return rc;
    if (cudaMemcpyAsync(mean, c->mean_tmp, V * sizeof(double), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
        return fail_cuda(c);
    if (m2 && cudaMemcpyAsync(m2, c->m2_tmp, V * sizeof(double), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
        return fail_cuda(c);
    return check_device_error(c);
}

int sl_get_samples(sl_ctx *c, int s0, int count, double *out)
{
    if (!c || !out || s0 < 0 || count < 0 || s0 + count > c->M) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    const size_t V = size_t(c->vals);  // values per sample (components x nodes)
    const size_t n = V * count;
    if (c->precision == SL_FP64) {
        if (cudaMemcpyAsync(out, static_cast<double *>(c->Q) + V * s0, n * sizeof(double), cudaMemcpyDeviceToHost,
                            c->st) != cudaSuccess)
            return fail_cuda(c);
    } else {
        std::vector<float2> tmp(n);
        if (cudaMemcpyAsync(tmp.data(), static_cast<float2 *>(c->Q) + V * s0, n * sizeof(float2),
                            cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
            cudaStreamSynchronize(c->st) != cudaSuccess)
            return fail_cuda(c);
        for (size_t i = 0; i < n; ++i) out[i] = double(tmp[i].x) + double(tmp[i].y);
    }
    return check_device_error(c);
}

int sl_set_samples(sl_ctx *c, int s0, int count, const double *in)
{
    if (!c || !in || s0 < 0 || count < 0 || s0 + count > c->M) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    const size_t V = size_t(c->vals);  // values per sample (components x nodes)
    const size_t n = V * count;
    cudaError_t e;
    if (c->precision == SL_FP64) {
        e = cudaMemcpyAsync(static_cast<double *>(c->Q) + V * s0, in, n * sizeof(double), cudaMemcpyHostToDevice,
                            c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    } else {
        std::vector<float2> tmp(n);
        for (size_t i = 0; i < n; ++i) {
            const float hi = float(in[i]);
            tmp[i] = make_float2(hi, float(in[i] - double(hi)));
        }
        e = cudaMemcpyAsync(static_cast<float2 *>(c->Q) + V * s0, tmp.data(), n * sizeof(float2),
                            cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    }
    return e == cudaSuccess ? SL_OK : fail_cuda(c);
}

int sl_profile(sl_ctx *c, int enable)
{
    if (!c) return SL_ERR_ARG;
    c->profiling = enable ? 1 : 0;
    return SL_OK;
}

int sl_profile_read(sl_ctx *c, double *kernel_ms, long long *launches)
{
    if (!c || !kernel_ms || !launches) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    double total = 0.0;
    for (auto &ev : c->events) {
        float ms = 0.f;
        if (cudaEventSynchronize(ev.second) != cudaSuccess || cudaEventElapsedTime(&ms, ev.first, ev.second) != cudaSuccess)
            return fail_cuda(c);
        total += ms;
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    *kernel_ms = total;
    *launches = (long long)c->events.size();
    c->events.clear();
    return SL_OK;
}

int sl_wiener(sl_ctx *c, long long step0, int nsteps, double dt, double *out)
{
    if (!c || !out || nsteps < 0 || step0 < 0 || !(dt > 0.0)) return SL_ERR_ARG;
    if (c->poisoned) return SL_ERR_STATE;
    const size_t n = size_t(nsteps) * c->M * c->m.dim;
    if (n == 0) return SL_OK;
    double *d = nullptr;
    if (sl::ctx_alloc(c, reinterpret_cast<void **>(&d), n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return SL_ERR_OOM;
    }
    cudaError_t e = sl::launch_wiener(c->seed, step0, c->sample0, nsteps, c->M, c->m.dim, std::sqrt(dt), d, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, n * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    sl::ctx_free(c, d);
    return e == cudaSuccess ? SL_OK : fail_cuda(c);
}

}  // extern "C"
