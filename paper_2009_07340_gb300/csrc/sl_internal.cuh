// sl_internal.cuh -- context layout and launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sl.h"

namespace sl {

// NVTX range over a host API call: the solver's entry points appear as named
// ranges in Nsight tools (ncu --nvtx filters on them); without a tool
// attached a push / pop is a cheap no-op.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

constexpr int kMaxN = 16;           // nodes per direction per element
constexpr int kMaxThreads1D = 256;  // elements (threads) per CTA in the 1D kernel
constexpr int kMaxCluster1D = 8;    // CTAs per sample field (portable cluster size)

// Field descriptor copied to the device for the initialisation kernels.
struct FieldDev {
    int kind;
    double p[40];
    const double *nodal;  // nodal drift / diffusion: device copy of the node values
    const double *face;   // and of the interface table (nullptr: derived from the traces)
    int *err;             // diffusion tables read in place: D < 0 sets bit 4 here (else null)
};

struct Mesh {
    int dim, N, n;  // n = N^dim nodes per element
    int K[2];       // elements per direction (K[1] = 1 in 1D)
    int E;          // elements
    double lo[2], hi[2], h[2];
    int periodic;   // 1: periodic in every direction; 0: Dirichlet boundaries
};

// Kernel arguments of the 1D step (one launch advances `nsteps` steps).
struct Step1DArgs {
    int K, M;         // elements, samples
    int S;            // samples per CTA (cluster size 1) ; 1 when clustered
    int C;            // CTAs per sample field (cluster size)
    int T;            // thread slots per sample per CTA (>= elements per CTA)
    int nsteps;
    double dt, h;
    double inv_w2;         // 1 / w^2 of the boundary rows (0: hard constraints)
    int periodic;          // 0: Dirichlet boundaries with the ghost values below
    int ncomp;             // scalar fields per sample (1 or 2), state [M][ncomp][K][N]
    const double *ghost;   // [nsteps][2] boundary values at x = lo, hi after each step (Dirichlet)
    const double *xi;      // [N] reference nodes on [0,1]
    const double *nodeU;   // [K][N] drift at the nodes
    const double *nodeB;   // [K][N] sqrt(2 D) at the nodes
    const double *nodeDiv; // [K][N] du/dx at the nodes
    const double *faceU;   // [K + 1] drift at interface k (left face of element k; K: x = hi)
    const double *faceB;   // [K + 1] sqrt(2 D) at interface k
    const double *dW;      // [nsteps][M] Wiener increments
    void *Q;               // [M][K][N] state (double for SL_FP64, float otherwise)
    int *err;              // device error word (bit 0: non-finite remap)
};

// Kernel arguments of the 2D step.
// Bounded queue depth for chunked launches: before launch number i, the host
// waits (blocking-sync event) until launch i - kDepth has completed, so a
// stream never holds more than kDepth queued launches.  CUDA multiplexes
// streams onto a few in-order hardware queues; a stream with a deep queue of
// dependent launches would block every other stream that shares its queue.
struct LaunchThrottle {
    static constexpr int kDepth = 2;
    cudaEvent_t ev[kDepth] = {};
    long long n = 0;  // launches recorded
    cudaError_t before() const { return n >= kDepth ? cudaEventSynchronize(ev[n % kDepth]) : cudaSuccess; }
    cudaError_t after(cudaStream_t st)
    {
        const cudaError_t e = cudaEventRecord(ev[n % kDepth], st);
        ++n;
        return e;
    }
};

struct Step2DArgs {
    int Kx, Ky, M;
    int nsteps;
    double dt, hx, hy;
    double s4x, s4y;       // 4 / hx, 4 / hy (displacements in scaled element units)
    const double *xi;
    const double *tab;     // [N N + 5 N] node tables: 4 (xi_i - xi_m), barycentric weights of the
                           // scaled nodes, h_i(0), h_i(1), -4 xi_i, 4 (1 - xi_i)
    unsigned char *fb;     // [M][E]: groups the iterative solve left to the direct one
    unsigned long long *fbcount = nullptr;  // [2]: per phase, groups so left, cumulative (may be null)
    // the direct kernel's CTA slots holding a flagged group (in a batch, those
    // of args[0] serve the class): slot_mark [slots] 1 while listed,
    // slot_list [slots], slot_ctl [2] = list length, CTAs finished; all zero
    // between launches
    unsigned *slot_mark = nullptr, *slot_list = nullptr, *slot_ctl = nullptr;
    int f64_factor = 0;  // host: the FP32 remap factors its capacitance matrix in FP64 (SL_MIXED)
    const void *coef;      // [5][E][n] in the kernel's precision: 4 u_x dt / hx, 4 u_y dt / hy,
                           // 4 b / hx, 4 b / hy (b = sqrt(2 D)), dt du_j/dx_j (launch_coef2d)
    const double *nodeU;   // [2][E][n]
    const double *nodeB;   // [E][n]
    const double *nodeDiv; // [E][n]
    const double *faceU;   // [2][E][N]: vertical (u_x at x-face of e), horizontal (u_y)
    const double *faceB;   // [2][E][N]
    const double *dW;      // [nsteps][M][2]
    void *Q;               // [M][E][n]
    void *faces;           // scratch [M][E][4N] face values of the advected interpolant
    void *alpha;           // scratch [M][NCOMP][E][n] (FP32 modes: float): phase 1's advected interpolant
                           // relative to the element reference, phase 2's first iterate
    int *err;
    double w;              // weight of the face rows (1 unless the caller set one)
    int periodic;          // 0: Dirichlet boundaries on all four sides
    const double *ghost;   // [nsteps][ghost_w] boundary values (left, right, bottom, top face points)
    int ghost_w;           // 2 (Kx + Ky) N
    const double *faceUhi; // [Ky][N] u_x on x = hi, then [Kx][N] u_y on y = hi (Dirichlet)
    const double *faceBhi; // the same for sqrt(2 D)
    long long chunk;       // element-sample groups per launch (0: all in one launch)
    long long g0, g1;      // groups [g0, g1) of this launch (set by the launcher)
    LaunchThrottle *throttle;  // host object; with chunk > 0: bounded queue depth (may be null)
};

// Persistent batched 1D launch: `ninst` instances of one order N, work
// items (instance, sample slot) numbered by prefix[0..ninst].
struct Batch1DLaunch {
    const Step1DArgs *args;  // device [ninst]
    const int *prefix;       // device [ninst + 1]
    int ninst;
    int *counter;            // device work counter (reset by the launcher)
    int grid;                // persistent CTAs
    size_t smem;             // dynamic shared memory per CTA
};
cudaError_t launch_step1d_batch_fp64(const Batch1DLaunch &b, int N, cudaStream_t st);
cudaError_t launch_step1d_batch_mixed(const Batch1DLaunch &b, int N, cudaStream_t st);
cudaError_t launch_step1d_batch_fp32(const Batch1DLaunch &b, int N, cudaStream_t st);
cudaError_t launch_step1d_fp64(const Step1DArgs &a, int N, cudaStream_t st);
cudaError_t launch_step1d_mixed(const Step1DArgs &a, int N, cudaStream_t st);
cudaError_t launch_step1d_fp32(const Step1DArgs &a, int N, cudaStream_t st);
size_t step1d_smem_bytes_fp64(int N, int S, int T);
size_t step1d_smem_bytes_mixed(int N, int S, int T);
size_t step1d_smem_bytes_fp32(int N, int S, int T);
// Batched 2D launch: `ninst` instances of one order N; instance i owns the
// element-sample groups [prefix[i], prefix[i+1]).
struct Batch2DLaunch {
    const Step2DArgs *args;    // device [ninst]
    const long long *prefix;   // device [ninst + 1]
    int ninst;
    long long total_groups;
    int nsteps;
    int f64_factor = 0;        // SL_MIXED: capacitance matrix factored in FP64
};
cudaError_t launch_step2d_batch_fp64(const Batch2DLaunch &b, int N, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32(const Batch2DLaunch &b, int N, cudaStream_t st);
cudaError_t launch_step2d_fp64(const Step2DArgs &a, int N, cudaStream_t st);
cudaError_t launch_step2d_fp32(const Step2DArgs &a, int N, cudaStream_t st);
// two fields per sample (Q [M][2][E][n], faces [M][2][E][4N]), N <= 8
cudaError_t launch_step2d_c2(const Step2DArgs &a, int N, bool fp64, cudaStream_t st);
// The context's 2D advance coefficients for step size dt (once per step size and fields).
cudaError_t ensure_coef2d(sl_ctx *c, double dt);
// The 2D advance coefficients of step size dt (Step2DArgs::coef), FP64 or float.
cudaError_t launch_coef2d(const double *nodeU, const double *nodeB, const double *nodeDiv, long long V, double dt,
                          double s4x, double s4y, bool fp64, void *out, cudaStream_t st);
// Host-side node tables of a 2D order (Step2DArgs::tab) from the nodes xi[N].
void node_tables2d(int N, const double *xi, double *tab);
cudaError_t launch_init_fields(const Mesh &m, const FieldDev &u, const FieldDev &D, const FieldDev &phi0,
                               const double *phi0_nodal_dev, double *xi, double *nodeU, double *nodeB,
                               double *nodeDiv, double *faceU, double *faceB, void *Q, int M,
                               int state_is_double, cudaStream_t st);
cudaError_t launch_wiener(unsigned long long seed, long long step0, long long sample0, int nsteps, int M, int dim,
                          double sqrt_dt, double *out, cudaStream_t st);
cudaError_t launch_moments(const void *Q, int state_is_double, int M, long long V, int chunk,
                           double *psum, double *psq, double *mean, double *m2, cudaStream_t st);
// The first pass alone: per-chunk sums and sums of squares [ceil(M/chunk)][V].
cudaError_t launch_moment_partials(const void *Q, int state_is_double, int M, long long V, int chunk,
                                   double *psum, double *psq, cudaStream_t st);
// The second pass alone: chunk partials [nc][V] added in ascending c, / M.
cudaError_t launch_moments_combine(const double *psum, const double *psq, int nc, long long V, long long M,
                                   double *mean, double *m2, cudaStream_t st);
// Per-node histogram of the samples into B bins over [lo, hi] (device [V][B]).
cudaError_t launch_pdf(const void *Q, int state_is_double, int M, long long V, int B, double lo, double hi,
                       unsigned int *counts, cudaStream_t st);
// 2D coefficients on the faces x = hi ([Ky][N], u_x) and y = hi ([Kx][N], u_y).
cudaError_t launch_init_faces_hi(const Mesh &m, const FieldDev &u, const FieldDev &D, double *faceUhi, double *faceBhi,
                                 cudaStream_t st);
// Every sample set to `mean` (Eq. re-seed).
cudaError_t launch_reseed(void *Q, int state_is_double, int M, long long V, const double *mean, cudaStream_t st);

// Module loading.  With lazy loading (the default), the first launch of a
// kernel loads it, and a load may synchronise the whole device: a request
// whose kernel is first launched while another request's long kernels run
// would wait for them.  Each unit's preload function prepares every kernel
// it holds (prepare_kernel: load, shared-memory limit); ensure_loaded() runs
// them all once per device, before any launch.
template <typename F>
cudaError_t prepare_kernel(F f)
{
    // Loads kernel f and lets its launches use the device's whole opt-in
    // shared memory.  The limit is set here once: changing a kernel's
    // attribute while an instance of it runs can wait for that instance,
    // which would stall a launch from one request behind another's kernel.
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    int dev = 0, optin = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - int(fa.sharedSizeBytes));
    return e;
}
cudaError_t preload_step1d_fp64();
cudaError_t preload_step1d_mixed();
cudaError_t preload_step1d_fp32();
cudaError_t preload_step2d_fp64();
cudaError_t preload_step2d_fp32();
cudaError_t preload_step2d_c2();
cudaError_t preload_setup();
cudaError_t ensure_loaded();

}  // namespace sl

// Solver context (opaque in the ABI).
struct sl_ctx {
    sl::Mesh m;
    int M = 0;
    int precision = SL_FP64;
    int strict_dt = 0;
    unsigned long long seed = 0;
    long long sample0 = 0;
    cudaStream_t st = nullptr;
    int device = 0;
    long long step = 0;
    int poisoned = 0;
    int bounds_stale = 0; // fields changed on the device: dtmax / dtedge recomputed when asked
    double dtmax = 0.0;   // Eq. (1d_timestep) with the smallest node gap
    double dtedge = 0.0;  // the same with the first node's distance to the element face
    // device memory owned by the context
    double *xi = nullptr, *nodeU = nullptr, *nodeB = nullptr, *nodeDiv = nullptr;
    double *faceU = nullptr, *faceB = nullptr;
    void *Q = nullptr;
    size_t state_elem = 8;
    double *dW = nullptr;
    int dW_cap = 0;  // steps the Wiener scratch holds
    double *psum = nullptr, *psq = nullptr, *mean_tmp = nullptr, *m2_tmp = nullptr;
    int mom_chunk = 64;
    int *err = nullptr;
    void *faces2d = nullptr;  // 2D face-value scratch
    void *alpha2d = nullptr;  // 2D: phase 1's interpolant at the nodes (Step2DArgs::alpha)
    void *coef2d = nullptr;   // 2D: the advance coefficients of one step size (Step2DArgs::coef)
    double coef2d_dt = 0.0;   // the step size they hold (0: none yet)
    long long fields_version = 0, coef2d_version = -1;  // fields changed since they were formed?
    double *tab2d = nullptr;  // 2D node tables of the order (Step2DArgs::tab)
    unsigned char *fb2d = nullptr;  // 2D: groups left to the direct solve, [M][E]
    unsigned long long *fbcount2d = nullptr;  // 2D: their cumulative count per phase [2]
    unsigned *slots2d = nullptr;  // 2D: [2 M E + 2] slot marks, slot list, list control (Step2DArgs::slot_*)
    long long launch_chunk = 0;  // 2D: element-sample groups per kernel launch (0: all)
    double bc_weight = 1.0;       // weight w of the remap's boundary rows (INFINITY: hard, 1D)
    double inv_w2 = 1.0;          // 1 / w^2 (0 for hard constraints)
    int periodic = 1;             // 0: 1D Dirichlet boundaries
    int ncomp = 1;                // scalar fields per sample (state [M][ncomp][E][n])
    int ghost_w = 2;              // boundary values per step: 1D 2, 2D 2 (Kx + Ky) N
    double *faceUhi = nullptr, *faceBhi = nullptr;  // 2D faces x = hi, y = hi
    long long vals = 0;           // values per sample: ncomp E n
    int reseed_every = 0;         // > 0: samples set to their mean after every such step count
    double *ghost = nullptr;      // device [ghost_cap][2] boundary values (Dirichlet)
    long long ghost_cap = 0, ghost_base = 0, ghost_count = 0;  // rows, first step, steps covered
    sl::LaunchThrottle throttle;  // events created when launch_chunk > 0
    // 1D launch geometry
    int S = 1, C = 1, T = 1;
    // kernel timing hook
    int profiling = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
};

namespace sl {
// Wiener increments of one instance in a batched launch.
struct WienerJob {
    unsigned long long seed;
    long long sample0;
    int M, dim;
    double sqrt_dt;
    double *out;  // [nsteps][M][dim]
};
cudaError_t launch_wiener_batch(const WienerJob *jobs, const long long *prefix, int njobs, int nsteps,
                                const long long *steps, long long total, cudaStream_t st);
cudaError_t launch_advance_counters(long long *steps, int n, int by, cudaStream_t st);
}  // namespace sl

namespace sl {
// Context memory comes from the library's stream-ordered memory pool of the
// context's device (created by ensure_loaded): allocating and releasing it
// never synchronises the device, so contexts created and freed while other
// work runs (the server) do not wait for that work.  The pool keeps freed
// memory mapped for reuse (cudaMemPoolTrimTo releases it) and reuses a block
// on another stream only once its free has executed.
cudaMemPool_t device_pool(int device);
inline cudaError_t ctx_alloc(const sl_ctx *c, void **p, size_t bytes)
{
    return cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 1, device_pool(c->device), c->st);
}
inline void ctx_free(const sl_ctx *c, void *p)
{
    if (p) cudaFreeAsync(p, c->st);
}
}  // namespace sl
