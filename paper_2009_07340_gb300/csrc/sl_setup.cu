// sl_setup.cu -- device kernels around the step: reference nodes, prescribed
// fields at the nodes and faces, the initial state (Section 5.1), the Wiener
// increments (Section 5.2) and the sample moments (Section 5.4).
#include <cmath>
#include <cstdint>

#include <algorithm>

#include <type_traits>

#include "sl_internal.cuh"
#include "sl_rng.cuh"

namespace sl {

// Chebyshev-Gauss nodes on [0,1]: xi_i = (1 - cos((i + 1/2) pi / N)) / 2
// (Eq. gaussquad with (i+1/2)/N, interleaved with the Lobatto nodes).
__device__ __forceinline__ double gauss_node(int i, int N) { return 0.5 * (1.0 - cospi((i + 0.5) / N)); }

// d h_m / d xi at x for the Lagrange basis on the Gauss nodes (product rule).
__device__ double lagrange_deriv(int N, int m, double x)
{
    double sum = 0.0;
    const double xm = gauss_node(m, N);
    for (int k = 0; k < N; ++k) {
        if (k == m) continue;
        double v = 1.0 / (xm - gauss_node(k, N));
        for (int l = 0; l < N; ++l)
            if (l != m && l != k) v *= (x - gauss_node(l, N)) / (xm - gauss_node(l, N));
        sum += v;
    }
    return sum;
}

__device__ void drift_at(const FieldDev &f, double x, double y, double &ux, double &uy)
{
    const double *p = f.p;
    switch (f.kind) {
    case SL_U_CONST: ux = p[0]; uy = p[1]; break;
    case SL_U_SIN: ux = p[0] + p[1] * sin(p[2] * M_PI * x); uy = 0.0; break;
    default: ux = -p[0] * (y - p[2]); uy = p[0] * (x - p[1]); break;  // SL_U_ROTATION
    }
}

__device__ double diffusion_at(const FieldDev &f, double x, double y)
{
    const double *p = f.p;
    switch (f.kind) {
    case SL_D_CONST: return p[0];
    case SL_D_COS: return p[0] * (1.0 + p[1] * cos(p[2] * M_PI * x));
    default: return p[0] * (1.0 + p[1] * sin(p[2] * M_PI * x) * sin(p[3] * M_PI * y));  // SL_D_SINSIN
    }
}

// h_l(x): the Lagrange basis polynomial l on the Gauss nodes (product form).
__device__ double lagrange_at(int N, int l, double x)
{
    const double xl = gauss_node(l, N);
    double v = 1.0;
    for (int k = 0; k < N; ++k)
        if (k != l) v *= (x - gauss_node(k, N)) / (xl - gauss_node(k, N));
    return v;
}

// Nodal fields (node values handed over by a field solver, Section 5.2).
// Value at node v = e n + p; the drift's y component follows its x block.
__device__ __forceinline__ void node_drift(const FieldDev &f, const Mesh &m, long long v, double x, double y,
                                           double &ux, double &uy)
{
    if (f.kind == SL_U_NODAL) {
        ux = f.nodal[v];
        uy = m.dim == 2 ? f.nodal[(long long)m.E * m.n + v] : 0.0;
    } else {
        drift_at(f, x, y, ux, uy);
    }
}

__device__ __forceinline__ double node_diffusion(const FieldDev &f, long long v, double x, double y)
{
    return f.kind == SL_D_NODAL ? f.nodal[v] : diffusion_at(f, x, y);
}

// Trace of element e's nodal interpolant of vals ([E][n]) on its face
// xi_dir = side, at the face's Gauss point pt (0 in 1D).
__device__ double trace_of(const Mesh &m, const double *vals, int e, int dir, double side, int pt)
{
    const int N = m.N;
    double s = 0.0;
    for (int l = 0; l < N; ++l) {
        const int node = m.dim == 1 ? l : (dir == 0 ? pt * N + l : l * N + pt);
        s += lagrange_at(N, l, side) * vals[(long long)e * m.n + node];
    }
    return s;
}

// A nodal field at point pt of interface idx (0..K along dir) on grid line
// `line` (the element row for dir 0, the column for dir 1): the interface
// table when given (1D [K+1]; 2D vertical [K1][K0+1][N] then horizontal
// [K1+1][K0][N]), else the mean of the traces of the elements on both sides,
// the inside one alone at a Dirichlet boundary.  On a periodic mesh
// interface K is interface 0.
__device__ double iface_nodal(const Mesh &m, const double *vals, const double *face, int dir, int line, int idx,
                              int pt)
{
    const int K = m.K[dir];
    if (m.periodic && idx == K) idx = 0;
    if (face) {
        if (m.dim == 1) return face[idx];
        if (dir == 0) return face[((long long)line * (m.K[0] + 1) + idx) * m.N + pt];
        return face[(long long)m.K[1] * (m.K[0] + 1) * m.N + ((long long)idx * m.K[0] + line) * m.N + pt];
    }
    const bool has_l = idx > 0 || m.periodic, has_r = idx < K;
    const int kl = (idx - 1 + K) % K;
    const int el = dir == 0 ? line * m.K[0] + kl : kl * m.K[0] + line;
    const int er = dir == 0 ? line * m.K[0] + idx : idx * m.K[0] + line;
    const double l = has_l ? trace_of(m, vals, el, dir, 1.0, pt) : 0.0;
    const double r = has_r ? trace_of(m, vals, er, dir, 0.0, pt) : 0.0;
    if (has_l && has_r) return 0.5 * (l + r);
    return has_l ? l : r;
}

// Normal drift u_dir and sqrt(2 D) at an interface point at (x, y); nodal
// kinds through iface_nodal, a derived D clipped at 0 (D >= 0 on the nodes
// does not bound the interpolant's trace).
__device__ void face_fields(const FieldDev &fu, const FieldDev &fD, const Mesh &m, int dir, int line, int idx,
                            int pt, double x, double y, double &un, double &b)
{
    if (fu.kind == SL_U_NODAL) {
        un = iface_nodal(m, fu.nodal + (long long)dir * m.E * m.n, fu.face, dir, line, idx, pt);
    } else {
        double ux, uy;
        drift_at(fu, x, y, ux, uy);
        un = dir == 0 ? ux : uy;
    }
    double D;
    if (fD.kind == SL_D_NODAL) {
        D = iface_nodal(m, fD.nodal, fD.face, dir, line, idx, pt);
        if (fD.face && fD.err && !(D >= 0.0)) atomicOr(fD.err, 4);  // a given value below 0
        D = fmax(D, 0.0);  // a derived trace may undershoot
    } else {
        D = diffusion_at(fD, x, y);
    }
    b = sqrt(2.0 * D);
}

__device__ double phi0_at(const FieldDev &f, const Mesh &m, double x, double y)
{
    const double *p = f.p;
    switch (f.kind) {
    case SL_PHI_GAUSS: {
        const double Lx = m.hi[0] - m.lo[0], Ly = m.hi[1] - m.lo[1];
        const int ny = m.dim == 2 ? 1 : 0;
        double v = 0.0;
        for (int ix = -1; ix <= 1; ++ix)
            for (int iy = -ny; iy <= ny; ++iy) {
                const double dx = x - p[2] + ix * Lx;
                double r2 = dx * dx;
                if (m.dim == 2) {
                    const double dy = y - p[3] + iy * Ly;
                    r2 += dy * dy;
                }
                v += exp(-r2 / (2.0 * p[1] * p[1]));
            }
        return p[0] * v;
    }
    case SL_PHI_FOURIER: {
        double v = p[0];
        const int nk = int(p[2]);
        for (int k = 1; k <= nk; ++k)
            v += p[3 + 2 * (k - 1)] * cos(k * p[1] * M_PI * x) + p[4 + 2 * (k - 1)] * sin(k * p[1] * M_PI * x);
        return v;
    }
    case SL_PHI_SINE: return p[0] + p[1] * sin(2.0 * M_PI * p[2] * x);
    default: return p[0] + p[1] * sin(2.0 * M_PI * p[2] * x) * sin(2.0 * M_PI * p[2] * y);  // SL_PHI_SINSIN
    }
}

// One thread per node (e, p): physical coordinates, drift, sqrt(2D), the
// divergence of the drift by spectral differentiation along the element's
// grid lines (the paper takes du/dx from the DSEM solver, Section 5.2), and
// the initial value written to every sample.
__device__ __forceinline__ void store_state(double *Q, long long i, double v) { Q[i] = v; }
__device__ __forceinline__ void store_state(float2 *Q, long long i, double v)
{
    const float hi = float(v);
    Q[i] = make_float2(hi, float(v - double(hi)));
}
__device__ __forceinline__ double load_state(const double *Q, long long i) { return Q[i]; }
__device__ __forceinline__ double load_state(const float2 *Q, long long i)
{
    const float2 v = Q[i];
    return double(v.x) + double(v.y);
}

template <typename State>
__global__ void init_nodes_kernel(Mesh m, FieldDev fu, FieldDev fD, FieldDev fphi, const double *phi0_nodal,
                                  double *xi, double *nodeU, double *nodeB, double *nodeDiv, State *Q, int M)
{
    const long long V = (long long)m.E * m.n;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < m.N && blockIdx.x == 0) xi[v] = gauss_node(int(v), m.N);
    if (v >= V) return;
    const int e = int(v / m.n), p = int(v % m.n);
    const int N = m.N;
    const int kx = e % m.K[0], ky = e / m.K[0];
    const int i = p % N, j = p / N;
    const double x = m.lo[0] + (kx + gauss_node(i, N)) * m.h[0];
    const double y = m.dim == 2 ? m.lo[1] + (ky + gauss_node(j, N)) * m.h[1] : 0.0;
    double ux, uy;
    node_drift(fu, m, v, x, y, ux, uy);
    nodeU[v] = ux;
    if (m.dim == 2) nodeU[V + v] = uy;
    const double Dv = node_diffusion(fD, v, x, y);
    if (fD.err && !(Dv >= 0.0)) atomicOr(fD.err, 4);  // tables read in place are checked here
    nodeB[v] = sqrt(2.0 * Dv);
    // divergence
    const long long ve = (long long)e * m.n;
    double dx = 0.0, dy = 0.0;
    for (int l = 0; l < N; ++l) {
        double uxl, uyl, dummy;
        if (m.dim == 1) {
            node_drift(fu, m, ve + l, m.lo[0] + (kx + gauss_node(l, N)) * m.h[0], 0.0, uxl, dummy);
            dx += lagrange_deriv(N, l, gauss_node(i, N)) * uxl;
        } else {
            node_drift(fu, m, ve + j * N + l, m.lo[0] + (kx + gauss_node(l, N)) * m.h[0], y, uxl, dummy);
            dx += lagrange_deriv(N, l, gauss_node(i, N)) * uxl;
            node_drift(fu, m, ve + l * N + i, x, m.lo[1] + (ky + gauss_node(l, N)) * m.h[1], dummy, uyl);
            dy += lagrange_deriv(N, l, gauss_node(j, N)) * uyl;
        }
    }
    nodeDiv[v] = dx / m.h[0] + (m.dim == 2 ? dy / m.h[1] : 0.0);
    if (!Q) return;  // coefficients only (new fields between steps)
    const double phi = phi0_nodal ? phi0_nodal[v] : phi0_at(fphi, m, x, y);
    for (int s = 0; s < M; ++s) store_state(Q, (long long)s * V + v, phi);
}

// Interface coefficients.  1D: interface f (left face of element f) at
// x_f = lo + f h.  2D: for each element the N points of its low-x face
// (normal drift u_x) and of its low-y face (u_y), at the Gauss-node positions.
__global__ void init_faces_kernel(Mesh m, FieldDev fu, FieldDev fD, double *faceU, double *faceB)
{
    const int nf = m.dim == 1 ? m.E + 1 : m.E * m.N;  // 1D: interfaces 0..K (K: x = hi)
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nf) return;
    if (m.dim == 1) {
        const double xf = v == m.E ? m.hi[0] : m.lo[0] + v * m.h[0];  // v = E: the boundary x = hi
        face_fields(fu, fD, m, 0, 0, v, 0, xf, 0.0, faceU[v], faceB[v]);
        return;
    }
    const int e = v / m.N, f = v % m.N;
    const int kx = e % m.K[0], ky = e / m.K[0];
    const double xv = m.lo[0] + kx * m.h[0], yv = m.lo[1] + (ky + gauss_node(f, m.N)) * m.h[1];
    face_fields(fu, fD, m, 0, ky, kx, f, xv, yv, faceU[v], faceB[v]);
    const double xh = m.lo[0] + (kx + gauss_node(f, m.N)) * m.h[0], yh = m.lo[1] + ky * m.h[1];
    face_fields(fu, fD, m, 1, kx, ky, f, xh, yh, faceU[nf + v], faceB[nf + v]);
}

cudaError_t launch_init_fields(const Mesh &m, const FieldDev &u, const FieldDev &D, const FieldDev &phi0,
                               const double *phi0_nodal_dev, double *xi, double *nodeU, double *nodeB,
                               double *nodeDiv, double *faceU, double *faceB, void *Q, int M,
                               int state_is_double, cudaStream_t st)
{
    const long long V = (long long)m.E * m.n;
    const int tb = 128;
    const unsigned nb = unsigned((V + tb - 1) / tb);
    if (state_is_double)
        init_nodes_kernel<double><<<nb, tb, 0, st>>>(m, u, D, phi0, phi0_nodal_dev, xi, nodeU, nodeB, nodeDiv,
                                                     static_cast<double *>(Q), M);
    else
        init_nodes_kernel<float2><<<nb, tb, 0, st>>>(m, u, D, phi0, phi0_nodal_dev, xi, nodeU, nodeB, nodeDiv,
                                                     static_cast<float2 *>(Q), M);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nf = m.dim == 1 ? m.E + 1 : m.E * m.N;
    init_faces_kernel<<<(nf + tb - 1) / tb, tb, 0, st>>>(m, u, D, faceU, faceB);
    return cudaGetLastError();
}

// dW[t][s][d] = sqrt(dt) z_d for step counter step0 + t and sample
// sample0 + s.
__global__ void wiener_kernel(unsigned long long seed, long long step0, long long sample0, int nsteps, int M,
                              int dim, double sqrt_dt, double *out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nsteps * M) return;
    const int t = int(idx / M), s = int(idx % M);
    const double2 z = normal_pair(seed, uint32_t(step0 + t), uint32_t(sample0 + s), 0u);
    out[idx * dim] = __dmul_rn(sqrt_dt, z.x);
    if (dim == 2) out[idx * dim + 1] = __dmul_rn(sqrt_dt, z.y);
}

cudaError_t launch_wiener(unsigned long long seed, long long step0, long long sample0, int nsteps, int M,
                          int dim, double sqrt_dt, double *out, cudaStream_t st)
{
    const long long n = (long long)nsteps * M;
    if (n == 0) return cudaSuccess;
    const int tb = 128;
    wiener_kernel<<<unsigned((n + tb - 1) / tb), tb, 0, st>>>(seed, step0, sample0, nsteps, M, dim, sqrt_dt, out);
    return cudaGetLastError();
}

// Batched Wiener increments: job i covers [prefix[i], prefix[i+1]) =
// nsteps x M_i entries, for the step counters steps[i] .. steps[i]+nsteps-1
// (read on the device, so a captured graph replays with advancing counters).
__global__ void wiener_batch_kernel(const WienerJob *__restrict__ jobs, const long long *__restrict__ prefix, int njobs,
                                    int nsteps, const long long *__restrict__ steps, long long total)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= idx) lo = mid;
        else hi = mid - 1;
    }
    const WienerJob j = jobs[lo];
    const long long local = idx - prefix[lo];
    const int t = int(local / j.M), s = int(local % j.M);
    const double2 z = normal_pair(j.seed, uint32_t(steps[lo] + t), uint32_t(j.sample0 + s), 0u);
    j.out[local * j.dim] = __dmul_rn(j.sqrt_dt, z.x);
    if (j.dim == 2) j.out[local * j.dim + 1] = __dmul_rn(j.sqrt_dt, z.y);
}

cudaError_t launch_wiener_batch(const WienerJob *jobs, const long long *prefix, int njobs, int nsteps,
                                const long long *steps, long long total, cudaStream_t st)
{
    if (total == 0) return cudaSuccess;
    const int tb = 256;
    wiener_batch_kernel<<<unsigned((total + tb - 1) / tb), tb, 0, st>>>(jobs, prefix, njobs, nsteps, steps, total);
    return cudaGetLastError();
}

__global__ void advance_counters_kernel(long long *steps, int n, int by)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) steps[i] += by;
}

cudaError_t launch_advance_counters(long long *steps, int n, int by, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    advance_counters_kernel<<<(n + 255) / 256, 256, 0, st>>>(steps, n, by);
    return cudaGetLastError();
}

// Moments, Eq. (averaged), in a fixed summation order.  A warp owns
// kMomVL x W consecutive values (W = 2 when V is even and the state is
// 16-byte aligned: one 16-byte load per value lane) and chunk c = blockIdx.y
// of `chunk` consecutive samples.  Its lanes form kMomSL sample lanes of
// kMomVL value lanes: sample lane j adds samples s0 + j, s0 + j + kMomSL,
// ... in ascending order (each warp load reads kMomSL rows of 128
// contiguous bytes), and the sample lanes' sums are then added by a
// butterfly of warp shuffles (lanes j and j ^ 1, then j ^ 2), which lands
// the same bits in every lane.  psum/psq [c][V] receive the chunk sums; the
// final pass adds them in ascending c in FP64.
//
// Running sums: FP64 for FP64 states.  For float-pair states (value hi +
// lo) float pairs kept exact to about 2^-48 relative by error-free
// transformations (TwoSum, and the FMA product error), on the FP32 pipe:
// FP64 arithmetic runs at 1/64 of the FP32 rate on GB300, and FP64 adds per
// loaded value made the pass FP64-bound.  The pairs are rounded to FP64
// once per chunk.
constexpr int kMomThreads = 128;
constexpr int kMomSL = 4;            // sample lanes per warp
constexpr int kMomVL = 32 / kMomSL;  // value lanes per warp

struct PairSum {  // s = hi + lo, |lo| <= ulp(hi) / 2
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float xh, float xl)
    {
        const float t = __fadd_rn(hi, xh);
        const float bb = __fsub_rn(t, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(xh, bb));  // TwoSum(hi, xh)
        const float e = __fadd_rn(err, __fadd_rn(lo, xl));
        hi = __fadd_rn(t, e);
        lo = __fsub_rn(e, __fsub_rn(hi, t));  // FastTwoSum(t, e)
    }
    // x = xh + xl squared: xh^2 exactly as a pair (FMA), the rest (below
    // 2^-24 of it) in FP32
    __device__ __forceinline__ void add_square(float xh, float xl)
    {
        const float p = __fmul_rn(xh, xh);
        const float pe = __fmaf_rn(xh, xh, -p);
        add(p, __fmaf_rn(__fadd_rn(xh, xh), xl, __fmaf_rn(xl, xl, pe)));
    }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

template <typename State, int W>
struct MomLoad;
template <>
struct MomLoad<double, 1> {
    using T = double;
    __device__ static void get(const T &v, double *x) { x[0] = v; }
};
template <>
struct MomLoad<double, 2> {
    using T = double2;
    __device__ static void get(const T &v, double *x) { x[0] = v.x, x[1] = v.y; }
};
template <>
struct MomLoad<float2, 1> {
    using T = float2;
    __device__ static void get(const T &v, float *h, float *l) { h[0] = v.x, l[0] = v.y; }
};
template <>
struct MomLoad<float2, 2> {
    using T = float4;
    __device__ static void get(const T &v, float *h, float *l) { h[0] = v.x, l[0] = v.y, h[1] = v.z, l[1] = v.w; }
};

template <typename State, int W>
__global__ void __launch_bounds__(kMomThreads) moments_partial_kernel(const State *__restrict__ Q, int M, long long V,
                                                                      int chunk, double *__restrict__ psum,
                                                                      double *__restrict__ psq)
{
    using L = MomLoad<State, W>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = lane / kMomVL, i = lane % kMomVL;  // sample lane, value lane
    const long long v0 = (((long long)blockIdx.x * (kMomThreads / 32) + warp) * kMomVL + i) * W;
    const bool live = v0 < V;  // W = 2 only for even V: a live lane's pair lies inside [0, V)
    const int c = blockIdx.y;
    const long long s0 = (long long)c * chunk + j, s1 = min((long long)M, (long long)c * chunk + chunk);
    const typename L::T *q = reinterpret_cast<const typename L::T *>(Q + (live ? v0 : 0));
    const long long stride = V / W;  // one sample, in loads
    double a[W], b[W];
    if constexpr (std::is_same<State, double>::value) {
#pragma unroll
        for (int k = 0; k < W; ++k) a[k] = b[k] = 0.0;
        if (live) {
#pragma unroll 4
            for (long long s = s0; s < s1; s += kMomSL) {
                double x[W];
                L::get(q[s * stride], x);
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    a[k] += x[k];
                    b[k] = fma(x[k], x[k], b[k]);
                }
            }
        }
#pragma unroll
        for (int off = kMomVL; off < 32; off <<= 1)
#pragma unroll
            for (int k = 0; k < W; ++k) {
                a[k] += __shfl_xor_sync(0xffffffffu, a[k], off);
                b[k] += __shfl_xor_sync(0xffffffffu, b[k], off);
            }
    } else {
        PairSum pa[W], pb[W];
        if (live) {
#pragma unroll 4
            for (long long s = s0; s < s1; s += kMomSL) {
                float h[W], l[W];
                L::get(q[s * stride], h, l);
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    pa[k].add(h[k], l[k]);
                    pb[k].add_square(h[k], l[k]);
                }
            }
        }
#pragma unroll
        for (int off = kMomVL; off < 32; off <<= 1)
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const float ah = __shfl_xor_sync(0xffffffffu, pa[k].hi, off);
                const float al = __shfl_xor_sync(0xffffffffu, pa[k].lo, off);
                const float bh = __shfl_xor_sync(0xffffffffu, pb[k].hi, off);
                const float bl = __shfl_xor_sync(0xffffffffu, pb[k].lo, off);
                pa[k].add(ah, al);
                pb[k].add(bh, bl);
            }
#pragma unroll
        for (int k = 0; k < W; ++k) a[k] = pa[k].value(), b[k] = pb[k].value();
    }
    if (live && j == 0)
#pragma unroll
        for (int k = 0; k < W; ++k) {
            psum[(long long)c * V + v0 + k] = a[k];
            psq[(long long)c * V + v0 + k] = b[k];
        }
}

// The final pass: a block owns 32 consecutive values (one per lane) and its
// kFinWarps warps split the chunks, warp w adding chunks w, w + kFinWarps,
// ... in ascending order; warp 0 then adds the warps' sums in ascending w.
constexpr int kFinWarps = 8;

__global__ void __launch_bounds__(32 * kFinWarps)
    moments_final_kernel(const double *__restrict__ psum, const double *__restrict__ psq, int nc, long long V,
                         double M, double *__restrict__ mean, double *__restrict__ m2)
{
    __shared__ double sa[kFinWarps][32], sb[kFinWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long v = (long long)blockIdx.x * 32 + lane;
    double a = 0.0, b = 0.0;
    if (v < V) {
#pragma unroll 4
        for (int c = w; c < nc; c += kFinWarps) {
            a += psum[(long long)c * V + v];
            b += psq[(long long)c * V + v];
        }
    }
    sa[w][lane] = a;
    sb[w][lane] = b;
    __syncthreads();
    if (w == 0 && v < V) {
        double ta = sa[0][lane], tb = sb[0][lane];
#pragma unroll
        for (int k = 1; k < kFinWarps; ++k) {
            ta += sa[k][lane];
            tb += sb[k][lane];
        }
        mean[v] = ta / M;
        if (m2) m2[v] = tb / M;
    }
}

// 2D faces on the upper domain boundaries (used with Dirichlet boundaries):
// x = hi at the Gauss nodes of each row, then y = hi at those of each column.
__global__ void init_faces_hi_kernel(Mesh m, FieldDev fu, FieldDev fD, double *faceUhi, double *faceBhi)
{
    const int nx = m.K[1] * m.N, ny = m.K[0] * m.N;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nx + ny) return;
    if (v < nx) {  // x = hi at the Gauss nodes of element row v / N
        const double y = m.lo[1] + (v / m.N + gauss_node(v % m.N, m.N)) * m.h[1];
        face_fields(fu, fD, m, 0, v / m.N, m.K[0], v % m.N, m.hi[0], y, faceUhi[v], faceBhi[v]);
    } else {  // y = hi at the Gauss nodes of element column w / N
        const int w = v - nx;
        const double x = m.lo[0] + (w / m.N + gauss_node(w % m.N, m.N)) * m.h[0];
        face_fields(fu, fD, m, 1, w / m.N, m.K[1], w % m.N, x, m.hi[1], faceUhi[v], faceBhi[v]);
    }
}

cudaError_t launch_init_faces_hi(const Mesh &m, const FieldDev &u, const FieldDev &D, double *faceUhi, double *faceBhi,
                                 cudaStream_t st)
{
    const int total = (m.K[0] + m.K[1]) * m.N;
    init_faces_hi_kernel<<<(total + 127) / 128, 128, 0, st>>>(m, u, D, faceUhi, faceBhi);
    return cudaGetLastError();
}

// Histogram of the M samples at every node (recovery of the PDF by binning
// the samples, Section 5.4): bin b = floor((x - lo) * scale), scale = B /
// (hi - lo), in FP64; x = hi goes to the last bin; x outside [lo, hi] (or
// NaN) is not counted.  A block owns `npb` consecutive nodes and counts in
// shared memory; consecutive threads read consecutive nodes of one sample.
template <typename State>
__global__ void pdf_kernel(const State *__restrict__ Q, int M, long long V, int B, double lo, double hi,
                           double scale, int npb, unsigned int *__restrict__ counts)
{
    extern __shared__ unsigned int hist[];  // [npb][B]
    const long long v0 = (long long)blockIdx.x * npb;
    const int nb = int(min((long long)npb, V - v0));
    for (int i = threadIdx.x; i < nb * B; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const long long work = (long long)nb * M;
    for (long long i = threadIdx.x; i < work; i += blockDim.x) {
        const int j = int(i % nb);
        const long long s = i / nb;
        const double x = load_state(Q, s * V + v0 + j);
        if (!(x >= lo && x <= hi)) continue;
        int b = int(floor((x - lo) * scale));
        if (b > B - 1) b = B - 1;
        atomicAdd(&hist[j * B + b], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb * B; i += blockDim.x) counts[v0 * B + i] = hist[i];
}

cudaError_t launch_pdf(const void *Q, int state_is_double, int M, long long V, int B, double lo, double hi,
                       unsigned int *counts, cudaStream_t st)
{
    const int npb = std::max(1, std::min(64, int((48 * 1024 / 4) / B)));
    const size_t smem = size_t(npb) * B * sizeof(unsigned int);
    const unsigned grid = unsigned((V + npb - 1) / npb);
    const double scale = double(B) / (hi - lo);
    if (V == 0) return cudaSuccess;
    if (state_is_double)
        pdf_kernel<double><<<grid, 256, smem, st>>>(static_cast<const double *>(Q), M, V, B, lo, hi, scale, npb, counts);
    else
        pdf_kernel<float2><<<grid, 256, smem, st>>>(static_cast<const float2 *>(Q), M, V, B, lo, hi, scale, npb, counts);
    return cudaGetLastError();
}

// Eq. re-seed: every sample of every node set to the node's sample mean.
template <typename State>
__global__ void reseed_kernel(State *Q, const double *__restrict__ mean, int M, long long V)
{
    const long long total = (long long)M * V;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        store_state(Q, i, mean[i % V]);
}

cudaError_t launch_reseed(void *Q, int state_is_double, int M, long long V, const double *mean, cudaStream_t st)
{
    const int tb = 256;
    const long long total = (long long)M * V;
    const unsigned grid = unsigned(std::min<long long>((total + tb - 1) / tb, 152LL * 16));
    if (total == 0) return cudaSuccess;
    if (state_is_double)
        reseed_kernel<double><<<grid, tb, 0, st>>>(static_cast<double *>(Q), mean, M, V);
    else
        reseed_kernel<float2><<<grid, tb, 0, st>>>(static_cast<float2 *>(Q), mean, M, V);
    return cudaGetLastError();
}

cudaError_t launch_moment_partials(const void *Q, int state_is_double, int M, long long V, int chunk, double *psum,
                                   double *psq, cudaStream_t st)
{
    const int nc = (M + chunk - 1) / chunk;
    if (nc > 65535) return cudaErrorInvalidValue;  // chunks are the grid's y dimension
    // two values per thread where V is even and the state starts on a
    // 16-byte boundary (then every sample row does: 16-byte loads)
    const bool two = V % 2 == 0 && reinterpret_cast<uintptr_t>(Q) % 16 == 0;
    const long long per_block = (kMomThreads / 32) * kMomVL * (two ? 2 : 1);  // values per block
    const dim3 g1(unsigned((V + per_block - 1) / per_block), unsigned(nc));
    if (state_is_double) {
        const double *q = static_cast<const double *>(Q);
        if (two) moments_partial_kernel<double, 2><<<g1, kMomThreads, 0, st>>>(q, M, V, chunk, psum, psq);
        else moments_partial_kernel<double, 1><<<g1, kMomThreads, 0, st>>>(q, M, V, chunk, psum, psq);
    } else {
        const float2 *q = static_cast<const float2 *>(Q);
        if (two) moments_partial_kernel<float2, 2><<<g1, kMomThreads, 0, st>>>(q, M, V, chunk, psum, psq);
        else moments_partial_kernel<float2, 1><<<g1, kMomThreads, 0, st>>>(q, M, V, chunk, psum, psq);
    }
    return cudaGetLastError();
}

cudaError_t launch_moments_combine(const double *psum, const double *psq, int nc, long long V, long long M,
                                   double *mean, double *m2, cudaStream_t st)
{
    moments_final_kernel<<<unsigned((V + 31) / 32), 32 * kFinWarps, 0, st>>>(psum, psq, nc, V, double(M), mean, m2);
    return cudaGetLastError();
}

cudaError_t launch_moments(const void *Q, int state_is_double, int M, long long V, int chunk, double *psum,
                           double *psq, double *mean, double *m2, cudaStream_t st)
{
    const int nc = (M + chunk - 1) / chunk;
    const cudaError_t e = launch_moment_partials(Q, state_is_double, M, V, chunk, psum, psq, st);
    return e != cudaSuccess ? e : launch_moments_combine(psum, psq, nc, V, M, mean, m2, st);
}

// Advance coefficients of the 2D step for step size dt, formed once per
// step size and field change instead of in every step of every sample: the
// particle displacement is then one FMA per direction, dx = ax + bx dW, in
// the kernel's own precision (FP64 arithmetic is 1/64 of the FP32 rate).
template <typename R>
__global__ void coef2d_kernel(const double *__restrict__ nodeU, const double *__restrict__ nodeB,
                              const double *__restrict__ nodeDiv, long long V, double dt, double s4x, double s4y,
                              R *__restrict__ out)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const double b = nodeB[v];
    out[v] = R(__dmul_rn(__dmul_rn(nodeU[v], dt), s4x));
    out[V + v] = R(__dmul_rn(__dmul_rn(nodeU[V + v], dt), s4y));
    out[2 * V + v] = R(__dmul_rn(b, s4x));
    out[3 * V + v] = R(__dmul_rn(b, s4y));
    out[4 * V + v] = R(__dmul_rn(dt, nodeDiv[v]));
}

cudaError_t launch_coef2d(const double *nodeU, const double *nodeB, const double *nodeDiv, long long V, double dt,
                          double s4x, double s4y, bool fp64, void *out, cudaStream_t st)
{
    const unsigned grid = unsigned((V + 255) / 256);
    if (fp64)
        coef2d_kernel<double><<<grid, 256, 0, st>>>(nodeU, nodeB, nodeDiv, V, dt, s4x, s4y, static_cast<double *>(out));
    else
        coef2d_kernel<float><<<grid, 256, 0, st>>>(nodeU, nodeB, nodeDiv, V, dt, s4x, s4y, static_cast<float *>(out));
    return cudaGetLastError();
}

void node_tables2d(int N, const double *xi, double *tab)
{
    // the same FP64 expressions, in the same order, as the step kernels used
    // when they formed these tables themselves
    double *Z = tab, *lam = tab + N * N, *h0 = lam + N, *h1 = h0 + N, *x0 = h1 + N, *x1 = x0 + N;
    for (int i = 0; i < N; ++i)
        for (int m = 0; m < N; ++m) Z[i * N + m] = 4.0 * (xi[i] - xi[m]);
    for (int j = 0; j < N; ++j) {
        double l = 1.0, l0 = 1.0, l1 = 1.0;
        for (int m = 0; m < N; ++m)
            if (m != j) {
                l /= 4.0 * (xi[j] - xi[m]);
                l0 *= (0.0 - xi[m]) / (xi[j] - xi[m]);
                l1 *= (1.0 - xi[m]) / (xi[j] - xi[m]);
            }
        lam[j] = l;
        h0[j] = l0;
        h1[j] = l1;
        x0[j] = -4.0 * xi[j];
        x1[j] = 4.0 * (1.0 - xi[j]);
    }
}

cudaError_t preload_setup()
{
    cudaError_t e = prepare_kernel(init_nodes_kernel<double>);
    if (e == cudaSuccess) e = prepare_kernel(init_nodes_kernel<float2>);
    if (e == cudaSuccess) e = prepare_kernel(init_faces_kernel);
    if (e == cudaSuccess) e = prepare_kernel(wiener_kernel);
    if (e == cudaSuccess) e = prepare_kernel(wiener_batch_kernel);
    if (e == cudaSuccess) e = prepare_kernel(advance_counters_kernel);
    if (e == cudaSuccess) e = prepare_kernel(moments_partial_kernel<double, 1>);
    if (e == cudaSuccess) e = prepare_kernel(moments_partial_kernel<double, 2>);
    if (e == cudaSuccess) e = prepare_kernel(moments_partial_kernel<float2, 1>);
    if (e == cudaSuccess) e = prepare_kernel(moments_partial_kernel<float2, 2>);
    if (e == cudaSuccess) e = prepare_kernel(moments_final_kernel);
    if (e == cudaSuccess) e = prepare_kernel(coef2d_kernel<double>);
    if (e == cudaSuccess) e = prepare_kernel(coef2d_kernel<float>);
    if (e == cudaSuccess) e = prepare_kernel(reseed_kernel<double>);
    if (e == cudaSuccess) e = prepare_kernel(init_faces_hi_kernel);
    if (e == cudaSuccess) e = prepare_kernel(pdf_kernel<double>);
    if (e == cudaSuccess) e = prepare_kernel(pdf_kernel<float2>);
    if (e == cudaSuccess) e = prepare_kernel(reseed_kernel<float2>);
    return e;
}

}  // namespace sl
