// sl_step2d.cuh -- 2D semi-Lagrangian Monte-Carlo step on tensor-product
// elements (n = N^2 Gauss nodes per element, nodes p = j*N + i, x fastest).
//
// Per element-sample and step (Sections 5.2-5.3 in tensor form; the paper
// defers the multi-dimensional remap to the authors' earlier deterministic
// paper, so the reading is: tensor Lagrange basis on the scattered advected
// particles, 4N face rows at the Gauss-node positions of the four faces):
//   particle p moves from its node by (dx_p, dy_p) = (u_x dt + b dW_x,
//   u_y dt + b dW_y) / h  (Eq. def_dx, one dW per sample and dimension);
//   phi*_p = Q_p - dt (div u)_p Q_p                     (Eq. advection_phi);
//   V[p][(i',j')] = h_i'(x*_p) h_j'(y*_p) (Gauss-node basis at the particles);
//   phase 1: alpha = V^{-1} phi* (nodal values of the advected interpolant),
//            face values B alpha at the 4N face points  (Eq. remap_bnd);
//   phase 2: upwind face values g (Eq. bnd_update) and
//            q = argmin |V q - phi*|^2 + |B q - g|^2     (Section 5.3).
// The two phases are two launches per step: phase 2 of an element needs its
// neighbours' phase-1 face values.
//
// Mapping: a group of n threads (rounded up to a warp multiple, its own named
// barrier) per element-sample; thread p owns particle p.  Rows of the stacked
// system [V; B] (B only in phase 2) are staged in shared memory; thread c
// builds row c of the Gram matrix G = [V;B]^T [V;B] in registers and the
// group solves G x = [V;B]^T rhs by Gauss-Jordan elimination without
// pivoting (G is SPD), one broadcast pivot row per step.  Everything is
// relative to the element reference value c (the middle node's state):
// [V;B] 1 = 1 (partition of unity), so the unknown is q - c.  The FP32 mode
// keeps the state and face values as float pairs (as in 1D) and applies one
// step of iterative refinement of the stacked least-squares residual against
// the original rows, replaying the stored elimination multipliers.
#pragma once
#include <cooperative_groups.h>

#include <algorithm>

#include <type_traits>

#include "sl_internal.cuh"

namespace sl {

constexpr int kGroupThreads2D = 256;  // threads per CTA

__device__ __forceinline__ void two_sum2d(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// A boundary value as a face value: FP64, or the float pair hi + lo.
template <typename FaceT>
__device__ __forceinline__ FaceT ghost_face2d(double g)
{
    if constexpr (std::is_same<FaceT, double>::value) {
        return g;
    } else {
        const float hi = float(g);
        return make_float2(hi, float(g - double(hi)));
    }
}

__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// 16-byte vectors of R for shared-memory rows (every row and sub-array of a
// group starts on a 16-byte boundary; rows are LD >= n (rounded to 4) long).
template <typename R>
struct Vec16;
template <>
struct Vec16<float> {
    using T = float4;
    static constexpr int W = 4;
    __device__ static float at(const float4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
    __device__ static float4 make(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};
template <>
struct Vec16<double> {
    using T = double2;
    static constexpr int W = 2;
    __device__ static double at(const double2 &v, int i) { return i == 0 ? v.x : v.y; }
    __device__ static double2 make(double a, double b, double, double) { return make_double2(a, b); }
};

// Lanes per Gram row: one while a row of n values fits in a thread's
// registers (FP32 n <= 81, FP64 n <= 64); above that the row's columns are
// split over SP adjacent lanes of one warp, which exchange the pivot-column
// entries by shuffles.  FP32 N = 10 would fit in one lane but runs faster on
// two (more warps per SM); N = 9 runs faster on one.  FP32 N = 12 on two
// lanes at two CTAs per SM keeps its row in local memory (7.5x slower), so
// it takes four lanes and one CTA.
template <int N, typename R>
constexpr int split2d()
{
    return std::is_same<R, float>::value ? (N <= 9 ? 1 : (N <= 11 ? 2 : 4)) : (N <= 8 ? 1 : (N <= 10 ? 2 : 4));
}

template <int N, typename R, int NCOMP = 1>
struct Geo2D {
    static constexpr int n = N * N;
    static constexpr int SP = split2d<N, R>();                  // lanes per row
    static constexpr int VWg = sizeof(R) == 4 ? 4 : 2;          // values per 16 bytes
    // columns per lane (SP > 1), widened by one 16-byte vector where a lane's
    // block would span a multiple of 128 bytes: the lanes of a row then read
    // a shared row at offsets in different banks
    static constexpr int NC0 = ((n + SP - 1) / SP + VWg - 1) / VWg * VWg;
    static constexpr int NC = (NC0 * int(sizeof(R))) % 128 == 0 ? NC0 + VWg : NC0;
    static constexpr int GS = (SP * n + 31) / 32 * 32;          // threads per group
    static constexpr int GPC = GS >= kGroupThreads2D ? 1 : kGroupThreads2D / GS;  // groups per CTA
    static constexpr int kBlock = GPC * GS;                     // threads per CTA
    static constexpr int LD = (SP == 1 ? n : (n > SP * NC ? n : SP * NC)) + 3 & ~3;  // row stride (16-byte rows)
    static constexpr int P = n + 4 * N;                         // stacked rows
    // per-group shared memory (elements of R)
    static constexpr int P4 = (P + 3) & ~3;                     // P rounded to 16-byte multiples
    // rhs, vec and res hold one P4-long array per field
    static constexpr int kRows = P * LD, kRhs = NCOMP * P4, kPiv = 2 * (LD + 4), kVec = NCOMP * P4, kRes = NCOMP * P4;
    static constexpr int kGroup = (kRows + kRhs + kPiv + kVec + kRes + 3) & ~3;  // keeps rows 16-byte aligned
    // per-CTA tables: Z [N][N], lambda [N], h0 [N], h1 [N]
    static constexpr int kTables = N * N + 3 * N;
};

// CTAs per SM the register budget is sized for: three for FP32 N <= 6
// (1.14-1.31x over two), two where shared memory allows two and the row
// still fits (FP32 N <= 11, FP64 N = 9), one otherwise.  At one CTA the high
// orders ran one element-sample group per SM: two made FP32 N = 9 1.66x,
// N = 10 1.73x, N = 11 2.2x and FP64 N = 9 1.10x faster.  FP64 N <= 6 gained
// nothing from two (FP64-pipe bound).
template <int N, typename R>
constexpr int min_ctas2d()
{
    return std::is_same<R, float>::value ? (N <= 6 ? 3 : (N <= 11 ? 2 : 1)) : (N == 9 ? 2 : 1);
}

// BATCH = false: one instance (a0), group g = element-sample g.
// BATCH = true: `ninst` instances of the same N, instance i owning groups
// [prefix[i], prefix[i+1]) (its E*M element-samples).
// NCOMP = 2: two fields per sample ([M][2][E][n]) on the same particles, so
// one Gram matrix, one elimination and one upwind choice serve both; each
// field has its own right-hand side, refinement, faces and state.
template <int N, typename R, int PHASE, bool BATCH, int NCOMP = 1>
__global__ void __launch_bounds__(Geo2D<N, R>::kBlock, min_ctas2d<N, R>()) sl2d_step_kernel(const Step2DArgs a0, const Step2DArgs *__restrict__ args,
                                                                    const long long *__restrict__ prefix, int ninst, int t)
{
    using G = Geo2D<N, R, NCOMP>;
    constexpr int P4 = G::P4;  // stride of the per-field arrays
    constexpr int n = G::n, LD = G::LD, SP = G::SP, NC = G::NC;
    constexpr int P = PHASE == 1 ? n : G::P;  // rows of the system solved in this phase
    using VV = Vec16<R>;
    using VT = typename VV::T;
    constexpr int VW = VV::W;
    constexpr bool kPair = !std::is_same<R, double>::value;
    using State = typename std::conditional<kPair, float2, double>::type;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *tab = reinterpret_cast<R *>(smem_raw);
    R *sZ = tab;              // [N][N] 4 (xi_i - xi_m)
    R *slam = sZ + N * N;     // [N] barycentric weights of the (scaled) Gauss nodes
    R *sh0 = slam + N;        // [N] h_i(0)
    R *sh1 = sh0 + N;         // [N] h_i(1)
    const int grp = threadIdx.x / G::GS;
    const int tig = threadIdx.x - grp * G::GS;  // thread in the group
    const int c = tig / SP;                     // thread's node / row / column index
    const int h = tig - c * SP;                 // column block of the row (SP > 1)
    const bool lead = h == 0;                   // the row's lane for per-row work
    const int rowbase = (threadIdx.x & 31) - h; // lane of the row's first thread
    R *gbase = tab + ((G::kTables + 3) & ~3) + grp * G::kGroup;
    R *Vs = gbase;                 // [P][LD] stacked rows
    R *rhs = Vs + G::kRows;        // [NCOMP][P4] right-hand sides (relative to c)
    R *piv = rhs + G::kRhs;        // [2][LD + 4] pivot rows (+ b of field 0 at LD, 1 / pivot, b of field 1)
    R *vec = piv + G::kPiv;        // [NCOMP][P4] broadcast vectors
    R *res = vec + G::kVec;        // [NCOMP][P4] residuals

    // node tables depend on N only (every instance of a batch class shares them)
    const double *xi = BATCH ? args[0].xi : a0.xi;
    if (threadIdx.x < N * N) {
        const int i = threadIdx.x / N, m = threadIdx.x % N;
        sZ[threadIdx.x] = R(4.0 * (xi[i] - xi[m]));
    }
    if (threadIdx.x < N) {
        const int j = threadIdx.x;
        double lam = 1.0, l0 = 1.0, l1 = 1.0;
        for (int m = 0; m < N; ++m)
            if (m != j) {
                lam /= 4.0 * (xi[j] - xi[m]);
                l0 *= (0.0 - xi[m]) / (xi[j] - xi[m]);
                l1 *= (1.0 - xi[m]) / (xi[j] - xi[m]);
            }
        slam[j] = R(lam);
        sh0[j] = R(l0);
        sh1[j] = R(l1);
    }
    __syncthreads();

    const long long ggid = (BATCH ? 0 : a0.g0) + (long long)blockIdx.x * G::GPC + grp;
    int inst = 0;
    if constexpr (BATCH) {
        int lo = 0, hi = ninst - 1;  // last instance with prefix[i] <= ggid
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= ggid) lo = mid;
            else hi = mid - 1;
        }
        inst = lo;
    }
    const Step2DArgs a = BATCH ? args[inst] : a0;
    const long long gid = BATCH ? ggid - prefix[inst] : ggid;
    const int E = a.Kx * a.Ky;
    const bool group_active = BATCH ? ggid < prefix[ninst] : gid < a.g1;
    const int s = group_active ? int(gid / E) : 0;
    const int e = group_active ? int(gid % E) : 0;
    const int kx = e % a.Kx, ky = e / a.Kx;
    const bool real = group_active && c < n;     // every lane of a real row
    const bool real_lead = real && lead;          // its per-row work
    const int bar_id = 1 + grp;

    // reference values and own state, per field
    State *Qg = reinterpret_cast<State *>(a.Q);
    long long qoff[NCOMP];
    R ch[NCOMP], cl[NCOMP], qh[NCOMP], ql[NCOMP];
#pragma unroll
    for (int cc = 0; cc < NCOMP; ++cc) {
        qoff[cc] = (((long long)s * NCOMP + cc) * E + e) * n;
        cl[cc] = qh[cc] = ql[cc] = R(0);
        const State cv = Qg[qoff[cc] + n / 2];
        if constexpr (kPair) {
            ch[cc] = cv.x;
            cl[cc] = cv.y;
        } else {
            ch[cc] = cv;
        }
        if (real_lead) {
            const State qv = Qg[qoff[cc] + c];
            if constexpr (kPair) {
                qh[cc] = qv.x;
                ql[cc] = qv.y;
            } else {
                qh[cc] = qv;
            }
        }
    }
    const int ip = c % N, jp = c / N;
    R hx[N], hy[N];
    R ph[NCOMP];
#pragma unroll
    for (int cc = 0; cc < NCOMP; ++cc) ph[cc] = R(0);
    if (real_lead) {
        const long long V = (long long)E * n;
        const double dWx = a.dW[((long long)t * a.M + s) * 2 + 0];
        const double dWy = a.dW[((long long)t * a.M + s) * 2 + 1];
        const double ux = a.nodeU[(long long)e * n + c], uy = a.nodeU[V + (long long)e * n + c];
        const double b = a.nodeB[(long long)e * n + c];
        // explicit unfused products: the compiler may not contract these
        // differently in the batched and single kernels
        const R dx = R(__dmul_rn(4.0, __dadd_rn(__dmul_rn(ux, a.dt), __dmul_rn(b, dWx))) / a.hx);
        const R dy = R(__dmul_rn(4.0, __dadd_rn(__dmul_rn(uy, a.dt), __dmul_rn(b, dWy))) / a.hy);
        const R gam = R(a.dt * a.nodeDiv[(long long)e * n + c]);
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) {
            R dq = qh[cc] - ch[cc];
            if constexpr (kPair) dq += ql[cc] - cl[cc];
            if constexpr (kPair)
                ph[cc] = dq - __fmul_rn(gam, qh[cc]);
            else
                ph[cc] = dq - __dmul_rn(gam, qh[cc]);
        }
        // Gauss-node basis at the particle: h_i'(x) = lam_i' prod_{m != i'} (x - zeta_m),
        // x - zeta_m = Z[ip][m] + dx (node difference plus displacement)
        R pre = R(1);
#pragma unroll
        for (int m = 0; m < N; ++m) {
            hx[m] = pre;
            pre *= sZ[ip * N + m] + dx;
        }
        R suf = R(1);
#pragma unroll
        for (int m = N - 1; m >= 0; --m) {
            hx[m] *= suf * slam[m];
            suf *= sZ[ip * N + m] + dx;
        }
        pre = R(1);
#pragma unroll
        for (int m = 0; m < N; ++m) {
            hy[m] = pre;
            pre *= sZ[jp * N + m] + dy;
        }
        suf = R(1);
#pragma unroll
        for (int m = N - 1; m >= 0; --m) {
            hy[m] *= suf * slam[m];
            suf *= sZ[jp * N + m] + dy;
        }
        // row c of V and its right-hand side
        // (row c of V: entry q = jj N + ii is hx[ii] hy[jj]; 16-byte stores,
        // the padding past n is never read)
#pragma unroll
        for (int q = 0; q < n; q += VW) {
            R v4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) v4[i] = (i < VW && q + i < n) ? hx[(q + i) % N] * hy[(q + i) / N] : R(0);
            *reinterpret_cast<VT *>(Vs + c * LD + q) = VV::make(v4[0], v4[1], v4[2], v4[3]);
        }
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) rhs[cc * P4 + c] = ph[cc];
    }

    using FaceT = typename std::conditional<kPair, float2, double>::type;
    FaceT *faces = reinterpret_cast<FaceT *>(a.faces);
    long long fbase[NCOMP];  // [M][NCOMP][E][4N]
#pragma unroll
    for (int cc = 0; cc < NCOMP; ++cc) fbase[cc] = ((long long)s * NCOMP + cc) * E;
    if constexpr (PHASE == 2) {
        // face rows of B and the upwinded face values g (Eq. bnd_update)
        if (group_active && lead && c < 4 * N) {
            const int side = c / N, f = c % N;
            R *row = Vs + (n + c) * LD;
#pragma unroll
            for (int q = 0; q < n; q += VW) *reinterpret_cast<VT *>(row + q) = VV::make(R(0), R(0), R(0), R(0));
            const double dW = a.dW[((long long)t * a.M + s) * 2 + (side < 2 ? 0 : 1)];
            int e_face;  // element whose low face is this interface
            if (side == 0) e_face = e;
            else if (side == 1) e_face = ky * a.Kx + (kx + 1) % a.Kx;
            else if (side == 2) e_face = e;
            else e_face = ((ky + 1) % a.Ky) * a.Kx + kx;
            // a face on a Dirichlet domain boundary: the ghost value takes the
            // place of the missing neighbour (low side at x = lo / y = lo, high
            // side at x = hi / y = hi); the faces x = hi, y = hi have their own
            // coefficients
            const bool dir = !a.periodic;
            const bool ghost_low = dir && ((side == 0 && kx == 0) || (side == 2 && ky == 0));
            const bool ghost_high = dir && ((side == 1 && kx == a.Kx - 1) || (side == 3 && ky == a.Ky - 1));
            const long long fidx = (long long)(side < 2 ? 0 : 1) * E * N + (long long)e_face * N + f;
            double af, bf;
            if (ghost_high) {
                const long long hidx = side == 1 ? (long long)ky * N + f : (long long)a.Ky * N + (long long)kx * N + f;
                af = a.faceUhi[hidx] * a.dt;
                bf = a.faceBhi[hidx];
            } else {
                af = a.faceU[fidx] * a.dt;
                bf = a.faceB[fidx];
            }
            bool from_low;  // take the value from the element on the low side
            if constexpr (kPair)
                from_low = fmaf(float(bf), float(dW), float(af)) > 0.f;
            else
                from_low = __dadd_rn(af, __dmul_rn(bf, dW)) > 0.0;
            int e_low, e_high;
            if (side == 0) {
                e_low = ky * a.Kx + (kx - 1 + a.Kx) % a.Kx;
                e_high = e;
            } else if (side == 1) {
                e_low = e;
                e_high = e_face;
            } else if (side == 2) {
                e_low = ((ky - 1 + a.Ky) % a.Ky) * a.Kx + kx;
                e_high = e;
            } else {
                e_low = e;
                e_high = e_face;
            }
            const bool xface = side < 2;
            // low element's far face (right / top) or high element's near face (left / bottom)
            // the face rows and values carry the boundary weight w (1 by default)
            const R w = R(a.w);
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) {  // (two fields: periodic meshes only, no ghosts)
                FaceT gv;
                if (from_low && ghost_low)  // left [Ky][N] or bottom [Kx][N] boundary values
                    gv = ghost_face2d<FaceT>(a.ghost[t * a.ghost_w + (side == 0 ? (long long)ky * N + f
                                                                            : 2LL * a.Ky * N + (long long)kx * N + f)]);
                else if (!from_low && ghost_high)  // right [Ky][N] or top [Kx][N]
                    gv = ghost_face2d<FaceT>(a.ghost[t * a.ghost_w + (side == 1 ? (long long)a.Ky * N + (long long)ky * N + f
                                                                            : 2LL * a.Ky * N + (long long)a.Kx * N +
                                                                                  (long long)kx * N + f)]);
                else
                    gv = from_low ? faces[(fbase[cc] + e_low) * 4 * N + (xface ? N : 3 * N) + f]
                                  : faces[(fbase[cc] + e_high) * 4 * N + (xface ? 0 : 2 * N) + f];
                R gr;
                if constexpr (kPair)
                    gr = (gv.x - ch[cc]) + (gv.y - cl[cc]);
                else
                    gr = gv - ch[cc];
                rhs[cc * P4 + n + c] = w * gr;
            }
            if (side == 0)
#pragma unroll
                for (int ii = 0; ii < N; ++ii) row[f * N + ii] = w * sh0[ii];
            else if (side == 1)
#pragma unroll
                for (int ii = 0; ii < N; ++ii) row[f * N + ii] = w * sh1[ii];
            else if (side == 2)
#pragma unroll
                for (int jj = 0; jj < N; ++jj) row[jj * N + f] = w * sh0[jj];
            else
#pragma unroll
                for (int jj = 0; jj < N; ++jj) row[jj * N + f] = w * sh1[jj];
        }
    }
    group_sync(bar_id, G::GS);

    // Gram row c: G[c][c'] = sum_p S[p][c] S[p][c'], b_c = sum_p S[p][c] rhs_p
    // (SP > 1: lane h holds the columns c' = h NC + j, j < NC, of row c)
    constexpr int NG = SP == 1 ? n : NC;
    const int col0 = h * NC;  // first column of this lane (SP > 1)
    R gr[NG];
#pragma unroll
    for (int q = 0; q < NG; ++q) gr[q] = R(0);
    R bc[NCOMP];
#pragma unroll
    for (int cc = 0; cc < NCOMP; ++cc) bc[cc] = R(0);
    if (real) {
        for (int p = 0; p < P; ++p) {
            const R vpc = Vs[p * LD + c];
            const R *rowp = Vs + p * LD;
            if constexpr (SP == 1) {
#pragma unroll
                for (int q = 0; q < n; q += VW) {
                    const VT v = *reinterpret_cast<const VT *>(rowp + q);
#pragma unroll
                    for (int i = 0; i < VW; ++i)
                        if (q + i < n) gr[q + i] = fma(vpc, VV::at(v, i), gr[q + i]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < NC; j += VW) {
                    const VT v = *reinterpret_cast<const VT *>(rowp + col0 + j);
#pragma unroll
                    for (int i = 0; i < VW; ++i)
                        if (col0 + j + i < n) gr[j + i] = fma(vpc, VV::at(v, i), gr[j + i]);
                }
            }
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) bc[cc] = fma(vpc, rhs[cc * P4 + p], bc[cc]);
        }
    }

    // Gauss-Jordan elimination without pivoting (G is SPD); multipliers are
    // kept in the eliminated positions for the refinement replay
    R diag = R(1);
    bool bad = false;
    // entry k of row c, from the lane holding column k (SP > 1: a shuffle
    // executed by every lane of the warp; k is a compile-time index)
    auto row_entry = [&](const int k) -> R {
        if constexpr (SP == 1) {
            return gr[k];
        } else {
            const R mine = h == k / NC ? gr[k % NC] : R(0);
            return __shfl_sync(0xffffffffu, mine, rowbase + k / NC);
        }
    };
#pragma unroll
    for (int k = 0; k < n; ++k) {
        R *pr = piv + (k & 1) * (LD + 4);
        if constexpr (SP == 1) {
            if (c == k) {
#pragma unroll
                for (int q = 0; q < n; q += VW) {
                    R v4[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) v4[i] = (i < VW && q + i < n) ? gr[q + i] : R(0);
                    *reinterpret_cast<VT *>(pr + q) = VV::make(v4[0], v4[1], v4[2], v4[3]);
                }
                pr[LD] = bc[0];
                if constexpr (NCOMP > 1) pr[LD + 2] = bc[1];
                pr[LD + 1] = R(1) / gr[k];
                diag = gr[k];
            }
        } else {
            if (c == k) {  // every lane of the pivot row publishes its columns
#pragma unroll
                for (int j = 0; j < NC; j += VW) {
                    R v4[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) v4[i] = i < VW ? gr[j + i] : R(0);
                    *reinterpret_cast<VT *>(pr + col0 + j) = VV::make(v4[0], v4[1], v4[2], v4[3]);
                }
                if (lead) {
                    pr[LD] = bc[0];
                    if constexpr (NCOMP > 1) pr[LD + 2] = bc[1];
                }
                if (h == k / NC) {
                    pr[LD + 1] = R(1) / gr[k % NC];
                    diag = gr[k % NC];
                }
            }
        }
        group_sync(bar_id, G::GS);
        const R gk = row_entry(k);
        if (real && c != k) {
            const R l = gk * pr[LD + 1];
            // columns < k hold multipliers (eliminated); only q > k change
            if constexpr (SP == 1) {
#pragma unroll
                for (int q = 0; q < n; q += VW) {
                    if (q + VW <= k + 1) continue;  // chunk entirely at or before the pivot column
                    const VT v = *reinterpret_cast<const VT *>(pr + q);
#pragma unroll
                    for (int i = 0; i < VW; ++i)
                        if (q + i > k && q + i < n) gr[q + i] = fma(-l, VV::at(v, i), gr[q + i]);
                }
                gr[k] = l;
            } else {
#pragma unroll
                for (int j = 0; j < NC; j += VW) {
                    const VT v = *reinterpret_cast<const VT *>(pr + col0 + j);
#pragma unroll
                    for (int i = 0; i < VW; ++i) {
                        const int q = col0 + j + i;
                        if (q > k && q < n) gr[j + i] = fma(-l, VV::at(v, i), gr[j + i]);
                    }
                }
                if (h == k / NC) gr[k % NC] = l;
            }
            bc[0] = fma(-l, pr[LD], bc[0]);
            if constexpr (NCOMP > 1) bc[1] = fma(-l, pr[LD + 2], bc[1]);
        }
    }
    if constexpr (SP > 1) diag = __shfl_sync(0xffffffffu, diag, rowbase + (c < n ? c : 0) / NC);  // the row's pivot
    R x[NCOMP];
#pragma unroll
    for (int cc = 0; cc < NCOMP; ++cc) x[cc] = real_lead ? bc[cc] / diag : R(0);
    bad |= real_lead && !(diag > R(0));

    if constexpr (kPair) {
        // one step of iterative refinement of the stacked least-squares
        // residual: r = S^T (rhs - S x), G dx = r, x += dx (per field)
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc)
            if (c < n && lead) vec[cc * P4 + c] = x[cc];  // the group may have more threads than nodes
        group_sync(bar_id, G::GS);
        if (real_lead) {
            // (V x)_c from the particle's basis values: sum_j' hy_j' sum_i' hx_i' x[j'N + i']
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) {
                R t2[N];
#pragma unroll
                for (int jj = 0; jj < N; ++jj) t2[jj] = R(0);
#pragma unroll
                for (int q = 0; q < n; q += VW) {
                    const VT v = *reinterpret_cast<const VT *>(vec + cc * P4 + q);
#pragma unroll
                    for (int i = 0; i < VW; ++i)
                        if (q + i < n) t2[(q + i) / N] = fma(hx[(q + i) % N], VV::at(v, i), t2[(q + i) / N]);
                }
                R vx = R(0);
#pragma unroll
                for (int jj = 0; jj < N; ++jj) vx = fma(hy[jj], t2[jj], vx);
                res[cc * P4 + c] = rhs[cc * P4 + c] - vx;
            }
        }
        if (PHASE == 2 && group_active && lead && c < 4 * N) {
            const R *row = Vs + (n + c) * LD;
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) {
                R bx = R(0);
#pragma unroll
                for (int q = 0; q < n; q += VW) {
                    const VT rv = *reinterpret_cast<const VT *>(row + q);
                    const VT xv = *reinterpret_cast<const VT *>(vec + cc * P4 + q);
#pragma unroll
                    for (int i = 0; i < VW; ++i)
                        if (q + i < n) bx = fma(VV::at(rv, i), VV::at(xv, i), bx);
                }
                res[cc * P4 + n + c] = rhs[cc * P4 + n + c] - bx;
            }
        }
        group_sync(bar_id, G::GS);
        R rc[NCOMP];
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) rc[cc] = R(0);
        if (real_lead)
            for (int p = 0; p < P; p += VW) {
#pragma unroll
                for (int cc = 0; cc < NCOMP; ++cc) {
                    const VT rv = *reinterpret_cast<const VT *>(res + cc * P4 + p);
#pragma unroll
                    for (int i = 0; i < VW; ++i)
                        if (p + i < P) rc[cc] = fma(Vs[(p + i) * LD + c], VV::at(rv, i), rc[cc]);
                }
            }
#pragma unroll
        for (int k = 0; k < n; ++k) {
            R *pr = piv + (k & 1) * (LD + 4);
            if (c == k && lead)
#pragma unroll
                for (int cc = 0; cc < NCOMP; ++cc) pr[cc] = rc[cc];
            group_sync(bar_id, G::GS);
            const R gk = row_entry(k);
            if (real_lead && c != k)
#pragma unroll
                for (int cc = 0; cc < NCOMP; ++cc) rc[cc] = fma(-gk, pr[cc], rc[cc]);
        }
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) x[cc] += real_lead ? rc[cc] / diag : R(0);
    }
#pragma unroll
    for (int cc = 0; cc < NCOMP; ++cc) bad |= real_lead && !isfinite(x[cc]);

    if constexpr (PHASE == 1) {
        // face values of the advected interpolant (alpha - c = x) at the 4N face points
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc)
            if (c < n && lead) vec[cc * P4 + c] = x[cc];  // the group may have more threads than nodes
        group_sync(bar_id, G::GS);
        if (group_active && lead && c < 4 * N) {
            const int side = c / N, f = c % N;
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) {
                const R *vc = vec + cc * P4;
                R v = R(0);
                if (side < 2) {
                    const R *h = side == 0 ? sh0 : sh1;
#pragma unroll
                    for (int ii = 0; ii < N; ++ii) v = fma(h[ii], vc[f * N + ii], v);
                } else {
                    const R *h = side == 2 ? sh0 : sh1;
#pragma unroll
                    for (int jj = 0; jj < N; ++jj) v = fma(h[jj], vc[jj * N + f], v);
                }
                FaceT out;
                if constexpr (kPair) {
                    two_sum2d(ch[cc], v, out.x, out.y);
                    out.y += cl[cc];
                } else {
                    out = ch[cc] + v;
                }
                faces[(fbase[cc] + e) * 4 * N + c] = out;
            }
        }
    } else {
        if (real_lead) {
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) {
                if constexpr (kPair) {
                    float hi, lo;
                    two_sum2d(ch[cc], x[cc], hi, lo);
                    Qg[qoff[cc] + c] = make_float2(hi, lo + cl[cc]);
                } else {
                    Qg[qoff[cc] + c] = ch[cc] + x[cc];
                }
            }
        }
    }
    if (bad) atomicOr(a.err, 1);
}

template <int N, typename R, int NCOMP = 1>
cudaError_t launch_step2d_n(const Step2DArgs &a, cudaStream_t st)
{
    using G = Geo2D<N, R, NCOMP>;
    const size_t smem = sizeof(R) * (((G::kTables + 3) & ~3) + size_t(G::GPC) * G::kGroup);
    const long long groups = (long long)a.Kx * a.Ky * a.M;
    // a launch covers at most `chunk` groups (a multiple of the groups per CTA)
    const long long chunk =
        a.chunk > 0 ? std::min(groups, (a.chunk + G::GPC - 1) / G::GPC * G::GPC) : groups;
    const unsigned block = unsigned(G::kBlock);
    auto k1 = sl2d_step_kernel<N, R, 1, false, NCOMP>;
    auto k2 = sl2d_step_kernel<N, R, 2, false, NCOMP>;
    Step2DArgs b = a;
    LaunchThrottle *th = a.chunk > 0 ? a.throttle : nullptr;
    for (int t = 0; t < a.nsteps; ++t) {
        for (int phase = 1; phase <= 2; ++phase)  // every group's faces before any remap
            for (long long g0 = 0; g0 < groups; g0 += chunk) {
                if (th) {
                    const cudaError_t e = th->before();
                    if (e != cudaSuccess) return e;
                }
                b.g0 = g0;
                b.g1 = std::min(groups, g0 + chunk);
                const unsigned grid = unsigned((b.g1 - g0 + G::GPC - 1) / G::GPC);
                if (phase == 1) k1<<<grid, block, smem, st>>>(b, nullptr, nullptr, 0, t);
                else k2<<<grid, block, smem, st>>>(b, nullptr, nullptr, 0, t);
                if (th) {
                    const cudaError_t e = th->after(st);
                    if (e != cudaSuccess) return e;
                }
            }
    }
    return cudaGetLastError();
}

// Prepares the two single-instance kernels of one order for two fields.
template <int N, typename R>
cudaError_t preload_step2d_c2_n()
{
    cudaError_t e = prepare_kernel(sl2d_step_kernel<N, R, 1, false, 2>);
    if (e == cudaSuccess) e = prepare_kernel(sl2d_step_kernel<N, R, 2, false, 2>);
    return e;
}

// Prepares the four kernels of one order (two phases, single and batched).
template <int N, typename R>
cudaError_t preload_step2d_n()
{
    cudaError_t e = prepare_kernel(sl2d_step_kernel<N, R, 1, false>);
    if (e == cudaSuccess) e = prepare_kernel(sl2d_step_kernel<N, R, 2, false>);
    if (e == cudaSuccess) e = prepare_kernel(sl2d_step_kernel<N, R, 1, true>);
    if (e == cudaSuccess) e = prepare_kernel(sl2d_step_kernel<N, R, 2, true>);
    return e;
}

// All instances of one order N, `nsteps` steps: two launches per step.
template <int N, typename R>
cudaError_t launch_step2d_batch_n(const Batch2DLaunch &b, cudaStream_t st)
{
    using G = Geo2D<N, R>;
    const size_t smem = sizeof(R) * (((G::kTables + 3) & ~3) + size_t(G::GPC) * G::kGroup);
    const unsigned grid = unsigned((b.total_groups + G::GPC - 1) / G::GPC);
    const unsigned block = unsigned(G::kBlock);
    auto k1 = sl2d_step_kernel<N, R, 1, true>;
    auto k2 = sl2d_step_kernel<N, R, 2, true>;
    Step2DArgs none = {};
    for (int t = 0; t < b.nsteps; ++t) {
        k1<<<grid, block, smem, st>>>(none, b.args, b.prefix, b.ninst, t);
        k2<<<grid, block, smem, st>>>(none, b.args, b.prefix, b.ninst, t);
    }
    return cudaGetLastError();
}

}  // namespace sl
