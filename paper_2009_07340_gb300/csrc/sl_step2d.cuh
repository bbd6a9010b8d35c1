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
// The two phases are two launches each per step: phase 2 of an element needs
// its neighbours' phase-1 face values.
//
// Mapping: a group of threads (its own named barrier) per element-sample;
// thread p owns particle p.  Everything is relative to the element reference
// value c (the middle node's state): [V;B] 1 = 1 (partition of unity), so the
// unknown is q - c.  The FP32 mode keeps the state and face values as float
// pairs (as in 1D).  Each phase runs two kernels:
//  - the fast kernel (MODE 1, one thread per node, every order): the
//    iteration preconditioned by the tensor product V0 = Vy (x) Vx of two 1D
//    advected bases (the particle rows' and columns' mean positions), in
//    phase 2 with the face rows through the 4N x 4N capacitance matrix.  A
//    group whose conditioning test fails, or which has not converged within
//    its iteration limit, is flagged for
//  - the direct kernel (MODE 2, the flagged groups only; SP lanes per row):
//    phase 1 by Gauss-Jordan elimination of V with partial pivoting (orders
//    with one lane per row) or of the Gram matrix V^T V; phase 2 by the Gram
//    matrix G = [V;B]^T [V;B], Gauss-Jordan without pivoting (G is SPD), and
//    in FP32 one step of iterative refinement of the stacked least-squares
//    residual against the original rows.
#pragma once
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

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

// Quotients inside the fast path's preconditioner (the tensor factors Wx, Wy,
// the face basis and the inverse of C): FP32 takes the fast approximate
// division (__fdividef, within a few ulp for these magnitudes), which changes
// only how fast the iteration converges, never what it converges to; FP64
// divides exactly.
__device__ __forceinline__ float pdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double pdiv(double a, double b) { return a / b; }

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

template <int N, typename R, int NCOMP = 1, bool FASTONLY = false>
struct Geo2D {
    static constexpr int n = N * N;
    // lanes per row (the fast-path kernel holds no rows: one thread per node)
    static constexpr int SP = FASTONLY ? 1 : split2d<N, R>();
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
    static constexpr int HXS = (2 * N + 3) & ~3;                // stride of the particles' basis-value table
    // the order has the tensor-preconditioned fast path (one or two fields)
    static constexpr bool kFast = N <= 12 && NCOMP <= 2;
    __host__ __device__ static constexpr int r4(int v) { return (v + 3) & ~3; }
    // row stride (elements) for v values read by 16-byte loads from
    // consecutive rows: an odd number of 16-byte units, so that the eight
    // rows of one quarter-warp fall in eight different groups of four banks
    __host__ __device__ static constexpr int odd16(int v)
    {
        const int u = (v * int(sizeof(R)) + 15) / 16;
        return (u | 1) * 16 / int(sizeof(R));
    }
    static constexpr int NTP = odd16(n);      // rows of the particles' basis values by node (hxT, hyT)
    // rows of C^{-1} (FP64 N = 10 unpadded: the padding would leave room for
    // one CTA per SM instead of two)
    static constexpr int CIS = sizeof(R) == 8 && N == 10 ? r4(4 * N) : odd16(4 * N);
    // pivot block of the inversion of C (divides 4N; the published block rows
    // fit in the space of C^{-1}).  Measured on 16 x 16 meshes: 4 x 4 blocks
    // are 3-9 % faster than 2 x 2 for FP32 N = 8, 9, and 4-7 % slower in FP64
    // (its extra FP64 block inversions); below N = 8 a tie.  From N = 10 the
    // rows of C are split over two or three threads, each of which inverts
    // every pivot block: there 2 x 2 blocks are 3-9 % faster.
    static constexpr int kCB = sizeof(R) == 4 && (N == 8 || N == 9) ? 4 : 2;
    // threads per row of C in its assembly and inversion (measured on 16 x 16
    // meshes in FP32): one up to N = 9, two at N = 10 and 11 (5 and 8 %
    // faster than one), three at N = 12 (7 % faster than one, level with
    // two).  At N = 8 two were 11 % slower than one (the 32 rows then need a
    // group barrier per step instead of __syncwarp), at N = 9 two and at
    // N = 10 three 7 % slower.
    static constexpr int kQB = N <= 9 ? 1 : (N == 12 ? 3 : 2);
    // its buffers after the basis-value table: hxT, hyT [N][NTP]; Wx, Mx = Wx Wx^T, Wy, My [N][N];
    // gx0, gx1, gy0, gy1, dbx, dby [N]; tA, tB [NTP]; u4, mu4 [4N];
    // convergence slots [2][GS / 32][2]; C^{-1} [4N][CIS]
    static constexpr int kFastBuf = FASTONLY ? 2 * N * NTP + 4 * r4(N * N) + 6 * r4(N) + 2 * NTP + 2 * r4(4 * N) +
                                                   r4(4 * (GS / 32) + 1) + 4 * N * CIS
                                             : 0;
    static_assert((4 * N) % kCB == 0 && 2 * kCB * r4(4 * N) <= 4 * N * CIS, "pivot blocks of C");
    // the mixed form's FP64 factor (MODE 3), per group after all groups (floats):
    // [4][N][N] and [4][2][N] and [8][N] doubles, 88 doubles, [4][N][N] + [4N][4] + 56 floats
    // (FP64 kernels: [4][N][N], [4][2][N], [8][N], 88, then [4N][4] and 56 doubles, the
    // rounded copy of the inverses being the inverses themselves)
    static constexpr int kX3 = !FASTONLY ? 0
                               : sizeof(R) == 4 ? r4(2 * (4 * N * N + 8 * N + 8 * N + 88) + 4 * N * N + 16 * N + 56)
                                                : r4(4 * N * N + 16 * N + 88 + 16 * N + 56);
    // the FP64 kernels invert C by the same structure (about (4N)^3 / 8 FP64
    // FMA less), except at N = 5, 7, 10, where its buffers would cost a CTA per SM
    static constexpr bool kStructC64 = sizeof(R) == 8 && N != 5 && N != 7 && N != 10;
    // rhs, vec and res hold one P4-long array per field
    static constexpr int kRows0 = P * LD;
    // the fast-path kernel holds no stacked rows: only the basis values and its buffers
    static constexpr int kRows = FASTONLY ? r4(n * HXS + kFastBuf) : kRows0;
    static constexpr int kRhs = NCOMP * P4, kPiv = 2 * (LD + 4), kVec = NCOMP * P4, kRes = NCOMP * P4;
    static constexpr int kGroup = (kRows + kRhs + kPiv + kVec + kRes + 3) & ~3;  // keeps rows 16-byte aligned
    // per-CTA tables: Z [N][N], lambda [N], h0 [N], h1 [N], -4 xi [N], 4 (1 - xi) [N]
    static constexpr int kTables = N * N + 5 * N;
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

// CTAs per SM of the fast-path kernel (MODE 1): it holds no Gram or pivot
// rows, so FP32 fits three CTAs (85 registers at 256 threads) where the
// direct solve fits two, and four of the smaller CTAs of N = 9 (192 threads,
// 80 registers) and N = 12 (160 threads, 96 registers; the compiler spills
// no more there than at three); FP64 keeps two, and one at N = 11, whose
// 151 KB of shared memory per CTA leave room for no second.
template <int N, typename R>
constexpr int min_ctas2d_fast()
{
    return std::is_same<R, float>::value ? (N == 9 || N == 12 ? 4 : 3) : (N <= 10 ? 2 : 1);
}

// BATCH = false: one instance (a0), group g = element-sample g.
// BATCH = true: `ninst` instances of the same N, instance i owning groups
// [prefix[i], prefix[i+1]) (its E*M element-samples).
// NCOMP = 2: two fields per sample ([M][2][E][n]) on the same particles, so
// one Gram matrix, one elimination and one upwind choice serve both; each
// field has its own right-hand side, refinement, faces and state.
// MODE 1: the fast path only; a group it does not finish is flagged in fb,
//         and its direct-kernel CTA slot is listed (Step2DArgs::slot_*).
// MODE 2: the direct solve for the groups MODE 1 flagged, CTA slot by slot
//         from that list.
// MODE 3: MODE 1 of the FP32 remap (phase 2) with the capacitance matrix C
//         factored (inverted) in FP64 and C^{-1} rounded to FP32 for its
//         applications: the mixed-precision form (SL_MIXED).
// One CTA slot: groups [g0 + cta GPC, g0 + (cta + 1) GPC) (g0 = 0 in a batch),
// the node tables already in shared memory.
template <int N, typename R, int PHASE, bool BATCH, int NCOMP, int MODE>
__device__ __forceinline__ void sl2d_cta(const Step2DArgs &a0, const Step2DArgs *__restrict__ args,
                                         const long long *__restrict__ prefix, int ninst, int t, long long cta)
{
    using G = Geo2D<N, R, NCOMP, MODE != 2>;
    static_assert(MODE >= 1 && MODE <= 3 && G::kFast, "the fast path and its fallback: N <= 12, one or two fields");
    static_assert(MODE != 3 || (PHASE == 2 && std::is_same<R, float>::value), "an FP64 capacitance factor: FP32 remap");
    constexpr int P4 = G::P4;  // stride of the per-field arrays
    constexpr int n = G::n, LD = G::LD, SP = G::SP, NC = G::NC;
    constexpr int HXS = G::HXS;  // stride of the phase-2 basis-value table (16-byte rows)
    static_assert(n * HXS <= G::kRows, "basis-value table fits in the rows' space");
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
    R *sX0 = sh1 + N;         // [N] -4 xi_m (scaled face x = 0 minus node m)
    R *sX1 = sX0 + N;         // [N] 4 (1 - xi_m)
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

    const long long ggid = (BATCH ? 0 : a0.g0) + cta * G::GPC + grp;
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
    if constexpr (MODE == 2) {
        if (!(group_active && a.fb[gid] != 0)) return;  // finished by the fast path
    }

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
    R dxp = R(0), dyp = R(0);  // the particle's displacement in scaled element units (4 / h)
    R ph[NCOMP];
#pragma unroll
    for (int cc = 0; cc < NCOMP; ++cc) ph[cc] = R(0);
    if (real_lead) {
        const long long V = (long long)E * n, pe = (long long)e * n + c;
        const R dWx = R(a.dW[((long long)t * a.M + s) * 2 + 0]);
        const R dWy = R(a.dW[((long long)t * a.M + s) * 2 + 1]);
        const R *cf = static_cast<const R *>(a.coef);
        // displacement dx = 4 (u dt + b dW) / h as one explicit FMA of the
        // step's coefficients (the same rounding in the batched and single kernels)
        const R dx = fma(cf[2 * V + pe], dWx, cf[pe]);
        const R dy = fma(cf[3 * V + pe], dWy, cf[V + pe]);
        dxp = dx;
        dyp = dy;
        const R gam = cf[4 * V + pe];
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
        if constexpr (SP > 1) {
            // row c of V (entry q = jj N + ii is hx[ii] hy[jj]) for the lanes
            // of the row; 16-byte stores, the padding past n is never read
#pragma unroll
            for (int q = 0; q < n; q += VW) {
                R v4[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) v4[i] = (i < VW && q + i < n) ? hx[(q + i) % N] * hy[(q + i) / N] : R(0);
                *reinterpret_cast<VT *>(Vs + c * LD + q) = VV::make(v4[0], v4[1], v4[2], v4[3]);
            }
        } else if constexpr (PHASE == 2) {
            // the particle's basis values, hx then hy ([n][HXS] table at Vs):
            // the Gram matrix is formed from them in tensor form
#pragma unroll
            for (int q = 0; q < 2 * N; q += VW) {
                R v4[4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    v4[i] = (i < VW && q + i < 2 * N) ? (q + i < N ? hx[q + i] : hy[q + i - N]) : R(0);
                *reinterpret_cast<VT *>(Vs + c * HXS + q) = VV::make(v4[0], v4[1], v4[2], v4[3]);
            }
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
            if constexpr (SP > 1)
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
            if constexpr (SP > 1) {
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
    }
    group_sync(bar_id, G::GS);

    bool bad = false;
    constexpr int NG = SP == 1 ? n : NC;  // row entries a lane holds
    const int col0 = h * NC;  // first column of this lane (SP > 1)
    // ---------------------------------------------------------------- fast path
    // Within an element the particles of a sample move almost alike (one
    // Wiener increment per sample, fields that vary little across an
    // element), so V is close to a tensor product V0 of two 1D advected-basis
    // matrices: with x~_a the mean x of particle column a and y~_b the mean y
    // of particle row b, V0[(b,a)][(j,i)] = h_i(x~_a) h_j(y~_b).  Its inverse
    // is the tensor product of the 1D interpolation matrices Wx[i][a] =
    // l~_a(xi_i) (the Lagrange basis on the x~, evaluated at the nodes) and Wy.
    // Phase 1 iterates alpha += V0^{-1} (phi* - V alpha).  Phase 2 iterates
    // q += G0^{-1} S^T (rhs - S q) on the stacked system S = [V; w B], with
    // G0 = V0^T (I + w^2 E0^T E0) V0, E0 = B V0^{-1}, applied in the stable
    // order V0^{-1} (I - E0^T C^{-1} E0) V0^{-T}, C = w^{-2} I + E0 E0^T
    // (4N x 4N, assembled from 1D products and inverted by its 4N row
    // threads).  Both converge to the direct solution.  A group whose tensor
    // factors are ill-conditioned (||Wx|| ||Wy|| above kFastCond: particles
    // far outside the element) or whose iteration has not converged after
    // kFastIters is flagged for the direct kernel.
    bool done = false;
    if constexpr (G::kFast && MODE != 2) {
        constexpr int NW = G::GS / 32;
        constexpr int NT = G::NTP, R4N = G::r4(N);
        // largest ||Wx|| ||Wy|| tried: in a model of config-3 elements every
        // case converged below these in the given iteration count (FP32 phase 2
        // stops converging first)
        constexpr float kFastCond = kPair ? (PHASE == 1 ? 512.0f : 160.0f) : 4096.0f;
        constexpr int kFastIters = kPair ? 8 : 16;
        const float kFastTol = kPair ? 1e-6f : 1e-13f;
        R *hxT = Vs + n * HXS;          // [N][NT]: hx_p[i] at [i][p]
        R *hyT = hxT + N * NT;          // [N][NT]
        R *Wx = hyT + N * NT;           // [N][N]: Wx[i][a]
        R *Mx = Wx + G::r4(N * N);      // [N][N]: Wx Wx^T
        R *Wy = Mx + G::r4(N * N);
        R *My = Wy + G::r4(N * N);      // [N][N]: Wy Wy^T
        R *gx0 = My + G::r4(N * N);     // [N] l~_a(0); then l~_a(1), and the same in y
        R *gx1 = gx0 + R4N;
        R *gy0 = gx1 + R4N;
        R *gy1 = gy0 + R4N;
        R *dbx = gy1 + R4N;             // [N] mean x displacement of particle column a
        R *dby = dbx + R4N;             // [N] mean y displacement of particle row b
        R *tA = dby + R4N;              // [NT] work vectors
        R *tB = tA + NT;
        R *u4 = tB + NT;                // [4N]
        R *mu4 = u4 + G::r4(4 * N);     // [4N]
        R *uu4 = piv;                   // [4N] u = E0 t, in the direct solve's pivot rows (unused here)
        static_assert(G::kPiv >= G::r4(4 * N), "u fits in the pivot rows");
        unsigned *red = reinterpret_cast<unsigned *>(mu4 + G::r4(4 * N));  // [2][NW][2] maxima, [1] decision
        R *Ci = mu4 + G::r4(4 * N) + G::r4(4 * NW + 1);  // [4N][CIS] C^{-1}
        static_assert(n * HXS + G::kFastBuf <= G::kRows, "fast-path buffers fit in the rows' space");
        const int lane = threadIdx.x & 31, wig = tig >> 5;
        R cref = R(0);  // |c| of the field being iterated

        // displacements (and, in phase 2, the particles' basis values) to shared memory
        if (c < n) {
            tA[c] = dxp;
            tB[c] = dyp;
            if constexpr (PHASE == 2) {
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    hxT[i * NT + c] = hx[i];
                    hyT[i * NT + c] = hy[i];
                }
            }
        }
        group_sync(bar_id, G::GS);
        if (c < N) {
            R sx = R(0);
#pragma unroll
            for (int b = 0; b < N; ++b) sx += tA[b * N + c];
            dbx[c] = sx / R(N);
        } else if (c < 2 * N) {
            R sy = R(0);
#pragma unroll
            for (int a2 = 0; a2 < N; ++a2) sy += tB[(c - N) * N + a2];
            dby[c - N] = sy / R(N);
        }
        group_sync(bar_id, G::GS);
        // the 1D inverse factors and the tilde basis at the faces; every
        // difference is a node difference plus a displacement difference
        if (c < n) {
            const int i = c / N, a2 = c % N;
            R nx = R(1), dx_ = R(1), ny = R(1), dy_ = R(1);
#pragma unroll
            for (int m = 0; m < N; ++m)
                if (m != a2) {
                    nx *= sZ[i * N + m] - dbx[m];
                    dx_ *= sZ[a2 * N + m] + (dbx[a2] - dbx[m]);
                    ny *= sZ[i * N + m] - dby[m];
                    dy_ *= sZ[a2 * N + m] + (dby[a2] - dby[m]);
                }
            // the preconditioner's factors: an FP32 quotient within a few ulp serves
            // as well as the correctly rounded one (the iteration's residual decides)
            const R wx = pdiv(nx, dx_), wy = pdiv(ny, dy_);
            Wx[i * N + a2] = wx;
            Wy[i * N + a2] = wy;
        }
        if (c < 4 * N) {
            const int s2 = c / N, a2 = c % N;
            const R *db = s2 < 2 ? dbx : dby;
            const R *X = (s2 & 1) ? sX1 : sX0;
            R num = R(1), den = R(1);
#pragma unroll
            for (int m = 0; m < N; ++m)
                if (m != a2) {
                    num *= X[m] - db[m];
                    den *= sZ[a2 * N + m] + (db[a2] - db[m]);
                }
            gx0[s2 * R4N + a2] = pdiv(num, den);
        }
        group_sync(bar_id, G::GS);
        {
            // conditioning of the tensor factors: ||Wx||_inf ||Wy||_inf
            R sx = R(0), sy = R(0);
            if (c < N) {
#pragma unroll
                for (int a2 = 0; a2 < N; ++a2) {
                    sx += fabs(Wx[c * N + a2]);
                    sy += fabs(Wy[c * N + a2]);
                }
            }
            const unsigned kx = __reduce_max_sync(0xffffffffu, __float_as_uint(float(sx)));
            const unsigned ky = __reduce_max_sync(0xffffffffu, __float_as_uint(float(sy)));
            if (tig == 0) red[4 * NW] = __uint_as_float(kx) * __uint_as_float(ky) <= kFastCond ? 1u : 0u;
        }
        group_sync(bar_id, G::GS);
        if (red[4 * NW] != 0u) {
            // group maxima of |d| and |x| of one iteration, through the slots of buffer it & 1
            auto publish_maxima = [&](const int it, const R d, const R x) {
                const unsigned kd = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(float(d))));
                const unsigned kxm = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(float(x))));
                if (lane == 0) {
                    red[(it & 1) * 2 * NW + 2 * wig] = kd;
                    red[(it & 1) * 2 * NW + 2 * wig + 1] = kxm;
                }
            };
            auto converged = [&](const int it) -> bool {  // read after a group barrier
                unsigned md = 0u, mx = 0u;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    md = max(md, red[(it & 1) * 2 * NW + 2 * w]);
                    mx = max(mx, red[(it & 1) * 2 * NW + 2 * w + 1]);
                }
                return __uint_as_float(md) <= kFastTol * (__uint_as_float(mx) + float(cref));
            };
            if constexpr (PHASE == 1) {
                // one field after the other, each with exactly the arithmetic
                // and the stopping decision of a single-field run
                bool all = true;
                for (int cc = 0; cc < NCOMP && all; ++cc) {
                    R *vc = vec + cc * P4, *rs = res + cc * P4;
                    const R *hs = rhs + cc * P4;
                    cref = fabs(ch[cc]);
                    R x = R(0);                  // alpha - c at node c
                    R r = real ? hs[c] : R(0);   // phi* - V alpha at particle c
                    bool conv = false;
                    for (int it = 0; it < kFastIters; ++it) {
                        if (c < n) rs[c] = r;
                        group_sync(bar_id, G::GS);
                        // V0^{-1} r: [(b, i)] = sum_a Wx[i][a] r[(b, a)] (stored at [i][b]), then sum_b Wy[j][b] [(b, i)]
                        if (c < n) {
                            const int i = c % N, b = c / N;
                            R t = R(0);
#pragma unroll
                            for (int a2 = 0; a2 < N; ++a2) t = fma(Wx[i * N + a2], rs[b * N + a2], t);
                            tA[i * N + b] = t;
                        }
                        group_sync(bar_id, G::GS);
                        R d = R(0);
                        if (c < n) {
                            const int i = c % N, j = c / N;
#pragma unroll
                            for (int b = 0; b < N; ++b) d = fma(Wy[j * N + b], tA[i * N + b], d);
                            x += d;
                            vc[c] = x;
                        }
                        publish_maxima(it, d, x);
                        group_sync(bar_id, G::GS);
                        if (converged(it)) {
                            conv = true;
                            break;
                        }
                        if (real) {  // the new residual at particle c, from every node's x
                            R t2[N];
#pragma unroll
                            for (int jj = 0; jj < N; ++jj) t2[jj] = R(0);
#pragma unroll
                            for (int q = 0; q < n; q += VW) {
                                const VT v = *reinterpret_cast<const VT *>(vc + q);
#pragma unroll
                                for (int i = 0; i < VW; ++i)
                                    if (q + i < n) t2[(q + i) / N] = fma(hx[(q + i) % N], VV::at(v, i), t2[(q + i) / N]);
                            }
                            R vx = R(0);
#pragma unroll
                            for (int jj = 0; jj < N; ++jj) vx = fma(hy[jj], t2[jj], vx);
                            r = hs[c] - vx;
                        }
                    }
                    if (conv && real)  // phase 2 starts from it
                        static_cast<R *>(a.alpha)[(((long long)s * NCOMP + cc) * E + e) * n + c] = x;
                    all = all && conv;
                }
                done = all;
            } else {
                R *const gvec = vec, *const gres = res;
                const R *const grhs = rhs;
                const R wb = R(a.w), wi2 = R(1) / (wb * wb);
                // products for C: Mx = Wx Wx^T, My = Wy Wy^T (kept for the iteration), and
                // hvx[s][i] = sum_a Wx[i][a] gx_s[a] at u4[s N + i], hvy[s][j] = sum_b Wy[j][b] gy_s[b] at u4[(2 + s) N + j]
                if (c < n) {
                    const int i = c / N, i2 = c % N;
                    R sxx = R(0), syy = R(0);
#pragma unroll
                    for (int a2 = 0; a2 < N; ++a2) {
                        sxx = fma(Wx[i * N + a2], Wx[i2 * N + a2], sxx);
                        syy = fma(Wy[i * N + a2], Wy[i2 * N + a2], syy);
                    }
                    Mx[c] = sxx;
                    My[c] = syy;
                }
                if (c < 4 * N) {
                    const int s2 = c / N, k = c % N;
                    const R *W = s2 < 2 ? Wx : Wy;
                    const R *g = gx0 + s2 * R4N;
                    R v = R(0);
#pragma unroll
                    for (int m = 0; m < N; ++m) v = fma(W[k * N + m], g[m], v);
                    u4[c] = v;
                }
                group_sync(bar_id, G::GS);
                if constexpr (!(MODE == 3 || (MODE == 1 && G::kStructC64))) {
                // C's rows are held by QB threads each (thread c: row c / QB, its
                // columns [q CW, q CW + CW), q = c % QB), which assemble them from
                // the 1D products and invert C in place (C is symmetric positive
                // definite, eigenvalues >= w^-2).  4N QB <= 32: one warp,
                // synchronised per step by __syncwarp; above that the group
                // barrier.
                constexpr int QB = G::kQB;
                constexpr int CW = G::r4((4 * N + QB - 1) / QB);  // columns per thread
                constexpr bool kOneWarp = 4 * N * QB <= 32;
                using RC = R;
                using VC = Vec16<RC>;
                using VCT = typename VC::T;
                constexpr int VWC = VC::W;
                const bool crow = c < 4 * N * QB;  // a thread holding part of a row of C
                const int row = c / QB, col0 = (c - row * QB) * CW;
                RC creg[CW];
#pragma unroll
                for (int jj = 0; jj < CW; ++jj) creg[jj] = RC(0);
                if (crow) {
                    const int f = row;
                    const bool fx = f < 2 * N;
                    const int s = (f / N) & 1, k = f % N;
                    const R *g = fx ? gx0 + s * R4N : gy0 + s * R4N;
                    const R *g0 = fx ? gx0 : gy0;
                    const R *g1 = fx ? gx1 : gy1;
                    R gg0 = R(0), gg1 = R(0);
#pragma unroll
                    for (int m = 0; m < N; ++m) {
                        gg0 = fma(g[m], g0[m], gg0);
                        gg1 = fma(g[m], g1[m], gg1);
                    }
                    const R *Mw = fx ? My : Mx;  // Wy Wy^T along x faces, Wx Wx^T along y faces
#pragma unroll
                    for (int jj = 0; jj < CW; ++jj) {
                        const int f2 = col0 + jj;
                        if (QB == 1 || f2 < 4 * N) {
                            const bool f2x = f2 < 2 * N;
                            const int s2 = (f2 / N) & 1, k2 = f2 % N;
                            R v;
                            if (fx == f2x) v = (s2 == 0 ? gg0 : gg1) * Mw[k * N + k2];
                            else if (fx) v = u4[(2 + s2) * N + k] * u4[s * N + k2];
                            else v = u4[(2 + s) * N + k2] * u4[s2 * N + k];
                            creg[jj] = f2 == f ? RC(v) + RC(wi2) : RC(v);
                        }
                    }
                }
                // Block Gauss-Jordan inversion in place with CB x CB pivot blocks
                // (every pivot block of an SPD matrix is SPD: no pivoting).  Step K:
                // the CB pivot rows publish themselves; after one barrier every
                // thread inverts the pivot block P in registers and forms CB
                // coefficients w: pivot row t takes row t of P^{-1}, any other row
                // w = -C[r][K] P^{-1}; then C[r][j] <- C[r][j] + sum_m w_m C[K_m][j]
                // outside the block (the pivot rows start from 0 instead of C[r][j])
                // and C[r][K] <- w.  A thread reads its row's entries C[r][K] from
                // the published rows: the partly inverted SPD matrix keeps
                // C[r][k] = C[k][r] while r is not yet eliminated and
                // C[r][k] = -C[k][r] once it is.  The published rows are
                // double-buffered in the space of C^{-1}, written only after the
                // last step.
                constexpr int CB = G::kCB;
                // published rows: column block q at q (CW + GAP), the gap putting the
                // blocks that threads of one row read at the same time in different banks
                constexpr int GAP = QB > 1 ? 4 : 0;
                constexpr int CR = G::r4(QB * (CW + GAP));  // stride of the published rows (elements of RC)
                auto pcol = [&](int j) { return j + (j / CW) * GAP; };  // column j's place in a published row
                const int pcol0 = pcol(col0);
                static_assert(2 * CB * CR * sizeof(RC) <= 4 * N * G::CIS * sizeof(R), "published rows fit in C^{-1}");
                if (!kOneWarp || wig == 0)  // uniform per warp; above one warp, every thread
#pragma unroll
                for (int K = 0; K < 4 * N; K += CB) {
                    RC *pb = reinterpret_cast<RC *>(Ci) + ((K / CB) & 1) * CB * CR;
                    const bool pivot = crow && row >= K && row < K + CB;
                    if (pivot)
#pragma unroll
                        for (int jj = 0; jj < CW; jj += VWC) {
                            RC v4[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) v4[i] = i < VWC ? creg[jj + i] : RC(0);
                            *reinterpret_cast<VCT *>(pb + (row - K) * CR + pcol0 + jj) =
                                VC::make(v4[0], v4[1], v4[2], v4[3]);
                        }
                    if constexpr (kOneWarp) __syncwarp();
                    else group_sync(bar_id, G::GS);
                    if (crow) {
                        RC Pm[CB][CB];  // the pivot block, then its inverse
#pragma unroll
                        for (int t2 = 0; t2 < CB; ++t2)
#pragma unroll
                            for (int m = 0; m < CB; ++m) Pm[t2][m] = pb[t2 * CR + pcol(K) + m];
#pragma unroll
                        for (int p = 0; p < CB; ++p) {
                            const RC d = pdiv(RC(1), Pm[p][p]);
#pragma unroll
                            for (int m = 0; m < CB; ++m) Pm[p][m] = m == p ? d : Pm[p][m] * d;
#pragma unroll
                            for (int q2 = 0; q2 < CB; ++q2)
                                if (q2 != p) {
                                    const RC l = Pm[q2][p];
#pragma unroll
                                    for (int m = 0; m < CB; ++m) Pm[q2][m] = m == p ? -l * d : fma(-l, Pm[p][m], Pm[q2][m]);
                                }
                        }
                        const RC sgn = row >= K ? RC(1) : RC(-1);
                        RC w[CB];
#pragma unroll
                        for (int m = 0; m < CB; ++m) {
                            RC other = RC(0), own = RC(0);
#pragma unroll
                            for (int t2 = 0; t2 < CB; ++t2) {
                                other = fma(-sgn * pb[t2 * CR + pcol(row)], Pm[t2][m], other);
                                own = row == K + t2 ? Pm[t2][m] : own;
                            }
                            w[m] = pivot ? own : other;
                        }
#pragma unroll
                        for (int jj = 0; jj < CW; jj += VWC) {
                            VCT v[CB];
#pragma unroll
                            for (int m = 0; m < CB; ++m) v[m] = *reinterpret_cast<const VCT *>(pb + m * CR + pcol0 + jj);
#pragma unroll
                            for (int i = 0; i < VWC; ++i) {
                                const int j = col0 + jj + i;
                                if (QB == 1 || j < 4 * N) {
                                    if (j >= K && j < K + CB) {
                                        RC wj = w[0];
#pragma unroll
                                        for (int m = 1; m < CB; ++m) wj = j == K + m ? w[m] : wj;
                                        creg[jj + i] = wj;
                                    } else {
                                        RC acc = pivot ? RC(0) : creg[jj + i];
#pragma unroll
                                        for (int m = 0; m < CB; ++m) acc = fma(w[m], VC::at(v[m], i), acc);
                                        creg[jj + i] = acc;
                                    }
                                }
                            }
                        }
                    }
                }
                // the last step's published rows are read before C^{-1} overwrites them
                if constexpr (kOneWarp) {
                    if (wig == 0) __syncwarp();
                } else {
                    group_sync(bar_id, G::GS);
                }
                if (crow)  // this thread's part of row `row` of C^{-1} (16-byte stores)
#pragma unroll
                    for (int jj = 0; jj < CW; jj += VW)
                        if (col0 + jj < 4 * N) {
                            R v4[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) v4[i] = i < VW ? R(creg[jj + i]) : R(0);
                            *reinterpret_cast<VT *>(Ci + row * G::CIS + col0 + jj) = VV::make(v4[0], v4[1], v4[2], v4[3]);
                        }
                } else {
                // MODE 3 (and the FP64 kernels): C^{-1} from its structure, the factors
                // in FP64.  C =
                // w^-2 I + [[Gx (x) My, Cxy], [Cxy^T, Gy (x) Mx]] with Gx = [gx_s . gx_s']
                // (2 x 2), My = Wy Wy^T and Cxy of rank 4 (its (s, s') blocks are
                // hvy_s' hvx_s^T).  The Kronecker blocks invert through the
                // eigenvectors Q of Gx and Gy: (w^-2 I + Gx (x) My)^{-1} =
                // sum_t q_t q_t^T (x) (w^-2 I + lambda_t My)^{-1}, four N x N
                // inverses; the coupling enters by block elimination and the
                // Woodbury identity on the Schur complement, with 4 x 4 matrices
                // P = A^T Cxx^{-1} A, Qm = B^T Cyy^{-1} B (Cxy = A B^T) and
                // T = P^{-1} - Qm.  The N x N and 4 x 4 inverses and the products
                // that form P and Qm run in FP64; C^{-1}'s entries are assembled
                // from them in the kernel's precision.  Same result as the inverse of the dense C
                // (checked in a NumPy model with these index conventions).
                double *xd = reinterpret_cast<double *>(tab + ((G::kTables + 3) & ~3) + G::GPC * G::kGroup +
                                                        grp * G::kX3);
                double *Ainv = xd;                 // [4][N][N]: (w^-2 I + lx_t My)^{-1}, t = 0, 1; then the y side
                double *piv64 = Ainv + 4 * N * N;  // [4][2][N] pivot rows of their Gauss-Jordan
                double *yz = piv64 + 8 * N;        // [8][N]: y_{t,tp} = Ainv_t hvy_tp, z_{t,tg} = Ainv_{2+t} hvx_tg
                double *sm64 = yz + 8 * N;         // Qx [2][2], lx [2], Qy [2][2], ly [2], then warp-0 scratch
                constexpr bool kAlias = std::is_same<R, double>::value;  // FP64: Ainv is its own copy
                R *A32 = kAlias ? reinterpret_cast<R *>(Ainv) : reinterpret_cast<R *>(sm64 + 88);  // [4][N][N] Ainv in R
                R *Z32 = kAlias ? reinterpret_cast<R *>(sm64 + 88) : A32 + 4 * N * N;  // [4N][4]: rows of Cxx^{-1} A, Cyy^{-1} B
                R *s32 = Z32 + 16 * N;             // Qx [4], Qy [4], Mxx [16], M1 [16], Ti [16]
                const R *hvx = u4, *hvy = u4 + 2 * N;  // hvx[s N + i] = (Wx gx_s)_i, hvy[s N + j] = (Wy gy_s)_j
                // GB300 runs FP64 at 2 lanes per clock per SM, so a warp-wide FP64
                // instruction costs the same whatever its active lanes: the small
                // FP64 steps below spread their work over the lanes of warp 0.
                double *w64 = sm64 + 12;  // warp-0 scratch: [6] Gram entries, then [16] dots, [3][16] 4 x 4 matrices
                if (wig == 0) {  // the 2 x 2 eigen-decompositions (a Jacobi rotation each)
                    if (lane < 6) {  // lane 3 d + e: d = 0 x, 1 y; e = 0: g0.g0, 1: g0.g1, 2: g1.g1
                        const int d = lane / 3, e = lane - 3 * d;
                        const R *ga = d == 0 ? (e == 2 ? gx1 : gx0) : (e == 2 ? gy1 : gy0);
                        const R *gb = d == 0 ? (e == 0 ? gx0 : gx1) : (e == 0 ? gy0 : gy1);
                        double acc = 0.0;
#pragma unroll
                        for (int m = 0; m < N; ++m) acc = fma(double(ga[m]), double(gb[m]), acc);
                        w64[lane] = acc;
                    }
                    __syncwarp();
                    if (lane < 2) {
                        const int d = lane;
                        const double g00 = w64[3 * d], g01 = w64[3 * d + 1], g11 = w64[3 * d + 2];
                        double cs = 1.0, sn = 0.0, l0 = g00, l1 = g11;
                        if (g01 != 0.0) {
                            const double tau = (g11 - g00) / (2.0 * g01);
                            const double tn = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(fma(tau, tau, 1.0)));
                            cs = 1.0 / sqrt(fma(tn, tn, 1.0));
                            sn = tn * cs;
                            l0 = fma(-tn, g01, g00);
                            l1 = fma(tn, g01, g11);
                        }
                        double *q = sm64 + 6 * d;  // Q = [[cs, sn], [-sn, cs]]: column t the eigenvector of l_t
                        q[0] = cs;
                        q[1] = sn;
                        q[2] = -sn;
                        q[3] = cs;
                        q[4] = l0;
                        q[5] = l1;
                        s32[4 * d + 0] = R(cs);
                        s32[4 * d + 1] = R(sn);
                        s32[4 * d + 2] = R(-sn);
                        s32[4 * d + 3] = R(cs);
                    }
                }
                group_sync(bar_id, G::GS);
                {  // the four N x N inverses, Gauss-Jordan in FP64, each matrix's rows in one warp
                    constexpr bool kOneWarp3 = 4 * N <= 32;
                    int mat = -1, row = 0;
                    if constexpr (kOneWarp3) {
                        if (tig < 4 * N) mat = tig / N, row = tig % N;
                    } else {
                        if (wig < 2 && lane < 2 * N) mat = 2 * wig + lane / N, row = lane % N;
                    }
                    double arow[N];
                    if (mat >= 0) {
                        const double lam = sm64[(mat >> 1) * 6 + 4 + (mat & 1)];
                        const R *M = mat < 2 ? My : Mx;  // My for the x faces, Mx for the y faces
#pragma unroll
                        for (int j = 0; j < N; ++j)
                            arow[j] = j == row ? fma(lam, double(M[row * N + j]), double(wi2)) : lam * double(M[row * N + j]);
                    }
                    if (kOneWarp3 ? wig == 0 : wig < 2) {  // uniform per warp
#pragma unroll
                        for (int k = 0; k < N; ++k) {
                            // the pivot row publishes itself unscaled; every row then takes
                            // one FMA per entry (the pivot row from zero), so that the
                            // warp's FP64 instructions are not split by the pivot's scaling
                            double *pr = piv64 + ((mat < 0 ? 0 : mat) * 2 + (k & 1)) * N;
                            if (mat >= 0 && row == k)
#pragma unroll
                                for (int j = 0; j < N; ++j) pr[j] = arow[j];
                            __syncwarp();
                            if (mat >= 0) {
                                const double pinv = 1.0 / pr[k];
                                const bool own = row == k;
                                const double coef = own ? pinv : -arow[k] * pinv;
#pragma unroll
                                for (int j = 0; j < N; ++j)
                                    arow[j] = j == k ? (own ? pinv : coef) : fma(coef, pr[j], own ? 0.0 : arow[j]);
                            }
                        }
                    }
                    if (mat >= 0)
#pragma unroll
                        for (int j = 0; j < N; ++j) {
                            Ainv[(mat * N + row) * N + j] = arow[j];
                            if constexpr (!kAlias) A32[(mat * N + row) * N + j] = R(arow[j]);
                        }
                }
                group_sync(bar_id, G::GS);
                for (int e2 = tig; e2 < 8 * N; e2 += G::GS) {  // y and z, FP64
                    const int v = e2 / N, k = e2 - v * N;
                    const int mat = v < 4 ? v >> 1 : 2 + ((v - 4) >> 1);
                    const R *h = v < 4 ? hvy + (v & 1) * N : hvx + (v & 1) * N;
                    double acc = 0.0;
#pragma unroll
                    for (int k2 = 0; k2 < N; ++k2) acc = fma(Ainv[(mat * N + k) * N + k2], double(h[k2]), acc);
                    yz[e2] = acc;
                }
                group_sync(bar_id, G::GS);
                if (wig == 0) {  // P, Qm and the 4 x 4 algebra, FP64, one entry per lane
                    double *dyz = w64 + 6;   // [16]: dy[t][a1][a2] = hvy_a1 . y_{t,a2} at 4t + 2a1 + a2, dz at 8 + ...
                    double *Pm = dyz + 16;   // [16] P, then P^{-1}, then T^{-1}
                    double *Qm = Pm + 16;    // [16]
                    double *QT = Qm + 16;    // [16] Qm T^{-1}
                    if (lane < 16) {
                        const bool isz = lane >= 8;
                        const int t = (lane >> 2) & 1, a1 = (lane >> 1) & 1, a2 = lane & 1;
                        const R *h = isz ? hvx + a1 * N : hvy + a1 * N;
                        const double *v = yz + ((isz ? 4 : 0) + 2 * t + a2) * N;
                        double acc = 0.0;
#pragma unroll
                        for (int k = 0; k < N; ++k) acc = fma(double(h[k]), v[k], acc);
                        dyz[lane] = acc;
                    }
                    __syncwarp();
                    const int e = lane & 15, i4 = e >> 2, j4 = e & 3;
                    {
                        const double *Qx = sm64, *Qy = sm64 + 6;
                        const int sg = i4 >> 1, sp = i4 & 1, tg = j4 >> 1, tp = j4 & 1;
                        double v = 0.0;
#pragma unroll
                        for (int t = 0; t < 2; ++t)
                            v = lane < 16 ? fma(Qx[2 * sg + t] * Qx[2 * tg + t], dyz[4 * t + 2 * sp + tp], v)
                                          : fma(Qy[2 * sp + t] * Qy[2 * tp + t], dyz[8 + 4 * t + 2 * sg + tg], v);
                        (lane < 16 ? Pm : Qm)[e] = v;
                    }
                    __syncwarp();
                    auto inv4w = [&](double *A) {  // in place, one entry per lane (both half-warps alike)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const double p = A[5 * k], aik = A[4 * i4 + k], akj = A[4 * k + j4], aij = A[e];
                            __syncwarp();
                            const double pinv = 1.0 / p;
                            const double v = i4 == k ? (j4 == k ? pinv : akj * pinv)
                                                     : (j4 == k ? -aik * pinv : fma(-aik, akj * pinv, aij));
                            if (lane < 16) A[e] = v;
                            __syncwarp();
                        }
                    };
                    inv4w(Pm);
                    if (lane < 16) Pm[e] -= Qm[e];  // T = P^{-1} - Qm
                    __syncwarp();
                    inv4w(Pm);                      // T^{-1}
                    double qt = 0.0;
#pragma unroll
                    for (int m = 0; m < 4; ++m) qt = fma(Qm[4 * i4 + m], Pm[4 * m + j4], qt);
                    if (lane < 16) QT[e] = qt;
                    __syncwarp();
                    double mxx = Qm[e];
#pragma unroll
                    for (int m = 0; m < 4; ++m) mxx = fma(QT[4 * i4 + m], Qm[4 * m + j4], mxx);
                    if (lane < 16) {
                        s32[8 + e] = R(mxx);                                   // Mxx = Qm + Qm T^-1 Qm
                        s32[24 + e] = R((i4 == j4 ? 1.0 : 0.0) + QT[e]);      // M1 = I + Qm T^-1
                        s32[40 + e] = R(Pm[e]);                                // T^-1
                    }
                }
                if (c < 4 * N) {  // row c of Cxx^{-1} A (x faces) or Cyy^{-1} B (y faces)
                    const int f = c, s = (f / N) & 1, k = f % N;
                    const double *Qd = f < 2 * N ? sm64 : sm64 + 6;
                    R zr[4];
#pragma unroll
                    for (int a1 = 0; a1 < 2; ++a1)
#pragma unroll
                        for (int a2 = 0; a2 < 2; ++a2) {
                            double acc = 0.0;
#pragma unroll
                            for (int t = 0; t < 2; ++t)
                                acc = f < 2 * N ? fma(Qd[2 * s + t] * Qd[2 * a1 + t], yz[(2 * t + a2) * N + k], acc)
                                                : fma(Qd[2 * s + t] * Qd[2 * a2 + t], yz[(4 + 2 * t + a1) * N + k], acc);
                            zr[2 * a1 + a2] = R(acc);
                        }
#pragma unroll
                    for (int i = 0; i < 4; i += VW)
                        *reinterpret_cast<VT *>(Z32 + 4 * f + i) = VV::make(zr[i], zr[(i + 1) & 3], zr[(i + 2) & 3], zr[(i + 3) & 3]);
                }
                group_sync(bar_id, G::GS);
                auto load4 = [&](const R *p, R (&z)[4]) {  // four values from a 16-byte-aligned row
#pragma unroll
                    for (int i = 0; i < 4; i += VW) {
                        const VT v = *reinterpret_cast<const VT *>(p + i);
#pragma unroll
                        for (int i2 = 0; i2 < VW; ++i2) z[i + i2] = VV::at(v, i2);
                    }
                };
                if (c < 4 * N) {  // row c of C^{-1}, assembled in the kernel's precision
                    const int f = c, s = (f / N) & 1, k = f % N;
                    const bool fx = f < 2 * N;
                    R zr[4];
                    load4(Z32 + 4 * f, zr);
                    const R *Mxx = s32 + 8, *M1 = s32 + 24, *Tinv = s32 + 40;
                    R rr[4], rp[4];  // the row's coefficients for its own block and the other
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        R a1 = R(0), a2 = R(0);
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            a1 = fma(zr[m], fx ? Mxx[4 * m + j] : Tinv[4 * m + j], a1);
                            a2 = fma(zr[m], fx ? M1[4 * m + j] : M1[4 * j + m], a2);
                        }
                        rr[j] = a1;
                        rp[j] = -a2;
                    }
                    const R *Q32 = fx ? s32 : s32 + 4;
                    R cq[2][2];  // Q[s][t] Q[s2][t]
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
                        for (int t = 0; t < 2; ++t) cq[s2][t] = Q32[2 * s + t] * Q32[2 * s2 + t];
                    const R *Ab = A32 + (fx ? 0 : 2) * N * N + k * N;  // row k of the block's inverses t = 0, 1
#pragma unroll
                    for (int f2 = 0; f2 < 4 * N; f2 += 4) {
                        R v4[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int g2 = f2 + i, s2 = (g2 / N) & 1, k2 = g2 % N;
                            const bool same = fx == (g2 < 2 * N);
                            R z2[4];
                            load4(Z32 + 4 * g2, z2);
                            const R *cf = same ? rr : rp;
                            R v = cf[0] * z2[0];
                            v = fma(cf[1], z2[1], v);
                            v = fma(cf[2], z2[2], v);
                            v = fma(cf[3], z2[3], v);
                            if (same) {
                                v = fma(cq[s2][0], Ab[k2], v);
                                v = fma(cq[s2][1], Ab[N * N + k2], v);
                            }
                            v4[i] = v;
                        }
#pragma unroll
                        for (int i = 0; i < 4; i += VW)
                            *reinterpret_cast<VT *>(Ci + f * G::CIS + f2 + i) =
                                VV::make(v4[i], v4[(i + 1) & 3], v4[(i + 2) & 3], v4[(i + 3) & 3]);
                    }
                }
                }
                R qf[NCOMP];  // q - c at node c, per field
                bool all = true;
                for (int cc = 0; cc < NCOMP && all; ++cc) {
                R *vec = gvec + cc * P4, *res = gres + cc * P4;
                const R *rhs = grhs + cc * P4;
                cref = fabs(ch[cc]);
                // phase 1's interpolant: the remap differs from it only by the face correction
                R q = real ? static_cast<const R *>(a.alpha)[(((long long)s * NCOMP + cc) * E + e) * n + c] : R(0);
                bool conv = false;
                for (int it = 0; it <= kFastIters; ++it) {
                    if (c < n) vec[c] = q;
                    group_sync(bar_id, G::GS);
                    if (it > 0 && converged(it - 1)) {
                        conv = true;
                        break;
                    }
                    if (it == kFastIters) break;
                    // stacked residual: particles phi* - V q, face points w (g - c) - w B q
                    if (real) {
                        R t2[N];
#pragma unroll
                        for (int jj = 0; jj < N; ++jj) t2[jj] = R(0);
#pragma unroll
                        for (int qq = 0; qq < n; qq += VW) {
                            const VT v = *reinterpret_cast<const VT *>(vec + qq);
#pragma unroll
                            for (int i = 0; i < VW; ++i)
                                if (qq + i < n) t2[(qq + i) / N] = fma(hx[(qq + i) % N], VV::at(v, i), t2[(qq + i) / N]);
                        }
                        R vq = R(0);
#pragma unroll
                        for (int jj = 0; jj < N; ++jj) vq = fma(hy[jj], t2[jj], vq);
                        res[c] = rhs[c] - vq;
                    }
                    if (group_active && c < 4 * N) {
                        const int side = c / N, f = c % N;
                        R bq = R(0);
                        if (side < 2) {
                            const R *hf = side == 0 ? sh0 : sh1;
#pragma unroll
                            for (int ii = 0; ii < N; ++ii) bq = fma(hf[ii], vec[f * N + ii], bq);
                        } else {
                            const R *hf = side == 2 ? sh0 : sh1;
#pragma unroll
                            for (int jj = 0; jj < N; ++jj) bq = fma(hf[jj], vec[jj * N + f], bq);
                        }
                        res[n + c] = rhs[n + c] - wb * bq;
                    }
                    group_sync(bar_id, G::GS);
                    // z = S^T res at node c = (i, j)
                    if (c < n) {
                        const int i = c % N, j = c / N;
                        R z = R(0);
#pragma unroll
                        for (int p2 = 0; p2 < n; p2 += VW) {
                            const VT xv = *reinterpret_cast<const VT *>(hxT + i * NT + p2);
                            const VT yv = *reinterpret_cast<const VT *>(hyT + j * NT + p2);
                            const VT rv = *reinterpret_cast<const VT *>(res + p2);
#pragma unroll
                            for (int e2 = 0; e2 < VW; ++e2)
                                if (p2 + e2 < n) z = fma(VV::at(xv, e2) * VV::at(yv, e2), VV::at(rv, e2), z);
                        }
                        z = fma(wb * sh0[i], res[n + j], z);
                        z = fma(wb * sh1[i], res[n + N + j], z);
                        z = fma(wb * sh0[j], res[n + 2 * N + i], z);
                        z = fma(wb * sh1[j], res[n + 3 * N + i], z);
                        tA[c] = z;
                    }
                    group_sync(bar_id, G::GS);
                    // V0^{-T} z, first pass: [(j, a)] = sum_i Wx[i][a] z[(j, i)] (stored at [a][j]).
                    // With it, the face rows' u = E0 V0^{-T} z comes from z directly: since
                    // the rows of E0 are outer products, u on x face s at node k is
                    // (My rx_s)_k with rx_s[j] = sum_i hvx_s[i] z[(j, i)], and on y face s
                    // (Mx ry_s)_k with ry_s[i] = sum_j hvy_s[j] z[(j, i)]: first r, here
                    if (c < n) {
                        const int a2 = c % N, j = c / N;
                        R t = R(0);
#pragma unroll
                        for (int i = 0; i < N; ++i) t = fma(Wx[i * N + a2], tA[j * N + i], t);
                        tB[a2 * N + j] = t;
                    }
                    if (c < 4 * N) {
                        R r4v = R(0);
                        if (c < 2 * N) {
                            const R *hv = u4 + (c / N) * N;
                            const int j = c % N;
#pragma unroll
                            for (int i = 0; i < N; ++i) r4v = fma(hv[i], tA[j * N + i], r4v);
                        } else {
                            const R *hv = u4 + (c / N) * N;  // hvy_s at u4 + (2 + s) N
                            const int i = c % N;
#pragma unroll
                            for (int j = 0; j < N; ++j) r4v = fma(hv[j], tA[j * N + i], r4v);
                        }
                        mu4[c] = r4v;
                    }
                    group_sync(bar_id, G::GS);
                    // second pass: t[(b, a)] = sum_j Wy[j][b] [(j, a)]; and u from r
                    if (c < n) {
                        const int a2 = c % N, b = c / N;
                        R tv = R(0);
#pragma unroll
                        for (int j = 0; j < N; ++j) tv = fma(Wy[j * N + b], tB[a2 * N + j], tv);
                        tA[c] = tv;
                    }
                    if (c < 4 * N) {
                        const R *Mm = c < 2 * N ? My : Mx;
                        const R *rv = mu4 + (c / N) * N;
                        const int k = c % N;
                        R uv = R(0);
#pragma unroll
                        for (int m = 0; m < N; ++m) uv = fma(Mm[k * N + m], rv[m], uv);
                        uu4[c] = uv;
                    }
                    group_sync(bar_id, G::GS);
                    // V0^{-1} t, first pass: [(b, i)] = sum_a Wx[i][a] t[(b, a)] (stored at [i][b]);
                    // and mu = C^{-1} u
                    if (c < n) {
                        const int i = c % N, b = c / N;
                        R t = R(0);
#pragma unroll
                        for (int a2 = 0; a2 < N; ++a2) t = fma(Wx[i * N + a2], tA[b * N + a2], t);
                        tB[i * N + b] = t;
                    }
                    if (c < 4 * N) {
                        R m = R(0);
#pragma unroll
                        for (int f2 = 0; f2 < 4 * N; f2 += VW) {
                            const VT cv = *reinterpret_cast<const VT *>(Ci + c * G::CIS + f2);
                            const VT uv = *reinterpret_cast<const VT *>(uu4 + f2);
#pragma unroll
                            for (int i = 0; i < VW; ++i)
                                if (f2 + i < 4 * N) m = fma(VV::at(cv, i), VV::at(uv, i), m);
                        }
                        mu4[c] = m;  // r was last read in the previous stage
                    }
                    group_sync(bar_id, G::GS);
                    // second pass, less V0^{-1} E0^T mu, which at node (i, j) is
                    // sum_s (My mu_x,s)_j hvx_s[i] + hvy_s[j] (Mx mu_y,s)_i
                    R d = R(0);
                    if (c < n) {
                        const int i = c % N, j = c / N;
#pragma unroll
                        for (int b = 0; b < N; ++b) d = fma(Wy[j * N + b], tB[i * N + b], d);
                        R mx0 = R(0), mx1 = R(0), my0 = R(0), my1 = R(0);
#pragma unroll
                        for (int k = 0; k < N; ++k) {
                            mx0 = fma(My[j * N + k], mu4[k], mx0);
                            mx1 = fma(My[j * N + k], mu4[N + k], mx1);
                            my0 = fma(Mx[i * N + k], mu4[2 * N + k], my0);
                            my1 = fma(Mx[i * N + k], mu4[3 * N + k], my1);
                        }
                        R corr = mx0 * u4[i];
                        corr = fma(mx1, u4[N + i], corr);
                        corr = fma(u4[2 * N + j], my0, corr);
                        corr = fma(u4[3 * N + j], my1, corr);
                        d -= corr;
                        q += d;
                    }
                    publish_maxima(it, d, q);
                }
                qf[cc] = q;
                all = all && conv;
                }
                if (all) {
                    done = true;
                    if (real)
#pragma unroll
                        for (int cc = 0; cc < NCOMP; ++cc) {
                            if constexpr (kPair) {
                                float hi, lo;
                                two_sum2d(ch[cc], qf[cc], hi, lo);
                                Qg[qoff[cc] + c] = make_float2(hi, lo + cl[cc]);
                            } else {
                                Qg[qoff[cc] + c] = ch[cc] + qf[cc];
                            }
                        }
                }
            }
        }
    }
    if constexpr (MODE != 2) {  // a group the fast path did not finish goes to the direct solve
        if (group_active && tig == 0) {
            a.fb[gid] = done ? 0 : 1;
            if (!done) {
                if (a.fbcount) atomicAdd(a.fbcount + (PHASE - 1), 1ull);
                // its direct-kernel CTA slot, listed once however many of its groups are flagged
                const Step2DArgs &L = BATCH ? args[0] : a0;
                const long long slot = ggid / Geo2D<N, R, NCOMP, false>::GPC;
                if (atomicExch(L.slot_mark + slot, 1u) == 0u) L.slot_list[atomicAdd(L.slot_ctl, 1u)] = unsigned(slot);
            }
        }
        if (!done) return;
    }
    // ---------------------------------------------------------------- direct path
    if constexpr (MODE == 2) {
    if constexpr (PHASE == 1 && SP == 1) {
        // Phase 1: alpha = V^{-1} phi* by Gauss-Jordan elimination of the
        // square advected-basis matrix V itself, with partial (row) pivoting.
        // Row c (particle c) lives in the registers of its lanes.  At step k
        // every warp nominates its not yet pivoted row of largest |V[.][k]| (a
        // warp max-reduction of the magnitudes' bit patterns) and publishes
        // it; after one group barrier every thread takes the nominee of
        // largest magnitude (the lowest warp on ties) as the pivot row.  Every
        // other row eliminates column k and keeps its multiplier there.  Node
        // k's alpha is its pivot row's right-hand side over the pivot.
        constexpr int NW = G::GS / 32;  // warps per group
        static_assert(2 * NW * (LD + 4) + 2 * NW <= 4 * N * LD, "pivot nominees fit in the face rows' space");
        R *cnd = Vs + n * LD;                                                     // [2][NW][LD + 4] nominated rows
        unsigned *mags = reinterpret_cast<unsigned *>(cnd + 2 * NW * (LD + 4));  // [2][NW] their keys
        const int wig = tig >> 5, lane = threadIdx.x & 31;
        R gr[NG];
        if constexpr (SP == 1) {  // row c of V from the particle's own basis values
#pragma unroll
            for (int q = 0; q < n; ++q) gr[q] = real ? hx[q % N] * hy[q / N] : R(0);
        } else {  // this lane's columns of row c, staged by the row's first lane
#pragma unroll
            for (int q = 0; q < NG; q += VW) {
                VT v = VV::make(R(0), R(0), R(0), R(0));
                if (real) v = *reinterpret_cast<const VT *>(Vs + c * LD + col0 + q);
#pragma unroll
                for (int i = 0; i < VW; ++i)
                    if (q + i < NG) gr[q + i] = col0 + q + i < n ? VV::at(v, i) : R(0);
            }
        }
        R bc[NCOMP];
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) bc[cc] = real ? rhs[cc * P4 + c] : R(0);
        int mypiv = -1;  // the column this row pivots, once chosen
        R diag = R(1);
        // entry k of this thread's row, from the lane holding column k (SP > 1:
        // a shuffle executed by every lane of the warp; k is a compile-time index)
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
            const int buf = k & 1;
            const int hk = SP == 1 ? 0 : k / NC;  // lane of a row holding column k
            const int jk = SP == 1 ? k : k % NC;  // its register
            unsigned key = 0u;                    // 0: no candidate
            if (real && mypiv < 0 && h == hk) key = __float_as_uint(fabsf(float(gr[jk]))) + 1u;
            const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
            const unsigned ball = __ballot_sync(0xffffffffu, key != 0u && key == kmax);
            const int wl = __ffs(ball) - 1;  // the lowest lane holding the warp's largest entry
            const bool nominee = ball != 0u && lane - h == wl - hk;  // a lane of the warp's nominated row
            R *slot = cnd + (buf * NW + wig) * (LD + 4);
            if (nominee) {
#pragma unroll
                for (int q = 0; q < NG; q += VW) {
                    R v4[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) v4[i] = (i < VW && q + i < NG) ? gr[q + i] : R(0);
                    *reinterpret_cast<VT *>(slot + col0 + q) = VV::make(v4[0], v4[1], v4[2], v4[3]);
                }
                if (lead) {
                    slot[LD] = bc[0];
                    if constexpr (NCOMP > 1) slot[LD + 2] = bc[1];
                }
                if (h == hk) slot[LD + 1] = R(1) / gr[jk];
            }
            if (lane == 0) mags[buf * NW + wig] = kmax;
            group_sync(bar_id, G::GS);
            int wstar = 0;
            unsigned best = mags[buf * NW];
#pragma unroll
            for (int w = 1; w < NW; ++w) {
                const unsigned m = mags[buf * NW + w];
                if (m > best) {
                    best = m;
                    wstar = w;
                }
            }
            const R *pr = cnd + (buf * NW + wstar) * (LD + 4);
            const bool is_piv = nominee && wig == wstar;
            if (is_piv) {
                mypiv = k;
                if (h == hk) diag = gr[jk];
            }
            bad |= real_lead && best == 0u;  // no non-zero entry left in column k: V is singular
            const R gk = row_entry(k);
            if (real && !is_piv) {
                const R l = gk * pr[LD + 1];
                // columns < k hold multipliers (or this row's pivot); only q > k change
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
                    if (h == hk) gr[jk] = l;
                }
                bc[0] = fma(-l, pr[LD], bc[0]);
                if constexpr (NCOMP > 1) bc[1] = fma(-l, pr[LD + 2], bc[1]);
            }
        }
        if constexpr (SP > 1) diag = __shfl_sync(0xffffffffu, diag, rowbase + (mypiv >= 0 ? mypiv : 0) / NC);
        const bool has = real_lead && mypiv >= 0;
        bad |= real_lead && mypiv < 0;
        R x[NCOMP];
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) x[cc] = has ? bc[cc] / diag : R(0);

        if constexpr (kPair) {
            // one step of iterative refinement: r = phi* - V x from the
            // particle's basis values, V dx = r by replaying the elimination's
            // multipliers (pivot rows in the same order), x += dx
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc)
                if (has) vec[cc * P4 + mypiv] = x[cc];
            group_sync(bar_id, G::GS);
            R rc[NCOMP];
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) rc[cc] = R(0);
            if (real_lead) {
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
                    rc[cc] = rhs[cc * P4 + c] - vx;
                }
            }
#pragma unroll
            for (int k = 0; k < n; ++k) {
                R *pr = piv + (k & 1) * (LD + 4);
                if (lead && mypiv == k)
#pragma unroll
                    for (int cc = 0; cc < NCOMP; ++cc) pr[cc] = rc[cc];
                group_sync(bar_id, G::GS);
                const R gk = row_entry(k);
                if (real_lead && mypiv != k)
#pragma unroll
                    for (int cc = 0; cc < NCOMP; ++cc) rc[cc] = fma(-gk, pr[cc], rc[cc]);
            }
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) x[cc] += has ? rc[cc] / diag : R(0);
        }
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) bad |= real_lead && !isfinite(x[cc]);
        // face values of the advected interpolant (alpha - c = x, node-indexed) at the 4N face points
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc)
            if (has) {
                vec[cc * P4 + mypiv] = x[cc];
                if constexpr (MODE == 2)  // the fast phase 2 starts from it
                    static_cast<R *>(a.alpha)[(((long long)s * NCOMP + cc) * E + e) * n + mypiv] = x[cc];
            }
        group_sync(bar_id, G::GS);
    } else {
        // Gram row c: G[c][c'] = sum_p S[p][c] S[p][c'], b_c = sum_p S[p][c] rhs_p
        // (SP > 1: lane h holds the columns c' = h NC + j, j < NC, of row c)
        R gr[NG];
#pragma unroll
        for (int q = 0; q < NG; ++q) gr[q] = R(0);
        R bc[NCOMP];
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) bc[cc] = R(0);
        const int ic = c % N, jc = c / N;  // node (i, j) of row c
        // face-row weight w and the Gauss-node basis at the faces
        const R wb = R(a.w);
        if (SP == 1 && real) {
            // G = V^T V + B^T B in tensor form.  V[p][(i',j')] = hx_p[i'] hy_p[j'], so
            // row c = (i, j) of V^T V is sum_p V[p][c] (hx_p (x) hy_p), and B's rows
            // (w h_i'(0 or 1) along one face) give w^2 (h0[i] h0[i'] + h1[i] h1[i'])
            // on the entries (i', j) and the same in y on (i, j').
            for (int p = 0; p < n; ++p) {
                const R *hp = Vs + p * HXS;
                R hxp[N], hyp[N];
#pragma unroll
                for (int q = 0; q < 2 * N; q += VW) {
                    const VT v = *reinterpret_cast<const VT *>(hp + q);
#pragma unroll
                    for (int i = 0; i < VW; ++i) {
                        if (q + i < N) hxp[q + i] = VV::at(v, i);
                        else if (q + i < 2 * N) hyp[q + i - N] = VV::at(v, i);
                    }
                }
                const R vpc = hp[ic] * hp[N + jc];
                R u[N];
#pragma unroll
                for (int ii = 0; ii < N; ++ii) u[ii] = vpc * hxp[ii];
#pragma unroll
                for (int jj = 0; jj < N; ++jj)
#pragma unroll
                    for (int ii = 0; ii < N; ++ii) gr[jj * N + ii] = fma(u[ii], hyp[jj], gr[jj * N + ii]);
#pragma unroll
                for (int cc = 0; cc < NCOMP; ++cc) bc[cc] = fma(vpc, rhs[cc * P4 + p], bc[cc]);
            }
            const R w2 = wb * wb;
            const R x0 = w2 * sh0[ic], x1 = w2 * sh1[ic], y0 = w2 * sh0[jc], y1 = w2 * sh1[jc];
#pragma unroll
            for (int jj = 0; jj < N; ++jj)
                if (jj == jc)
#pragma unroll
                    for (int ii = 0; ii < N; ++ii) gr[jj * N + ii] = fma(x1, sh1[ii], fma(x0, sh0[ii], gr[jj * N + ii]));
#pragma unroll
            for (int ii = 0; ii < N; ++ii)
                if (ii == ic)
#pragma unroll
                    for (int jj = 0; jj < N; ++jj) gr[jj * N + ii] = fma(y1, sh1[jj], fma(y0, sh0[jj], gr[jj * N + ii]));
            const R b0x = wb * sh0[ic], b1x = wb * sh1[ic], b0y = wb * sh0[jc], b1y = wb * sh1[jc];
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) {
                const R *rf = rhs + cc * P4 + n;  // w (g - c) per face point: sides x=0, x=1, y=0, y=1
                bc[cc] = fma(b0x, rf[jc], bc[cc]);
                bc[cc] = fma(b1x, rf[N + jc], bc[cc]);
                bc[cc] = fma(b0y, rf[2 * N + ic], bc[cc]);
                bc[cc] = fma(b1y, rf[3 * N + ic], bc[cc]);
            }
        } else if (real) {
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
            if (PHASE == 2 && SP == 1 && group_active && lead && c < 4 * N) {
                // (B x) at face point c: w times the trace of x along the face
                const int side = c / N, f = c % N;
#pragma unroll
                for (int cc = 0; cc < NCOMP; ++cc) {
                    const R *vc = vec + cc * P4;
                    R bx = R(0);
                    if (side < 2) {
                        const R *hf = side == 0 ? sh0 : sh1;
#pragma unroll
                        for (int ii = 0; ii < N; ++ii) bx = fma(hf[ii], vc[f * N + ii], bx);
                    } else {
                        const R *hf = side == 2 ? sh0 : sh1;
#pragma unroll
                        for (int jj = 0; jj < N; ++jj) bx = fma(hf[jj], vc[jj * N + f], bx);
                    }
                    res[cc * P4 + n + c] = rhs[cc * P4 + n + c] - wb * bx;
                }
            } else if (PHASE == 2 && SP > 1 && group_active && lead && c < 4 * N) {
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
            if (SP == 1 && real_lead) {
                // S^T r for row c = (i, j): sum_p V[p][c] r_p, then the four face terms
                for (int p = 0; p < n; ++p) {
                    const R vpc = Vs[p * HXS + ic] * Vs[p * HXS + N + jc];
#pragma unroll
                    for (int cc = 0; cc < NCOMP; ++cc) rc[cc] = fma(vpc, res[cc * P4 + p], rc[cc]);
                }
                const R b0x = wb * sh0[ic], b1x = wb * sh1[ic], b0y = wb * sh0[jc], b1y = wb * sh1[jc];
#pragma unroll
                for (int cc = 0; cc < NCOMP; ++cc) {
                    const R *rf = res + cc * P4 + n;
                    rc[cc] = fma(b0x, rf[jc], rc[cc]);
                    rc[cc] = fma(b1x, rf[N + jc], rc[cc]);
                    rc[cc] = fma(b0y, rf[2 * N + ic], rc[cc]);
                    rc[cc] = fma(b1y, rf[3 * N + ic], rc[cc]);
                }
            } else if (real_lead)
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
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc)
                if (c < n && lead) {  // the group may have more threads than nodes
                    vec[cc * P4 + c] = x[cc];
                    if constexpr (MODE == 2)  // the fast phase 2 starts from it
                        static_cast<R *>(a.alpha)[(((long long)s * NCOMP + cc) * E + e) * n + c] = x[cc];
                }
            group_sync(bar_id, G::GS);
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
    }
    }  // direct path
    if constexpr (PHASE == 1) {
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
    }
    if (bad) atomicOr(a.err, 1);
}

// The step kernel of one phase (see sl2d_cta).  MODE 1 runs one CTA slot per
// CTA.  MODE 2 is a persistent grid over the slot list MODE 1 left: with no
// flagged group it reads the list's length and exits; the last CTA to finish
// empties the list for the next launch.
template <int N, typename R, int PHASE, bool BATCH, int NCOMP = 1, int MODE = 1>
__global__ void __launch_bounds__(Geo2D<N, R, NCOMP, MODE != 2>::kBlock,
                                  MODE == 1 ? min_ctas2d_fast<N, R>() : (MODE == 3 ? 2 : min_ctas2d<N, R>()))
    sl2d_step_kernel(const Step2DArgs a0, const Step2DArgs *__restrict__ args, const long long *__restrict__ prefix,
                     int ninst, int t)
{
    using G = Geo2D<N, R, NCOMP, MODE != 2>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *tab = reinterpret_cast<R *>(smem_raw);
    // node tables depend on N only (every instance of a batch class shares
    // them); computed once per context on the host (node_tables2d)
    const double *tabsrc = BATCH ? args[0].tab : a0.tab;
    if constexpr (MODE != 2) {
        for (int k = threadIdx.x; k < G::kTables; k += blockDim.x) tab[k] = R(tabsrc[k]);
        __syncthreads();
        sl2d_cta<N, R, PHASE, BATCH, NCOMP, MODE>(a0, args, prefix, ninst, t, blockIdx.x);
    } else {
        const Step2DArgs &L = BATCH ? args[0] : a0;
        const unsigned count = *static_cast<volatile const unsigned *>(L.slot_ctl);
        const long long slot0 = BATCH ? 0 : a0.g0 / G::GPC;  // a launch starts on a slot boundary
        if (blockIdx.x < count) {
            for (int k = threadIdx.x; k < G::kTables; k += blockDim.x) tab[k] = R(tabsrc[k]);
            __syncthreads();
            for (unsigned i = blockIdx.x; i < count; i += gridDim.x) {
                const long long slot = L.slot_list[i];
                sl2d_cta<N, R, PHASE, BATCH, NCOMP, MODE>(a0, args, prefix, ninst, t, slot - slot0);
                __syncthreads();  // the slot's shared memory is free again
                if (threadIdx.x == 0) L.slot_mark[slot] = 0u;
            }
        }
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(L.slot_ctl + 1, 1u) == gridDim.x - 1) {  // every other CTA has read the length
                L.slot_ctl[0] = 0u;
                L.slot_ctl[1] = 0u;
            }
        }
    }
}

template <int N, typename R, int NCOMP, int MODE>
size_t smem2d()
{
    using G = Geo2D<N, R, NCOMP, MODE != 2>;
    constexpr bool kX = MODE == 3 || (MODE == 1 && G::kStructC64);
    return sizeof(R) * (((G::kTables + 3) & ~3) + size_t(G::GPC) * (G::kGroup + (kX ? G::kX3 : 0)));
}

// One phase over groups [g0, g1): for orders with the fast path, the fast
// kernel and then the direct kernel for the groups it flagged.
// CTAs of kernel K resident on the device at once (at least one per SM).
template <auto K>
unsigned resident_ctas(int block, size_t smem)
{
    static std::atomic<int> per_sm{0};  // queried once the kernel has been prepared
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        nsm = 1;
    if (per_sm.load() == 0) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, K, block, smem) == cudaSuccess && per > 0)
            per_sm.store(per);
        else
            cudaGetLastError();
    }
    return unsigned(std::max(1, nsm) * std::max(1, per_sm.load()));
}

// The fast kernel runs one CTA per slot of its own geometry (one thread per
// node); the direct kernel (SP lanes per row, fewer groups per CTA) is a
// persistent grid over the slots the fast kernel listed, at most one CTA
// per slot of the launch and no more than fit on the device at once.
// The mixed-precision form (an FP64 capacitance factor, MODE 3) exists for
// the FP32 remap (one or two fields).
template <typename R, int NCOMP>
constexpr bool kHasMode3 = std::is_same<R, float>::value && NCOMP <= 2;

template <int N, typename R, int NCOMP, bool BATCH>
cudaError_t launch_phase2d(int phase, long long groups, const Step2DArgs &b, const Step2DArgs *args,
                           const long long *prefix, int ninst, int t, bool f64c, cudaStream_t st,
                           LaunchThrottle *th)
{
    auto one = [&](auto kernel, auto geo, size_t smem, unsigned cap) -> cudaError_t {
        using G = decltype(geo);
        if (th) {
            const cudaError_t e = th->before();
            if (e != cudaSuccess) return e;
        }
        const unsigned grid = std::min(unsigned((groups + G::GPC - 1) / G::GPC), cap);
        kernel<<<grid, unsigned(G::kBlock), smem, st>>>(b, args, prefix, ninst, t);
        return th ? th->after(st) : cudaSuccess;
    };
    using GF = Geo2D<N, R, NCOMP, true>;
    using GD = Geo2D<N, R, NCOMP, false>;
    constexpr unsigned kAll = ~0u;
    cudaError_t e;
    if (phase == 1) {
        constexpr auto k2 = sl2d_step_kernel<N, R, 1, BATCH, NCOMP, 2>;
        e = one(sl2d_step_kernel<N, R, 1, BATCH, NCOMP, 1>, GF{}, smem2d<N, R, NCOMP, 1>(), kAll);
        if (e == cudaSuccess)
            e = one(k2, GD{}, smem2d<N, R, NCOMP, 2>(), resident_ctas<k2>(GD::kBlock, smem2d<N, R, NCOMP, 2>()));
    } else {
        constexpr auto k2 = sl2d_step_kernel<N, R, 2, BATCH, NCOMP, 2>;
        if constexpr (kHasMode3<R, NCOMP>) {
            e = f64c ? one(sl2d_step_kernel<N, R, 2, BATCH, NCOMP, 3>, GF{}, smem2d<N, R, NCOMP, 3>(), kAll)
                     : one(sl2d_step_kernel<N, R, 2, BATCH, NCOMP, 1>, GF{}, smem2d<N, R, NCOMP, 1>(), kAll);
        } else {
            e = one(sl2d_step_kernel<N, R, 2, BATCH, NCOMP, 1>, GF{}, smem2d<N, R, NCOMP, 1>(), kAll);
        }
        if (e == cudaSuccess)
            e = one(k2, GD{}, smem2d<N, R, NCOMP, 2>(), resident_ctas<k2>(GD::kBlock, smem2d<N, R, NCOMP, 2>()));
    }
    return e;
}

template <int N, typename R, int NCOMP = 1>
cudaError_t launch_step2d_n(const Step2DArgs &a, cudaStream_t st)
{
    using G = Geo2D<N, R, NCOMP>;
    const long long groups = (long long)a.Kx * a.Ky * a.M;
    // a launch covers at most `chunk` groups (a multiple of the groups per CTA)
    const long long chunk =
        a.chunk > 0 ? std::min(groups, (a.chunk + G::GPC - 1) / G::GPC * G::GPC) : groups;
    Step2DArgs b = a;
    LaunchThrottle *th = a.chunk > 0 ? a.throttle : nullptr;
    for (int t = 0; t < a.nsteps; ++t) {
        for (int phase = 1; phase <= 2; ++phase)  // every group's faces before any remap
            for (long long g0 = 0; g0 < groups; g0 += chunk) {
                b.g0 = g0;
                b.g1 = std::min(groups, g0 + chunk);
                const cudaError_t e = launch_phase2d<N, R, NCOMP, false>(phase, b.g1 - g0, b, nullptr, nullptr, 0, t,
                                                                         a.f64_factor != 0, st, th);
                if (e != cudaSuccess) return e;
            }
    }
    return cudaGetLastError();
}

template <int N, typename R, int NCOMP, bool BATCH>
cudaError_t preload_phases2d()
{
    cudaError_t e = cudaSuccess;
    for (auto k : {sl2d_step_kernel<N, R, 1, BATCH, NCOMP, 1>, sl2d_step_kernel<N, R, 1, BATCH, NCOMP, 2>,
                   sl2d_step_kernel<N, R, 2, BATCH, NCOMP, 1>, sl2d_step_kernel<N, R, 2, BATCH, NCOMP, 2>})
        if (e == cudaSuccess) e = prepare_kernel(k);
    if constexpr (kHasMode3<R, NCOMP>)
        if (e == cudaSuccess) e = prepare_kernel(sl2d_step_kernel<N, R, 2, BATCH, NCOMP, 3>);
    return e;
}

// Prepares the single-instance kernels of one order for two fields.
template <int N, typename R>
cudaError_t preload_step2d_c2_n()
{
    return preload_phases2d<N, R, 2, false>();
}

// Prepares the kernels of one order (both phases, single and batched).
template <int N, typename R>
cudaError_t preload_step2d_n()
{
    cudaError_t e = preload_phases2d<N, R, 1, false>();
    if (e == cudaSuccess) e = preload_phases2d<N, R, 1, true>();
    return e;
}

// All instances of one order N, `nsteps` steps: per step both phases, each
// one launch (two with the fast path) over every instance's groups.
template <int N, typename R>
cudaError_t launch_step2d_batch_n(const Batch2DLaunch &b, cudaStream_t st)
{
    Step2DArgs none = {};
    for (int t = 0; t < b.nsteps; ++t)
        for (int phase = 1; phase <= 2; ++phase) {
            const cudaError_t e = launch_phase2d<N, R, 1, true>(phase, b.total_groups, none, b.args, b.prefix, b.ninst,
                                                                t, b.f64_factor != 0, st, nullptr);
            if (e != cudaSuccess) return e;
        }
    return cudaGetLastError();
}

}  // namespace sl
