// sl_step1d.cuh -- 1D semi-Lagrangian Monte-Carlo step, sample field resident
// on chip for all steps of a launch.
//
// Mapping.  One thread owns one element of one sample and keeps its N nodal
// values in registers across the whole step loop.  A CTA holds S complete
// sample fields (K <= 256 elements), or, for K > 256, a thread-block cluster
// of C CTAs holds one sample field and exchanges face values through
// distributed shared memory.  Per step the only communication is the two
// face values per element (Eq. remap_bnd) needed by the neighbours' upwind
// choice (Eq. bnd_update): one barrier per step, double-buffered faces.
//
// Per element-sample and step (Sections 5.2-5.3), in element coordinates
// scaled by 4 (zeta = 4 xi, exact; it keeps every product of N-1 node
// differences O(N) so the batch inversion below cannot overflow in FP32).
// A particle is its Gauss node plus a displacement and is never formed as one
// number: every difference is (zeta_i - zeta_m) [table Z] + displacement
// difference, so a displacement ~1e-4 of the node coordinate keeps its full
// relative precision (rounding zeta + delta would bias the drift by up to
// ulp(zeta)/delta per step, a systematic error that grows with the step count).
//   delta_j  = 4 u_j dt / h + (4 b_j / h) dW                     Eq. def_dx
//   phi*_j   = Q_j - (dt du/dx|_j) Q_j                           Eq. advection_phi
//   w_j      = 1 / prod_{m != j} (Z_jm + delta_j - delta_m)  (barycentric
//              weights of the advected nodes; one division per element by
//              batch inversion)
//   E_bj     = w_j prod_{m != j} (zeta_b - zeta_m - delta_m), zeta_b = 0, 4:
//              advected Lagrange basis (Eq. h_star) at the faces
//   e_b      = sum_j phi*_j E_bj                                  Eq. remap_bnd
//   g        = upwind face values                                 Eq. bnd_update
//   q        = argmin |V q - phi*|^2 + |B q - g|^2               Section 5.3
// The remap uses the reduced form of that least-squares problem: with
// H* = V^{-1} (the advected basis at the Gauss nodes) and E = B V^{-1},
//   mu = (I + E E^T)^{-1} (E phi* - g),   q = H* (phi* - E^T mu),
// a 2x2 SPD "capacitance" solve (the factor) and one evaluation of the
// advected interpolant at the N Gauss nodes.  Values enter relative to an
// element reference value c (the middle node's state), using sum_j h*_j = 1,
// which keeps the rounding of the FP32 forms proportional to the variation
// inside the element.
//
// State precision.  SL_FP64 keeps the state in FP64.  The FP32 modes keep it
// as an unevaluated pair hi + lo of floats: all samples hold nearly the same
// values, so the rounding of a plain FP32 state is correlated across samples
// and steps, does not average out in the moments, and grows linearly with the
// step count.  Each node is updated as q = c + A with c the element's
// reference value (a pair) and A the FP32 remap correction, by an exact
// TwoSum; face values are exchanged as pairs and jumps e - g are formed from
// the pair parts, so every FP32 quantity is a small difference.
//
// Each evaluation sum_j c_j prod_{m != j}(z - zeta*_m) uses the division-free
// recurrence A <- A d_k + c_k P, P <- P d_k (4 operations per term).  Work per
// element-sample and step: ~6 N^2 + 22 N operations.
#pragma once
#include <cooperative_groups.h>

#include <type_traits>

#include "sl_internal.cuh"

// CTAs per SM the FP32 modes are compiled for (register budget 256 threads x 2).
#ifndef SL1D_FP32_MIN_BLOCKS
#define SL1D_FP32_MIN_BLOCKS 2
#endif

namespace sl {

namespace cg = cooperative_groups;

template <int MODE>
struct Prec1D;
template <>
struct Prec1D<SL_FP64> {
    using R = double;      // basis evaluation and contractions
    using State = double;  // resident state
    using Fac = double;    // 2x2 capacitance factor
};
template <>
struct Prec1D<SL_MIXED> {
    using R = float;
    using State = float2;  // hi + lo
    using Fac = double;
};
template <>
struct Prec1D<SL_FP32> {
    using R = float;
    using State = float2;
    using Fac = float;
};

// s + e = a + b exactly (Knuth's TwoSum; no magnitude ordering needed).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// A boundary value as a face value: FP64, or the float pair hi + lo.
template <typename FaceT>
__device__ __forceinline__ FaceT ghost_face(double g)
{
    if constexpr (std::is_same<FaceT, double>::value) {
        return g;
    } else {
        const float hi = float(g);
        return make_float2(hi, float(g - double(hi)));
    }
}

// Row of a shared-memory table into registers with 16-byte loads.
// Compile-time node tables of the FP32 kernels (values the compiler folds
// into the instructions, so the step loop loads no node table): 4 (xi_i -
// xi_m), -4 xi_m and 4 (1 - xi_m), with xi_i = (1 - cos((i + 1/2) pi / N)) / 2.
// cos and sin by their Taylor series on [0, pi/4] after the exact reductions
// cos(pi t) = -cos(pi (1 - t)) and cos(pi t) = sin(pi (1/2 - t)); for
// N = 2..16 every entry equals the float of the same expression with libm's
// cos.  Measured 3-6 % faster per step than the shared-memory tables (which
// the FP64 kernels keep); a __constant__-memory table had been slower, since
// the compiler held its values in registers.
constexpr double kPiCt = 3.141592653589793238462643383279502884;
constexpr double ct_cos_series(double x)
{
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k <= 12; ++k) {
        term *= -x2 / double((2 * k - 1) * (2 * k));
        sum += term;
    }
    return sum;
}
constexpr double ct_sin_series(double x)
{
    double x2 = x * x, term = x, sum = x;
    for (int k = 1; k <= 12; ++k) {
        term *= -x2 / double((2 * k) * (2 * k + 1));
        sum += term;
    }
    return sum;
}
constexpr double ct_cospi(double t)  // t in [0, 1]
{
    if (t > 0.5) return -ct_cospi(1.0 - t);
    if (t > 0.25) return ct_sin_series(kPiCt * (0.5 - t));
    return ct_cos_series(kPiCt * t);
}
template <int N>
struct NodeTab1D {
    float z[N][N];
    float f0[N], f1[N];
    constexpr NodeTab1D() : z(), f0(), f1()
    {
        double xi[N] = {};
        for (int i = 0; i < N; ++i) xi[i] = 0.5 * (1.0 - ct_cospi((i + 0.5) / N));
        for (int i = 0; i < N; ++i)
            for (int m = 0; m < N; ++m) z[i][m] = float(4.0 * (xi[i] - xi[m]));
        for (int m = 0; m < N; ++m) {
            f0[m] = float(-4.0 * xi[m]);
            f1[m] = float(4.0 * (1.0 - xi[m]));
        }
    }
};

template <int NP>
__device__ __forceinline__ void load_row(const float *src, float (&z)[NP])
{
#pragma unroll
    for (int m = 0; m < NP; m += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(src + m);
        z[m] = v.x;
        z[m + 1] = v.y;
        z[m + 2] = v.z;
        z[m + 3] = v.w;
    }
}
template <int NP>
__device__ __forceinline__ void load_row(const double *src, double (&z)[NP])
{
#pragma unroll
    for (int m = 0; m < NP; m += 2) {
        const double2 v = *reinterpret_cast<const double2 *>(src + m);
        z[m] = v.x;
        z[m + 1] = v.y;
    }
}

// NCOMP scalar fields per sample share the particles and so the advance, the
// weights, the advected face basis, the upwind choice and the capacitance
// factor (Section 5.3: the remap cost does not grow with the number of
// components); the compositional update, face values, jumps, mu and the
// final evaluation are per component.  State layout [M][NCOMP][K][N].
template <int N, int MODE, int NCOMP>
__device__ __forceinline__ void step1d_body(const Step1DArgs &a, const int slot)
{
    using R = typename Prec1D<MODE>::R;
    using State = typename Prec1D<MODE>::State;
    using Fac = typename Prec1D<MODE>::Fac;
    constexpr bool kPair = !std::is_same<R, double>::value;
    using FaceT = typename std::conditional<kPair, float2, double>::type;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = a.T, S = a.S, K = a.K;
    constexpr int NP = (N + 3) & ~3;            // padded row of the Z table
    // face pairs first (8-byte aligned for any S, T), then the 16-byte
    // aligned Z table (4 S T faces of 8 bytes = a multiple of 32 bytes)
    FaceT *sface = reinterpret_cast<FaceT *>(smem_raw);           // [2 buf][2 side][NCOMP][S][T]
    R *sZ = reinterpret_cast<R *>(smem_raw + sizeof(FaceT) * 4 * NCOMP * S * T);  // [N][NP] zeta_i - zeta_m
    R *sal = sZ + N * NP;                      // [N][T] 4 u dt / h
    R *sbe = sal + N * T;                      // [N][T] 4 b / h
    R *sga = sbe + N * T;                      // [N][T] dt du/dx
    R *sF0 = sga + N * T;                      // [N] 0 - zeta_m
    R *sF1 = sF0 + N;                          // [N] 4 - zeta_m
    R *sfa = sF1 + N;                          // [T + 1] u dt at the interfaces k0 .. k1
    R *sfb = sfa + (T + 1);                    // [T + 1] sqrt(2 D)
    constexpr NodeTab1D<N> kTab{};
    auto F0 = [&](int m) -> R { if constexpr (kPair) return kTab.f0[m]; else return sF0[m]; };
    auto F1 = [&](int m) -> R { if constexpr (kPair) return kTab.f1[m]; else return sF1[m]; };

    cg::cluster_group cluster = cg::this_cluster();
    const int C = a.C;
    const int rank = C > 1 ? int(cluster.block_rank()) : 0;
    const int k0 = int((long long)K * rank / C);
    const int k1 = int((long long)K * (rank + 1) / C);
    const int Kc = k1 - k0;

    // dt-dependent coefficient tables of this CTA's elements
    for (int idx = threadIdx.x; idx < N * T; idx += blockDim.x) {
        const int j = idx / T, kl = idx - j * T;
        double al = 0.0, be = 0.0, ga = 0.0;  // idle slots: unmoved nodes
        if (kl < Kc) {
            const int k = k0 + kl;
            al = 4.0 * a.nodeU[k * N + j] * a.dt / a.h;
            be = 4.0 * a.nodeB[k * N + j] / a.h;
            ga = a.dt * a.nodeDiv[k * N + j];
        }
        sal[idx] = R(al);
        sbe[idx] = R(be);
        sga[idx] = R(ga);
    }
    for (int idx = threadIdx.x; idx < N * NP; idx += blockDim.x) {
        const int i = idx / NP, m = idx - i * NP;
        sZ[idx] = m < N ? R(4.0 * (a.xi[i] - a.xi[m])) : R(0);
    }
    for (int idx = threadIdx.x; idx <= Kc; idx += blockDim.x) {
        const int f = a.periodic ? (k0 + idx) % K : k0 + idx;  // interface f: left face of element f
        sfa[idx] = R(a.faceU[f] * a.dt);
        sfb[idx] = R(a.faceB[f]);
    }
    if (threadIdx.x < N) {
        sF0[threadIdx.x] = R(-4.0 * a.xi[threadIdx.x]);
        sF1[threadIdx.x] = R(4.0 * (1.0 - a.xi[threadIdx.x]));
    }

    const int sl = threadIdx.x / T;
    const int kl = threadIdx.x - sl * T;
    const int s = slot * S + sl;
    const bool active = sl < S && kl < Kc && s < a.M;

    State *Qg = reinterpret_cast<State *>(a.Q);
    R Q[NCOMP][N], Ql[NCOMP][N];  // state (hi part in Q; lo part used by the pair modes only)
#pragma unroll
    for (int cc = 0; cc < NCOMP; ++cc)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            Q[cc][j] = R(0);
            Ql[cc][j] = R(0);
        }
    if (active) {
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) {
            const State *src = Qg + (((long long)s * NCOMP + cc) * K + (k0 + kl)) * N;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                if constexpr (kPair) {
                    const float2 v = src[j];
                    Q[cc][j] = v.x;
                    Ql[cc][j] = v.y;
                } else {
                    Q[cc][j] = src[j];
                }
            }
        }
    }
    // neighbour slots for the upwind choice
    const int sbase = (sl < S ? sl : 0) * T;  // threads beyond S*T read slot 0, never write
    int lnb_rank = rank, lnb_idx = kl - 1;
    int rnb_rank = rank, rnb_idx = kl + 1;
    if (kl == 0) {
        if (C == 1)
            lnb_idx = Kc - 1;
        else {
            lnb_rank = (rank - 1 + C) % C;
            const int pk0 = int((long long)K * lnb_rank / C), pk1 = int((long long)K * (lnb_rank + 1) / C);
            lnb_idx = pk1 - pk0 - 1;
        }
    }
    if (kl == Kc - 1) {
        if (C == 1)
            rnb_idx = 0;
        else {
            rnb_rank = (rank + 1) % C;
            rnb_idx = 0;
        }
    }
    bool bad = false;

    if (C > 1)
        cluster.sync();
    else
        __syncthreads();

    double dWn = (active && a.nsteps > 0) ? a.dW[s] : 0.0;
    for (int t = 0; t < a.nsteps; ++t) {
        const double dW = dWn;
        if (active && t + 1 < a.nsteps) dWn = a.dW[(long long)(t + 1) * a.M + s];
        const R dWr = R(dW);

        // advance (Eq. def_dx) and compositional update (Eq. advection_phi)
        // every value enters relative to c = Q_ref (the middle node's state):
        // ph_j = phi*_j - c = (Q_j - c) - (dt du/dx)_j Q_j
        R dl[N], ph[NCOMP][N], ch[NCOMP], cl[NCOMP];
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) {
            ch[cc] = Q[cc][N / 2];
            cl[cc] = Ql[cc][N / 2];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            dl[j] = fma(sbe[j * T + kl], dWr, sal[j * T + kl]);
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) {
                R dq = Q[cc][j] - ch[cc];
                if constexpr (kPair) dq += Ql[cc][j] - cl[cc];
                ph[cc][j] = fma(-sga[j * T + kl], Q[cc][j], dq);
            }
        }

        // barycentric weights of the advected nodes
        R w[N];
#pragma unroll
        for (int j = 0; j < N; ++j) w[j] = R(1);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R z[NP];
            if constexpr (kPair) {
#pragma unroll
                for (int m = 0; m < N; ++m) z[m] = kTab.z[j][m];
            } else {
                load_row<NP>(sZ + j * NP, z);
            }
#pragma unroll
            for (int m = j + 1; m < N; ++m) {
                const R d = z[m] + (dl[j] - dl[m]);
                w[j] *= d;
                w[m] *= -d;
            }
        }
        {
            R pp[N];
            pp[0] = w[0];
#pragma unroll
            for (int j = 1; j < N; ++j) pp[j] = pp[j - 1] * w[j];
            R inv = R(1) / pp[N - 1];
#pragma unroll
            for (int j = N - 1; j >= 1; --j) {
                const R pj = w[j];
                w[j] = inv * pp[j - 1];
                inv *= pj;
            }
            w[0] = inv;
        }

        // advected basis at the two faces and the face values
        R E0[N], E1[N];
        R e0[NCOMP], e1[NCOMP];
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) e0[cc] = e1[cc] = R(0);
        {
            R pre[N];
            pre[0] = R(1);
#pragma unroll
            for (int m = 1; m < N; ++m) pre[m] = pre[m - 1] * (F0(m - 1) - dl[m - 1]);
            R suf = R(1);
#pragma unroll
            for (int j = N - 1; j >= 0; --j) {
                E0[j] = w[j] * (pre[j] * suf);
                suf *= F0(j) - dl[j];
            }
            pre[0] = R(1);
#pragma unroll
            for (int m = 1; m < N; ++m) pre[m] = pre[m - 1] * (F1(m - 1) - dl[m - 1]);
            suf = R(1);
#pragma unroll
            for (int j = N - 1; j >= 0; --j) {
                E1[j] = w[j] * (pre[j] * suf);
                suf *= F1(j) - dl[j];
            }
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc)
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    e0[cc] = fma(ph[cc][j], E0[j], e0[cc]);  // face values relative to c
                    e1[cc] = fma(ph[cc][j], E1[j], e1[cc]);
                }
        }
        FaceT f0[NCOMP], f1[NCOMP];  // absolute face values
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) {
            if constexpr (kPair) {
                two_sum(ch[cc], e0[cc], f0[cc].x, f0[cc].y);
                f0[cc].y += cl[cc];
                two_sum(ch[cc], e1[cc], f1[cc].x, f1[cc].y);
                f1[cc].y += cl[cc];
            } else {
                f0[cc] = ch[cc] + e0[cc];
                f1[cc] = ch[cc] + e1[cc];
            }
        }

        const int buf = t & 1;
        FaceT *fL = sface + (buf * 2 + 0) * NCOMP * S * T;  // value at xi = 0 of each element, [NCOMP][S][T]
        FaceT *fR = sface + (buf * 2 + 1) * NCOMP * S * T;  // value at xi = 1
        if (sl < S) {
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) {
                fL[cc * S * T + sbase + kl] = f0[cc];
                fR[cc * S * T + sbase + kl] = f1[cc];
            }
        }
        if (C > 1)
            cluster.sync();
        else
            __syncthreads();

        // upwind interface values (Eq. bnd_update): at interface f take the
        // left element's value when u dt + sqrt(2D) dW > 0
        FaceT gL[NCOMP], gR[NCOMP];
        {
            R sigL, sigR;
            if constexpr (sizeof(R) == 8) {  // same operation order as the definition
                sigL = __dadd_rn(sfa[kl], __dmul_rn(sfb[kl], dWr));
                sigR = __dadd_rn(sfa[kl + 1], __dmul_rn(sfb[kl + 1], dWr));
            } else {
                sigL = fmaf(sfb[kl], dWr, sfa[kl]);
                sigR = fmaf(sfb[kl + 1], dWr, sfa[kl + 1]);
            }
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) {
                FaceT left_e1, right_e0;
                if (C > 1) {
                    left_e1 = *cluster.map_shared_rank(fR + cc * S * T + lnb_idx, lnb_rank);
                    right_e0 = *cluster.map_shared_rank(fL + cc * S * T + rnb_idx, rnb_rank);
                } else {
                    left_e1 = fR[cc * S * T + sbase + lnb_idx];
                    right_e0 = fL[cc * S * T + sbase + rnb_idx];
                }
                if (!a.periodic) {  // a domain boundary: the ghost value takes the missing neighbour's place
                    if (k0 + kl == 0) left_e1 = ghost_face<FaceT>(a.ghost[2 * t + 0]);
                    if (k0 + kl == K - 1) right_e0 = ghost_face<FaceT>(a.ghost[2 * t + 1]);
                }
                gL[cc] = sigL > R(0) ? left_e1 : f0[cc];
                gR[cc] = sigR > R(0) ? f1[cc] : right_e0;
            }
        }

        // 2x2 capacitance solve: (I + E E^T) mu = E phi* - g
        R mu0[NCOMP], mu1[NCOMP];
        {
            R g00 = R(0), g01 = R(0), g11 = R(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                g00 = fma(E0[j], E0[j], g00);
                g01 = fma(E0[j], E1[j], g01);
                g11 = fma(E1[j], E1[j], g11);
            }
            // I / w^2 + E E^T (w = 1 unless the caller weights the boundary rows)
            const Fac G00 = Fac(a.inv_w2) + Fac(g00), G01 = Fac(g01), G11 = Fac(a.inv_w2) + Fac(g11);
            const Fac det = G00 * G11 - G01 * G01;
            const Fac idet = Fac(1) / det;
            bad |= !(det > Fac(0));
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) {
                Fac r0, r1;  // jumps E phi* - g
                if constexpr (kPair) {
                    r0 = Fac((f0[cc].x - gL[cc].x) + (f0[cc].y - gL[cc].y));
                    r1 = Fac((f1[cc].x - gR[cc].x) + (f1[cc].y - gR[cc].y));
                } else {
                    r0 = f0[cc] - gL[cc];
                    r1 = f1[cc] - gR[cc];
                }
                const Fac m0 = (G11 * r0 - G01 * r1) * idet;
                const Fac m1 = (G00 * r1 - G01 * r0) * idet;
                mu0[cc] = R(m0);
                mu1[cc] = R(m1);
                bad |= !isfinite(m0) || !isfinite(m1);
            }
        }

        // q_i = c + sum_j (phi*_j - c - E0_j mu0 - E1_j mu1) h*_j(xi_i)
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc)
#pragma unroll
            for (int j = 0; j < N; ++j) ph[cc][j] = (ph[cc][j] - fma(E0[j], mu0[cc], E1[j] * mu1[cc])) * w[j];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            R z[NP];
            if constexpr (kPair) {
#pragma unroll
                for (int m = 0; m < N; ++m) z[m] = kTab.z[i][m];
            } else {
                load_row<NP>(sZ + i * NP, z);
            }
            R A[NCOMP];
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) A[cc] = ph[cc][0];
            R P = z[0] - dl[0];
#pragma unroll
            for (int k = 1; k < N; ++k) {
                const R d = z[k] - dl[k];
#pragma unroll
                for (int cc = 0; cc < NCOMP; ++cc) A[cc] = fma(A[cc], d, ph[cc][k] * P);
                if (k + 1 < N) P *= d;
            }
#pragma unroll
            for (int cc = 0; cc < NCOMP; ++cc) {
                if constexpr (kPair) {
                    two_sum(ch[cc], A[cc], Q[cc][i], Ql[cc][i]);
                    Ql[cc][i] += cl[cc];
                } else {
                    Q[cc][i] = ch[cc] + A[cc];
                }
            }
        }
    }

    if (active) {
#pragma unroll
        for (int cc = 0; cc < NCOMP; ++cc) {
            State *dst = Qg + (((long long)s * NCOMP + cc) * K + (k0 + kl)) * N;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                if constexpr (kPair)
                    dst[j] = make_float2(Q[cc][j], Ql[cc][j]);
                else
                    dst[j] = Q[cc][j];
            }
        }
        if (bad) atomicOr(a.err, 1);
    }
    // no CTA may leave while a cluster peer can still read its faces
    if (C > 1) cluster.sync();
}

// One launch: CTA (or cluster) b advances sample slot b / C.
template <int N, int MODE>
__global__ void __launch_bounds__(kMaxThreads1D, MODE == SL_FP64 ? 1 : SL1D_FP32_MIN_BLOCKS) sl1d_step_kernel(const Step1DArgs a)
{
    step1d_body<N, MODE, 1>(a, int(blockIdx.x) / a.C);
}

// Two scalar fields per sample sharing the remap factorization.
template <int N, int MODE>
__global__ void __launch_bounds__(kMaxThreads1D, MODE == SL_FP64 ? 1 : SL1D_FP32_MIN_BLOCKS) sl1d_step_kernel_c2(const Step1DArgs a)
{
    step1d_body<N, MODE, 2>(a, int(blockIdx.x) / a.C);
}

// Persistent batched launch over many instances of one order N (K <= 256,
// no clusters): each CTA takes work items (instance, sample slot) from an
// atomic counter and runs every step of the item resident on chip.
template <int N, int MODE>
__global__ void __launch_bounds__(kMaxThreads1D, MODE == SL_FP64 ? 1 : SL1D_FP32_MIN_BLOCKS) sl1d_step_kernel_batch(const Step1DArgs *__restrict__ args,
                                                   const int *__restrict__ item_prefix, int ninst,
                                                   int *__restrict__ counter)
{
    __shared__ int s_item;
    const int total = item_prefix[ninst];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= total) return;
        int lo = 0, hi = ninst - 1;  // last instance with item_prefix[i] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (item_prefix[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const Step1DArgs ai = args[lo];
        step1d_body<N, MODE, 1>(ai, item - item_prefix[lo]);
        __syncthreads();  // shared tables of this item are dead before the next fill
    }
}

template <int MODE>
size_t step1d_smem_bytes_t(int N, int S, int T, int ncomp = 1)
{
    using R = typename Prec1D<MODE>::R;
    const int NP = (N + 3) & ~3;
    return sizeof(R) * (size_t(N) * NP + size_t(3) * N * T + 2 * N + 2 * (T + 1)) + size_t(8) * 4 * ncomp * S * T;
}

template <int N, int MODE>
cudaError_t launch_step1d_n(const Step1DArgs &a, cudaStream_t st)
{
    const size_t smem = step1d_smem_bytes_t<MODE>(N, a.S, a.T, a.ncomp);
    auto kern = a.ncomp == 2 ? sl1d_step_kernel_c2<N, MODE> : sl1d_step_kernel<N, MODE>;
    cudaLaunchConfig_t cfg = {};
    const int slots = (a.M + a.S - 1) / a.S;
    cfg.gridDim = dim3(unsigned(slots * a.C));
    cfg.blockDim = dim3(unsigned(a.S * a.T));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(a.C);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int MODE>
cudaError_t launch_step1d_mode(const Step1DArgs &a, int N, cudaStream_t st)
{
    switch (N) {
    case 2: return launch_step1d_n<2, MODE>(a, st);
    case 3: return launch_step1d_n<3, MODE>(a, st);
    case 4: return launch_step1d_n<4, MODE>(a, st);
    case 5: return launch_step1d_n<5, MODE>(a, st);
    case 6: return launch_step1d_n<6, MODE>(a, st);
    case 7: return launch_step1d_n<7, MODE>(a, st);
    case 8: return launch_step1d_n<8, MODE>(a, st);
    case 9: return launch_step1d_n<9, MODE>(a, st);
    case 10: return launch_step1d_n<10, MODE>(a, st);
    case 11: return launch_step1d_n<11, MODE>(a, st);
    case 12: return launch_step1d_n<12, MODE>(a, st);
    case 13: return launch_step1d_n<13, MODE>(a, st);
    case 14: return launch_step1d_n<14, MODE>(a, st);
    case 15: return launch_step1d_n<15, MODE>(a, st);
    case 16: return launch_step1d_n<16, MODE>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int N, int MODE>
cudaError_t launch_sl1d_step_kernel_batch_n(const Batch1DLaunch &b, cudaStream_t st)
{
    auto kern = sl1d_step_kernel_batch<N, MODE>;
    cudaError_t e = cudaMemsetAsync(b.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<b.grid, kMaxThreads1D, b.smem, st>>>(b.args, b.prefix, b.ninst, b.counter);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_sl1d_step_kernel_batch_mode(const Batch1DLaunch &b, int N, cudaStream_t st)
{
    switch (N) {
    case 2: return launch_sl1d_step_kernel_batch_n<2, MODE>(b, st);
    case 3: return launch_sl1d_step_kernel_batch_n<3, MODE>(b, st);
    case 4: return launch_sl1d_step_kernel_batch_n<4, MODE>(b, st);
    case 5: return launch_sl1d_step_kernel_batch_n<5, MODE>(b, st);
    case 6: return launch_sl1d_step_kernel_batch_n<6, MODE>(b, st);
    case 7: return launch_sl1d_step_kernel_batch_n<7, MODE>(b, st);
    case 8: return launch_sl1d_step_kernel_batch_n<8, MODE>(b, st);
    case 9: return launch_sl1d_step_kernel_batch_n<9, MODE>(b, st);
    case 10: return launch_sl1d_step_kernel_batch_n<10, MODE>(b, st);
    case 11: return launch_sl1d_step_kernel_batch_n<11, MODE>(b, st);
    case 12: return launch_sl1d_step_kernel_batch_n<12, MODE>(b, st);
    case 13: return launch_sl1d_step_kernel_batch_n<13, MODE>(b, st);
    case 14: return launch_sl1d_step_kernel_batch_n<14, MODE>(b, st);
    case 15: return launch_sl1d_step_kernel_batch_n<15, MODE>(b, st);
    case 16: return launch_sl1d_step_kernel_batch_n<16, MODE>(b, st);
    default: return cudaErrorInvalidValue;
    }
}

// Prepares the step kernels of one mode for every order.
template <int MODE, int... I>
cudaError_t preload_step1d_seq(std::integer_sequence<int, I...>)
{
    cudaError_t e = cudaSuccess;
    auto one = [&](auto f) {
        if (e == cudaSuccess) e = prepare_kernel(f);
    };
    (one(sl1d_step_kernel<I + 2, MODE>), ...);
    (one(sl1d_step_kernel_c2<I + 2, MODE>), ...);
    (one(sl1d_step_kernel_batch<I + 2, MODE>), ...);
    return e;
}

template <int MODE>
cudaError_t preload_step1d_mode()
{
    return preload_step1d_seq<MODE>(std::make_integer_sequence<int, kMaxN - 1>{});
}

}  // namespace sl
