// sl_step1d_f2.cuh -- the FP32 modes (SL_MIXED, SL_FP32) of the 1D step with
// packed f32x2 arithmetic (FFMA2 / FADD2 / FMUL2, sm_100 and later).
//
// Same method, same mapping and same arithmetic decisions as sl_step1d.cuh
// (reduced constrained least-squares remap, displacement kept apart from the
// node position, values relative to the element reference c, FP32-pair state
// updated by an exact TwoSum); only the instruction form changes.  Two lanes
// carry two independent chains in one instruction, which halves the issue
// slots of the O(N^2) parts:
//   - advance / compositional update / state update: node pairs (2p, 2p+1);
//   - barycentric weights: for each advected node j, the products over
//     m-pairs of (Z_jm + delta_j - delta_m) (the m = j lane multiplies by 1);
//   - face bases: lane 0 = face xi = 0, lane 1 = face xi = 1;
//   - remap: k outer over the advected nodes, pairs of Gauss nodes inner,
//     with d'_ik = Z_ki + delta_k = -(zeta_i - zeta*_k); the recurrence on d'
//     returns (-1)^(N-1) times the sum, a compile-time sign.
// For odd N the last pair has one virtual lane (tables hold 0 there); it is
// never read back.
#pragma once
#include "sl_step1d.cuh"

namespace sl {

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <int J>
__device__ __forceinline__ float lane(const float2 *v)
{
    return (J & 1) ? v[J >> 1].y : v[J >> 1].x;
}
__device__ __forceinline__ float lane_rt(const float2 &v, int odd) { return odd ? v.y : v.x; }

template <int N, int MODE>
__device__ __forceinline__ void step1d_f2_body(const Step1DArgs &a, const int slot)
{
    using Fac = typename Prec1D<MODE>::Fac;
    constexpr int NE = N + (N & 1);     // padded to an even count
    constexpr int NH = NE / 2;          // node pairs
    constexpr int NP = (NE + 3) & ~3;   // Z row length (float4 loads)
    constexpr float kSign = (N & 1) ? 1.f : -1.f;  // (-1)^(N-1)

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = a.T, S = a.S, K = a.K;
    float2 *sface = reinterpret_cast<float2 *>(smem_raw);                 // [2 buf][2 side][S][T] pairs
    float *sZ = reinterpret_cast<float *>(sface + 4 * S * T);             // [N][NP] zeta_j - zeta_m
    float2 *sal = reinterpret_cast<float2 *>(sZ + N * NP);                // [NH][T] 4 u dt / h
    float2 *sbe = sal + NH * T;                                           // [NH][T] 4 b / h
    float2 *sng = sbe + NH * T;                                           // [NH][T] -dt du/dx
    float2 *sF = sng + NH * T;                                            // [N] (0 - zeta_m, 4 - zeta_m)
    float *sfa = reinterpret_cast<float *>(sF + N);                       // [T + 1] u dt at interfaces
    float *sfb = sfa + (T + 1);                                           // [T + 1] sqrt(2 D)
    // node tables as compile-time constants (see NodeTab1D): rows of Z padded
    // with zeros past N, face pairs (0 - zeta_m, 4 - zeta_m)
    constexpr NodeTab1D<N> kTab{};
    auto zrow = [&](int j, float (&zr)[NP]) {
#pragma unroll
        for (int m = 0; m < NP; ++m) zr[m] = m < N ? kTab.z[j][m] : 0.f;
    };
    auto Fp = [&](int m) { return make_float2(kTab.f0[m], kTab.f1[m]); };

    cg::cluster_group cluster = cg::this_cluster();
    const int C = a.C;
    const int rank = C > 1 ? int(cluster.block_rank()) : 0;
    const int k0 = int((long long)K * rank / C);
    const int k1 = int((long long)K * (rank + 1) / C);
    const int Kc = k1 - k0;

    for (int idx = threadIdx.x; idx < NH * T; idx += blockDim.x) {
        const int p = idx / T, kl = idx - p * T;
        float v[3][2];
        for (int l = 0; l < 2; ++l) {
            const int j = 2 * p + l;
            double al = 0.0, be = 0.0, ga = 0.0;
            if (kl < Kc && j < N) {
                const int k = k0 + kl;
                al = 4.0 * a.nodeU[k * N + j] * a.dt / a.h;
                be = 4.0 * a.nodeB[k * N + j] / a.h;
                ga = a.dt * a.nodeDiv[k * N + j];
            }
            v[0][l] = float(al);
            v[1][l] = float(be);
            v[2][l] = float(-ga);
        }
        sal[idx] = make_float2(v[0][0], v[0][1]);
        sbe[idx] = make_float2(v[1][0], v[1][1]);
        sng[idx] = make_float2(v[2][0], v[2][1]);
    }
    for (int idx = threadIdx.x; idx < N * NP; idx += blockDim.x) {
        const int j = idx / NP, m = idx - j * NP;
        sZ[idx] = m < N ? float(4.0 * (a.xi[j] - a.xi[m])) : 0.f;
    }
    for (int idx = threadIdx.x; idx <= Kc; idx += blockDim.x) {
        const int f = a.periodic ? (k0 + idx) % K : k0 + idx;  // K: the boundary x = hi
        sfa[idx] = float(a.faceU[f] * a.dt);
        sfb[idx] = float(a.faceB[f]);
    }
    if (threadIdx.x < N)
        sF[threadIdx.x] = make_float2(float(-4.0 * a.xi[threadIdx.x]), float(4.0 * (1.0 - a.xi[threadIdx.x])));

    const int sl = threadIdx.x / T;
    const int kl = threadIdx.x - sl * T;
    const int s = slot * S + sl;
    const bool active = sl < S && kl < Kc && s < a.M;

    float2 *Qg = reinterpret_cast<float2 *>(a.Q);
    float2 Qh[NH], Ql[NH];  // state pairs: hi parts and lo parts of nodes (2p, 2p+1)
#pragma unroll
    for (int p = 0; p < NH; ++p) {
        Qh[p] = make_float2(0.f, 0.f);
        Ql[p] = make_float2(0.f, 0.f);
    }
    if (active) {
        const float2 *src = Qg + ((long long)s * K + (k0 + kl)) * N;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const float2 v = src[j];
            if (j & 1) {
                Qh[j >> 1].y = v.x;
                Ql[j >> 1].y = v.y;
            } else {
                Qh[j >> 1].x = v.x;
                Ql[j >> 1].x = v.y;
            }
        }
    }
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
        const float dWr = float(dWn);
        if (active && t + 1 < a.nsteps) dWn = a.dW[(long long)(t + 1) * a.M + s];

        // advance and compositional update, relative to c = Q_{N/2}
        const float ch = lane_rt(Qh[(N / 2) >> 1], (N / 2) & 1);
        const float cl = lane_rt(Ql[(N / 2) >> 1], (N / 2) & 1);
        float2 dl[NH], ndl[NH], ph[NH];
        const float2 nch = bc2(-ch), ncl = bc2(-cl);
#pragma unroll
        for (int p = 0; p < NH; ++p) {
            dl[p] = fma2(sbe[p * T + kl], bc2(dWr), sal[p * T + kl]);
            ndl[p] = mul2(dl[p], bc2(-1.f));
            const float2 dq = add2(add2(Qh[p], nch), add2(Ql[p], ncl));
            ph[p] = fma2(sng[p * T + kl], Qh[p], dq);
        }

        // barycentric weights w_j = 1 / prod_{m != j}(Z_jm + delta_j - delta_m)
        float w[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            float zr[NP];
            zrow(j, zr);
            const float dj = lane_rt(dl[j >> 1], j & 1);
            float2 acc = make_float2(1.f, 1.f);
#pragma unroll
            for (int p = 0; p < NH; ++p) {
                float2 d = add2(make_float2(zr[2 * p], zr[2 * p + 1]), add2(bc2(dj), ndl[p]));
                if (2 * p == j) d.x = 1.f;
                if (2 * p + 1 == j || 2 * p + 1 >= N) d.y = 1.f;
                acc = mul2(acc, d);
            }
            w[j] = acc.x * acc.y;
        }
        {
            float pp[N];
            pp[0] = w[0];
#pragma unroll
            for (int j = 1; j < N; ++j) pp[j] = pp[j - 1] * w[j];
            float inv = 1.f / pp[N - 1];
#pragma unroll
            for (int j = N - 1; j >= 1; --j) {
                const float pj = w[j];
                w[j] = inv * pp[j - 1];
                inv *= pj;
            }
            w[0] = inv;
        }

        // advected basis at both faces at once: E[j] = (E0_j, E1_j)
        float2 E[N];
        float2 e = make_float2(0.f, 0.f);
        {
            float2 pre[N];
            pre[0] = make_float2(1.f, 1.f);
#pragma unroll
            for (int m = 1; m < N; ++m)
                pre[m] = mul2(pre[m - 1], add2(Fp(m - 1), bc2(lane_rt(ndl[(m - 1) >> 1], (m - 1) & 1))));
            float2 suf = make_float2(1.f, 1.f);
#pragma unroll
            for (int j = N - 1; j >= 0; --j) {
                E[j] = mul2(mul2(bc2(w[j]), pre[j]), suf);
                if (j > 0) suf = mul2(suf, add2(Fp(j), bc2(lane_rt(ndl[j >> 1], j & 1))));
            }
#pragma unroll
            for (int j = 0; j < N; ++j) e = fma2(bc2(lane_rt(ph[j >> 1], j & 1)), E[j], e);
        }
        float2 f0, f1;  // absolute face values as (hi, lo) pairs
        two_sum(ch, e.x, f0.x, f0.y);
        f0.y += cl;
        two_sum(ch, e.y, f1.x, f1.y);
        f1.y += cl;

        const int buf = t & 1;
        float2 *fL = sface + (buf * 2 + 0) * S * T;
        float2 *fR = sface + (buf * 2 + 1) * S * T;
        if (sl < S) {
            fL[sbase + kl] = f0;
            fR[sbase + kl] = f1;
        }
        if (C > 1)
            cluster.sync();
        else
            __syncthreads();

        float2 gL, gR;
        {
            const float sigL = fmaf(sfb[kl], dWr, sfa[kl]);
            const float sigR = fmaf(sfb[kl + 1], dWr, sfa[kl + 1]);
            float2 left_e1, right_e0;
            if (C > 1) {
                left_e1 = *cluster.map_shared_rank(fR + lnb_idx, lnb_rank);
                right_e0 = *cluster.map_shared_rank(fL + rnb_idx, rnb_rank);
            } else {
                left_e1 = fR[sbase + lnb_idx];
                right_e0 = fL[sbase + rnb_idx];
            }
            if (!a.periodic) {  // a domain boundary: the ghost value takes the missing neighbour's place
                if (k0 + kl == 0) left_e1 = ghost_face<float2>(a.ghost[2 * t + 0]);
                if (k0 + kl == K - 1) right_e0 = ghost_face<float2>(a.ghost[2 * t + 1]);
            }
            gL = sigL > 0.f ? left_e1 : f0;
            gR = sigR > 0.f ? f1 : right_e0;
        }

        // 2x2 capacitance solve (I + E E^T) mu = E phi* - g
        float mu0, mu1;
        {
            float2 gd = make_float2(0.f, 0.f);
            float g01 = 0.f;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                gd = fma2(E[j], E[j], gd);
                g01 = fmaf(E[j].x, E[j].y, g01);
            }
            // I / w^2 + E E^T (w = 1 unless the caller weights the boundary rows)
            const Fac G00 = Fac(a.inv_w2) + Fac(gd.x), G01 = Fac(g01), G11 = Fac(a.inv_w2) + Fac(gd.y);
            const Fac r0 = Fac((f0.x - gL.x) + (f0.y - gL.y));
            const Fac r1 = Fac((f1.x - gR.x) + (f1.y - gR.y));
            const Fac det = G00 * G11 - G01 * G01;
            const Fac idet = Fac(1) / det;
            const Fac m0 = (G11 * r0 - G01 * r1) * idet;
            const Fac m1 = (G00 * r1 - G01 * r0) * idet;
            mu0 = float(m0);
            mu1 = float(m1);
            bad |= !(det > Fac(0)) || !isfinite(m0) || !isfinite(m1);
        }

        // rw_j = (phi*_j - c - E0_j mu0 - E1_j mu1) w_j
        float rw[N];
#pragma unroll
        for (int j = 0; j < N; ++j)
            rw[j] = (lane_rt(ph[j >> 1], j & 1) - fmaf(E[j].x, mu0, E[j].y * mu1)) * w[j];

        // remap to the Gauss nodes, pairs of nodes per instruction
        float2 A[NH], P[NH];
        {
            float zr[NP];
            zrow(0, zr);
            const float d0 = lane_rt(dl[0], 0);
#pragma unroll
            for (int p = 0; p < NH; ++p) {
                A[p] = bc2(rw[0]);
                P[p] = add2(make_float2(zr[2 * p], zr[2 * p + 1]), bc2(d0));
            }
        }
#pragma unroll
        for (int k = 1; k < N; ++k) {
            float zr[NP];
            zrow(k, zr);
            const float2 dk = bc2(lane_rt(dl[k >> 1], k & 1));
            const float2 rk = bc2(rw[k]);
#pragma unroll
            for (int p = 0; p < NH; ++p) {
                const float2 d = add2(make_float2(zr[2 * p], zr[2 * p + 1]), dk);
                A[p] = fma2(A[p], d, mul2(rk, P[p]));
                if (k + 1 < N) P[p] = mul2(P[p], d);
            }
        }
        // q = c + sign * A as an exact pair (TwoSum, two lanes per instruction)
#pragma unroll
        for (int p = 0; p < NH; ++p) {
            const float2 b = mul2(A[p], bc2(kSign));
            const float2 sm = add2(bc2(ch), b);
            const float2 bb = fma2(bc2(ch), bc2(-1.f), sm);          // s - a
            const float2 ta = fma2(bb, bc2(-1.f), sm);               // s - bb
            const float2 ea = fma2(ta, bc2(-1.f), bc2(ch));          // a - (s - bb)
            const float2 eb = fma2(bb, bc2(-1.f), b);                // b - bb
            Qh[p] = sm;
            Ql[p] = add2(add2(ea, eb), bc2(cl));
        }
    }

    if (active) {
        float2 *dst = Qg + ((long long)s * K + (k0 + kl)) * N;
#pragma unroll
        for (int j = 0; j < N; ++j)
            dst[j] = (j & 1) ? make_float2(Qh[j >> 1].y, Ql[j >> 1].y) : make_float2(Qh[j >> 1].x, Ql[j >> 1].x);
        if (bad) atomicOr(a.err, 1);
    }
    if (C > 1) cluster.sync();
}

// One launch: CTA (or cluster) b advances sample slot b / C.
template <int N, int MODE>
__global__ void __launch_bounds__(kMaxThreads1D, SL1D_FP32_MIN_BLOCKS) sl1d_step_kernel_f2(const Step1DArgs a)
{
    step1d_f2_body<N, MODE>(a, int(blockIdx.x) / a.C);
}

// Persistent batched launch over many instances of one order N (K <= 256,
// no clusters): each CTA takes work items (instance, sample slot) from an
// atomic counter and runs every step of the item resident on chip.
template <int N, int MODE>
__global__ void __launch_bounds__(kMaxThreads1D, SL1D_FP32_MIN_BLOCKS) sl1d_step_kernel_f2_batch(const Step1DArgs *__restrict__ args,
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
        step1d_f2_body<N, MODE>(ai, item - item_prefix[lo]);
        __syncthreads();  // shared tables of this item are dead before the next fill
    }
}

template <int MODE>
size_t step1d_f2_smem_bytes(int N, int S, int T)
{
    const int NE = N + (N & 1), NH = NE / 2, NP = (NE + 3) & ~3;
    return sizeof(float2) * (size_t(4) * S * T) + sizeof(float) * size_t(N) * NP +
           sizeof(float2) * (size_t(3) * NH * T + N) + sizeof(float) * 2 * (T + 1);
}

template <int N, int MODE>
cudaError_t launch_step1d_f2_n(const Step1DArgs &a, cudaStream_t st)
{
    const size_t smem = step1d_f2_smem_bytes<MODE>(N, a.S, a.T);
    auto kern = sl1d_step_kernel_f2<N, MODE>;
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
cudaError_t launch_step1d_f2_mode(const Step1DArgs &a, int N, cudaStream_t st)
{
    switch (N) {
    case 2: return launch_step1d_f2_n<2, MODE>(a, st);
    case 3: return launch_step1d_f2_n<3, MODE>(a, st);
    case 4: return launch_step1d_f2_n<4, MODE>(a, st);
    case 5: return launch_step1d_f2_n<5, MODE>(a, st);
    case 6: return launch_step1d_f2_n<6, MODE>(a, st);
    case 7: return launch_step1d_f2_n<7, MODE>(a, st);
    case 8: return launch_step1d_f2_n<8, MODE>(a, st);
    case 9: return launch_step1d_f2_n<9, MODE>(a, st);
    case 10: return launch_step1d_f2_n<10, MODE>(a, st);
    case 11: return launch_step1d_f2_n<11, MODE>(a, st);
    case 12: return launch_step1d_f2_n<12, MODE>(a, st);
    case 13: return launch_step1d_f2_n<13, MODE>(a, st);
    case 14: return launch_step1d_f2_n<14, MODE>(a, st);
    case 15: return launch_step1d_f2_n<15, MODE>(a, st);
    case 16: return launch_step1d_f2_n<16, MODE>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int N, int MODE>
cudaError_t launch_sl1d_step_kernel_f2_batch_n(const Batch1DLaunch &b, cudaStream_t st)
{
    auto kern = sl1d_step_kernel_f2_batch<N, MODE>;
    cudaError_t e = cudaMemsetAsync(b.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<b.grid, kMaxThreads1D, b.smem, st>>>(b.args, b.prefix, b.ninst, b.counter);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_sl1d_step_kernel_f2_batch_mode(const Batch1DLaunch &b, int N, cudaStream_t st)
{
    switch (N) {
    case 2: return launch_sl1d_step_kernel_f2_batch_n<2, MODE>(b, st);
    case 3: return launch_sl1d_step_kernel_f2_batch_n<3, MODE>(b, st);
    case 4: return launch_sl1d_step_kernel_f2_batch_n<4, MODE>(b, st);
    case 5: return launch_sl1d_step_kernel_f2_batch_n<5, MODE>(b, st);
    case 6: return launch_sl1d_step_kernel_f2_batch_n<6, MODE>(b, st);
    case 7: return launch_sl1d_step_kernel_f2_batch_n<7, MODE>(b, st);
    case 8: return launch_sl1d_step_kernel_f2_batch_n<8, MODE>(b, st);
    case 9: return launch_sl1d_step_kernel_f2_batch_n<9, MODE>(b, st);
    case 10: return launch_sl1d_step_kernel_f2_batch_n<10, MODE>(b, st);
    case 11: return launch_sl1d_step_kernel_f2_batch_n<11, MODE>(b, st);
    case 12: return launch_sl1d_step_kernel_f2_batch_n<12, MODE>(b, st);
    case 13: return launch_sl1d_step_kernel_f2_batch_n<13, MODE>(b, st);
    case 14: return launch_sl1d_step_kernel_f2_batch_n<14, MODE>(b, st);
    case 15: return launch_sl1d_step_kernel_f2_batch_n<15, MODE>(b, st);
    case 16: return launch_sl1d_step_kernel_f2_batch_n<16, MODE>(b, st);
    default: return cudaErrorInvalidValue;
    }
}

// Prepares the packed step kernels of one mode for every order.
template <int MODE, int... I>
cudaError_t preload_step1d_f2_seq(std::integer_sequence<int, I...>)
{
    cudaError_t e = cudaSuccess;
    auto one = [&](auto f) {
        if (e == cudaSuccess) e = prepare_kernel(f);
    };
    (one(sl1d_step_kernel_f2<I + 2, MODE>), ...);
    (one(sl1d_step_kernel_f2_batch<I + 2, MODE>), ...);
    return e;
}

}  // namespace sl
