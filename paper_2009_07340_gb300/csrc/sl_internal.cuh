// sl_internal.cuh -- context layout and launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/sl.h"

namespace sl {

constexpr int kMaxN = 16;           // nodes per direction per element
constexpr int kMaxThreads1D = 256;  // elements (threads) per CTA in the 1D kernel
constexpr int kMaxCluster1D = 8;    // CTAs per sample field (portable cluster size)

// Field descriptor copied to the device for the initialisation kernels.
struct FieldDev {
    int kind;
    double p[40];
};

struct Mesh {
    int dim, N, n;  // n = N^dim nodes per element
    int K[2];       // elements per direction (K[1] = 1 in 1D)
    int E;          // elements
    double lo[2], hi[2], h[2];
};

// Kernel arguments of the 1D step (one launch advances `nsteps` steps).
struct Step1DArgs {
    int K, M;         // elements, samples
    int S;            // samples per CTA (cluster size 1) ; 1 when clustered
    int C;            // CTAs per sample field (cluster size)
    int T;            // thread slots per sample per CTA (>= elements per CTA)
    int nsteps;
    double dt, h;
    const double *xi;      // [N] reference nodes on [0,1]
    const double *nodeU;   // [K][N] drift at the nodes
    const double *nodeB;   // [K][N] sqrt(2 D) at the nodes
    const double *nodeDiv; // [K][N] du/dx at the nodes
    const double *faceU;   // [K] drift at interface k (left face of element k)
    const double *faceB;   // [K] sqrt(2 D) at interface k
    const double *dW;      // [nsteps][M] Wiener increments
    void *Q;               // [M][K][N] state (double for SL_FP64, float otherwise)
    int *err;              // device error word (bit 0: non-finite remap)
};

// Kernel arguments of the 2D step.
struct Step2DArgs {
    int Kx, Ky, M;
    int nsteps;
    double dt, hx, hy;
    const double *xi;
    const double *nodeU;   // [2][E][n]
    const double *nodeB;   // [E][n]
    const double *nodeDiv; // [E][n]
    const double *faceU;   // [2][E][N]: vertical (u_x at x-face of e), horizontal (u_y)
    const double *faceB;   // [2][E][N]
    const double *dW;      // [nsteps][M][2]
    void *Q;               // [M][E][n]
    void *faces;           // scratch [M][E][4N] face values of the advected interpolant
    int *err;
};

cudaError_t launch_step1d_fp64(const Step1DArgs &a, int N, cudaStream_t st);
cudaError_t launch_step1d_mixed(const Step1DArgs &a, int N, cudaStream_t st);
cudaError_t launch_step1d_fp32(const Step1DArgs &a, int N, cudaStream_t st);
size_t step1d_smem_bytes_fp64(int N, int S, int T);
size_t step1d_smem_bytes_mixed(int N, int S, int T);
size_t step1d_smem_bytes_fp32(int N, int S, int T);
cudaError_t launch_step2d_fp64(const Step2DArgs &a, int N, cudaStream_t st);
cudaError_t launch_step2d_fp32(const Step2DArgs &a, int N, cudaStream_t st);
cudaError_t launch_init_fields(const Mesh &m, const FieldDev &u, const FieldDev &D, const FieldDev &phi0,
                               const double *phi0_nodal_dev, double *xi, double *nodeU, double *nodeB,
                               double *nodeDiv, double *faceU, double *faceB, void *Q, int M,
                               int state_is_double, cudaStream_t st);
cudaError_t launch_wiener(unsigned long long seed, long long step0, long long sample0, int nsteps, int M, int dim,
                          double sqrt_dt, double *out, cudaStream_t st);
cudaError_t launch_moments(const void *Q, int state_is_double, int M, long long V, int chunk,
                           double *psum, double *psq, double *mean, double *m2, cudaStream_t st);

}  // namespace sl
