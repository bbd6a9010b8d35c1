// 2D step kernels in FP64 (see sl_step2d.cuh); N <= 8 keep a Gram row of up
// to 64 doubles in one thread's registers, N = 9..11 split it over two or
// four lanes (sl_step2d_fp64_nNN.cu).  N = 12 would need 228 KB of shared
// memory per element-sample, above the per-CTA limit.
#include "sl_step2d.cuh"

namespace sl {
cudaError_t launch_step2d_fp64_n9(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp64_n9(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t preload_step2d_fp64_n9();
cudaError_t launch_step2d_fp64_n10(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp64_n10(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t preload_step2d_fp64_n10();
cudaError_t launch_step2d_fp64_n11(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp64_n11(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t preload_step2d_fp64_n11();

cudaError_t launch_step2d_fp64(const Step2DArgs &a, int N, cudaStream_t st)
{
    switch (N) {
    case 2: return launch_step2d_n<2, double>(a, st);
    case 3: return launch_step2d_n<3, double>(a, st);
    case 4: return launch_step2d_n<4, double>(a, st);
    case 5: return launch_step2d_n<5, double>(a, st);
    case 6: return launch_step2d_n<6, double>(a, st);
    case 7: return launch_step2d_n<7, double>(a, st);
    case 8: return launch_step2d_n<8, double>(a, st);
    case 9: return launch_step2d_fp64_n9(a, st);
    case 10: return launch_step2d_fp64_n10(a, st);
    case 11: return launch_step2d_fp64_n11(a, st);
    default: return cudaErrorNotSupported;
    }
}
cudaError_t preload_step2d_fp64()
{
    cudaError_t e = preload_step2d_n<2, double>();
    if (e == cudaSuccess) e = preload_step2d_n<3, double>();
    if (e == cudaSuccess) e = preload_step2d_n<4, double>();
    if (e == cudaSuccess) e = preload_step2d_n<5, double>();
    if (e == cudaSuccess) e = preload_step2d_n<6, double>();
    if (e == cudaSuccess) e = preload_step2d_n<7, double>();
    if (e == cudaSuccess) e = preload_step2d_n<8, double>();
    if (e == cudaSuccess) e = preload_step2d_fp64_n9();
    if (e == cudaSuccess) e = preload_step2d_fp64_n10();
    if (e == cudaSuccess) e = preload_step2d_fp64_n11();
    return e;
}
cudaError_t launch_step2d_batch_fp64(const Batch2DLaunch &b, int N, cudaStream_t st)
{
    switch (N) {
    case 2: return launch_step2d_batch_n<2, double>(b, st);
    case 3: return launch_step2d_batch_n<3, double>(b, st);
    case 4: return launch_step2d_batch_n<4, double>(b, st);
    case 5: return launch_step2d_batch_n<5, double>(b, st);
    case 6: return launch_step2d_batch_n<6, double>(b, st);
    case 7: return launch_step2d_batch_n<7, double>(b, st);
    case 8: return launch_step2d_batch_n<8, double>(b, st);
    case 9: return launch_step2d_batch_fp64_n9(b, st);
    case 10: return launch_step2d_batch_fp64_n10(b, st);
    case 11: return launch_step2d_batch_fp64_n11(b, st);
    default: return cudaErrorNotSupported;
    }
}
}  // namespace sl
