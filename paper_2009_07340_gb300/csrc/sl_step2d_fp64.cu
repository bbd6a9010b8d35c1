// 2D step kernels in FP64 (see sl_step2d.cuh); N <= 8 (a Gram row of 64
// doubles per thread stays in registers).
#include "sl_step2d.cuh"

namespace sl {
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
    default: return cudaErrorNotSupported;
    }
}
}  // namespace sl
