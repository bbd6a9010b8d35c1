// 2D FP32 step kernels for N = 11 (one order per translation unit keeps the
// heavily unrolled Gram / Gauss-Jordan code of the orders compiling in parallel).
#include "sl_step2d.cuh"

namespace sl {
cudaError_t launch_step2d_fp32_n11(const Step2DArgs &a, cudaStream_t st) { return launch_step2d_n<11, float>(a, st); }
cudaError_t launch_step2d_batch_fp32_n11(const Batch2DLaunch &b, cudaStream_t st) { return launch_step2d_batch_n<11, float>(b, st); }
cudaError_t preload_step2d_fp32_n11() { return preload_step2d_n<11, float>(); }
}  // namespace sl
