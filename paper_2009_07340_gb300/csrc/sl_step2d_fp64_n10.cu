// 2D FP64 step kernels for N = 10 (a Gram row of 100 doubles is split over
// several lanes; one order per translation unit compiles in parallel).
#include "sl_step2d.cuh"

namespace sl {
cudaError_t launch_step2d_fp64_n10(const Step2DArgs &a, cudaStream_t st) { return launch_step2d_n<10, double>(a, st); }
cudaError_t launch_step2d_batch_fp64_n10(const Batch2DLaunch &b, cudaStream_t st) { return launch_step2d_batch_n<10, double>(b, st); }
cudaError_t preload_step2d_fp64_n10() { return preload_step2d_n<10, double>(); }
}  // namespace sl
