// 2D FP64 step kernels for N = 9 (a Gram row of 81 doubles is split over
// several lanes; one order per translation unit compiles in parallel).
#include "sl_step2d.cuh"

namespace sl {
cudaError_t launch_step2d_fp64_n9(const Step2DArgs &a, cudaStream_t st) { return launch_step2d_n<9, double>(a, st); }
cudaError_t launch_step2d_batch_fp64_n9(const Batch2DLaunch &b, cudaStream_t st) { return launch_step2d_batch_n<9, double>(b, st); }
cudaError_t preload_step2d_fp64_n9() { return preload_step2d_n<9, double>(); }
}  // namespace sl
