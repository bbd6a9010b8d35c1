// 1D step kernels, precision mode SL_FP64 (see sl_step1d.cuh).
#include "sl_step1d.cuh"

namespace sl {
cudaError_t launch_step1d_fp64(const Step1DArgs &a, int N, cudaStream_t st) { return launch_step1d_mode<SL_FP64>(a, N, st); }
size_t step1d_smem_bytes_fp64(int N, int S, int T) { return step1d_smem_bytes_t<SL_FP64>(N, S, T); }
cudaError_t launch_step1d_batch_fp64(const Batch1DLaunch &b, int N, cudaStream_t st) { return launch_sl1d_step_kernel_batch_mode<SL_FP64>(b, N, st); }
cudaError_t preload_step1d_fp64() { return preload_step1d_mode<SL_FP64>(); }
}  // namespace sl
