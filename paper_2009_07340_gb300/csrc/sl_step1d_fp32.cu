// 1D step kernels, precision mode SL_FP32 (scalar FP32 kernel of sl_step1d.cuh;
// measured as fast as the packed form on GB300, where FFMA2 has the FFMA rate).
#include "sl_step1d.cuh"

namespace sl {
cudaError_t launch_step1d_fp32(const Step1DArgs &a, int N, cudaStream_t st) { return launch_step1d_mode<SL_FP32>(a, N, st); }
size_t step1d_smem_bytes_fp32(int N, int S, int T) { return step1d_smem_bytes_t<SL_FP32>(N, S, T); }
cudaError_t launch_step1d_batch_fp32(const Batch1DLaunch &b, int N, cudaStream_t st) { return launch_sl1d_step_kernel_batch_mode<SL_FP32>(b, N, st); }
cudaError_t preload_step1d_fp32() { return preload_step1d_mode<SL_FP32>(); }
}  // namespace sl
