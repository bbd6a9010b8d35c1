// 1D step kernels, precision mode SL_MIXED (packed FP32, see sl_step1d_f2.cuh;
// measured 8-17% faster than the scalar form for this mode at N = 8..16).
#include "sl_step1d_f2.cuh"

namespace sl {
cudaError_t launch_step1d_mixed(const Step1DArgs &a, int N, cudaStream_t st) { return launch_step1d_f2_mode<SL_MIXED>(a, N, st); }
size_t step1d_smem_bytes_mixed(int N, int S, int T) { return step1d_f2_smem_bytes<SL_MIXED>(N, S, T); }
cudaError_t launch_step1d_batch_mixed(const Batch1DLaunch &b, int N, cudaStream_t st) { return launch_sl1d_step_kernel_f2_batch_mode<SL_MIXED>(b, N, st); }
cudaError_t preload_step1d_mixed() { return preload_step1d_f2_seq<SL_MIXED>(std::make_integer_sequence<int, kMaxN - 1>{}); }
}  // namespace sl
