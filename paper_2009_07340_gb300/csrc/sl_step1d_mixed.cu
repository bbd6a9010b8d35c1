// 1D step kernels, precision mode SL_MIXED (see sl_step1d.cuh).
#include "sl_step1d.cuh"

namespace sl {
cudaError_t launch_step1d_mixed(const Step1DArgs &a, int N, cudaStream_t st) { return launch_step1d_mode<SL_MIXED>(a, N, st); }
size_t step1d_smem_bytes_mixed(int N, int S, int T) { return step1d_smem_bytes_t<SL_MIXED>(N, S, T); }
}  // namespace sl
