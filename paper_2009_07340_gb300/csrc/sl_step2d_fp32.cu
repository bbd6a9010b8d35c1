// 2D step kernels in FP32 with float-pair state and one refinement step
// (see sl_step2d.cuh); N <= 10 (a Gram row of up to 100 floats per thread).
// Both FP32 modes (SL_MIXED, SL_FP32) run this kernel in 2D: an FP64 Gram
// factor would cost ~n^3/2 FP64 operations per element-sample, at 1/64 of the
// FP32 rate on GB300.
#include "sl_step2d.cuh"

namespace sl {
cudaError_t launch_step2d_fp32(const Step2DArgs &a, int N, cudaStream_t st)
{
    switch (N) {
    case 2: return launch_step2d_n<2, float>(a, st);
    case 3: return launch_step2d_n<3, float>(a, st);
    case 4: return launch_step2d_n<4, float>(a, st);
    case 5: return launch_step2d_n<5, float>(a, st);
    case 6: return launch_step2d_n<6, float>(a, st);
    case 7: return launch_step2d_n<7, float>(a, st);
    case 8: return launch_step2d_n<8, float>(a, st);
    case 9: return launch_step2d_n<9, float>(a, st);
    case 10: return launch_step2d_n<10, float>(a, st);
    default: return cudaErrorNotSupported;
    }
}
}  // namespace sl
