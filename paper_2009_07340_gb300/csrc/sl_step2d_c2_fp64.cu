// 2D FP64 step kernels for two fields per sample, N <= 8 (see
// sl_step2d_c2.cu; a translation unit of their own so that the two
// precisions compile in parallel).
#include "sl_step2d.cuh"

namespace sl {
cudaError_t launch_step2d_c2_fp64(const Step2DArgs &a, int N, cudaStream_t st)
{
    switch (N) {
    case 2: return launch_step2d_n<2, double, 2>(a, st);
    case 3: return launch_step2d_n<3, double, 2>(a, st);
    case 4: return launch_step2d_n<4, double, 2>(a, st);
    case 5: return launch_step2d_n<5, double, 2>(a, st);
    case 6: return launch_step2d_n<6, double, 2>(a, st);
    case 7: return launch_step2d_n<7, double, 2>(a, st);
    case 8: return launch_step2d_n<8, double, 2>(a, st);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t preload_step2d_c2_fp64()
{
    cudaError_t e = cudaSuccess;
    for (auto f : {preload_step2d_c2_n<2, double>, preload_step2d_c2_n<3, double>, preload_step2d_c2_n<4, double>,
                   preload_step2d_c2_n<5, double>, preload_step2d_c2_n<6, double>, preload_step2d_c2_n<7, double>,
                   preload_step2d_c2_n<8, double>})
        if (e == cudaSuccess) e = f();
    return e;
}
}  // namespace sl
