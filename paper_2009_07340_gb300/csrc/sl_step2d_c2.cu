// 2D step kernels for two fields per sample sharing the particles (and so
// the Gram matrix and its elimination), FP32 and FP64, N <= 8.  Batches and
// served requests carry one field; these are the single-instance kernels.
#include "sl_step2d.cuh"

namespace sl {
cudaError_t launch_step2d_c2(const Step2DArgs &a, int N, bool fp64, cudaStream_t st)
{
    switch (N) {
    case 2: return fp64 ? launch_step2d_n<2, double, 2>(a, st) : launch_step2d_n<2, float, 2>(a, st);
    case 3: return fp64 ? launch_step2d_n<3, double, 2>(a, st) : launch_step2d_n<3, float, 2>(a, st);
    case 4: return fp64 ? launch_step2d_n<4, double, 2>(a, st) : launch_step2d_n<4, float, 2>(a, st);
    case 5: return fp64 ? launch_step2d_n<5, double, 2>(a, st) : launch_step2d_n<5, float, 2>(a, st);
    case 6: return fp64 ? launch_step2d_n<6, double, 2>(a, st) : launch_step2d_n<6, float, 2>(a, st);
    case 7: return fp64 ? launch_step2d_n<7, double, 2>(a, st) : launch_step2d_n<7, float, 2>(a, st);
    case 8: return fp64 ? launch_step2d_n<8, double, 2>(a, st) : launch_step2d_n<8, float, 2>(a, st);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t preload_step2d_c2()
{
    cudaError_t e = cudaSuccess;
    for (auto f : {preload_step2d_c2_n<2, float>, preload_step2d_c2_n<3, float>, preload_step2d_c2_n<4, float>,
                   preload_step2d_c2_n<5, float>, preload_step2d_c2_n<6, float>, preload_step2d_c2_n<7, float>,
                   preload_step2d_c2_n<8, float>, preload_step2d_c2_n<2, double>, preload_step2d_c2_n<3, double>,
                   preload_step2d_c2_n<4, double>, preload_step2d_c2_n<5, double>, preload_step2d_c2_n<6, double>,
                   preload_step2d_c2_n<7, double>, preload_step2d_c2_n<8, double>})
        if (e == cudaSuccess) e = f();
    return e;
}
}  // namespace sl
