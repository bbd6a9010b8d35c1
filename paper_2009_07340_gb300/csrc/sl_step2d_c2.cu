// 2D step kernels for two fields per sample sharing the particles (and so
// the fast path's preconditioner and capacitance inverse, and the direct
// path's Gram matrix and its elimination), N <= 8.  Batches and served
// requests carry one field; these are the single-instance kernels.  The
// FP64 kernels are compiled in sl_step2d_c2_fp64.cu.
#include "sl_step2d.cuh"

namespace sl {
cudaError_t launch_step2d_c2_fp64(const Step2DArgs &a, int N, cudaStream_t st);
cudaError_t preload_step2d_c2_fp64();

cudaError_t launch_step2d_c2(const Step2DArgs &a, int N, bool fp64, cudaStream_t st)
{
    if (fp64) return launch_step2d_c2_fp64(a, N, st);
    switch (N) {
    case 2: return launch_step2d_n<2, float, 2>(a, st);
    case 3: return launch_step2d_n<3, float, 2>(a, st);
    case 4: return launch_step2d_n<4, float, 2>(a, st);
    case 5: return launch_step2d_n<5, float, 2>(a, st);
    case 6: return launch_step2d_n<6, float, 2>(a, st);
    case 7: return launch_step2d_n<7, float, 2>(a, st);
    case 8: return launch_step2d_n<8, float, 2>(a, st);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t preload_step2d_c2()
{
    cudaError_t e = cudaSuccess;
    for (auto f : {preload_step2d_c2_n<2, float>, preload_step2d_c2_n<3, float>, preload_step2d_c2_n<4, float>,
                   preload_step2d_c2_n<5, float>, preload_step2d_c2_n<6, float>, preload_step2d_c2_n<7, float>,
                   preload_step2d_c2_n<8, float>})
        if (e == cudaSuccess) e = f();
    return e == cudaSuccess ? preload_step2d_c2_fp64() : e;
}
}  // namespace sl
