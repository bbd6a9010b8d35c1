// 2D step kernels of the FP32 remap with float-pair state (see
// sl_step2d.cuh), N <= 12.  Both FP32 modes run them; SL_MIXED differs only
// in the remap's fast kernel, which factors the capacitance matrix in FP64
// (MODE 3).  The orders are compiled in sl_step2d_fp32_nNN.cu.
#include "sl_internal.cuh"

namespace sl {
cudaError_t launch_step2d_fp32_n2(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32_n2(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t launch_step2d_fp32_n3(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32_n3(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t launch_step2d_fp32_n4(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32_n4(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t launch_step2d_fp32_n5(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32_n5(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t launch_step2d_fp32_n6(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32_n6(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t launch_step2d_fp32_n7(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32_n7(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t launch_step2d_fp32_n8(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32_n8(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t launch_step2d_fp32_n9(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32_n9(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t launch_step2d_fp32_n10(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32_n10(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t launch_step2d_fp32_n11(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32_n11(const Batch2DLaunch &b, cudaStream_t st);
cudaError_t launch_step2d_fp32_n12(const Step2DArgs &a, cudaStream_t st);
cudaError_t launch_step2d_batch_fp32_n12(const Batch2DLaunch &b, cudaStream_t st);

cudaError_t preload_step2d_fp32_n2();
cudaError_t preload_step2d_fp32_n3();
cudaError_t preload_step2d_fp32_n4();
cudaError_t preload_step2d_fp32_n5();
cudaError_t preload_step2d_fp32_n6();
cudaError_t preload_step2d_fp32_n7();
cudaError_t preload_step2d_fp32_n8();
cudaError_t preload_step2d_fp32_n9();
cudaError_t preload_step2d_fp32_n10();
cudaError_t preload_step2d_fp32_n11();
cudaError_t preload_step2d_fp32_n12();

cudaError_t launch_step2d_fp32(const Step2DArgs &a, int N, cudaStream_t st)
{
    switch (N) {
    case 2: return launch_step2d_fp32_n2(a, st);
    case 3: return launch_step2d_fp32_n3(a, st);
    case 4: return launch_step2d_fp32_n4(a, st);
    case 5: return launch_step2d_fp32_n5(a, st);
    case 6: return launch_step2d_fp32_n6(a, st);
    case 7: return launch_step2d_fp32_n7(a, st);
    case 8: return launch_step2d_fp32_n8(a, st);
    case 9: return launch_step2d_fp32_n9(a, st);
    case 10: return launch_step2d_fp32_n10(a, st);
    case 11: return launch_step2d_fp32_n11(a, st);
    case 12: return launch_step2d_fp32_n12(a, st);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t preload_step2d_fp32()
{
    cudaError_t e = cudaSuccess;
    for (auto f : {preload_step2d_fp32_n2, preload_step2d_fp32_n3, preload_step2d_fp32_n4, preload_step2d_fp32_n5, preload_step2d_fp32_n6, preload_step2d_fp32_n7, preload_step2d_fp32_n8, preload_step2d_fp32_n9, preload_step2d_fp32_n10, preload_step2d_fp32_n11, preload_step2d_fp32_n12})
        if (e == cudaSuccess) e = f();
    return e;
}

cudaError_t launch_step2d_batch_fp32(const Batch2DLaunch &b, int N, cudaStream_t st)
{
    switch (N) {
    case 2: return launch_step2d_batch_fp32_n2(b, st);
    case 3: return launch_step2d_batch_fp32_n3(b, st);
    case 4: return launch_step2d_batch_fp32_n4(b, st);
    case 5: return launch_step2d_batch_fp32_n5(b, st);
    case 6: return launch_step2d_batch_fp32_n6(b, st);
    case 7: return launch_step2d_batch_fp32_n7(b, st);
    case 8: return launch_step2d_batch_fp32_n8(b, st);
    case 9: return launch_step2d_batch_fp32_n9(b, st);
    case 10: return launch_step2d_batch_fp32_n10(b, st);
    case 11: return launch_step2d_batch_fp32_n11(b, st);
    case 12: return launch_step2d_batch_fp32_n12(b, st);
    default: return cudaErrorNotSupported;
    }
}
}  // namespace sl
