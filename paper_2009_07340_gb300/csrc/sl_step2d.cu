// 2D step kernels (tensor-product elements).
#include "sl_internal.cuh"

namespace sl {
cudaError_t launch_step2d(const Step2DArgs &, int, int, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace sl
