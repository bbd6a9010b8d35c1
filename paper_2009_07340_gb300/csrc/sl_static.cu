// sl_static.cu -- sample moments without any device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need the
// moments: a serving loop that reserved its whole HBM budget up front and
// admits work by footprint (a new allocation could exceed or fragment that
// budget), code that must not stall other streams (cudaMalloc / cudaFree can
// synchronise the device), or a host framework that owns every device byte
// through its own pool.  sl_moments_static gives them the moment reduction of
// sl_moments_device with its partial sums in a fixed, file-scope device array
// instead of memory allocated by a context.
#include <cuda_runtime.h>

#include <mutex>

#include "sl_internal.cuh"

namespace {

// Partial-sum scratch: 2^21 doubles (16 MiB), held by every GPU that loads
// the library until the process exits.  Shared by all calls on a device.
constexpr long long kStaticScratchDoubles = 1ll << 21;
__device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device; looked up once
// per device (the host-side name of the array is not a device address).
cudaError_t scratch_address(int dev, double **out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int sl_moments_static(const double *d_samples, int M, long long V, double *d_mean, double *d_m2,
                                 void *stream)
{
    if (!d_samples || !d_mean || M < 1 || V < 1) return SL_ERR_ARG;
    // partial sums need 2 * chunks * V doubles; use 64-sample chunks when
    // they fit, longer chunks otherwise
    long long max_chunks = kStaticScratchDoubles / (2 * V);
    if (max_chunks < 1) return SL_ERR_ARG;  // V above 2^20 nodes
    if (max_chunks > 65535) max_chunks = 65535;  // chunks are a grid dimension
    long long chunk = 64;
    if ((M + chunk - 1) / chunk > max_chunks) chunk = (M + max_chunks - 1) / max_chunks;
    const long long nc = (M + chunk - 1) / chunk;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SL_ERR_CUDA;
    double *scratch = nullptr;
    if (scratch_address(dev, &scratch) != cudaSuccess) return SL_ERR_CUDA;
    // every partial the final pass reads is written first by this call:
    // nothing in the scratch needs clearing
    const cudaError_t e = sl::launch_moments(d_samples, 1, M, V, int(chunk), scratch, scratch + nc * V, d_mean, d_m2,
                                             static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SL_OK : SL_ERR_CUDA;
}
