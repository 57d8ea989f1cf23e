// Allocation-free form of ddgi_image_metrics for callers that cannot call
// cudaMalloc (for example a plug-in whose host application owns the whole
// device-memory budget, or a real-time thread where an allocation and its
// implicit device synchronisation are not allowed).  The per-block partial
// sums live in a file-scope device array instead of caller scratch.
#include <mutex>

#include "internal.h"

namespace {

// 2 doubles per block for at most kMetricMaxBlocks blocks: 16 KiB, held by
// every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_metric_scratch[2 * kMetricMaxBlocks];

// Largest image this entry point accepts (pixels).
constexpr uint32_t kStaticMaxPixels = 1u << 26;
constexpr int kMaxDevices = 64;

std::mutex g_lock;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in, so the address is looked up once per device
// (with that device current) and cached.  The cache is never invalidated: a
// device reset that reloads the module could move the array, which is why
// the header rules out calls after a reset.
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_metric_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" ddgi_status ddgi_image_metrics_static(const float* img, const float* ref, uint32_t n,
                                                 double* out, void* stream) {
    if (!out || (n > 0 && (!img || !ref))) return DDGI_ERR_INVALID_ARG;
    if (n > kStaticMaxPixels) return DDGI_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(ref)) % 16 ||
        reinterpret_cast<uintptr_t>(out) % 8)
        return DDGI_ERR_INVALID_ARG;
    double* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return DDGI_ERR_CUDA;
    // every partial the second launch reads is written by the first one, so
    // nothing left by an earlier call needs clearing
    cudaError_t e = launch_metrics(reinterpret_cast<const float4*>(img),
                                   reinterpret_cast<const float4*>(ref), n, scratch, out,
                                   (cudaStream_t)stream);
    return e == cudaSuccess ? DDGI_OK : DDGI_ERR_CUDA;
}
