// Image error metrics of Sec. 4: mean squared error and mean absolute
// percentage error (epsilon 0.01) of a rendered radiance image against a
// reference, accumulated in fp64.  Two launches: per-block fp64 partial sums
// into a scratch array, then one block reduces the partials.
#include "internal.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block b accumulates pixels b, b + nblocks, ... (grid-stride over float4 records)
__global__ void __launch_bounds__(kThreads) k_metric_partials(const float4* __restrict__ img,
                                                              const float4* __restrict__ ref,
                                                              uint32_t n, double* __restrict__ part) {
    double se = 0.0, ape = 0.0;
    // 64-bit index: with a 32-bit one, i + stride wraps for n near 2^32 and
    // the loop would never end
    const size_t stride = (size_t)gridDim.x * kThreads;
    for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
        float4 a = img[i], b = ref[i];
        double d0 = (double)a.x - b.x, d1 = (double)a.y - b.y, d2 = (double)a.z - b.z;
        se += d0 * d0 + d1 * d1 + d2 * d2;
        ape += fabs(d0) / ((double)b.x + 0.01) + fabs(d1) / ((double)b.y + 0.01) +
               fabs(d2) / ((double)b.z + 0.01);
    }
    __shared__ double s_se[kThreads / 32], s_ape[kThreads / 32];
    se = warp_sum(se);
    ape = warp_sum(ape);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        s_se[w] = se;
        s_ape[w] = ape;
    }
    __syncthreads();
    if (w == 0) {
        se = l < kThreads / 32 ? s_se[l] : 0.0;
        ape = l < kThreads / 32 ? s_ape[l] : 0.0;
        se = warp_sum(se);
        ape = warp_sum(ape);
        if (l == 0) {
            part[2 * blockIdx.x] = se;
            part[2 * blockIdx.x + 1] = ape;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_metric_final(const double* __restrict__ part,
                                                           uint32_t nblocks, uint32_t n,
                                                           double* __restrict__ out) {
    double se = 0.0, ape = 0.0;
    for (uint32_t b = threadIdx.x; b < nblocks; b += kThreads) {
        se += part[2 * b];
        ape += part[2 * b + 1];
    }
    __shared__ double s_se[kThreads / 32], s_ape[kThreads / 32];
    se = warp_sum(se);
    ape = warp_sum(ape);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        s_se[w] = se;
        s_ape[w] = ape;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        se = 0.0;
        ape = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) {
            se += s_se[k];
            ape += s_ape[k];
        }
        double cnt = 3.0 * (double)n;
        out[0] = n ? se / cnt : 0.0;
        out[1] = n ? ape / cnt : 0.0;
    }
}

}  // namespace

uint32_t metric_blocks(uint32_t n) {
    uint32_t b = (n + 4 * kThreads - 1) / (4 * kThreads);
    return b < 1 ? 1 : (b > kMetricMaxBlocks ? kMetricMaxBlocks : b);
}

cudaError_t launch_metrics(const float4* img, const float4* ref, uint32_t n, double* scratch,
                           double* out, cudaStream_t st) {
    uint32_t nb = metric_blocks(n);
    k_metric_partials<<<nb, kThreads, 0, st>>>(img, ref, n, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_metric_final<<<1, kThreads, 0, st>>>(scratch, nb, n, out);
    return cudaGetLastError();
}

extern "C" ddgi_status ddgi_image_metrics(const float* img, const float* ref, uint32_t n,
                                          double* scratch, uint32_t scratch_doubles, double* out,
                                          void* stream) {
    if (!out || (n > 0 && (!img || !ref))) return DDGI_ERR_INVALID_ARG;
    if (!scratch || scratch_doubles < 2 * metric_blocks(n)) return DDGI_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(ref)) % 16 ||
        reinterpret_cast<uintptr_t>(scratch) % 8 || reinterpret_cast<uintptr_t>(out) % 8)
        return DDGI_ERR_INVALID_ARG;
    cudaError_t e = launch_metrics(reinterpret_cast<const float4*>(img),
                                   reinterpret_cast<const float4*>(ref), n, scratch, out,
                                   (cudaStream_t)stream);
    return e == cudaSuccess ? DDGI_OK : DDGI_ERR_CUDA;
}
