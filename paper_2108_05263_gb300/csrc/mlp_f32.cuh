// fp32 debug form of the learned target's network: the same 80-64-64-64-64-3
// MLP as the tensor-core kernels, evaluated on the CUDA cores in fp32 (fp32
// weights straight from the parameter array, fp32 activations, fp32
// accumulation), one thread per query.  It exists to check the network's
// gradients entry by entry against the fp64 oracle; the tensor-core kernels
// stay the product path.
#pragma once
#include "common.cuh"

#define MLP_F32_THREADS 128
#define MLP_F32_SMEM (MLP_NPARAM * 4)

// input row: sin / cos(2^k pi p'_a) for k = 0..11 and the three axes
// (axis-major, then frequency, then sin / cos), the normal, 5 zeros
__device__ __forceinline__ void mlp_f32_encode(const MLPView& m, f3 p, f3 n, float (&x)[MLP_IN]) {
    const float q[3] = {(p.x - m.lo[0]) * m.scale, (p.y - m.lo[1]) * m.scale, (p.z - m.lo[2]) * m.scale};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float sn, cs;
            sincospif(q[a] * (float)(1 << k), &sn, &cs);   // the product is exact (a power of two)
            x[24 * a + 2 * k] = sn;
            x[24 * a + 2 * k + 1] = cs;
        }
    x[72] = n.x;
    x[73] = n.y;
    x[74] = n.z;
#pragma unroll
    for (int i = 75; i < MLP_IN; ++i) x[i] = 0.f;
}

// one dense layer out = W in + b (ReLU unless it is the output layer), with
// W [outs][ins] row-major and b from the shared-memory parameter copy
template <int INS, int OUTS, bool RELU>
__device__ __forceinline__ void mlp_f32_layer(const float* __restrict__ sw, int l, const float* in, float* out) {
    const float* W = sw + mlp_off_w(l);
    const float* b = sw + mlp_off_b(l);
#pragma unroll 1
    for (int o = 0; o < OUTS; ++o) {
        float acc = b[o];
#pragma unroll 8
        for (int i = 0; i < INS; ++i) acc = fmaf(W[o * INS + i], in[i], acc);
        out[o] = RELU ? fmaxf(acc, 0.f) : acc;
    }
}

template <class Q>
__global__ void __launch_bounds__(MLP_F32_THREADS) k_mlp_infer_f32(MLPView m, Q q, uint32_t n) {
    extern __shared__ float sw[];
    for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) sw[i] = m.params[i];
    __syncthreads();
    const uint32_t i = blockIdx.x * MLP_F32_THREADS + threadIdx.x;
    if (i >= n) return;
    f3 p = {0.f, 0.f, 0.f}, nr = {0.f, 0.f, 1.f};
    const bool valid = q.query(i, p, nr);
    float x[MLP_IN], h[MLP_H], g[MLP_H], out[3];
    mlp_f32_encode(m, p, nr, x);
    mlp_f32_layer<MLP_IN, MLP_H, true>(sw, 0, x, h);
    mlp_f32_layer<MLP_H, MLP_H, true>(sw, 1, h, g);
    mlp_f32_layer<MLP_H, MLP_H, true>(sw, 2, g, h);
    mlp_f32_layer<MLP_H, MLP_H, true>(sw, 3, h, g);
    mlp_f32_layer<MLP_H, 3, false>(sw, 4, g, out);
    q.store(i, valid, f3{out[0], out[1], out[2]});
}

template <class Q>
cudaError_t launch_mlp_infer_f32(const MLPView& m, const Q& q, uint32_t n, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_infer_f32<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             MLP_F32_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_mlp_infer_f32<Q><<<(n + MLP_F32_THREADS - 1) / MLP_F32_THREADS, MLP_F32_THREADS, MLP_F32_SMEM, st>>>(m, q, n);
    return cudaGetLastError();
}
