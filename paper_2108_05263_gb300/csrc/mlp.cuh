// Learned target form: a 80-64-64-64-64-3 MLP evaluated with warp-level
// tensor-core MMAs (m16n8k16, fp16 operands, fp32 accumulation).
//
// Parameter layout (fp32 master, gradients and Adam moments share it; the
// fp16 copy holds the weights only):
//   W1 [64][80] @0, W2 [64][64] @5120, W3 @9216, W4 @13312, W5 [8][64] @17408
//   (rows 3..7 of W5 stay 0), b1..b4 [64] @17920.., b5 [8] @18176; 18184 floats.
// Shared-memory weights use padded row strides (88 / 72 halves) so that the
// fragment loads of a warp hit distinct banks.
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"

#define MLP_IN 80
#define MLP_H 64
#define MLP_OUTP 8
#define MLP_NPARAM 18184
#define MLP_NW 17920
#define MLP_BATCH 16384u   // training samples per Adam step
#define MLP_LD_IN 88
#define MLP_LD_H 72
#define MLP_SW_HALVES (64 * 88 + 3 * 64 * 72 + 8 * 72)   // 20032

__host__ __device__ constexpr int mlp_off_w(int l) {
    return l == 0 ? 0 : (l == 1 ? 5120 : (l == 2 ? 9216 : (l == 3 ? 13312 : 17408)));
}
__host__ __device__ constexpr int mlp_off_b(int l) { return 17920 + 64 * l; }
__host__ __device__ constexpr int mlp_in(int l) { return l == 0 ? 80 : 64; }
__host__ __device__ constexpr int mlp_out(int l) { return l == 4 ? 8 : 64; }
__host__ __device__ constexpr int mlp_ld(int l) { return l == 0 ? MLP_LD_IN : MLP_LD_H; }
__host__ __device__ constexpr int mlp_soff(int l) {
    return l == 0 ? 0 : (l == 1 ? 5632 : (l == 2 ? 10240 : (l == 3 ? 14848 : 19456)));
}

// device-side optimiser / judge state
struct MLPState {
    float loss_scale;      // gradients are computed for loss * loss_scale
    uint32_t overflow;     // last step saw a non-finite gradient (skipped)
    uint32_t good;         // steps since the last loss-scale change
    uint32_t count;        // training samples of the current step
    double judge_mlp;      // held-out relative squared error of the network
    double judge_probe;    // ... and of the probe lookup
    uint32_t judge_n;      // held-out samples counted
    uint32_t use_mlp;      // 1: the network serves queries this frame
};

struct MLPView {
    const __half* w16;     // [MLP_NW] fp16 weights, unpadded rows
    const float* params;   // [MLP_NPARAM] fp32 master (biases read from here)
    float lo[3];           // position normalisation p' = (p - lo) * scale
    float scale;
};

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ uint32_t h2_from(__half a, __half b) {
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Copy the fp16 weights into padded shared rows and the biases (fp32).
__device__ __forceinline__ void mlp_load_smem(const MLPView& m, __half* sW, float* sb) {
    for (int e = threadIdx.x; e < MLP_NW; e += blockDim.x) {
        int l = e < 5120 ? 0 : (e < 9216 ? 1 : (e < 13312 ? 2 : (e < 17408 ? 3 : 4)));
        int r = e - mlp_off_w(l);
        int in = mlp_in(l);
        int o = r / in, i = r - o * in;
        sW[mlp_soff(l) + o * mlp_ld(l) + i] = m.w16[e];
    }
    for (int e = threadIdx.x; e < 264; e += blockDim.x) sb[e] = m.params[17920 + e];
}

// feature pair (c, c+1) of the input encoding (c even): sin / cos of
// 2^k pi p'_a for c < 72, the normal for c = 72, 74, zeros beyond
__device__ __forceinline__ uint32_t feature_pair(const float* q, int c) {
    if (c < 72) {
        int a = c / 24, k = (c % 24) >> 1;
        float sn, cs;
        sincospif(ldexpf(q[a], k), &sn, &cs);
        return pack_h2(sn, cs);
    }
    if (c == 72) return pack_h2(q[3], q[4]);
    if (c == 74) return pack_h2(q[5], 0.f);
    return 0u;
}

// A fragments of the encoded inputs of a warp's 32 samples (2 m-tiles);
// sq: per-sample (p'.xyz, n.xyz, valid, 0) rows of 8 floats.
__device__ __forceinline__ void mlp_input_frags(const float* sq, uint32_t (&a)[2][5][4], int g, int t) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const float* q0 = sq + (mt * 16 + g) * 8;
        const float* q1 = sq + (mt * 16 + g + 8) * 8;
#pragma unroll
        for (int kt = 0; kt < 5; ++kt) {
            int c = kt * 16 + 2 * t;
            a[mt][kt][0] = feature_pair(q0, c);
            a[mt][kt][1] = feature_pair(q1, c);
            a[mt][kt][2] = feature_pair(q0, c + 8);
            a[mt][kt][3] = feature_pair(q1, c + 8);
        }
    }
}

// acc = bias + A x W^T for one layer (KT k-tiles of the input, NT n-tiles of
// the output), W in shared memory [out][ld] fp16
template <int KT, int NT>
__device__ __forceinline__ void mlp_layer(const __half* __restrict__ sW, int ld, const float* __restrict__ sb,
                                          const uint32_t (&a)[2][KT][4], float (&acc)[2][NT][4], int g, int t) {
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        float b0 = sb[nt * 8 + 2 * t], b1 = sb[nt * 8 + 2 * t + 1];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            acc[mt][nt][0] = b0;
            acc[mt][nt][1] = b1;
            acc[mt][nt][2] = b0;
            acc[mt][nt][3] = b1;
        }
    }
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const __half* w = sW + (nt * 8 + g) * ld + kt * 16 + 2 * t;
            uint32_t b0 = *reinterpret_cast<const uint32_t*>(w);
            uint32_t b1 = *reinterpret_cast<const uint32_t*>(w + 8);
            mma16816(acc[0][nt], a[0][kt], b0, b1);
            mma16816(acc[1][nt], a[1][kt], b0, b1);
        }
    }
}

// ReLU and conversion of an output (D) fragment set into the A fragments of
// the next layer: output n-tiles 2k and 2k+1 form input k-tile k.
template <int NT>
__device__ __forceinline__ void relu_to_frags(const float (&acc)[2][NT][4], uint32_t (&a)[2][NT / 2][4]) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int k = 0; k < NT / 2; ++k) {
            const float* lo = acc[mt][2 * k];
            const float* hi = acc[mt][2 * k + 1];
            a[mt][k][0] = pack_h2(fmaxf(lo[0], 0.f), fmaxf(lo[1], 0.f));
            a[mt][k][1] = pack_h2(fmaxf(lo[2], 0.f), fmaxf(lo[3], 0.f));
            a[mt][k][2] = pack_h2(fmaxf(hi[0], 0.f), fmaxf(hi[1], 0.f));
            a[mt][k][3] = pack_h2(fmaxf(hi[2], 0.f), fmaxf(hi[3], 0.f));
        }
}

// Full forward pass of a warp's 32 samples; out: acc of the output layer
// (rows g / g+8 of each m-tile, columns 2t, 2t+1 of 8).
__device__ __forceinline__ void mlp_forward(const __half* sW, const float* sb, const float* sq,
                                            float (&out)[2][1][4], int g, int t) {
    uint32_t a0[2][5][4];
    mlp_input_frags(sq, a0, g, t);
    float acc[2][8][4];
    uint32_t a[2][4][4];
    mlp_layer<5, 8>(sW + mlp_soff(0), MLP_LD_IN, sb, a0, acc, g, t);
    relu_to_frags<8>(acc, a);
#pragma unroll
    for (int l = 1; l < 4; ++l) {
        mlp_layer<4, 8>(sW + mlp_soff(l), MLP_LD_H, sb + 64 * l, a, acc, g, t);
        relu_to_frags<8>(acc, a);
    }
    mlp_layer<4, 1>(sW + mlp_soff(4), MLP_LD_H, sb + 256, a, out, g, t);
}

#define MLP_INFER_THREADS 128

// ---------------------------------------------------------------------------
// inference: Q::query(i, p, n) -> valid, Q::store(i, valid, rgb)
// ---------------------------------------------------------------------------
inline size_t mlp_infer_smem() { return MLP_SW_HALVES * 2 + 264 * 4 + 4 * 32 * 8 * 4 + 4 * 32 * 4 * 4; }

template <class Q>
__global__ void __launch_bounds__(MLP_INFER_THREADS) k_mlp_infer(MLPView m, Q q, uint32_t n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __half* sW = reinterpret_cast<__half*>(smem_raw);
    float* sb = reinterpret_cast<float*>(sW + MLP_SW_HALVES);
    float* sq_all = sb + 264;
    float* so_all = sq_all + 4 * 32 * 8;
    mlp_load_smem(m, sW, sb);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float* sq = sq_all + warp * 256;
    float* so = so_all + warp * 128;
    for (uint32_t base = blockIdx.x * MLP_INFER_THREADS; base < n; base += gridDim.x * MLP_INFER_THREADS) {
        const uint32_t i = base + warp * 32 + lane;
        f3 p = {0.f, 0.f, 0.f}, nr = {0.f, 0.f, 1.f};
        bool valid = i < n && q.query(i, p, nr);
        float* r = sq + lane * 8;
        r[0] = (p.x - m.lo[0]) * m.scale;
        r[1] = (p.y - m.lo[1]) * m.scale;
        r[2] = (p.z - m.lo[2]) * m.scale;
        r[3] = nr.x;
        r[4] = nr.y;
        r[5] = nr.z;
        __syncwarp();
        float out[2][1][4];
        mlp_forward(sW, sb, sq, out, g, t);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            int r0 = mt * 16 + g, r1 = r0 + 8;
            if (2 * t < 3) {
                so[r0 * 4 + 2 * t] = out[mt][0][0];
                so[r1 * 4 + 2 * t] = out[mt][0][2];
            }
            if (2 * t + 1 < 3) {
                so[r0 * 4 + 2 * t + 1] = out[mt][0][1];
                so[r1 * 4 + 2 * t + 1] = out[mt][0][3];
            }
        }
        __syncwarp();
        if (i < n) q.store(i, valid, f3{so[lane * 4], so[lane * 4 + 1], so[lane * 4 + 2]});
        __syncwarp();
    }
}


// Launches k_mlp_infer over n queries (a few blocks per SM, grid-stride).
template <class Q>
cudaError_t launch_mlp_infer(const MLPView& m, const Q& q, uint32_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_infer<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)mlp_infer_smem());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    uint32_t tiles = (n + MLP_INFER_THREADS - 1) / MLP_INFER_THREADS;
    uint32_t grid = tiles < 1216u ? tiles : 1216u;
    k_mlp_infer<Q><<<grid, MLP_INFER_THREADS, mlp_infer_smem(), st>>>(m, q, n);
    return cudaGetLastError();
}
