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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

#define MLP_IN 80
#define MLP_H 64
#define MLP_OUTP 8
#define MLP_NPARAM 18184
#define MLP_NW 17920
#define MLP_BATCH 16384u   // training samples per Adam step

__host__ __device__ constexpr int mlp_off_w(int l) {
    return l == 0 ? 0 : (l == 1 ? 5120 : (l == 2 ? 9216 : (l == 3 ? 13312 : 17408)));
}
__host__ __device__ constexpr int mlp_off_b(int l) { return 17920 + 64 * l; }
__host__ __device__ constexpr int mlp_in(int l) { return l == 0 ? 80 : 64; }

// device-side optimiser / judge state
struct MLPState {
    float loss_scale;      // gradients are computed for loss * loss_scale
    uint32_t overflow;     // last step saw a non-finite gradient (skipped)
    uint32_t good;         // steps since the last loss-scale change
    uint32_t count;        // training samples of the last Adam step
    double judge_mlp;      // held-out relative squared error of the network
    double judge_probe;    // ... and of the probe lookup
    uint32_t judge_n;      // held-out samples counted
    uint32_t use_mlp;      // 1: the network serves queries this frame
    uint32_t acc;          // training samples of the step in progress
    uint32_t done;         // optimiser CTAs finished (the last one resets it)
    uint32_t adam_t;       // Adam steps applied (a skipped step does not count)
};

struct MLPView {
    const uint16_t* w16;   // [MLP_NW] 16-bit weights (fp16 or bf16 bits), unpadded rows
    const float* params;   // [MLP_NPARAM] fp32 master (biases read from here)
    float lo[3];           // position normalisation p' = (p - lo) * scale
    float scale;
    uint32_t* err;         // device error word (bounded waits)
    int bf16;              // 1: weights and activations are bf16, else fp16
    int fp32;              // 1: fp32 CUDA-core debug form (params only; w16 unused)
};

// The network's 16-bit formats: fp16 (BF = false) or bf16 (BF = true), both
// with fp32 accumulation.  Values travel as raw 16-bit words.
template <bool BF>
struct H16;

template <>
struct H16<false> {
    static constexpr uint32_t umma_fmt = 0u;   // kind::f16 operand format code
    __device__ static __forceinline__ uint32_t pack(float a, float b) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
    __device__ static __forceinline__ uint16_t bits(float a) { return __half_as_ushort(__float2half_rn(a)); }
    __device__ static __forceinline__ float val(uint16_t b) { return __half2float(__ushort_as_half(b)); }
    // two fp32 -> packed pair with ReLU (negative values and -0 become +0)
    __device__ static __forceinline__ uint32_t relu2(uint32_t lo, uint32_t hi) {
        uint32_t r;
        asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(r) : "r"(hi), "r"(lo));
        return r;
    }
};

template <>
struct H16<true> {
    static constexpr uint32_t umma_fmt = 1u;
    __device__ static __forceinline__ uint32_t pack(float a, float b) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
    __device__ static __forceinline__ uint16_t bits(float a) { return __bfloat16_as_ushort(__float2bfloat16_rn(a)); }
    __device__ static __forceinline__ float val(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
    __device__ static __forceinline__ uint32_t relu2(uint32_t lo, uint32_t hi) {
        uint32_t r;
        asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "r"(hi), "r"(lo));
        return r;
    }
};

// ---------------------------------------------------------------------------
// inference on the 5th-generation tensor cores: Q::query(i, p, n) -> valid,
// Q::store(i, valid, rgb)
//
// One CTA per SM of 6 warpgroups; each warpgroup runs its own stream of
// 128-query tiles (thread = row), so that one stream's epilogue overlaps the
// others' MMAs.  Every layer is a K = 80 product: the activation tile keeps
// the layer-1 input in columns 64..79, whose column 75 is the constant 1, and
// each layer's weights carry its bias in column 75 and zeros in the other
// columns past its real inputs, so the tensor cores add the bias and the
// epilogue is a tensor-memory load, a ReLU-rounding conversion to fp16 and
// shared-memory stores.  Operands sit in shared memory in the canonical
// K-major layout without swizzle (core matrices of 8 rows x 16 bytes; the
// next 8 k at +128 B, the next 8 rows at +1280 B).  One thread per warpgroup
// issues tcgen05.mma (M = 128, N = 64 or 16, K = 16 per instruction, fp16 in,
// fp32 accumulate) into the warpgroup's 64 tensor-memory columns and commits
// to its mbarrier; the warpgroup's warps read their 32 rows back with
// tcgen05.ld.  Every wait is bounded: past the bound the warpgroup sets
// ERRBIT_MMA_WAIT, waits (bounded again) for the products it committed, and
// stops; the CTA then frees its tensor memory.
// ---------------------------------------------------------------------------
#define MLP_TC_WG 6                       // warpgroups (tile streams) per CTA
#define MLP_TC_THREADS (128 * MLP_TC_WG)
#define MLP_TC_COLS 512                   // tensor-memory columns per CTA: 64 per warpgroup (384 used)
#define MLP_TC_K 80
#define MLP_TC_WAIT_SPINS (1u << 22)

// shared-memory map (bytes): W1..W4 [64 x 80], W5 [16 x 80], activation
// tiles [128 x 80] per warpgroup, mbarriers
#define MLP_TC_W_OFF(l) (10240 * (l))        // W5 [16 x 80] = 2560 B ends at 43520
#define MLP_TC_A_OFF(g) (43520 + 20480 * (g))
#define MLP_TC_BAR_OFF (43520 + 20480 * MLP_TC_WG)
#define MLP_TC_SMEM (MLP_TC_BAR_OFF + 8 * MLP_TC_WG)
#define MLP_TC_ONE_COL 75                  // input column holding the constant 1

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) in a K-major no-swizzle tile with K = 80
__device__ __forceinline__ uint32_t kmajor_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1280 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: fp32 accumulator, A and B of the
// given format (0 fp16, 1 bf16) at bits 7 and 10, both K-major, N >> 3 at
// bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t umma_idesc_f16(int M, int N, uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < MLP_TC_WAIT_SPINS && !done; ++it)
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
    return done != 0;
}

// After a wait gave up: the products committed to `bar` may still be
// writing tensor memory, so wait for that commit once more, with a bound 16x
// the first, before the columns are freed.  Returns whether it arrived; if it
// did not, the error bit the caller sets is fatal for the context.
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
    for (int k = 0; k < 16; ++k)
        if (mbar_wait(bar, parity)) return true;
    return false;
}

// barrier of one warpgroup (ids 1..MLP_TC_WG; 0 is __syncthreads)
__device__ __forceinline__ void wg_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory"); }
__device__ __forceinline__ int wg_or(int g, int pred) {
    int r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.s32 p, %2, 0;\nbar.red.or.pred q, %1, 128, p;\nselp.s32 %0, 1, 0, q;\n}\n"
                 : "=r"(r)
                 : "r"(g + 1), "r"(pred)
                 : "memory");
    return r;
}


#define TMEM_LD_X16(taddr, v, o)                                                                          \
    asm volatile(                                                                                        \
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, " \
        "[%16];"                                                                                         \
        : "=r"(v[o + 0]), "=r"(v[o + 1]), "=r"(v[o + 2]), "=r"(v[o + 3]), "=r"(v[o + 4]), "=r"(v[o + 5]),  \
          "=r"(v[o + 6]), "=r"(v[o + 7]), "=r"(v[o + 8]), "=r"(v[o + 9]), "=r"(v[o + 10]), "=r"(v[o + 11]), \
          "=r"(v[o + 12]), "=r"(v[o + 13]), "=r"(v[o + 14]), "=r"(v[o + 15])                             \
        : "r"(taddr))

// weights of layer l as [rows][80] fp16 tiles in the canonical layout, copied
// in 16-byte chunks of the weight rows (8 inputs each): the real inputs, the
// bias (fp16) in input 75, zeros elsewhere.  The chunk of inputs 72..79 is
// rebuilt: layer 0 keeps its inputs 72..74 there, the hidden layers have none.
// W5 is padded to 16 rows; rows past a layer's outputs stay zero.
template <bool BF>
__device__ __forceinline__ void mlp_tc_load_weights(const MLPView& m, uint8_t* sm) {
    for (int e = threadIdx.x; e < 4 * 64 * 10 + 16 * 10; e += blockDim.x) {
        const int l = e < 2560 ? e / 640 : 4;
        const int rem = e < 2560 ? e - l * 640 : e - 2560;
        const int r = rem / 10, c = rem - r * 10;
        const int K = mlp_in(l), rows = l == 4 ? 3 : 64;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < rows) {
            if (8 * c < K) v = __ldg(reinterpret_cast<const uint4*>(m.w16 + mlp_off_w(l) + r * K + 8 * c));
            if (c == 9) {
                const uint32_t b = H16<BF>::bits(m.params[mlp_off_b(l) + r]);
                v.y = (l == 0 ? (v.y & 0xFFFFu) : 0u) | (b << 16);
                v.x = l == 0 ? v.x : 0u;
                v.z = 0u;
                v.w = 0u;
            }
        }
        *reinterpret_cast<uint4*>(sm + MLP_TC_W_OFF(l) + kmajor_off(r, 8 * c)) = v;
    }
}

// this thread's row of the layer-1 input: 12-frequency sin / cos of the
// normalised position (0..71), the normal (72..74), the constant 1 (75),
// zeros (76..79).  sin / cos(2^k pi x) is exact (sincospif) for k = 0, 4, 8
// and doubled for the three frequencies after each (sin 2a = 2 sin a cos a,
// cos 2a = (cos a - sin a)(cos a + sin a)): a few ulp of fp32, far below the
// fp16 rounding of the features.
template <bool BF>
__device__ __forceinline__ void mlp_tc_encode_row(uint8_t* sA, int r, const float (&q)[6]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        uint32_t w[12];
#pragma unroll
        for (int k0 = 0; k0 < 12; k0 += 4) {
            float sn, cs;
            sincospif(q[a] * (float)(1 << k0), &sn, &cs);
            w[k0] = H16<BF>::pack(sn, cs);
#pragma unroll
            for (int d = 1; d < 4; ++d) {
                const float s2 = 2.f * sn * cs, c2 = (cs - sn) * (cs + sn);
                sn = s2;
                cs = c2;
                w[k0 + d] = H16<BF>::pack(sn, cs);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
            *reinterpret_cast<uint4*>(sA + kmajor_off(r, 24 * a + 8 * c)) =
                make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
    }
    *reinterpret_cast<uint4*>(sA + kmajor_off(r, 72)) =
        make_uint4(H16<BF>::pack(q[3], q[4]), H16<BF>::pack(q[5], 1.f), 0u, 0u);
}

template <class Q, bool BF>
__global__ void __launch_bounds__(MLP_TC_THREADS, 1) k_mlp_infer(MLPView m, Q q, uint32_t n) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint32_t s_taddr;
    const int t = threadIdx.x & 127, g = threadIdx.x >> 7, w = threadIdx.x >> 5;
    uint8_t* sA = sm + MLP_TC_A_OFF(g);
    const uint32_t bar = smem_u32(sm + MLP_TC_BAR_OFF + 8 * g);
    mlp_tc_load_weights<BF>(m, sm);
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(MLP_TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tacc = s_taddr + 64u * (uint32_t)g;                 // this warpgroup's columns
    const uint32_t trow = tacc + ((uint32_t)(32 * (w & 3)) << 16);     // this warp's 32 lanes
    const uint32_t a_addr = smem_u32(sA), w_addr = smem_u32(sm);
    uint32_t phase = 0;
    bool failed = false;
    const uint32_t ntiles = (n + 127) / 128, streams = gridDim.x * MLP_TC_WG;
    // the query of a tile is fetched while the previous tile's first layer
    // runs on the tensor cores
    uint32_t tile = blockIdx.x * MLP_TC_WG + g;
    f3 p = {0.f, 0.f, 0.f}, nr = {0.f, 0.f, 1.f};
    bool valid = false;
    if (tile < ntiles) {
        const uint32_t i = tile * 128 + t;
        valid = i < n && q.query(i, p, nr);
    }
    for (; tile < ntiles; tile += streams) {
        const uint32_t i = tile * 128 + t;
        const bool vcur = valid;
        {
            const float qv[6] = {(p.x - m.lo[0]) * m.scale, (p.y - m.lo[1]) * m.scale,
                                 (p.z - m.lo[2]) * m.scale, nr.x, nr.y, nr.z};
            mlp_tc_encode_row<BF>(sA, t, qv);
        }
        f3 out = {0.f, 0.f, 0.f};
#pragma unroll 1
        for (int l = 0; l < 5; ++l) {
            // the layer input is in shared memory for the tensor cores
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            wg_sync(g);
            if (t == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t idesc =
                    l == 4 ? umma_idesc_f16(128, 16, H16<BF>::umma_fmt) : umma_idesc_f16(128, 64, H16<BF>::umma_fmt);
                const uint32_t wl = w_addr + (uint32_t)MLP_TC_W_OFF(l);
#pragma unroll
                for (int s = 0; s < MLP_TC_K / 16; ++s)
                    umma_f16(tacc, umma_sdesc(a_addr + 256u * s, 128u, 1280u), umma_sdesc(wl + 256u * s, 128u, 1280u),
                             idesc, s > 0 ? 1u : 0u);
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                             : "memory");
            }
            if (l == 0) {
                const uint32_t nt = tile + streams;
                valid = false;
                p = {0.f, 0.f, 0.f};
                nr = {0.f, 0.f, 1.f};
                if (nt < ntiles) {
                    const uint32_t ni = nt * 128 + t;
                    valid = ni < n && q.query(ni, p, nr);
                }
            }
            const bool ok = mbar_wait(bar, phase);
            if (wg_or(g, !ok)) {
                mbar_drain(bar, phase);
                failed = true;
                break;
            }
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (l < 4) {
#pragma unroll
                for (int c2 = 0; c2 < 4; ++c2) {
                    uint32_t v[16];
                    TMEM_LD_X16(trow + 16u * c2, v, 0);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        *reinterpret_cast<uint4*>(sA + kmajor_off(t, 16 * c2 + 8 * h)) =
                            make_uint4(H16<BF>::relu2(v[8 * h], v[8 * h + 1]), H16<BF>::relu2(v[8 * h + 2], v[8 * h + 3]),
                                       H16<BF>::relu2(v[8 * h + 4], v[8 * h + 5]),
                                       H16<BF>::relu2(v[8 * h + 6], v[8 * h + 7]));
                }
            } else {
                uint32_t v[16];
                TMEM_LD_X16(trow, v, 0);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                out = {__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2])};
            }
        }
        if (failed) break;
        if (i < n) q.store(i, vcur, out);
    }
    if (failed && t == 0) atomicOr(m.err, ERRBIT_MMA_WAIT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_taddr), "r"(MLP_TC_COLS));
}

// Launches k_mlp_infer over n queries: one persistent CTA per SM (6 tile
// streams, 384 of the SM's 512 tensor-memory columns).
template <class Q, bool BF>
cudaError_t launch_mlp_infer_t(const MLPView& m, const Q& q, uint32_t n, cudaStream_t st) {
    static int sms = 0;
    if (!sms) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_infer<Q, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)MLP_TC_SMEM);
        if (e != cudaSuccess) return e;
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const uint32_t tiles = (n + 127) / 128;
    const uint32_t need = (tiles + MLP_TC_WG - 1) / MLP_TC_WG;
    const uint32_t grid = need < (uint32_t)sms ? need : (uint32_t)sms;
    k_mlp_infer<Q, BF><<<grid, MLP_TC_THREADS, MLP_TC_SMEM, st>>>(m, q, n);
    return cudaGetLastError();
}

#include "mlp_f32.cuh"

// Launches k_mlp_infer over n queries in the network's format: one
// persistent CTA per SM (6 tile streams, 384 of the SM's 512 tensor-memory
// columns); or the fp32 debug form when the view asks for it.
template <class Q>
cudaError_t launch_mlp_infer(const MLPView& m, const Q& q, uint32_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (m.fp32) return launch_mlp_infer_f32<Q>(m, q, n, st);
    return m.bf16 ? launch_mlp_infer_t<Q, true>(m, q, n, st) : launch_mlp_infer_t<Q, false>(m, q, n, st);
}
