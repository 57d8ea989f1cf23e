// Learned target form (the neural cache the paper names as interchangeable
// with the probes, Sec. 2 / Sec. 5): batched tensor-core inference, a fused
// forward + backward training step with fp32 gradient accumulation and
// dynamic loss scaling, Adam, and the generation of self-training samples
// from probe-origin rays with one cosine bounce.
#include "internal.h"
#include "mlp.cuh"
#include "trace_engine.cuh"

namespace {

// caller-provided queries: [n][8] floats (p.xyz, valid, n.xyz, 0) -> [n][4] (f.rgb, valid)
struct BufferQuery {
    const float4* in;
    float4* out;
    __device__ bool query(uint32_t i, f3& p, f3& n) const {
        float4 a = in[2 * i], b = in[2 * i + 1];
        p = xyz(a);
        n = xyz(b);
        return a.w != 0.f;
    }
    __device__ void store(uint32_t i, bool valid, f3 f) const {
        out[i] = make_float4(f.x, f.y, f.z, valid ? 1.f : 0.f);
    }
};

// ---------------------------------------------------------------------------
// training: fused forward + backward over tiles of 128 samples
// ---------------------------------------------------------------------------
constexpr int kTrainRows = 128;
constexpr int kLdD5 = 24;

size_t train_smem() {
    return MLP_SW_HALVES * 2 + 264 * 4 + kTrainRows * MLP_LD_IN * 2 + 4 * kTrainRows * MLP_LD_H * 2 +
           kTrainRows * MLP_LD_H * 2 + kTrainRows * kLdD5 * 2 + kTrainRows * 8 * 4 + kTrainRows * 4 * 4;
}

template <int KT>
__device__ __forceinline__ void store_frags(uint16_t* s, int ld, int rowbase, const uint32_t (&a)[2][KT][4],
                                            int g, int t) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        int r0 = rowbase + mt * 16 + g, r1 = r0 + 8;
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
            int c = kt * 16 + 2 * t;
            *reinterpret_cast<uint32_t*>(s + r0 * ld + c) = a[mt][kt][0];
            *reinterpret_cast<uint32_t*>(s + r1 * ld + c) = a[mt][kt][1];
            *reinterpret_cast<uint32_t*>(s + r0 * ld + c + 8) = a[mt][kt][2];
            *reinterpret_cast<uint32_t*>(s + r1 * ld + c + 8) = a[mt][kt][3];
        }
    }
}

// acc[m = samples][n = layer input] = d[m][k = layer output] x W[k][n];
// W in shared memory [out][ld]; rows >= OUT_ROWS read as 0
template <bool BF, int KT, int NT, int OUT_ROWS>
__device__ __forceinline__ void bwd_data(const uint16_t* __restrict__ sW, int ld, const uint32_t (&d)[2][KT][4],
                                         float (&acc)[2][NT][4], int g, int t) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.f;
    const uint16_t z = 0;
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
        const int k0 = kt * 16 + 2 * t;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int col = nt * 8 + g;
            uint16_t w0 = k0 < OUT_ROWS ? sW[k0 * ld + col] : z;
            uint16_t w1 = k0 + 1 < OUT_ROWS ? sW[(k0 + 1) * ld + col] : z;
            uint16_t w2 = k0 + 8 < OUT_ROWS ? sW[(k0 + 8) * ld + col] : z;
            uint16_t w3 = k0 + 9 < OUT_ROWS ? sW[(k0 + 9) * ld + col] : z;
            uint32_t b0 = h2_from(w0, w1), b1 = h2_from(w2, w3);
            H16<BF>::mma(acc[0][nt], d[0][kt], b0, b1);
            H16<BF>::mma(acc[1][nt], d[1][kt], b0, b1);
        }
    }
}

// ReLU derivative from the stored activations of the layer input, then the
// masked deltas as A fragments (k-tiles of 16 outputs) and into sD
template <bool BF, int NT>
__device__ __forceinline__ void mask_delta(const float (&acc)[2][NT][4], const uint16_t* sAct, int ld_act,
                                           uint16_t* sD, int ld_d, int rowbase, uint32_t (&d)[2][NT / 2][4],
                                           int g, int t) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        int r0 = rowbase + mt * 16 + g, r1 = r0 + 8;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            int c = nt * 8 + 2 * t;
            const uint16_t* a0 = sAct + r0 * ld_act + c;
            const uint16_t* a1 = sAct + r1 * ld_act + c;
            float v0 = H16<BF>::val(a0[0]) > 0.f ? acc[mt][nt][0] : 0.f;
            float v1 = H16<BF>::val(a0[1]) > 0.f ? acc[mt][nt][1] : 0.f;
            float v2 = H16<BF>::val(a1[0]) > 0.f ? acc[mt][nt][2] : 0.f;
            float v3 = H16<BF>::val(a1[1]) > 0.f ? acc[mt][nt][3] : 0.f;
            uint32_t p0 = H16<BF>::pack(v0, v1), p1 = H16<BF>::pack(v2, v3);
            *reinterpret_cast<uint32_t*>(sD + r0 * ld_d + c) = p0;
            *reinterpret_cast<uint32_t*>(sD + r1 * ld_d + c) = p1;
            d[mt][nt >> 1][(nt & 1) ? 2 : 0] = p0;
            d[mt][nt >> 1][(nt & 1) ? 3 : 1] = p1;
        }
    }
}

// weight gradient of one 16-row output tile: grad[o][i] += sum_s D[s][o] * A[s][i]
// over the 128 samples of the block (8 k-tiles)
template <bool BF, int NT>
__device__ __forceinline__ void wgrad_tile(const uint16_t* sD, int ld_d, int o0, int out_real, const uint16_t* sA,
                                           int ld_a, int in, float* grad_w, int g, int t) {
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll 2
    for (int kt = 0; kt < kTrainRows / 16; ++kt) {
        const int s0 = kt * 16 + 2 * t;
        uint32_t a[4];
        a[0] = h2_from(sD[s0 * ld_d + o0 + g], sD[(s0 + 1) * ld_d + o0 + g]);
        a[1] = h2_from(sD[s0 * ld_d + o0 + g + 8], sD[(s0 + 1) * ld_d + o0 + g + 8]);
        a[2] = h2_from(sD[(s0 + 8) * ld_d + o0 + g], sD[(s0 + 9) * ld_d + o0 + g]);
        a[3] = h2_from(sD[(s0 + 8) * ld_d + o0 + g + 8], sD[(s0 + 9) * ld_d + o0 + g + 8]);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int col = nt * 8 + g;
            uint32_t b0 = h2_from(sA[s0 * ld_a + col], sA[(s0 + 1) * ld_a + col]);
            uint32_t b1 = h2_from(sA[(s0 + 8) * ld_a + col], sA[(s0 + 9) * ld_a + col]);
            H16<BF>::mma(acc[nt], a, b0, b1);
        }
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        int i = nt * 8 + 2 * t;
        int r0 = o0 + g, r1 = o0 + g + 8;
        if (r0 < out_real) {
            atomicAdd(grad_w + r0 * in + i, acc[nt][0]);
            atomicAdd(grad_w + r0 * in + i + 1, acc[nt][1]);
        }
        if (r1 < out_real) {
            atomicAdd(grad_w + r1 * in + i, acc[nt][2]);
            atomicAdd(grad_w + r1 * in + i + 1, acc[nt][3]);
        }
    }
}

// bias gradient: column sums of the deltas; thread (o, part) sums the rows
// part, part + P, ... of output o, P = blockDim / 64 partial sums per output
template <bool BF>
__device__ __forceinline__ void bias_grad(const uint16_t* sD, int ld_d, int out_real, float* grad_b) {
    const int o = threadIdx.x & 63, part = threadIdx.x >> 6, P = blockDim.x >> 6;
    if (o >= out_real) return;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int r = part;
    for (; r + 3 * P < kTrainRows; r += 4 * P) {
        s0 += H16<BF>::val(sD[r * ld_d + o]);
        s1 += H16<BF>::val(sD[(r + P) * ld_d + o]);
        s2 += H16<BF>::val(sD[(r + 2 * P) * ld_d + o]);
        s3 += H16<BF>::val(sD[(r + 3 * P) * ld_d + o]);
    }
    for (; r < kTrainRows; r += P) s0 += H16<BF>::val(sD[r * ld_d + o]);
    atomicAdd(grad_b + o, (s0 + s1) + (s2 + s3));
}

// samples [n][3] float4: (y.xyz, _), (n.xyz, _), (target.rgb, weight); weight 0
// excludes a sample.  Gradients of sum_s w_s sum_c (f - t)^2 / (sg(f)^2 + 0.01)
// times the loss scale are added to grad; the weights are summed into
// st->count.
template <bool BF>
__global__ void __launch_bounds__(kTrainRows, 1) k_mlp_train(MLPView m, const float4* __restrict__ smp,
                                                            uint32_t n, MLPState* __restrict__ st,
                                                            float* __restrict__ grad) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t* sW = reinterpret_cast<uint16_t*>(smem_raw);
    float* sb = reinterpret_cast<float*>(sW + MLP_SW_HALVES);
    uint16_t* sA0 = reinterpret_cast<uint16_t*>(sb + 264);
    uint16_t* sA[5];
    sA[0] = sA0;
    sA[1] = sA0 + kTrainRows * MLP_LD_IN;
    for (int l = 2; l < 5; ++l) sA[l] = sA[l - 1] + kTrainRows * MLP_LD_H;
    uint16_t* sD = sA[4] + kTrainRows * MLP_LD_H;
    uint16_t* sD5 = sD + kTrainRows * MLP_LD_H;
    float* sq_all = reinterpret_cast<float*>(sD5 + kTrainRows * kLdD5);
    float* st_all = sq_all + kTrainRows * 8;

    mlp_load_smem(m, sW, sb);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int rowbase = warp * 32;
    const uint32_t s = blockIdx.x * kTrainRows + threadIdx.x;
    {
        float4 y = s < n ? smp[3 * (size_t)s] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 nn = s < n ? smp[3 * (size_t)s + 1] : make_float4(0.f, 0.f, 1.f, 0.f);
        float4 tg = s < n ? smp[3 * (size_t)s + 2] : make_float4(0.f, 0.f, 0.f, 0.f);
        unsigned cnt = __ballot_sync(0xffffffffu, tg.w > 0.f);
        if (lane == 0 && cnt) atomicAdd(&st->count, (unsigned)__popc(cnt));
        float* r = sq_all + threadIdx.x * 8;
        r[0] = (y.x - m.lo[0]) * m.scale;
        r[1] = (y.y - m.lo[1]) * m.scale;
        r[2] = (y.z - m.lo[2]) * m.scale;
        r[3] = nn.x;
        r[4] = nn.y;
        r[5] = nn.z;
        float* q = st_all + threadIdx.x * 4;
        q[0] = tg.x;
        q[1] = tg.y;
        q[2] = tg.z;
        q[3] = tg.w;
    }
    __syncthreads();
    const float* sq = sq_all + rowbase * 8;

    // ---- forward, keeping every layer input in shared memory ------------------
    float out[2][1][4];
    {
        uint32_t a0[2][5][4];
        mlp_input_frags<BF>(sq, a0, g, t);
        store_frags<5>(sA[0], MLP_LD_IN, rowbase, a0, g, t);
        float acc[2][8][4];
        uint32_t a[2][4][4];
        mlp_layer<BF, 5, 8>(sW + mlp_soff(0), MLP_LD_IN, sb, a0, acc, g, t);
        relu_to_frags<BF, 8>(acc, a);
        store_frags<4>(sA[1], MLP_LD_H, rowbase, a, g, t);
#pragma unroll
        for (int l = 1; l < 4; ++l) {
            mlp_layer<BF, 4, 8>(sW + mlp_soff(l), MLP_LD_H, sb + 64 * l, a, acc, g, t);
            relu_to_frags<BF, 8>(acc, a);
            store_frags<4>(sA[l + 1], MLP_LD_H, rowbase, a, g, t);
        }
        mlp_layer<BF, 4, 1>(sW + mlp_soff(4), MLP_LD_H, sb + 256, a, out, g, t);
    }

    // ---- output gradient (relative L2, denominator held constant) -------------
    const float S = st->loss_scale;
    uint32_t d5[2][1][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        int r0 = rowbase + mt * 16 + g, r1 = r0 + 8;
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int row = e < 2 ? r0 : r1;
            int col = 2 * t + (e & 1);
            float f = out[mt][0][e];
            const float* q = st_all + row * 4;
            v[e] = col < 3 ? q[3] * S * 2.f * (f - q[col]) / (f * f + 0.01f) : 0.f;
        }
        d5[mt][0][0] = H16<BF>::pack(v[0], v[1]);
        d5[mt][0][1] = H16<BF>::pack(v[2], v[3]);
        d5[mt][0][2] = 0u;
        d5[mt][0][3] = 0u;
        *reinterpret_cast<uint32_t*>(sD5 + r0 * kLdD5 + 2 * t) = d5[mt][0][0];
        *reinterpret_cast<uint32_t*>(sD5 + r1 * kLdD5 + 2 * t) = d5[mt][0][1];
        *reinterpret_cast<uint32_t*>(sD5 + r0 * kLdD5 + 8 + 2 * t) = 0u;
        *reinterpret_cast<uint32_t*>(sD5 + r1 * kLdD5 + 8 + 2 * t) = 0u;
    }
    __syncthreads();
    // output layer: M = 16 (3 real rows), N = 64, split over the 4 warps
    if (warp == 0) wgrad_tile<BF, 8>(sD5, kLdD5, 0, 3, sA[4], MLP_LD_H, 64, grad + mlp_off_w(4), g, t);
    bias_grad<BF>(sD5, kLdD5, 3, grad + mlp_off_b(4));

    // ---- hidden layers, last to first -----------------------------------------
    uint32_t d[2][4][4];
    {
        float acc[2][8][4];
        bwd_data<BF, 1, 8, 8>(sW + mlp_soff(4), MLP_LD_H, d5, acc, g, t);
        __syncthreads();
        mask_delta<BF, 8>(acc, sA[4], MLP_LD_H, sD, MLP_LD_H, rowbase, d, g, t);
    }
    for (int l = 3; l >= 0; --l) {
        __syncthreads();
        // gradient of layer l (input sA[l], output deltas in sD)
        if (l == 0)
            wgrad_tile<BF, 10>(sD, MLP_LD_H, warp * 16, 64, sA[0], MLP_LD_IN, 80, grad + mlp_off_w(0), g, t);
        else
            wgrad_tile<BF, 8>(sD, MLP_LD_H, warp * 16, 64, sA[l], MLP_LD_H, 64, grad + mlp_off_w(l), g, t);
        bias_grad<BF>(sD, MLP_LD_H, 64, grad + mlp_off_b(l));
        if (l == 0) break;
        float acc[2][8][4];
        bwd_data<BF, 4, 8, 64>(sW + mlp_soff(l), MLP_LD_H, d, acc, g, t);
        __syncthreads();
        mask_delta<BF, 8>(acc, sA[l], MLP_LD_H, sD, MLP_LD_H, rowbase, d, g, t);
    }
}

// ---------------------------------------------------------------------------
// optimiser: overflow check, Adam, fp16 copy, loss-scale update
// ---------------------------------------------------------------------------
__global__ void k_mlp_check(const float* __restrict__ grad, MLPState* st) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    int local = 0;
    for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) local |= !isfinite(grad[i]);
    if (local) atomicOr(&bad, 1);
    __syncthreads();
    if (threadIdx.x == 0) st->overflow = bad;
}

__global__ void k_mlp_adam(float* __restrict__ params, float* __restrict__ grad, float* __restrict__ mom,
                           float* __restrict__ vel, uint16_t* __restrict__ w16, int bf16, MLPState* st, float lr,
                           float b1, float b2, float eps, uint32_t step) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool overflow = st->overflow != 0;
    if (i < MLP_NPARAM) {
        if (!overflow) {
            const float denom = st->loss_scale * 3.f * (float)max(st->count, 1u);
            const float gr = grad[i] / denom;
            const float mm = b1 * mom[i] + (1.f - b1) * gr;
            const float vv = b2 * vel[i] + (1.f - b2) * gr * gr;
            mom[i] = mm;
            vel[i] = vv;
            const float mh = mm / (1.f - powf(b1, (float)step));
            const float vh = vv / (1.f - powf(b2, (float)step));
            const float p = params[i] - lr * mh / (sqrtf(vh) + eps);
            params[i] = p;
            if (i < MLP_NW) w16[i] = bf16 ? H16<true>::bits(p) : H16<false>::bits(p);
        }
        grad[i] = 0.f;
    }
    if (i == 0) {
        if (overflow) {
            st->loss_scale = fmaxf(st->loss_scale * 0.5f, 1.f / 1024.f);
            st->good = 0;
        } else if (++st->good >= 512u) {
            st->loss_scale = fminf(st->loss_scale * 2.f, 32768.f);
            st->good = 0;
        }
    }
}


// ---------------------------------------------------------------------------
// self-training samples: probe-origin rays hit y; a cosine bounce from y hits
// z; target = Le(z) + rho(z) * max(f(z), 0) (0 when z does not face y)
// ---------------------------------------------------------------------------
__device__ __forceinline__ f3 probe_center(const VolumeView& v, int p) {
    int i = p % v.counts.x, j = (p / v.counts.x) % v.counts.y, k = p / (v.counts.x * v.counts.y);
    return probe_pos(v, i, j, k, p);
}

__device__ __forceinline__ f3 train_ray_dir(const TrainParams& tp, uint32_t r) {
    float4 q = __ldg(tp.sf + r);
    return {tp.R[0] * q.x + tp.R[1] * q.y + tp.R[2] * q.z, tp.R[3] * q.x + tp.R[4] * q.y + tp.R[5] * q.z,
            tp.R[6] * q.x + tp.R[7] * q.y + tp.R[8] * q.z};
}

__device__ __forceinline__ f3 bounce_dir(const TrainParams& tp, uint32_t s, f3 n) {
    const uint32_t cp = rng_cand(rng_prefix(tp.seed, s, tp.frame, PASS_TRAIN_BOUNCE), 0u);
    float u0 = u01(rng_u32_dim(cp, 0)), u1 = u01(rng_u32_dim(cp, 1));
    float r = sqrtf(u0), sn, cs;
    sincospif(2.f * u1, &sn, &cs);
    return onb_to_world(n, r * cs, r * sn, sqrtf(fmaxf(0.f, 1.f - u0)));
}

__global__ void __launch_bounds__(128) k_train_primary(SceneView s, VolumeView v, TrainParams tp, float4* smp) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tp.samples) return;
    const uint32_t p = i / tp.per, r = i - p * tp.per;
    f3 P = probe_center(v, (int)p);
    f3 w = train_ray_dir(tp, r);
    Hit h = trace_spec<false>(s, Ray{P, w, DDGI_T_EPS, DDGI_MISS_T});   // probe-origin rays, as in the probe trace
    bool valid = false;
    f3 n = {0.f, 0.f, 1.f}, y = P;
    if (h.tri != DDGI_NONE) {
        n = xyz(__ldg(s.nrm + h.tri));
        valid = dot(n, w) < 0.f;
        y = P + w * h.t;
    }
    smp[3 * (size_t)i] = make_float4(y.x, y.y, y.z, valid ? 1.f : 0.f);
    smp[3 * (size_t)i + 1] = make_float4(n.x, n.y, n.z, 0.f);
    smp[3 * (size_t)i + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
}

struct BounceGen {
    const float4* smp;
    TrainParams tp;
    __device__ __forceinline__ bool ray(uint32_t i, Ray& r) const {
        r.tmax = DDGI_MISS_T;
        float4 y = smp[3 * (size_t)i];
        if (y.w == 0.f) return false;
        r.o = xyz(y);
        r.d = bounce_dir(tp, i, xyz(smp[3 * (size_t)i + 1]));
        r.tmin = DDGI_T_EPS;
        return true;
    }
};

// query at z; store writes the target and the training weight
struct TargetQuery {
    SceneView s;
    TrainParams tp;
    float4* smp;
    const float2* hits;
    __device__ bool front_hit(uint32_t i, f3& z, f3& nz, uint32_t& tri) const {
        float4 y = smp[3 * (size_t)i];
        if (y.w == 0.f) return false;
        float2 hv = hits[i];
        tri = __float_as_uint(hv.y);
        if (tri == DDGI_NONE) return false;
        f3 w = bounce_dir(tp, i, xyz(smp[3 * (size_t)i + 1]));
        nz = xyz(__ldg(s.nrm + tri));
        if (!(dot(nz, w) < 0.f)) return false;
        z = xyz(y) + w * hv.x;
        return true;
    }
    __device__ bool query(uint32_t i, f3& p, f3& n) const {
        uint32_t tri;
        if (!front_hit(i, p, n, tri)) return false;
        return any_pos(xyz(__ldg(s.alb + tri)));
    }
    __device__ void store(uint32_t i, bool valid, f3 f) const {
        f3 z, nz, tg = {0.f, 0.f, 0.f};
        uint32_t tri;
        const bool sample_ok = smp[3 * (size_t)i].w != 0.f;
        if (front_hit(i, z, nz, tri)) {
            tg = xyz(__ldg(s.emi + tri));
            if (valid) {
                f3 rho = xyz(__ldg(s.alb + tri));
                tg = tg + mul(rho, f3{fmaxf(f.x, 0.f), fmaxf(f.y, 0.f), fmaxf(f.z, 0.f)});
            }
        }
        const float w = (sample_ok && (i & 15u) != 15u) ? 1.f : 0.f;
        smp[3 * (size_t)i + 2] = make_float4(tg.x, tg.y, tg.z, w);
    }
};

// held-out samples (index 16 j + 15): relative squared error of the network
// and of the probe lookup against the one-bounce target.  The denominator,
// the mean of the two predictions squared plus 0.01, is common to both and
// independent of the target: the target's noise then adds the same amount to
// both sums, so their difference weighs only the two predictions' biases (a
// target-based denominator would reward predictions biased toward zero).
struct JudgeQuery {
    VolumeView v;
    TrainParams tp;
    const float4* smp;
    MLPState* st;
    __device__ bool query(uint32_t j, f3& p, f3& n) const {
        const uint32_t i = 16 * j + 15;
        float4 y = smp[3 * (size_t)i];
        if (y.w == 0.f) return false;
        p = xyz(y);
        n = xyz(smp[3 * (size_t)i + 1]);
        return true;
    }
    __device__ void store(uint32_t j, bool valid, f3 f) const {
        if (!valid) return;
        const uint32_t i = 16 * j + 15;
        f3 y = xyz(smp[3 * (size_t)i]), n = xyz(smp[3 * (size_t)i + 1]);
        f3 tg = xyz(smp[3 * (size_t)i + 2]);
        f3 P = probe_center(v, (int)(i / tp.per));
        f3 E = ddgi_irradiance_biased(v, y, n, P) * (1.f / DDGI_PI);
        f3 fm = {fmaxf(f.x, 0.f), fmaxf(f.y, 0.f), fmaxf(f.z, 0.f)};
        float em = 0.f, ep = 0.f;
        const float tv[3] = {tg.x, tg.y, tg.z}, mv[3] = {fm.x, fm.y, fm.z}, pv[3] = {E.x, E.y, E.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float den = 0.5f * (mv[c] * mv[c] + pv[c] * pv[c]) + 0.01f;
            em += (mv[c] - tv[c]) * (mv[c] - tv[c]) / den;
            ep += (pv[c] - tv[c]) * (pv[c] - tv[c]) / den;
        }
        atomicAdd(&st->judge_mlp, (double)em);
        atomicAdd(&st->judge_probe, (double)ep);
        atomicAdd(&st->judge_n, 1u);
    }
};

__global__ void k_mlp_begin(MLPState* st) {
    st->count = 0;
    st->judge_mlp = 0.0;
    st->judge_probe = 0.0;
    st->judge_n = 0;
}

// serve: 0 = the judge decides, 1 = always the network, 2 = always the probes
__global__ void k_mlp_count_reset(MLPState* st) { st->count = 0; }

__global__ void k_mlp_judge(MLPState* st, int serve) {
    if (serve == 1)
        st->use_mlp = 1u;
    else if (serve == 2)
        st->use_mlp = 0u;
    else
        st->use_mlp = (st->judge_n > 0 && st->judge_mlp <= st->judge_probe) ? 1u : 0u;
}

// served network: ema <- a ema + (1 - a) params, fp16 copy of its weights
__global__ void k_mlp_ema(const float* __restrict__ params, float* __restrict__ ema, uint16_t* __restrict__ w16s,
                          int bf16,
                          float a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_NPARAM) {
        const float e = a * ema[i] + (1.f - a) * params[i];
        ema[i] = e;
        if (i < MLP_NW) w16s[i] = bf16 ? H16<true>::bits(e) : H16<false>::bits(e);
    }
}

// gradient of the mean loss (unscaled) into out
__global__ void k_mlp_grad_out(const float* __restrict__ grad, const MLPState* st, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_NPARAM) out[i] = grad[i] / (st->loss_scale * 3.f * (float)max(st->count, 1u));
}

__global__ void k_zero(float* p, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0.f;
}

}  // namespace

cudaError_t launch_mlp_infer_buffer(const MLPView& m, const float* queries, float* out, uint32_t n,
                                    cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    return launch_mlp_infer(m, BufferQuery{reinterpret_cast<const float4*>(queries), reinterpret_cast<float4*>(out)},
                            n, st);
}

template <bool BF>
cudaError_t launch_mlp_grad_t(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* grad,
                              cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_train<BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)train_smem());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    uint32_t grid = (n + kTrainRows - 1) / kTrainRows;
    k_mlp_train<BF><<<grid, kTrainRows, train_smem(), st>>>(m, smp, n, state, grad);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* grad,
                            cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    return m.bf16 ? launch_mlp_grad_t<true>(m, smp, n, state, grad, st)
                  : launch_mlp_grad_t<false>(m, smp, n, state, grad, st);
}

cudaError_t launch_mlp_adam(float* params, float* grad, float* mom, float* vel, uint16_t* w16, int bf16,
                            MLPState* state, float lr, uint32_t step, cudaStream_t st) {
    k_mlp_check<<<1, 1024, 0, st>>>(grad, state);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(params, grad, mom, vel, w16, bf16, state, lr, 0.9f,
                                                           0.99f, 1e-8f, step);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train_frame(const SceneView& s, const VolumeView& v, const MLPView& m, const MLPView& ms,
                                   const TrainParams& tp, float4* smp, float2* hits, uint32_t* counter,
                                   MLPState* state, float* params, float* grad, float* mom, float* vel, uint16_t* w16,
                                   float* ema, uint16_t* w16s, float ema_a, float lr, uint32_t step, int serve,
                                   cudaStream_t st) {
    k_mlp_begin<<<1, 1, 0, st>>>(state);
    k_train_primary<<<(tp.samples + 127) / 128, 128, 0, st>>>(s, v, tp, smp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_trace<BounceGen, false>(s, BounceGen{smp, tp}, tp.samples, counter, hits, st);
    if (e != cudaSuccess) return e;
    e = launch_mlp_infer(ms, TargetQuery{s, tp, smp, hits}, tp.samples, st);
    if (e != cudaSuccess) return e;
    // minibatches of MLP_BATCH samples, one Adam step each
    for (uint32_t b0 = 0, k = 0; b0 < tp.samples; b0 += MLP_BATCH, ++k) {
        const uint32_t nb = min(MLP_BATCH, tp.samples - b0);
        k_mlp_count_reset<<<1, 1, 0, st>>>(state);
        e = launch_mlp_grad(m, smp + 3 * (size_t)b0, nb, state, grad, st);
        if (e != cudaSuccess) return e;
        e = launch_mlp_adam(params, grad, mom, vel, w16, m.bf16, state, lr, step + k, st);
        if (e != cudaSuccess) return e;
    }
    k_mlp_ema<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(params, ema, w16s, m.bf16, ema_a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the judge compares the served network with the probes on held-out samples
    e = launch_mlp_infer(ms, JudgeQuery{v, tp, smp, state}, tp.samples / 16, st);
    if (e != cudaSuccess) return e;
    k_mlp_judge<<<1, 1, 0, st>>>(state, serve);
    return cudaGetLastError();
}

cudaError_t launch_mlp_serve(MLPState* state, int serve, cudaStream_t st) {
    k_mlp_judge<<<1, 1, 0, st>>>(state, serve);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad_only(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* grad,
                                 float* out, cudaStream_t st) {
    k_zero<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(grad, MLP_NPARAM);
    k_mlp_begin<<<1, 1, 0, st>>>(state);
    cudaError_t e = launch_mlp_grad(m, smp, n, state, grad, st);
    if (e != cudaSuccess) return e;
    k_mlp_grad_out<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(grad, state, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_zero<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(grad, MLP_NPARAM);
    return cudaGetLastError();
}

cudaError_t launch_mlp_step(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* params,
                            float* grad, float* mom, float* vel, uint16_t* w16, float lr, uint32_t step,
                            cudaStream_t st) {
    k_mlp_begin<<<1, 1, 0, st>>>(state);
    cudaError_t e = launch_mlp_grad(m, smp, n, state, grad, st);
    if (e != cudaSuccess) return e;
    return launch_mlp_adam(params, grad, mom, vel, w16, m.bf16, state, lr, step, st);
}
