// Learned target form (the neural cache the paper names as interchangeable
// with the probes, Sec. 2 / Sec. 5): batched tensor-core inference, a fused
// forward + backward training step with fp32 gradient accumulation and
// dynamic loss scaling, Adam, and the generation of self-training samples
// from probe-origin rays with one cosine bounce.
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>

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
// optimiser: overflow check, Adam, fp16 copy, loss-scale update
// ---------------------------------------------------------------------------
// One Adam step, fused with the overflow check and the loss-scale update
// (dynamic loss scaling: a step whose gradient holds a non-finite value is
// skipped -- parameters and moments untouched, the scale halved -- and does
// not count in Adam's bias correction, which uses the steps applied).
// The gradient of optimiser step t (1-based, skipped steps included)
// accumulates in buffer t & 1 of grad2
// (two buffers of MLP_NPARAM floats).  Every CTA checks the whole buffer for
// non-finite values, so all CTAs agree on skipping the step without a
// grid-wide barrier, updates its slice of the parameters and zeroes its slice
// of the other buffer, which step t + 1 accumulates into and which nothing
// reads during this step.  The last CTA to finish (every CTA has read the
// loss scale and the sample count by then) updates the loss scale, records
// the step's sample count and resets the accumulator.
constexpr int kOptThreads = 512;
__global__ void __launch_bounds__(kOptThreads) k_mlp_opt(float* __restrict__ params, float* __restrict__ grad2,
                                                         float* __restrict__ mom, float* __restrict__ vel,
                                                         uint16_t* __restrict__ w16, int bf16, MLPState* st, float lr,
                                                         float b1, float b2, float eps, uint32_t step,
                                                         float* __restrict__ ema, uint16_t* __restrict__ w16s,
                                                         float ema_a) {
    __shared__ float s_scale;
    __shared__ uint32_t s_acc, s_t;
    __shared__ int s_last;
    const float* __restrict__ g = grad2 + (size_t)(step & 1u) * MLP_NPARAM;
    float* __restrict__ gz = grad2 + (size_t)((step + 1u) & 1u) * MLP_NPARAM;
    if (threadIdx.x == 0) {
        s_scale = st->loss_scale;
        s_acc = st->acc;
        s_t = st->adam_t + 1u;   // this step's index in Adam's bias correction
    }
    int bad = 0;
    for (int i = threadIdx.x; i < MLP_NPARAM / 4; i += blockDim.x) {
        const float4 v = reinterpret_cast<const float4*>(g)[i];
        bad |= !isfinite(v.x) | !isfinite(v.y) | !isfinite(v.z) | !isfinite(v.w);
    }
    const bool overflow = __syncthreads_or(bad) != 0;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_NPARAM) {
        float p = params[i];
        if (!overflow) {
            const float denom = s_scale * 3.f * (float)max(s_acc, 1u);
            const float gr = g[i] / denom;
            const float mm = b1 * mom[i] + (1.f - b1) * gr;
            const float vv = b2 * vel[i] + (1.f - b2) * gr * gr;
            mom[i] = mm;
            vel[i] = vv;
            const float mh = mm / (1.f - powf(b1, (float)s_t));
            const float vh = vv / (1.f - powf(b2, (float)s_t));
            p = p - lr * mh / (sqrtf(vh) + eps);
            params[i] = p;
            if (i < MLP_NW) w16[i] = bf16 ? H16<true>::bits(p) : H16<false>::bits(p);
        }
        gz[i] = 0.f;
        if (ema) {   // the frame's last step: the served moving average follows
            const float e = ema_a * ema[i] + (1.f - ema_a) * p;
            ema[i] = e;
            if (i < MLP_NW) w16s[i] = bf16 ? H16<true>::bits(e) : H16<false>::bits(e);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&st->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        st->done = 0;
        st->overflow = overflow ? 1u : 0u;
        st->count = s_acc;
        st->acc = 0;
        if (!overflow) st->adam_t = s_t;
        if (overflow) {
            st->loss_scale = fmaxf(s_scale * 0.5f, 1.f / 1024.f);
            st->good = 0;
        } else if (++st->good >= 512u) {
            st->loss_scale = fminf(s_scale * 2.f, 32768.f);
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

__global__ void __launch_bounds__(128) k_train_primary(SceneView s, VolumeView v, TrainParams tp, float4* smp,
                                                       MLPState* st) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {   // the frame's counters (nothing reads them before the training kernels)
        st->count = 0;
        st->acc = 0;
        st->done = 0;
        st->judge_mlp = 0.0;
        st->judge_probe = 0.0;
        st->judge_n = 0;
    }
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
        // one atomic per converged group of lanes: three same-address
        // atomics per sample serialise at one L2 slice
        namespace cg = cooperative_groups;
        const cg::coalesced_group grp = cg::coalesced_threads();
        const double sm = cg::reduce(grp, (double)em, cg::plus<double>());
        const double sp = cg::reduce(grp, (double)ep, cg::plus<double>());
        if (grp.thread_rank() == 0) {
            atomicAdd(&st->judge_mlp, sm);
            atomicAdd(&st->judge_probe, sp);
            atomicAdd(&st->judge_n, grp.size());
        }
    }
};

__global__ void k_mlp_begin(MLPState* st) {
    st->count = 0;
    st->acc = 0;
    st->done = 0;
    st->judge_mlp = 0.0;
    st->judge_probe = 0.0;
    st->judge_n = 0;
}

// serve: 0 = the judge decides, 1 = always the network, 2 = always the probes

__global__ void k_mlp_judge(MLPState* st, int serve) {
    if (serve == 1)
        st->use_mlp = 1u;
    else if (serve == 2)
        st->use_mlp = 0u;
    else
        st->use_mlp = (st->judge_n > 0 && st->judge_mlp <= st->judge_probe) ? 1u : 0u;
}

// served network: ema <- a ema + (1 - a) params, fp16 copy of its weights
// gradient of the mean loss (unscaled) into out
__global__ void k_mlp_grad_out(const float* grad, const MLPState* st, float* out) {   // may run in place
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_NPARAM) out[i] = grad[i] / (st->loss_scale * 3.f * (float)max(st->acc, 1u));
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

// ---------------------------------------------------------------------------
// training on the tensor cores (tcgen05): one CTA (two warpgroups) per tile of
// 128 samples.  Forward: the inference kernel's K = 80 products with the bias
// in column 75, every layer input kept in shared memory (X0..X4).  Backward,
// layer l = 4..0, two products per commit:
//   dW_l^T [in (padded to 128) x out] = X_l^T dZ_l   (A and B read MN-major:
//       the K-major tiles seen with the sample index as K);
//   dX_l [128 x 80] = dZ_l W_l                       (B = W_l read MN-major);
// row 75 of dW_l^T is the bias gradient (column 75 of X_l is the constant 1).
// The gradients accumulate in tensor memory in fp32 over the tile's 128
// samples and are added to the global sums with one atomic per entry.
// ---------------------------------------------------------------------------
#define TR_X_OFF(l) (43520 + 20480 * (l))      // layer inputs X0..X4 [128 x 80]
#define TR_DZ_OFF(b) (145920 + 20480 * (b))    // deltas, two buffers [128 x 80]
#define TR_BAR_OFF 186880
#define TR_SMEM (TR_BAR_OFF + 16)
#define TR_COLS 256                            // tensor memory: [0, 80) products, [128, 256) dW^T x 2

// MN-major operand bit (15: A, 16: B) of the kind::f16 instruction descriptor
__host__ __device__ constexpr uint32_t umma_idesc_f16_mn(int M, int N, uint32_t fmt, uint32_t a_mn, uint32_t b_mn) {
    return umma_idesc_f16(M, N, fmt) | (a_mn << 15) | (b_mn << 16);
}

// Weight and bias gradients of layer l from tensor memory (dW_l^T, lane =
// input index r) into the global sums: warpgroup g takes column half g (the
// output layer's 16 columns go to warpgroup 0).
template <int OUTS>
__device__ __forceinline__ void tc_grad_out(int l, uint32_t tcol, int r, int g, float* __restrict__ grad) {
    const int K = l == 0 ? 75 : 64, real_out = l == 4 ? 3 : 64;
    const bool wrow = r < K, brow = r == MLP_TC_ONE_COL;
    constexpr int PER = OUTS == 16 ? 16 : OUTS / 2;
    if (OUTS == 16 && g != 0) return;
    const int c_begin = OUTS == 16 ? 0 : PER * g;
#pragma unroll
    for (int c0 = c_begin; c0 < c_begin + PER; c0 += 16) {
        uint32_t v[16];
        TMEM_LD_X16(tcol + (uint32_t)c0, v, 0);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (wrow || brow) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int o = c0 + j;
                if (o < real_out) {
                    const float gv = __uint_as_float(v[j]);
                    if (wrow)
                        atomicAdd(grad + mlp_off_w(l) + o * mlp_in(l) + r, gv);
                    else
                        atomicAdd(grad + mlp_off_b(l) + o, gv);
                }
            }
        }
    }
}

// samples [n][3] float4: (y.xyz, _), (n.xyz, _), (target.rgb, weight); weight 0
// excludes a sample.  Gradients of sum_s w_s sum_c (f - t)^2 / (sg(f)^2 + 0.01)
// times the loss scale are added to grad; the weights are summed into
// st->acc.  Two warpgroups: thread t owns
// sample row r = t mod 128 (its tensor-memory lane) and column half g = t / 128
// of every epilogue.  The gradient atomics of layer l + 1 run while the tensor
// core computes layer l's products (dW^T alternates between columns 128 and
// 192 of tensor memory).
template <bool BF>
__global__ void __launch_bounds__(256, 1) k_mlp_train_tc(MLPView m, const float4* __restrict__ smp, uint32_t n,
                                                         MLPState* __restrict__ st, float* __restrict__ grad) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint32_t s_taddr;
    const int t = threadIdx.x, w = t >> 5, r = t & 127, g = t >> 7;
    const uint32_t bar = smem_u32(sm + TR_BAR_OFF);
    mlp_tc_load_weights<BF>(m, sm);
    float4 tg = make_float4(0.f, 0.f, 0.f, 0.f);
    if (g == 0) {
        // this thread's sample: encoded input row, target and weight
        const uint32_t s_i = blockIdx.x * 128u + (uint32_t)r;
        float4 y = make_float4(0.f, 0.f, 0.f, 0.f), nn = make_float4(0.f, 0.f, 1.f, 0.f);
        if (s_i < n) {
            y = smp[3 * (size_t)s_i];
            nn = smp[3 * (size_t)s_i + 1];
            tg = smp[3 * (size_t)s_i + 2];
        }
        const unsigned cnt = __ballot_sync(0xffffffffu, tg.w > 0.f);
        if ((t & 31) == 0 && cnt) atomicAdd(&st->acc, (unsigned)__popc(cnt));
        const float qv[6] = {(y.x - m.lo[0]) * m.scale, (y.y - m.lo[1]) * m.scale, (y.z - m.lo[2]) * m.scale,
                             nn.x, nn.y, nn.z};
        mlp_tc_encode_row<BF>(sm + TR_X_OFF(0), r, qv);
    } else {
        // columns 64..79 of the hidden layers' inputs: zeros and the constant 1;
        // both delta buffers zeroed (their unused columns stay zero)
        const uint32_t one = H16<BF>::pack(0.f, 0.f) | ((uint32_t)H16<BF>::bits(1.f) << 16);
        for (int l = 1; l < 5; ++l) {
            *reinterpret_cast<uint4*>(sm + TR_X_OFF(l) + kmajor_off(r, 64)) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(sm + TR_X_OFF(l) + kmajor_off(r, 72)) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint32_t*>(sm + TR_X_OFF(l) + kmajor_off(r, 74)) = one;   // (74, 75) = (0, 1)
        }
        for (int b = 0; b < 2; ++b)
            for (int k = 0; k < 80; k += 8)
                *reinterpret_cast<uint4*>(sm + TR_DZ_OFF(b) + kmajor_off(r, k)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(TR_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = s_taddr;
    const uint32_t trow = tbase + ((uint32_t)(32 * (w & 3)) << 16);   // this warp's 32 lanes
    const uint32_t base = smem_u32(sm);
    uint32_t phase = 0;
    bool failed = false;

    // ---- forward ----------------------------------------------------------------
    float out[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
    for (int l = 0; l < 5 && !failed; ++l) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = umma_idesc_f16(128, l == 4 ? 16 : 64, H16<BF>::umma_fmt);
            const uint32_t xa = base + TR_X_OFF(l), wl = base + MLP_TC_W_OFF(l);
#pragma unroll
            for (int s = 0; s < MLP_TC_K / 16; ++s)
                umma_f16(tbase, umma_sdesc(xa + 256u * s, 128u, 1280u), umma_sdesc(wl + 256u * s, 128u, 1280u), idesc,
                         s > 0 ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                         : "memory");
        }
        const bool ok = mbar_wait(bar, phase);
        if (__syncthreads_or(!ok)) {
            mbar_drain(bar, phase);
            failed = true;
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (l < 4) {
            uint8_t* xn = sm + TR_X_OFF(l + 1);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int c2 = 2 * g + i;
                uint32_t v[16];
                TMEM_LD_X16(trow + 16u * (uint32_t)c2, v, 0);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    *reinterpret_cast<uint4*>(xn + kmajor_off(r, 16 * c2 + 8 * h)) =
                        make_uint4(H16<BF>::relu2(v[8 * h], v[8 * h + 1]), H16<BF>::relu2(v[8 * h + 2], v[8 * h + 3]),
                                   H16<BF>::relu2(v[8 * h + 4], v[8 * h + 5]),
                                   H16<BF>::relu2(v[8 * h + 6], v[8 * h + 7]));
            }
        } else if (g == 0) {
            uint32_t v[16];
            TMEM_LD_X16(trow, v, 0);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            out[0] = __uint_as_float(v[0]);
            out[1] = __uint_as_float(v[1]);
            out[2] = __uint_as_float(v[2]);
        }
    }
    // ---- output gradient (relative L2, denominator held constant) ----------------
    if (!failed && g == 0) {
        const float S = st->loss_scale;
        const float tv[3] = {tg.x, tg.y, tg.z};
        float d[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) d[c] = tg.w * S * 2.f * (out[c] - tv[c]) / (out[c] * out[c] + 0.01f);
        *reinterpret_cast<uint4*>(sm + TR_DZ_OFF(0) + kmajor_off(r, 0)) =
            make_uint4(H16<BF>::pack(d[0], d[1]), H16<BF>::pack(d[2], 0.f), 0u, 0u);
    }
    // ---- backward ---------------------------------------------------------------
    int cur = 0;   // buffer holding dZ_l
#pragma unroll 1
    for (int l = 4; l >= 0 && !failed; --l) {
        const int outs = l == 4 ? 16 : 64;
        const uint32_t dw_col = 128u + 64u * (uint32_t)(l & 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (t == 0) {
            const uint32_t xa = base + TR_X_OFF(l), dz = base + TR_DZ_OFF(cur), wl = base + MLP_TC_W_OFF(l);
            // dW^T = X^T dZ: M = 128 (inputs, padded), N = outs, K = 128 samples (two 8-row groups per step)
            const uint32_t idw = umma_idesc_f16_mn(128, outs, H16<BF>::umma_fmt, 1u, 1u);
#pragma unroll
            for (int s = 0; s < 8; ++s)
                umma_f16(tbase + dw_col, umma_sdesc(xa + 2560u * s, 1280u, 128u), umma_sdesc(dz + 2560u * s, 1280u, 128u),
                         idw, s > 0 ? 1u : 0u);
            if (l > 0) {
                // dX = dZ W: M = 128 samples, N = 80 inputs, K = outs
                const uint32_t idx = umma_idesc_f16_mn(128, 80, H16<BF>::umma_fmt, 0u, 1u);
                for (int s = 0; s < outs / 16; ++s)
                    umma_f16(tbase, umma_sdesc(dz + 256u * s, 128u, 1280u), umma_sdesc(wl + 2560u * s, 1280u, 128u), idx,
                             s > 0 ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                         : "memory");
        }
        // the previous layer's gradients, while these products run
        if (l == 3)
            tc_grad_out<16>(4, trow + 128u, r, g, grad);
        else if (l < 3)
            tc_grad_out<64>(l + 1, trow + 128u + 64u * (uint32_t)((l + 1) & 1), r, g, grad);
        const bool ok = mbar_wait(bar, phase);
        if (__syncthreads_or(!ok)) {
            mbar_drain(bar, phase);
            failed = true;
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (l > 0) {
            // dZ_{l-1} = dX_l masked by the ReLU of X_l (its first 64 columns)
            const uint8_t* xl = sm + TR_X_OFF(l);
            uint8_t* dn = sm + TR_DZ_OFF(cur ^ 1);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int c2 = 2 * g + i;
                uint32_t v[16];
                TMEM_LD_X16(trow + 16u * (uint32_t)c2, v, 0);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k0 = 16 * c2 + 8 * h;
                    const uint4 xv = *reinterpret_cast<const uint4*>(xl + kmajor_off(r, k0));
                    const uint32_t xs[4] = {xv.x, xv.y, xv.z, xv.w};
                    uint32_t o4[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float a0 = __uint_as_float(v[8 * h + 2 * q]), a1 = __uint_as_float(v[8 * h + 2 * q + 1]);
                        const float m0 = H16<BF>::val((uint16_t)(xs[q] & 0xFFFFu)) > 0.f ? a0 : 0.f;
                        const float m1 = H16<BF>::val((uint16_t)(xs[q] >> 16)) > 0.f ? a1 : 0.f;
                        o4[q] = H16<BF>::pack(m0, m1);
                    }
                    *reinterpret_cast<uint4*>(dn + kmajor_off(r, k0)) = make_uint4(o4[0], o4[1], o4[2], o4[3]);
                }
            }
            cur ^= 1;
        } else {
            tc_grad_out<64>(0, trow + 128u, r, g, grad);
        }
    }
    if (failed && t == 0) atomicOr(m.err, ERRBIT_MMA_WAIT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TR_COLS));
}

template <bool BF>
cudaError_t launch_mlp_grad_t(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* grad,
                              cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_train_tc<BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, TR_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    uint32_t grid = (n + 127) / 128;
    k_mlp_train_tc<BF><<<grid, 256, TR_SMEM, st>>>(m, smp, n, state, grad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fp32 debug form of the gradient: the same samples, loss, loss scaling and
// counters as k_mlp_train_tc, computed on the CUDA cores in fp32, one thread
// per sample (forward with every layer input kept, then backward).  Each
// parameter's gradient is summed over a warp's 32 samples with shuffles and
// added to the global sum by one atomic.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(MLP_F32_THREADS) k_mlp_grad_f32(MLPView m, const float4* __restrict__ smp,
                                                                  uint32_t n, MLPState* __restrict__ st,
                                                                  float* __restrict__ grad) {
    extern __shared__ float sw[];
    for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) sw[i] = m.params[i];
    __syncthreads();
    const uint32_t s_i = blockIdx.x * MLP_F32_THREADS + threadIdx.x;
    const int lane = threadIdx.x & 31;
    float4 y = make_float4(0.f, 0.f, 0.f, 0.f), nn = make_float4(0.f, 0.f, 1.f, 0.f), tg = y;
    if (s_i < n) {   // threads past n carry weight 0 but join the warp's reductions
        y = smp[3 * (size_t)s_i];
        nn = smp[3 * (size_t)s_i + 1];
        tg = smp[3 * (size_t)s_i + 2];
    }
    const unsigned cnt = __ballot_sync(0xffffffffu, tg.w > 0.f);
    if (lane == 0 && cnt) atomicAdd(&st->acc, (unsigned)__popc(cnt));
    // a[0]: the encoded input; a[l]: the ReLU output of layer l - 1 (input of layer l)
    float a[5][MLP_IN];
    mlp_f32_encode(m, xyz(y), xyz(nn), a[0]);
    mlp_f32_layer<MLP_IN, MLP_H, true>(sw, 0, a[0], a[1]);
    mlp_f32_layer<MLP_H, MLP_H, true>(sw, 1, a[1], a[2]);
    mlp_f32_layer<MLP_H, MLP_H, true>(sw, 2, a[2], a[3]);
    mlp_f32_layer<MLP_H, MLP_H, true>(sw, 3, a[3], a[4]);
    float out[3];
    mlp_f32_layer<MLP_H, 3, false>(sw, 4, a[4], out);
    // output delta of the relative-L2 loss (denominator held constant), scaled
    float dz[MLP_H], da[MLP_H];
    const float S = st->loss_scale, tv[3] = {tg.x, tg.y, tg.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) dz[c] = tg.w * S * 2.f * (out[c] - tv[c]) / (out[c] * out[c] + 0.01f);
#pragma unroll 1
    for (int l = 4; l >= 0; --l) {
        const int ins = mlp_in(l), kin = l == 0 ? 75 : MLP_H, outs = l == 4 ? 3 : MLP_H;
        const float* W = sw + mlp_off_w(l);
#pragma unroll 1
        for (int o = 0; o < outs; ++o) {
            const float d = dz[o];
#pragma unroll 1
            for (int i = 0; i < kin; ++i) {
                const float v = warp_sum_f32(d * a[l][i]);
                if (lane == 0) atomicAdd(grad + mlp_off_w(l) + o * ins + i, v);
            }
            const float vb = warp_sum_f32(d);
            if (lane == 0) atomicAdd(grad + mlp_off_b(l) + o, vb);
        }
        if (l > 0) {
            // delta of layer l - 1's pre-activation: W_l^T dz, masked by its ReLU
#pragma unroll 1
            for (int i = 0; i < MLP_H; ++i) {
                float acc = 0.f;
                for (int o = 0; o < outs; ++o) acc = fmaf(W[o * ins + i], dz[o], acc);
                da[i] = a[l][i] > 0.f ? acc : 0.f;
            }
#pragma unroll 1
            for (int i = 0; i < MLP_H; ++i) dz[i] = da[i];
        }
    }
}

cudaError_t launch_mlp_grad_f32(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* grad,
                                cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_F32_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_mlp_grad_f32<<<(n + MLP_F32_THREADS - 1) / MLP_F32_THREADS, MLP_F32_THREADS, MLP_F32_SMEM, st>>>(m, smp, n,
                                                                                                     state, grad);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mlp_grad(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* grad,
                            cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (m.fp32) return launch_mlp_grad_f32(m, smp, n, state, grad, st);
    return m.bf16 ? launch_mlp_grad_t<true>(m, smp, n, state, grad, st)
                  : launch_mlp_grad_t<false>(m, smp, n, state, grad, st);
}

// grad2: the two gradient buffers (step t reads buffer t & 1)
cudaError_t launch_mlp_adam(float* params, float* grad2, float* mom, float* vel, uint16_t* w16, int bf16,
                            MLPState* state, float lr, uint32_t step, cudaStream_t st, float* ema, uint16_t* w16s,
                            float ema_a) {
    k_mlp_opt<<<(MLP_NPARAM + kOptThreads - 1) / kOptThreads, kOptThreads, 0, st>>>(
        params, grad2, mom, vel, w16, bf16, state, lr, 0.9f, 0.99f, 1e-8f, step, ema, w16s, ema_a);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train_frame(const SceneView& s, const VolumeView& v, const MLPView& m, const MLPView& ms,
                                   const TrainParams& tp, float4* smp, float2* hits, uint32_t* counter,
                                   MLPState* state, float* params, float* grad, float* mom, float* vel, uint16_t* w16,
                                   float* ema, uint16_t* w16s, float ema_a, float lr, uint32_t step, int serve,
                                   cudaStream_t st) {
    k_train_primary<<<(tp.samples + 127) / 128, 128, 0, st>>>(s, v, tp, smp, state);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_trace<BounceGen, false>(s, BounceGen{smp, tp}, tp.samples, counter, hits, st);
    if (e != cudaSuccess) return e;
    e = launch_mlp_infer(ms, TargetQuery{s, tp, smp, hits}, tp.samples, st);
    if (e != cudaSuccess) return e;
    // minibatches of MLP_BATCH samples, one Adam step each
    for (uint32_t b0 = 0, k = 0; b0 < tp.samples; b0 += MLP_BATCH, ++k) {
        const uint32_t nb = min(MLP_BATCH, tp.samples - b0);
        e = launch_mlp_grad(m, smp + 3 * (size_t)b0, nb, state, grad + (size_t)((step + k) & 1u) * MLP_NPARAM, st);
        if (e != cudaSuccess) return e;
        const bool last = b0 + MLP_BATCH >= tp.samples;
        e = launch_mlp_adam(params, grad, mom, vel, w16, m.bf16, state, lr, step + k, st, last ? ema : nullptr,
                            w16s, ema_a);
        if (e != cudaSuccess) return e;
    }
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

cudaError_t launch_mlp_grad_only(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* out,
                                 cudaStream_t st) {
    // accumulated in `out` itself, apart from the optimiser's buffers
    k_zero<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(out, MLP_NPARAM);
    k_mlp_begin<<<1, 1, 0, st>>>(state);
    cudaError_t e = launch_mlp_grad(m, smp, n, state, out, st);
    if (e != cudaSuccess) return e;
    k_mlp_grad_out<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(out, state, out);
    return cudaGetLastError();
}

cudaError_t launch_mlp_step(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* params,
                            float* grad, float* mom, float* vel, uint16_t* w16, float lr, uint32_t step,
                            cudaStream_t st) {
    k_mlp_begin<<<1, 1, 0, st>>>(state);
    cudaError_t e = launch_mlp_grad(m, smp, n, state, grad + (size_t)(step & 1u) * MLP_NPARAM, st);
    if (e != cudaSuccess) return e;
    return launch_mlp_adam(params, grad, mom, vel, w16, m.bf16, state, lr, step, st, nullptr, nullptr, 0.f);
}
