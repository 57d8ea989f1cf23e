// Probe update of Sec. 3.2 (Eq. probeUpdate): per-ray trace with the
// attenuated emission and the probe-augmented bounce, then a per-probe blend
// of irradiance and distance moments with hysteresis and border refresh.
#include <algorithm>

#include "internal.h"
#include "trace_engine.cuh"

namespace {

__device__ __forceinline__ f3 rotate(const ProbeParams& p, float4 s) {
    return {p.R[0] * s.x + p.R[1] * s.y + p.R[2] * s.z, p.R[3] * s.x + p.R[4] * s.y + p.R[5] * s.z,
            p.R[6] * s.x + p.R[7] * s.y + p.R[8] * s.z};
}

// distance from a probe to the boundary of its own cell along d
__device__ __forceinline__ float cell_exit(const VolumeView& v, f3 d) {
    float t = DDGI_MISS_T;
    if (d.x != 0.f) t = fminf(t, 0.5f * v.spacing.x / fabsf(d.x));
    if (d.y != 0.f) t = fminf(t, 0.5f * v.spacing.y / fabsf(d.y));
    if (d.z != 0.f) t = fminf(t, 0.5f * v.spacing.z / fabsf(d.z));
    return t;
}

__device__ __forceinline__ f3 probe_of(const VolumeView& v, int p) {
    int i = p % v.counts.x, j = (p / v.counts.x) % v.counts.y, k = p / (v.counts.x * v.counts.y);
    return probe_pos(v, i, j, k, p);
}

// one thread per (probe, ray): trace, then the radiance of Eq. probeUpdate
// (GLOSSY: with the glossy half of L_DDGI+ toward the probe, Sec. 3.3)
template <bool GLOSSY>
__global__ void __launch_bounds__(128) k_probe_trace(SceneView s, VolumeView v, ProbeParams pp,
                                                     const float4* __restrict__ sf,
                                                     float4* __restrict__ rays, int total) {
    int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= total) return;
    int R = (int)pp.rays;
    int p = tid / R;
    // thread -> ray: consecutive threads take neighbouring directions, so a
    // warp traverses one patch of the sphere (the results go to the ray's slot)
    int r = (int)__ldg(pp.order + (tid - p * R));
    f3 P = probe_of(v, p);
    f3 w = rotate(pp, __ldg(sf + r));
    // one origin per 32-lane warp, directions over the sphere: per-thread
    // traversal with the speculative descent of the persistent engine
    Hit h = trace_spec<false>(s, Ray{P, w, DDGI_T_EPS, DDGI_MISS_T});
    float4 out = make_float4(0.f, 0.f, 0.f, DDGI_MISS_T);
    if (h.tri != DDGI_NONE) {
        f3 n = xyz(__ldg(s.nrm + h.tri));
        if (dot(n, w) > 0.f) {
            out.w = -h.t;
        } else {
            out.w = h.t;
            float att = 1.f;
            if (pp.le_attenuation > 0.f) {
                const int td = v.depth_n + 2;
                float mu = sample_depth(v.depth + (size_t)p * td * td, v.depth_n, -w).x;
                float db = fminf(mu, cell_exit(v, -w));
                float f = h.t / (h.t + pp.le_attenuation * db);
                att = f * f;
            }
            f3 le = xyz(__ldg(s.emi + h.tri));
            f3 rho = xyz(__ldg(s.alb + h.tri));
            f3 L = le * att;
            if (any_pos(rho)) {
                f3 y = P + w * h.t;
                f3 E = ddgi_irradiance_biased(v, y, n, P);
                L = L + mul(rho, E) * (1.f / DDGI_PI);
            }
            if (GLOSSY) {
                const float4 spec = __ldg(s.spec + h.tri);
                if (is_glossy(spec)) {
                    const uint32_t cp = rng_cand(rng_prefix(pp.seed, (uint32_t)p, pp.frame, PASS_PROBE_GLOSSY),
                                                 (uint32_t)r);
                    const f3 q = biased_point(v, P + w * h.t, P);
                    L = L + glossy_ddgi(v, q, n, -w, spec, u01(rng_u32_dim(cp, 0)), u01(rng_u32_dim(cp, 1)));
                }
            }
            out.x = L.x;
            out.y = L.y;
            out.z = L.z;
        }
    }
    rays[(size_t)p * R + r] = out;
}

// padded-tile index of the texel whose value border texel (X, Y) repeats
__device__ __forceinline__ int border_source(int X, int Y, int n) {
    int w = n + 2;
    int sx = X, sy = Y;
    if (Y == 0 || Y == n + 1) {
        if (X == 0 || X == n + 1) {          // corners take the opposite corner
            sx = X == 0 ? n : 1;
            sy = Y == 0 ? n : 1;
        } else {
            sx = n + 1 - X;
            sy = Y == 0 ? 1 : n;
        }
    } else if (X == 0 || X == n + 1) {
        sx = X == 0 ? 1 : n;
        sy = n + 1 - Y;
    }
    return sy * w + sx;
}

// one CTA per probe; rays and directions staged in shared memory
__global__ void __launch_bounds__(512) k_probe_blend(VolumeView v, ProbeParams pp,
                                                     const float4* __restrict__ sf,
                                                     const float4* __restrict__ rays) {
    extern __shared__ float4 smem[];
    const int R = (int)pp.rays;
    float4* s_ray = smem;            // R: L.rgb, signed distance
    float4* s_dir = smem + R;        // R: direction
    const int ni = v.irr_n, nd = v.depth_n, ti = ni + 2, td = nd + 2;
    float4* s_irr = smem + 2 * R;                             // ti*ti
    float2* s_dep = reinterpret_cast<float2*>(s_irr + ti * ti);  // td*td
    const int p = blockIdx.x;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        s_ray[r] = rays[(size_t)p * R + r];
        f3 w = rotate(pp, __ldg(sf + r));
        s_dir[r] = make_float4(w.x, w.y, w.z, 0.f);
    }
    __syncthreads();
    float4* g_irr = v.irr + (size_t)p * ti * ti;
    float2* g_dep = v.depth + (size_t)p * td * td;
    const float a = pp.hysteresis;
    const int nirr = ni * ni, ntot = nirr + nd * nd;
    for (int k = threadIdx.x; k < ntot; k += blockDim.x) {
        if (k < nirr) {
            int i = k % ni, j = k / ni;
            f3 dt = texel_dir(i, j, ni);
            float sw = 0.f;
            f3 sl = {0.f, 0.f, 0.f};
            for (int r = 0; r < R; ++r) {
                float4 d = s_dir[r];
                float c = dt.x * d.x + dt.y * d.y + dt.z * d.z;
                if (c > 0.f) {
                    float4 L = s_ray[r];
                    sw += c;
                    sl = sl + f3{L.x, L.y, L.z} * c;
                }
            }
            int idx = (j + 1) * ti + (i + 1);
            float4 old = g_irr[idx];
            if (sw > 0.f) {
                float s = DDGI_PI / sw;
                old.x = a * old.x + (1.f - a) * (sl.x * s);
                old.y = a * old.y + (1.f - a) * (sl.y * s);
                old.z = a * old.z + (1.f - a) * (sl.z * s);
            }
            s_irr[idx] = old;
        } else {
            int kk = k - nirr;
            int i = kk % nd, j = kk / nd;
            f3 dt = texel_dir(i, j, nd);
            float sw = 0.f, s1 = 0.f, s2 = 0.f;
            for (int r = 0; r < R; ++r) {
                float4 d = s_dir[r];
                float c = dt.x * d.x + dt.y * d.y + dt.z * d.z;
                // weights below 2^-40 are skipped (no change at fp32 resolution);
                // a warp's texels face nearby directions, so whole warps skip most rays
                if (c > pp.depth_cmin && c > 0.f) {
                    float wr = __powf(c, pp.depth_sharpness);
                    float t = fminf(fabsf(s_ray[r].w), pp.depth_tmax);
                    sw += wr;
                    s1 += wr * t;
                    s2 += wr * t * t;
                }
            }
            int idx = (j + 1) * td + (i + 1);
            float2 old = g_dep[idx];
            if (sw > 0.f) {
                old.x = a * old.x + (1.f - a) * (s1 / sw);
                old.y = a * old.y + (1.f - a) * (s2 / sw);
            }
            s_dep[idx] = old;
        }
    }
    __syncthreads();
    // write the padded tiles, border texels repeating their fold partner
    for (int k = threadIdx.x; k < ti * ti; k += blockDim.x) {
        int X = k % ti, Y = k / ti;
        g_irr[k] = s_irr[border_source(X, Y, ni)];
    }
    for (int k = threadIdx.x; k < td * td; k += blockDim.x) {
        int X = k % td, Y = k / td;
        g_dep[k] = s_dep[border_source(X, Y, nd)];
    }
}

// lexicographic minimum of (t, ray index) across the warp
__device__ __forceinline__ void warp_min_idx(float& t, int& r) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float t2 = __shfl_xor_sync(0xffffffffu, t, o);
        int r2 = __shfl_xor_sync(0xffffffffu, r, o);
        if (t2 < t || (t2 == t && r2 < r)) {
            t = t2;
            r = r2;
        }
    }
}

// Probe relocation (cited probe volume; Majercik et al. 2021), one warp per
// probe over this frame's rays: more than a quarter back-face hits moves the
// probe through the closest back face by its distance + delta / 2; else a
// front face nearer than delta pushes it away by the shortfall; every axis of
// the offset is then clamped to +-0.45 spacing.
__global__ void __launch_bounds__(128) k_probe_relocate(ProbeParams pp, const float4* __restrict__ rays,
                                                        float4* __restrict__ offset, float3 spacing, float delta,
                                                        int P) {
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (p >= P) return;
    const int R = (int)pp.rays;
    int nback = 0, rb = INT_MAX, rf = INT_MAX;
    float tb = DDGI_MISS_T, tf = DDGI_MISS_T;
    for (int r = lane; r < R; r += 32) {
        const float t = __ldg(rays + (size_t)p * R + r).w;
        if (t >= DDGI_MISS_T) continue;
        if (t < 0.f) {
            ++nback;
            if (-t < tb) {
                tb = -t;
                rb = r;
            }
        } else if (t < tf) {
            tf = t;
            rf = r;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nback += __shfl_xor_sync(0xffffffffu, nback, o);
    warp_min_idx(tb, rb);
    warp_min_idx(tf, rf);
    if (lane != 0) return;
    float4 off = offset[p];
    if (4 * nback > R && rb != INT_MAX) {
        const f3 d = rotate(pp, __ldg(pp.sf + rb));
        const float s = tb + 0.5f * delta;
        off.x += d.x * s;
        off.y += d.y * s;
        off.z += d.z * s;
    } else if (rf != INT_MAX && tf < delta) {
        const f3 d = rotate(pp, __ldg(pp.sf + rf));
        const float s = delta - tf;
        off.x -= d.x * s;
        off.y -= d.y * s;
        off.z -= d.z * s;
    }
    off.x = fminf(fmaxf(off.x, -0.45f * spacing.x), 0.45f * spacing.x);
    off.y = fminf(fmaxf(off.y, -0.45f * spacing.y), 0.45f * spacing.y);
    off.z = fminf(fmaxf(off.z, -0.45f * spacing.z), 0.45f * spacing.z);
    offset[p] = off;
}

}  // namespace

cudaError_t launch_probe_relocate(const VolumeView& v, const ProbeParams& p, const float4* rays, float4* offset,
                                  cudaStream_t st) {
    int P = v.counts.x * v.counts.y * v.counts.z;
    if (P == 0) return cudaSuccess;
    k_probe_relocate<<<(P + 3) / 4, 128, 0, st>>>(p, rays, offset, v.spacing, 0.1f * v.min_spacing, P);
    return cudaGetLastError();
}

cudaError_t launch_probe_trace(const SceneView& s, const VolumeView& v, const ProbeParams& p,
                               float4* rays, float2* hits, uint32_t* counter, cudaStream_t st) {
    int P = v.counts.x * v.counts.y * v.counts.z;
    int total = P * (int)p.rays;
    if (total == 0) return cudaSuccess;
    if (s.spec)
        k_probe_trace<true><<<(total + 127) / 128, 128, 0, st>>>(s, v, p, p.sf, rays, total);
    else
        k_probe_trace<false><<<(total + 127) / 128, 128, 0, st>>>(s, v, p, p.sf, rays, total);
    return cudaGetLastError();
}

size_t probe_blend_smem(const VolumeView& v, uint32_t rays) {
    int ti = v.irr_n + 2, td = v.depth_n + 2;
    return sizeof(float4) * (2 * (size_t)rays + ti * ti) + sizeof(float2) * td * td;
}

cudaError_t launch_probe_blend(const VolumeView& v, const ProbeParams& p, const float4* rays,
                               cudaStream_t st) {
    int P = v.counts.x * v.counts.y * v.counts.z;
    if (P == 0) return cudaSuccess;
    size_t smem = probe_blend_smem(v, p.rays);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_probe_blend, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    // one thread per texel of both maps when they fit one CTA (320 for 8x8 +
    // 16x16), so that the texel loop runs once
    const int texels = v.irr_n * v.irr_n + v.depth_n * v.depth_n;
    const int threads = std::min(512, (texels + 31) / 32 * 32);
    k_probe_blend<<<P, threads, smem, st>>>(v, p, p.sf, rays);
    return cudaGetLastError();
}
