// Probe update of Sec. 3.2 (Eq. probeUpdate): per-ray trace with the
// attenuated emission and the probe-augmented bounce, then a per-probe blend
// of irradiance and distance moments with hysteresis and border refresh.
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
__global__ void __launch_bounds__(128) k_probe_trace(SceneView s, VolumeView v, ProbeParams pp,
                                                     const float4* __restrict__ sf,
                                                     float4* __restrict__ rays, int total) {
    int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= total) return;
    int R = (int)pp.rays;
    int p = tid / R, r = tid - p * R;
    f3 P = probe_of(v, p);
    f3 w = rotate(pp, __ldg(sf + r));
    // coherent rays (one origin per 32-lane warp): traversal in place
    Hit h = trace_bvh<false>(s, Ray{P, w, DDGI_T_EPS, DDGI_MISS_T});
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
            out.x = L.x;
            out.y = L.y;
            out.z = L.z;
        }
    }
    rays[tid] = out;
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
__global__ void __launch_bounds__(256) k_probe_blend(VolumeView v, ProbeParams pp,
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
                if (c > 0.f) {
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

}  // namespace

cudaError_t launch_probe_trace(const SceneView& s, const VolumeView& v, const ProbeParams& p,
                               float4* rays, float2* hits, uint32_t* counter, cudaStream_t st) {
    int P = v.counts.x * v.counts.y * v.counts.z;
    int total = P * (int)p.rays;
    if (total == 0) return cudaSuccess;
    k_probe_trace<<<(total + 127) / 128, 128, 0, st>>>(s, v, p, p.sf, rays, total);
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
    k_probe_blend<<<P, 256, smem, st>>>(v, p, p.sf, rays);
    return cudaGetLastError();
}
