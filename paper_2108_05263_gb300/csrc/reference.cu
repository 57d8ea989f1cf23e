// Path-traced reference for the error metrics of Sec. 4 (MAPE, MSE): an
// unbiased path tracer with next-event estimation toward area-sampled
// emitters, cosine-distributed continuation, Russian roulette after the 4th
// vertex, at most 64 vertices, accumulated per pixel in fp64.  One path per
// pixel and sample through the pixel centre (the resampled frames use the
// same centres), random numbers keyed (seed, pixel, sample, pass 8, vertex,
// dimension).
#include "internal.h"
#include "trace_engine.cuh"

namespace {

#define PASS_PT 8u

__device__ __forceinline__ f3 pt_camera_dir(const CamView& cam, int px, int py) {
    const float W = (float)cam.width, H = (float)cam.height;
    float sx = (2.f * (px + 0.5f) / W - 1.f) * cam.tan_half_fovy * (W / H);
    float sy = (1.f - 2.f * (py + 0.5f) / H) * cam.tan_half_fovy;
    f3 d = f3{cam.fwd.x, cam.fwd.y, cam.fwd.z} + f3{cam.right.x, cam.right.y, cam.right.z} * sx +
           f3{cam.up.x, cam.up.y, cam.up.z} * sy;
    return d * rsqrtf(dot(d, d));
}

__global__ void __launch_bounds__(128) k_pt(SceneView s, CamView cam, uint32_t seed, uint32_t sample0,
                                            uint32_t spp, uint32_t max_depth, double* __restrict__ accum,
                                            float4* __restrict__ mean) {
    int px = blockIdx.x * blockDim.x + threadIdx.x;
    int py = blockIdx.y * blockDim.y + threadIdx.y;
    if (px >= cam.width || py >= cam.height) return;
    const uint32_t pix = (uint32_t)py * cam.width + px;
    const f3 o0 = {cam.pos.x, cam.pos.y, cam.pos.z};
    const f3 d0 = pt_camera_dir(cam, px, py);
    double sr = 0.0, sg = 0.0, sb = 0.0;
    for (uint32_t k = 0; k < spp; ++k) {
        const uint32_t smp = sample0 + k;
        const uint32_t prefix = rng_prefix(seed, pix, smp, PASS_PT);
        f3 o = o0, d = d0, beta = {1.f, 1.f, 1.f}, L = {0.f, 0.f, 0.f};
        Hit h = trace_bvh<false>(s, Ray{o, d, DDGI_T_EPS, DDGI_MISS_T});
        for (uint32_t depth = 1; depth <= max_depth; ++depth) {
            if (h.tri == DDGI_NONE) break;
            const f3 n = xyz(__ldg(s.nrm + h.tri));
            if (!(dot(n, d) < 0.f)) break;                    // back face: opaque interior
            const f3 x = o + d * h.t;
            if (depth == 1) L = L + xyz(__ldg(s.emi + h.tri));
            const f3 rho = xyz(__ldg(s.alb + h.tri));
            if (!any_pos(rho)) break;
            const uint32_t cp = rng_cand(prefix, depth);
            // next-event estimation toward a point uniform in emitter area
            if (s.num_emitters > 0) {
                float u0 = u01(rng_u32_dim(cp, 0)), u1 = u01(rng_u32_dim(cp, 1)), u2 = u01(rng_u32_dim(cp, 2));
                const float4* rec = s.evert + 4 * (size_t)sample_emitter(s, u0);
                float4 q0 = __ldg(rec), q1 = __ldg(rec + 1), q2 = __ldg(rec + 2), q3 = __ldg(rec + 3);
                float sq = sqrtf(u1);
                f3 y = xyz(q0) + xyz(q1) * (sq * (1.f - u2)) + xyz(q2) * (sq * u2);
                f3 dv = y - x;
                float d2 = dot(dv, dv);
                if (d2 > 0.f) {
                    float l = sqrtf(d2);
                    f3 w = dv * (1.f / l);
                    float cx = dot(n, w), cy = -dot(xyz(q3), w);
                    if (cx > 0.f && cy > 0.f) {
                        Hit sh = trace_bvh<true>(s, Ray{x, w, DDGI_T_EPS, (1.f - 1e-4f) * l});
                        if (sh.tri == DDGI_NONE) {
                            float gfac = cx * cy / d2 * s.area_total * (1.f / DDGI_PI);
                            L = L + mul(beta, mul(rho, f3{q1.w, q2.w, q3.w})) * gfac;
                        }
                    }
                }
            }
            // cosine continuation: the throughput is multiplied by rho
            float u3 = u01(rng_u32_dim(cp, 3)), u4 = u01(rng_u32_dim(cp, 4));
            float r = sqrtf(u3), sn, cs;
            sincospif(2.f * u4, &sn, &cs);
            f3 w = onb_to_world(n, r * cs, r * sn, sqrtf(fmaxf(0.f, 1.f - u3)));
            beta = mul(beta, rho);
            if (depth >= 4) {
                float q = fminf(fmaxf(fmaxf(beta.x, beta.y), beta.z), 0.95f);
                if (u01(rng_u32_dim(cp, 5)) >= q) break;
                beta = beta * (1.f / q);
            }
            o = x;
            d = w;
            h = trace_spec<false>(s, Ray{o, d, DDGI_T_EPS, DDGI_MISS_T});   // incoherent bounces
        }
        sr += L.x;
        sg += L.y;
        sb += L.z;
    }
    double* a = accum + 4 * (size_t)pix;
    a[0] += sr;
    a[1] += sg;
    a[2] += sb;
    a[3] += (double)spp;
    if (mean) mean[pix] = make_float4((float)(a[0] / a[3]), (float)(a[1] / a[3]), (float)(a[2] / a[3]), 1.f);
}

}  // namespace

cudaError_t launch_reference(const SceneView& s, const CamView& cam, uint32_t seed, uint32_t sample0,
                             uint32_t spp, uint32_t max_depth, double* accum, float4* mean, cudaStream_t st) {
    if (cam.width == 0 || cam.height == 0) return cudaSuccess;
    dim3 b(16, 8);
    dim3 g((cam.width + 15) / 16, (cam.height + 7) / 8);
    k_pt<<<g, b, 0, st>>>(s, cam, seed, sample0, spp, max_depth, accum, mean);
    return cudaGetLastError();
}
