// Primary visibility (support pass) and the shading estimator of Sec. 3.1
// steps 3-4 / Eq. Algorithm: Le at x + residual + the resampled bounded term
// behind one shadow ray, with a fresh probe query at the selected point.
#include "internal.h"
#include "trace_engine.cuh"

namespace {

__device__ __forceinline__ f3 camera_dir(const CamView& cam, int px, int py) {
    const float W = (float)cam.width, H = (float)cam.height;
    const float aspect = W / H;
    float sx = (2.f * (px + 0.5f) / W - 1.f) * cam.tan_half_fovy * aspect;
    float sy = (1.f - 2.f * (py + 0.5f) / H) * cam.tan_half_fovy;
    f3 fwd = {cam.fwd.x, cam.fwd.y, cam.fwd.z}, right = {cam.right.x, cam.right.y, cam.right.z};
    f3 up = {cam.up.x, cam.up.y, cam.up.z};
    f3 d = fwd + right * sx + up * sy;
    return d * rsqrtf(dot(d, d));
}

__global__ void __launch_bounds__(128) k_gbuffer(SceneView s, CamView cam, CamView pc, int has_prev,
                                                 GBufView g) {
    int px = blockIdx.x * blockDim.x + threadIdx.x;
    int py = blockIdx.y * blockDim.y + threadIdx.y;
    if (px >= g.width || py >= g.height) return;
    uint32_t pix = (uint32_t)py * g.width + px;
    const float W = (float)cam.width, H = (float)cam.height;
    const float aspect = W / H;
    f3 o = {cam.pos.x, cam.pos.y, cam.pos.z};
    f3 d = camera_dir(cam, px, py);
    // coherent rays: traversal in place, warps stay on the same nodes
    Hit h = trace_bvh<false>(s, Ray{o, d, DDGI_T_EPS, DDGI_MISS_T});
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = make_float4(0.f, 0.f, 0.f, __uint_as_float(DDGI_NONE));
    float4 g2 = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    if (h.tri != DDGI_NONE) {
        f3 n = xyz(__ldg(s.nrm + h.tri));
        if (dot(n, d) <= 0.f) {
            f3 p = o + d * h.t;
            f3 a = xyz(__ldg(s.alb + h.tri));
            int prev = -1;
            if (has_prev) {
                bool moving;
                f3 v = prev_position(s, h.tri, p, &moving) - f3{pc.pos.x, pc.pos.y, pc.pos.z};
                float z = dot(v, f3{pc.fwd.x, pc.fwd.y, pc.fwd.z});
                if (z > 0.f) {
                    float qx = dot(v, f3{pc.right.x, pc.right.y, pc.right.z}) / z / (pc.tan_half_fovy * aspect);
                    float qy = dot(v, f3{pc.up.x, pc.up.y, pc.up.z}) / z / pc.tan_half_fovy;
                    float fx = (qx + 1.f) * 0.5f * W, fy = (1.f - qy) * 0.5f * H;
                    if (fx >= 0.f && fy >= 0.f && fx < W && fy < H)
                        prev = ((int)floorf(fy) * cam.width + (int)floorf(fx)) | (moving ? DDGI_PREV_MOVING : 0);
                }
            }
            g0 = make_float4(p.x, p.y, p.z, h.t);
            g1 = make_float4(n.x, n.y, n.z, __uint_as_float(h.tri));
            g2 = make_float4(a.x, a.y, a.z, __int_as_float(prev));
        }
    }
    g.g0[pix] = g0;
    g.g1[pix] = g1;
    g.g2[pix] = g2;
}

// shadow rays toward each pixel's selected sample, work item = pixel
struct ShadowGen {
    GBufView g;
    ResView r;
    __device__ __forceinline__ bool ray(uint32_t pix, Ray& ry) const {
        ry.tmax = 0.f;
        float4 g1 = g.g1[pix];
        if (__float_as_uint(g1.w) == DDGI_NONE) return false;
        // an empty reservoir has W = 0: the first half of the record decides
        const float4 r0 = __ldg(r.rec + 4 * (size_t)pix);
        if (!(r0.w > 0.f)) return false;
        f3 x = xyz(g.g0[pix]);
        f3 d = xyz(r0) - x;
        float d2 = dot(d, d);
        if (!(d2 > 0.f)) return false;
        float l = sqrtf(d2);
        f3 w = d * (1.f / l);
        if (!(dot(xyz(g1), w) > 0.f)) return false;
        ry.o = x;
        ry.d = w;
        ry.tmin = DDGI_T_EPS;
        ry.tmax = (1.f - 1e-4f) * l;
        return true;
    }
};

// network query at each visible selected sample (learned target form)
struct ShadeQuery {
    SceneView s;
    GBufView g;
    ResView r;
    const float2* vis;
    float4* ind;
    __device__ bool query(uint32_t pix, f3& p, f3& n) const {
        if (__float_as_uint(g.g1[pix].w) == DDGI_NONE) return false;
        const float4* rec = r.rec + 4 * (size_t)pix;
        float4 r0 = __ldg(rec);
        uint32_t ty = __float_as_uint(__ldg(rec + 3).x);
        if (ty == DDGI_NONE || !(r0.w > 0.f)) return false;
        if (__float_as_uint(vis[pix].y) != DDGI_NONE) return false;
        f3 ny = xyz(__ldg(s.nrm + ty));
        if (!(dot(ny, xyz(g.g0[pix]) - xyz(r0)) > 0.f) || !any_pos(xyz(__ldg(s.alb + ty)))) return false;
        p = xyz(r0);
        n = ny;
        return true;
    }
    __device__ void store(uint32_t pix, bool valid, f3 f) const {
        if (!valid) {
            ind[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
            return;
        }
        f3 rho = xyz(__ldg(s.alb + __float_as_uint(__ldg(r.rec + 4 * (size_t)pix + 3).x)));
        ind[pix] = make_float4(rho.x * fmaxf(f.x, 0.f), rho.y * fmaxf(f.y, 0.f), rho.z * fmaxf(f.z, 0.f), 1.f);
    }
};

// Radiance at the selected sample y (triangle tri) toward the shaded point x1
// (normal n1, camera at eye) with the specular recursion of Sec. 3.3: at each
// path vertex x_n (n >= 2) the emission and the diffuse half rho / pi E are
// added; the glossy half is estimated by one sample of Eq. lddgiplus once the
// path footprint a(x1..xn) exceeds c a0 (or at the last of SHADE_MAX_VERTS
// vertices), else traced on along the sampled direction.  The footprint
// (Bekaert et al., as the paper adopts it): sqrt(a) is the sum over the
// path's segments of sqrt(|x_i - x_{i+1}|^2 / (p_i <n_{i+1}, -w_i>)), p_1 the
// Lambertian density cos / pi at x1, p_i the glossy density beyond;
// a0 = |x0 - x1|^2 / (4 pi <n1, -w0>).  Keys: (seed, pixel, frame,
// PASS_SHADE, vertex n, dimension 0 / 1).
__device__ f3 shade_radiance(const SceneView& s, const VolumeView& v, const ShadeParams& sp, f3 eye, f3 x1, f3 n1,
                             f3 y, uint32_t tri, uint32_t pix) {
    const f3 e0 = eye - x1, d1 = y - x1;
    const float l0 = length(e0), l1 = length(d1);
    const float a0 = l0 * l0 / (4.f * DDGI_PI * (dot(n1, e0) / l0));
    const float alim = sp.footprint_c * a0;
    const f3 w1 = d1 * (1.f / l1);
    const float p1 = dot(n1, w1) * (1.f / DDGI_PI);
    float sa = sqrtf(l1 * l1 / (p1 * fabsf(dot(xyz(__ldg(s.nrm + tri)), w1))));
    const uint32_t prefix = rng_prefix(sp.seed, pix, sp.frame, PASS_SHADE);
    f3 thr = {1.f, 1.f, 1.f}, L = {0.f, 0.f, 0.f}, prev = x1, cur = y;
    uint32_t t = tri;
#pragma unroll 1
    for (int n = 2;; ++n) {
        const f3 nrm = xyz(__ldg(s.nrm + t));
        const f3 back = prev - cur;
        if (dot(nrm, back) <= 0.f) break;
        L = L + mul(thr, xyz(__ldg(s.emi + t)));
        const f3 rho = xyz(__ldg(s.alb + t));
        const float4 spec = __ldg(s.spec + t);
        const bool glossy = is_glossy(spec);
        if (!any_pos(rho) && !glossy) break;
        const f3 q = biased_point(v, cur, prev);
        if (any_pos(rho)) L = L + mul(thr, mul(rho, ddgi_irradiance(v, q, nrm))) * (1.f / DDGI_PI);
        if (!glossy) break;
        const uint32_t cp = rng_cand(prefix, (uint32_t)n);
        const f3 wo = back * rsqrtf(dot(back, back));
        f3 wi;
        float g, pdf;
        if (!glossy_sample(nrm, wo, spec.w, u01(rng_u32_dim(cp, 0)), u01(rng_u32_dim(cp, 1)), wi, g, pdf)) break;
        const f3 wgt = xyz(spec) * g;
        if (sp.footprint_c < 0.f || sa * sa > alim || n >= SHADE_MAX_VERTS) {
            L = L + mul(thr, mul(wgt, ddgi_irradiance(v, q, wi))) * (1.f / DDGI_PI);
            break;
        }
        const Hit h = trace_bvh<false>(s, Ray{cur, wi, DDGI_T_EPS, DDGI_MISS_T});
        if (h.tri == DDGI_NONE) break;
        const float c3 = -dot(xyz(__ldg(s.nrm + h.tri)), wi);
        if (!(c3 > 0.f)) break;
        sa += sqrtf(h.t * h.t / (pdf * c3));
        thr = mul(thr, wgt);
        prev = cur;
        cur = cur + wi * h.t;
        t = h.tri;
    }
    return L;
}

template <bool GLOSSY>
__device__ __forceinline__ void shade_pixel(SceneView s, VolumeView v, GBufView g, ResView r,
                                            const float4* __restrict__ resid, float4* __restrict__ radiance,
                                            const float2* __restrict__ vis, const float4* __restrict__ ind,
                                            const MLPState* __restrict__ mst, ShadeParams sp) {
    // rows bottom-up: the shadow-ray pass read the pixels' planes top-down,
    // so its last rows are still in L2
    int px = blockIdx.x * blockDim.x + threadIdx.x;
    int py = (gridDim.y - 1 - blockIdx.y) * blockDim.y + threadIdx.y;
    if (px >= g.width || py >= g.height) return;
    uint32_t pix = (uint32_t)py * g.width + px;
    float4 g1 = g.g1[pix];
    uint32_t xtri = __float_as_uint(g1.w);
    if (xtri == DDGI_NONE) {
        radiance[pix] = make_float4(0.f, 0.f, 0.f, 1.f);
        return;
    }
    float4 g0 = g.g0[pix], g2 = g.g2[pix];
    const f3 x = xyz(g0), nx = xyz(g1), rho = xyz(g2);
    f3 out = xyz(__ldg(s.emi + xtri)) + xyz(resid[pix]);
    const float4* rec = r.rec + 4 * (size_t)pix;
    float4 r0 = __ldg(rec);
    uint32_t ty = __float_as_uint(__ldg(rec + 3).x);
    if (ty != DDGI_NONE && r0.w > 0.f) {
        f3 y = xyz(r0);
        f3 d = y - x;
        float d2 = dot(d, d);
        if (d2 > 0.f) {
            float l = sqrtf(d2);
            f3 w = d * (1.f / l);
            float cx = dot(nx, w);
            if (cx > 0.f) {
                if (__float_as_uint(__ldg(vis + pix).y) == DDGI_NONE) {
                    f3 L;
                    if (mst != nullptr && mst->use_mlp) {
                        bool front = dot(xyz(__ldg(s.nrm + ty)), x - y) > 0.f;
                        L = front ? xyz(__ldg(s.emi + ty)) + xyz(__ldg(ind + pix)) : f3{0.f, 0.f, 0.f};
                    } else if constexpr (GLOSSY) {
                        L = shade_radiance(s, v, sp, f3{g.eye.x, g.eye.y, g.eye.z}, x, nx, y, ty, pix);
                    } else {
                        L = radiance_at(s, v, y, ty, x);
                    }
                    float cy = fabsf(dot(xyz(__ldg(s.nrm + ty)), w));
                    float G = cx * cy / d2;
                    out = out + mul(rho, L) * (fminf(G, 1.f) * r0.w * (1.f / DDGI_PI));
                }
            }
        }
    }
    radiance[pix] = make_float4(out.x, out.y, out.z, 1.f);
}

// Diffuse shading at eight CTAs per SM (64 registers, 4 bytes of spill:
// -3 us against seven at 72); the glossy form, whose recursion's traversal
// would spill 256 bytes there (and ran 45 us slower at four CTAs and 122
// registers), keeps the compiler's choice (96).
__global__ void __launch_bounds__(128, 8) k_shade(SceneView s, VolumeView v, GBufView g, ResView r,
                                                  const float4* __restrict__ resid, float4* __restrict__ radiance,
                                                  const float2* __restrict__ vis, const float4* __restrict__ ind,
                                                  const MLPState* __restrict__ mst, ShadeParams sp) {
    shade_pixel<false>(s, v, g, r, resid, radiance, vis, ind, mst, sp);
}
__global__ void __launch_bounds__(128) k_shade_glossy(SceneView s, VolumeView v, GBufView g, ResView r,
                                                      const float4* __restrict__ resid,
                                                      float4* __restrict__ radiance, const float2* __restrict__ vis,
                                                      const float4* __restrict__ ind,
                                                      const MLPState* __restrict__ mst, ShadeParams sp) {
    shade_pixel<true>(s, v, g, r, resid, radiance, vis, ind, mst, sp);
}

inline dim3 tile_grid(int w, int h, dim3 b) { return dim3((w + b.x - 1) / b.x, (h + b.y - 1) / b.y); }

}  // namespace

cudaError_t launch_gbuffer(const SceneView& s, const CamView& cam, const CamView* prev,
                           const GBufView& g, float2* hits, uint32_t* counter, cudaStream_t st) {
    if (g.width == 0 || g.height == 0) return cudaSuccess;
    dim3 b(16, 8);
    k_gbuffer<<<tile_grid(g.width, g.height, b), b, 0, st>>>(s, cam, prev ? *prev : cam, prev != nullptr, g);
    return cudaGetLastError();
}

cudaError_t launch_shade(const SceneView& s, const VolumeView& v, const GBufView& g,
                         const ResView& r, const float4* resid, float4* radiance, float2* hits,
                         uint32_t* counter, const MLPView* mlp, MLPState* mst, float4* ind,
                         const ShadeParams& sp, cudaStream_t st) {
    if (g.width == 0 || g.height == 0) return cudaSuccess;
    cudaError_t e = launch_trace<ShadowGen, true>(s, ShadowGen{g, r}, (uint32_t)g.width * g.height,
                                                  counter, hits, st);
    if (e != cudaSuccess) return e;
    if (mlp) {
        e = launch_mlp_infer(*mlp, ShadeQuery{s, g, r, hits, ind}, (uint32_t)g.width * g.height, st);
        if (e != cudaSuccess) return e;
    }
    dim3 b(32, 4);   // measured best for this kernel (16 x 8 slower)
    if (s.spec)
        k_shade_glossy<<<tile_grid(g.width, g.height, b), b, 0, st>>>(s, v, g, r, resid, radiance, hits, ind,
                                                                      mlp ? mst : nullptr, sp);
    else
        k_shade<<<tile_grid(g.width, g.height, b), b, 0, st>>>(s, v, g, r, resid, radiance, hits, ind,
                                                               mlp ? mst : nullptr, sp);
    return cudaGetLastError();
}
