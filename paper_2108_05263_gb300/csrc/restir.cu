// Reservoir resampling of Sec. 3.1 step 2 with candidates of step 1: the
// initial candidates on all surfaces (emitter points + BSDF rays, Sec. 3.5
// residual), temporal reuse and spatial reuse with the cached probe query of
// Sec. 3.6.  One thread per pixel; SoA planes read and written as 16-byte
// records.
#include "internal.h"
#include "trace.cuh"

namespace {

struct Sel {
    f3 y, L;
    uint32_t tri, tag;
    float p;   // target at the owning pixel
};

__device__ __forceinline__ uint32_t sample_emitter(const SceneView& s, float u) {
    // first emitter whose cumulative area exceeds u * total: start at the
    // guide entry of u (never past the answer) and scan forward
    const uint32_t E = s.num_emitters;
    const float target = u * __ldg(s.cdf + E - 1);
    uint32_t j = min((uint32_t)(u * (float)s.guide_size), s.guide_size - 1);
    uint32_t i = __ldg(s.guide + j);
    while (i < E - 1 && !(target < __ldg(s.cdf + i))) ++i;
    return i;
}

// orthonormal basis around n (Duff et al., JCGT 2017)
__device__ __forceinline__ f3 onb_to_world(f3 n, float lx, float ly, float lz) {
    float sign = n.z >= 0.f ? 1.f : -1.f;
    float a = -1.f / (sign + n.z);
    float b = n.x * n.y * a;
    f3 t = {1.f + sign * n.x * n.x * a, sign * b, -sign * n.x};
    f3 bt = {b, sign + n.y * n.y * a, -n.y};
    return t * lx + bt * ly + n * lz;
}

__global__ void __launch_bounds__(128) k_restir_initial(SceneView s, VolumeView v, RestirParams rp,
                                                        GBufView g, ResView out,
                                                        float4* __restrict__ resid, uint32_t frame) {
    int px = blockIdx.x * blockDim.x + threadIdx.x;
    int py = blockIdx.y * blockDim.y + threadIdx.y;
    if (px >= g.width || py >= g.height) return;
    uint32_t pix = (uint32_t)py * g.width + px;
    float4 g1 = g.g1[pix];
    uint32_t xtri = __float_as_uint(g1.w);
    const uint32_t NL = s.num_emitters > 0 ? rp.n_light : 0u;
    const uint32_t NB = rp.n_bsdf;
    const uint32_t M = NL + NB;
    if (xtri == DDGI_NONE) {
        out.r0[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
        out.r1[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
        out.r2[pix] = make_uint2(DDGI_NONE, 0u);
        resid[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float4 g0 = g.g0[pix], g2 = g.g2[pix];
    const f3 x = xyz(g0), nx = xyz(g1), rho = xyz(g2);
    const uint32_t prefix = rng_prefix(rp.seed, pix, frame, PASS_INITIAL);
    const float inv_area = 1.f / s.area_total;
    const float invM = 1.f / (float)M;
    float wsum = 0.f;
    Sel sel;
    sel.tri = DDGI_NONE;
    sel.tag = 0u;
    sel.p = 0.f;
    sel.y = sel.L = f3{0.f, 0.f, 0.f};
    f3 res = {0.f, 0.f, 0.f};
    for (uint32_t c = 0; c < M; ++c) {
        const uint32_t cp = rng_cand(prefix, c);
        f3 y, L;
        float d2, cx, cy, pL;
        uint32_t tri;
        if (c < NL) {
            pL = inv_area;
            float u0 = u01(rng_u32_dim(cp, 0)), u1 = u01(rng_u32_dim(cp, 1));
            float u2 = u01(rng_u32_dim(cp, 2));
            uint32_t e = sample_emitter(s, u0);
            const float4* rec = s.evert + 4 * (size_t)e;
            float4 q0 = __ldg(rec), q1 = __ldg(rec + 1), q2 = __ldg(rec + 2), q3 = __ldg(rec + 3);
            tri = __float_as_uint(q0.w);
            float sq = sqrtf(u1);
            float b1 = sq * (1.f - u2), b2 = sq * u2;
            y = xyz(q0) + xyz(q1) * b1 + xyz(q2) * b2;
            f3 d = y - x;
            d2 = dot(d, d);
            if (d2 <= 0.f) continue;
            f3 w = d * rsqrtf(d2);
            cx = dot(nx, w);
            f3 ny = xyz(q3);
            float cyn = dot(ny, w);
            cy = fabsf(cyn);
            if (s.emitters_reflect) {
                L = radiance_at(s, v, y, tri, x);
            } else {
                // pure emitter: one-sided Le toward x
                L = cyn < 0.f ? f3{q1.w, q2.w, q3.w} : f3{0.f, 0.f, 0.f};
            }
        } else {
            float u0 = u01(rng_u32_dim(cp, 0)), u1 = u01(rng_u32_dim(cp, 1));
            float r = sqrtf(u0);
            float sn, cs;
            sincospif(2.f * u1, &sn, &cs);
            f3 w = onb_to_world(nx, r * cs, r * sn, sqrtf(fmaxf(0.f, 1.f - u0)));
            Ray ray{x, w, DDGI_T_EPS, DDGI_MISS_T};
            Hit h = trace_bvh<false>(s, ray);
            if (h.tri == DDGI_NONE) continue;
            tri = h.tri;
            pL = __ldg(s.emi + tri).w > 0.f ? inv_area : 0.f;
            y = x + w * h.t;
            d2 = h.t * h.t;
            cx = dot(nx, w);
            cy = fabsf(dot(xyz(__ldg(s.nrm + tri)), w));
            L = radiance_at(s, v, y, tri, x);
            if (cx > 0.f) {
                float G = cx * cy / d2;
                if (G > 1.f) res = res + mul(rho, L) * ((1.f - 1.f / G) / (float)NB);
            }
        }
        if (cx <= 0.f) continue;
        float pB = cx * (1.f / DDGI_PI) * cy / d2;
        float pmix = ((float)NL * pL + (float)NB * pB) * invM;
        float G = cx * cy / d2;
        float ph = luminance(mul(rho, L)) * (fminf(G, 1.f) * (1.f / DDGI_PI));
        float wc = pmix > 0.f ? ph / pmix : 0.f;
        wsum += wc;
        float u3 = u01(rng_u32_dim(cp, 3));
        if (wc > 0.f && u3 * wsum < wc) {
            sel.y = y;
            sel.L = L;
            sel.tri = tri;
            sel.tag = pix * 64u + c;
            sel.p = ph;
        }
    }
    resid[pix] = make_float4(res.x, res.y, res.z, 0.f);
    if (sel.tri == DDGI_NONE) {
        out.r0[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
        out.r1[pix] = make_float4(0.f, 0.f, 0.f, (float)M);
        out.r2[pix] = make_uint2(DDGI_NONE, 0u);
        return;
    }
    float W = sel.p > 0.f ? wsum / ((float)M * sel.p) : 0.f;
    out.r0[pix] = make_float4(sel.y.x, sel.y.y, sel.y.z, W);
    out.r1[pix] = make_float4(sel.L.x, sel.L.y, sel.L.z, (float)M);
    out.r2[pix] = make_uint2(sel.tri, sel.tag);
}

__device__ __forceinline__ float res_target(const SceneView& s, f3 x, f3 nx, f3 rho, float4 r0,
                                            float4 r1, uint32_t tri) {
    return target_fn(s, x, nx, rho, xyz(r0), tri, xyz(r1));
}

__global__ void __launch_bounds__(256) k_restir_temporal(SceneView s, RestirParams rp, GBufView g,
                                                         GBufView gp, float3 cam_prev, ResView cur,
                                                         ResView prev, ResView out, uint32_t frame) {
    int px = blockIdx.x * blockDim.x + threadIdx.x;
    int py = blockIdx.y * blockDim.y + threadIdx.y;
    if (px >= g.width || py >= g.height) return;
    uint32_t pix = (uint32_t)py * g.width + px;
    float4 c0 = cur.r0[pix], c1 = cur.r1[pix];
    uint2 c2 = cur.r2[pix];
    float4 g1 = g.g1[pix];
    float4 g2 = g.g2[pix];
    int pq = __float_as_int(g2.w);
    bool merge = __float_as_uint(g1.w) != DDGI_NONE && pq >= 0 &&
                 pq < gp.width * gp.height;
    float4 p0, p1;
    uint2 p2;
    float4 g0;
    if (merge) {
        float4 h1 = gp.g1[pq];
        g0 = g.g0[pix];
        merge = __float_as_uint(h1.w) != DDGI_NONE &&
                dot(xyz(g1), xyz(h1)) > rp.normal_reject_cos;
        if (merge) {
            f3 dv = xyz(g0) - f3{cam_prev.x, cam_prev.y, cam_prev.z};
            float de = length(dv);
            float dp = gp.g0[pq].w;
            merge = fabsf(de - dp) <= rp.depth_reject_frac * de;
        }
    }
    if (!merge) {
        out.r0[pix] = c0;
        out.r1[pix] = c1;
        out.r2[pix] = c2;
        return;
    }
    p0 = prev.r0[pq];
    p1 = prev.r1[pq];
    p2 = prev.r2[pq];
    const f3 x = xyz(g0), nx = xyz(g1), rho = xyz(g2);
    float Mc = c1.w;
    float Mp = fminf(p1.w, rp.temporal_mcap * Mc);
    float pc = res_target(s, x, nx, rho, c0, c1, c2.x);
    float wsum = pc * c0.w * Mc;
    float pp = res_target(s, x, nx, rho, p0, p1, p2.x);
    float wp = pp * p0.w * Mp;
    wsum += wp;
    uint32_t h = rng_u32_dim(rng_cand(rng_prefix(rp.seed, pix, frame, PASS_TEMPORAL), 0u), 0u);
    float u = u01(h);
    float psel = pc;
    if (wp > 0.f && u * wsum < wp) {
        c0 = p0;
        c1 = p1;
        c2 = p2;
        psel = pp;
    }
    float Mo = Mc + Mp;
    c0.w = psel > 0.f ? wsum / (Mo * psel) : 0.f;
    c1.w = Mo;
    out.r0[pix] = c0;
    out.r1[pix] = c1;
    out.r2[pix] = c2;
}

__global__ void __launch_bounds__(128) k_restir_spatial(SceneView s, RestirParams rp, GBufView g,
                                                        ResView in, ResView out, uint32_t frame,
                                                        uint32_t pass) {
    int px = blockIdx.x * blockDim.x + threadIdx.x;
    int py = blockIdx.y * blockDim.y + threadIdx.y;
    if (px >= g.width || py >= g.height) return;
    uint32_t pix = (uint32_t)py * g.width + px;
    float4 s0 = in.r0[pix], s1 = in.r1[pix];
    uint2 s2 = in.r2[pix];
    float4 g1 = g.g1[pix];
    if (__float_as_uint(g1.w) == DDGI_NONE) {
        out.r0[pix] = s0;
        out.r1[pix] = s1;
        out.r2[pix] = s2;
        return;
    }
    float4 g0 = g.g0[pix], g2 = g.g2[pix];
    const f3 x = xyz(g0), nx = xyz(g1), rho = xyz(g2);
    const float dist = g0.w;
    float psel = res_target(s, x, nx, rho, s0, s1, s2.x);
    float wsum = psel * s0.w * s1.w;
    float M = s1.w;
    const uint32_t prefix = rng_prefix(rp.seed, pix, frame, PASS_SPATIAL0 + pass);
    const int R = (int)rp.spatial_radius;
    const uint32_t span = 2u * rp.spatial_radius + 1u;
    for (uint32_t j = 0; j < rp.spatial_neighbours; ++j) {
        const uint32_t cp = rng_cand(prefix, j);
        int dx = 0, dy = 0;
        bool ok = false;
        for (uint32_t a = 0; a < 8u; ++a) {
            uint32_t h = rng_u32_dim(cp, a);
            int ox = (int)((h & 0xFFFFu) % span) - R;
            int oy = (int)((h >> 16) % span) - R;
            if ((ox != 0 || oy != 0) && ox * ox + oy * oy <= R * R) {
                dx = ox;
                dy = oy;
                ok = true;
                break;
            }
        }
        if (!ok) continue;
        int qx = px + dx, qy = py + dy;
        if (qx < 0 || qy < 0 || qx >= g.width || qy >= g.height) continue;
        uint32_t q = (uint32_t)qy * g.width + qx;
        float4 h1 = g.g1[q];
        if (__float_as_uint(h1.w) == DDGI_NONE) continue;
        if (dot(nx, xyz(h1)) <= rp.normal_reject_cos) continue;
        if (fabsf(dist - g.g0[q].w) > rp.depth_reject_frac * dist) continue;
        float4 n0 = in.r0[q], n1 = in.r1[q];
        uint2 n2 = in.r2[q];
        float pn = res_target(s, x, nx, rho, n0, n1, n2.x);
        float wn = pn * n0.w * n1.w;
        wsum += wn;
        M += n1.w;
        float u = u01(rng_u32_dim(cp, 8u));
        if (wn > 0.f && u * wsum < wn) {
            s0 = n0;
            s1 = n1;
            s2 = n2;
            psel = pn;
        }
    }
    s0.w = psel > 0.f ? wsum / (M * psel) : 0.f;
    s1.w = M;
    out.r0[pix] = s0;
    out.r1[pix] = s1;
    out.r2[pix] = s2;
}

inline dim3 tile_grid(int w, int h, dim3 b) { return dim3((w + b.x - 1) / b.x, (h + b.y - 1) / b.y); }

}  // namespace

cudaError_t launch_restir_initial(const SceneView& s, const VolumeView& v, const RestirParams& rp,
                                  const GBufView& g, const ResView& out, float4* resid,
                                  uint32_t frame, cudaStream_t st) {
    if (g.width == 0 || g.height == 0) return cudaSuccess;
    dim3 b(16, 8);
    k_restir_initial<<<tile_grid(g.width, g.height, b), b, 0, st>>>(s, v, rp, g, out, resid, frame);
    return cudaGetLastError();
}

cudaError_t launch_restir_temporal(const SceneView& s, const RestirParams& rp, const GBufView& g,
                                   const GBufView& gp, float3 prev_cam, const ResView& cur,
                                   const ResView& prev, const ResView& out, uint32_t frame,
                                   cudaStream_t st) {
    if (g.width == 0 || g.height == 0) return cudaSuccess;
    dim3 b(32, 8);
    k_restir_temporal<<<tile_grid(g.width, g.height, b), b, 0, st>>>(s, rp, g, gp, prev_cam, cur,
                                                                      prev, out, frame);
    return cudaGetLastError();
}

cudaError_t launch_restir_spatial(const SceneView& s, const RestirParams& rp, const GBufView& g,
                                  const ResView& in, const ResView& out, uint32_t frame,
                                  uint32_t pass, cudaStream_t st) {
    if (g.width == 0 || g.height == 0) return cudaSuccess;
    dim3 b(16, 8);
    k_restir_spatial<<<tile_grid(g.width, g.height, b), b, 0, st>>>(s, rp, g, in, out, frame, pass);
    return cudaGetLastError();
}
