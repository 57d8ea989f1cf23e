// Device-side building blocks shared by the kernels: vector math, the
// counter-based random numbers, octahedral probe maps and the views of the
// scene / probe volume that kernels receive by value.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cfloat>

#define DDGI_PI 3.14159265358979323846f
#define DDGI_T_EPS 1e-4f
#define DDGI_MISS_T 1e30f
#define DDGI_NONE 0xFFFFFFFFu

// random-number pass ids (keys of the hash chain)
#define PASS_INITIAL 0u
#define PASS_SPATIAL0 1u
#define PASS_TEMPORAL 5u
#define PASS_PROBE_ROT 7u
#define PASS_SHADE 12u          // glossy directions of the shading recursion (candidate = path vertex)
#define PASS_PROBE_GLOSSY 13u   // glossy direction at a probe ray's hit (pixel = probe, candidate = ray)
#define SHADE_MAX_VERTS 8       // path vertices of the shading recursion, the shaded point included

// device error word bits
#define TRAV_MAX_VISITS (1 << 16)   // default node-visit cap of one ray's traversal
#define ERRBIT_TRAVERSAL 1u
#define ERRBIT_STACK 2u
#define ERRBIT_MMA_WAIT 4u   // a tensor-core completion wait ran past its bound

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 mk(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ f3 xyz(float4 a) { return {a.x, a.y, a.z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator-(f3 a) { return {-a.x, -a.y, -a.z}; }
__device__ __forceinline__ f3 operator*(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ f3 operator*(float s, f3 a) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ f3 mul(f3 a, f3 b) { return {a.x * b.x, a.y * b.y, a.z * b.z}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float length(f3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ float luminance(f3 c) { return 0.2126f * c.x + 0.7152f * c.y + 0.0722f * c.z; }
__device__ __forceinline__ bool any_pos(f3 c) { return c.x > 0.f || c.y > 0.f || c.z > 0.f; }

// ---------------------------------------------------------------------------
// PCG hash (Jarzynski & Olano, JCGT 2020) chained over the key tuple
// (seed, pixel, frame, pass, candidate, dimension).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
    uint32_t state = v * 747796405u + 2891336453u;
    uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}
// prefix of the chain up to the pass id; candidate and dimension follow
__device__ __forceinline__ uint32_t rng_prefix(uint32_t seed, uint32_t pixel, uint32_t frame,
                                               uint32_t pass) {
    uint32_t h = pcg_hash(seed);
    h = pcg_hash(h + pixel);
    h = pcg_hash(h + frame);
    return pcg_hash(h + pass);
}
__device__ __forceinline__ uint32_t rng_cand(uint32_t prefix, uint32_t cand) {
    return pcg_hash(prefix + cand);
}
__device__ __forceinline__ uint32_t rng_u32_dim(uint32_t cprefix, uint32_t dim) {
    return pcg_hash(cprefix + dim);
}
__device__ __forceinline__ float u01(uint32_t h) { return (float)(h >> 8) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------------------
// views passed to kernels by value
// ---------------------------------------------------------------------------
struct SceneView {
    const float4* nodes;     // BVH4 nodes, 8 float4 each
    const float4* tris;      // BVH-ordered triangles: (v0, orig idx bits), e1, e2
    const float4* nrm;       // per original triangle: unit normal, 0
    const float4* alb;       // albedo rgb, 0
    const float4* emi;       // emission rgb, emissive flag (1/0)
    const float* cdf;        // cumulative emitter area (float), [num_emitters]
    const uint32_t* etri;    // emitter triangle ids
    const float4* evert;     // per emitter: (v0, tri), (e1, Le.r), (e2, Le.g), (n, Le.b)
    const float4* evert3;    // the same without the normal and triangle: (v0, Le.b), (e1, Le.r), (e2, Le.g)
    const uint32_t* guide;   // emitter search start per 1/guide_size of the area
    uint32_t guide_size;
    uint32_t emitters_reflect;   // some emitter has albedo > 0
    uint32_t num_emitters;
    float area_total;
    uint32_t* err;           // device error word
    const int* tri_inst;     // rigid instance of each original triangle (-1 static); null: static scene
    uint32_t num_tris;
    const float4* inst_delta;   // per instance: rows of M_prev M_cur^-1 (current -> previous pose)
    int max_visits;             // BVH nodes one ray may visit (traversal_visit_cap)
    const float4* spec;         // per original triangle: glossy k_s.rgb, GGX alpha; null: a diffuse scene
};

// bit of the G-buffer's previous-pixel word marking a surface on a rigid
// instance (its previous position is M_prev M_cur^-1 x)
#define DDGI_PREV_MOVING 0x40000000

// previous-pose position of a point x on triangle tri
__device__ __forceinline__ f3 prev_position(const SceneView& s, uint32_t tri, f3 x, bool* moving) {
    *moving = false;
    if (!s.tri_inst || tri >= s.num_tris) return x;
    const int k = __ldg(s.tri_inst + tri);
    if (k < 0) return x;
    *moving = true;
    const float4 r0 = __ldg(s.inst_delta + 3 * k), r1 = __ldg(s.inst_delta + 3 * k + 1),
                 r2 = __ldg(s.inst_delta + 3 * k + 2);
    return {r0.x * x.x + r0.y * x.y + r0.z * x.z + r0.w, r1.x * x.x + r1.y * x.y + r1.z * x.z + r1.w,
            r2.x * x.x + r2.y * x.y + r2.z * x.z + r2.w};
}

struct VolumeView {
    float4* irr;             // [P][ti*ti] rgb, 0
    float2* depth;           // [P][td*td] mean, mean square
    // the query's copies: for each 2x2 block of a padded tile (top-left
    // texel (x0, y0), 0 <= x0, y0 <= n, block y0 * (n + 1) + x0) its four
    // bilinear taps (x0, y0), (x0 + 1, y0), (x0, y0 + 1), (x0 + 1, y0 + 1),
    // so that a probe's taps are one 32-byte (distance) and two 32-byte
    // (irradiance) loads; rebuilt from irr / depth whenever those change
    float4* irr_q;           // [P][(irr_n + 1)^2][4] rgb, 0
    float4* depth_q;         // [P][(depth_n + 1)^2][2] (mean, mean square) x 2 per float4
    const float4* offset;    // [P] xyz, 0
    int has_offset;          // 0 while every offset is zero (they are then not read)
    float3 origin, spacing;
    int3 counts;
    int irr_n, depth_n;      // interior texels per side
    float min_spacing, max_spacing;
};

// 32-byte (256-bit) accesses: one L1 sector access per record half
__device__ __forceinline__ void ld32(const float4* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// the same, issued where written (a load whose result the next loop
// iteration consumes: the request goes out before this iteration's work)
__device__ __forceinline__ void ld32_issue(const float4* p, float4& a, float4& b) {
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}
__device__ __forceinline__ void ld16_issue(const float4* p, float4& a) {
    asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w) : "l"(p));
}

// the same from L2 only (scattered neighbour records: L1 seldom hits), issued
// where written so that the loads start before the arithmetic that follows
__device__ __forceinline__ void ld32_l2(const float4* p, float4& a, float4& b) {
    asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}

__device__ __forceinline__ void st32(float4* p, float4 a, float4 b) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a.x), "f"(a.y),
                 "f"(a.z), "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

// ---------------------------------------------------------------------------
// octahedral maps with a one-texel border
// ---------------------------------------------------------------------------
__device__ __forceinline__ float signnz(float x) { return x >= 0.f ? 1.f : -1.f; }

__device__ __forceinline__ float2 oct_encode(f3 d) {
    float s = fabsf(d.x) + fabsf(d.y) + fabsf(d.z);
    float u = d.x / s, v = d.y / s;
    if (d.z < 0.f) {
        float fu = (1.f - fabsf(v)) * signnz(u);
        float fv = (1.f - fabsf(u)) * signnz(v);
        u = fu;
        v = fv;
    }
    return make_float2(u, v);
}

__device__ __forceinline__ f3 oct_decode(float u, float v) {
    float z = 1.f - fabsf(u) - fabsf(v);
    float x = u, y = v;
    if (z < 0.f) {
        x = (1.f - fabsf(v)) * signnz(u);
        y = (1.f - fabsf(u)) * signnz(v);
    }
    float l = rsqrtf(x * x + y * y + z * z);
    return {x * l, y * l, z * l};
}

__device__ __forceinline__ f3 texel_dir(int i, int j, int n) {
    return oct_decode(2.f * (i + 0.5f) / n - 1.f, 2.f * (j + 0.5f) / n - 1.f);
}

// bilinear taps of a padded (n+2)^2 tile in direction d: the 2x2 block of
// the query's copy (VolumeView) and the weights within it
struct Taps {
    int q00;   // index of the 2x2 tap block (top-left tap (x0, y0): y0 * (n + 1) + x0)
    float ax, ay;
};
__device__ __forceinline__ Taps oct_taps(f3 d, int n) {
    float2 uv = oct_encode(d);
    float fx = (uv.x + 1.f) * 0.5f * n + 0.5f;
    float fy = (uv.y + 1.f) * 0.5f * n + 0.5f;
    float x0f = floorf(fx), y0f = floorf(fy);
    Taps t;
    t.ax = fx - x0f;
    t.ay = fy - y0f;
    // |u| + |v| <= 1 puts fx and fy in [0.5, n + 0.5] (a fast reciprocal in
    // oct_encode can pass 1 by an ulp, which moves neither floor): the clamps
    // only keep the taps of a NaN direction inside the tile
    const int x0 = min(max((int)x0f, 0), n), y0 = min(max((int)y0f, 0), n);
    t.q00 = y0 * (n + 1) + x0;
    return t;
}

// bilinear blend of the four taps (a, b: row y0; c, e: row y0 + 1)
__device__ __forceinline__ float2 bilerp2(const Taps& t, float2 a, float2 b, float2 c, float2 e) {
    float w00 = (1.f - t.ax) * (1.f - t.ay), w10 = t.ax * (1.f - t.ay);
    float w01 = (1.f - t.ax) * t.ay, w11 = t.ax * t.ay;
    return make_float2(w00 * a.x + w10 * b.x + w01 * c.x + w11 * e.x,
                       w00 * a.y + w10 * b.y + w01 * c.y + w11 * e.y);
}

// distance moments in direction d from a probe's 2x2 tap blocks
// (depth_q + p * (n + 1)^2 * 2): one 32-byte load
__device__ __forceinline__ float2 sample_depth_q(const float4* blocks, int n, f3 d) {
    Taps t = oct_taps(d, n);
    float4 ab, ce;
    ld32(blocks + 2 * (size_t)t.q00, ab, ce);
    return bilerp2(t, make_float2(ab.x, ab.y), make_float2(ab.z, ab.w), make_float2(ce.x, ce.y),
                   make_float2(ce.z, ce.w));
}

__device__ __forceinline__ f3 probe_pos(const VolumeView& v, int i, int j, int k, int p) {
    const float4 o = v.has_offset ? __ldg(v.offset + p) : make_float4(0.f, 0.f, 0.f, 0.f);
    return {v.origin.x + v.spacing.x * i + o.x, v.origin.y + v.spacing.y * j + o.y,
            v.origin.z + v.spacing.z * k + o.z};
}

// ---------------------------------------------------------------------------
// probe query: irradiance E(q, n) blended from the 8 surrounding probes
// (trilinear x wrap shading x cubed Chebyshev visibility, crushed below 0.2)
// ---------------------------------------------------------------------------
// U: unroll factor of the loop over the 8 probes (kernels differ in which
// register / latency balance suits them)
template <int U = 1>
__device__ __forceinline__ f3 ddgi_irradiance(const VolumeView& v, f3 q, f3 n) {
    float g[3] = {(q.x - v.origin.x) / v.spacing.x, (q.y - v.origin.y) / v.spacing.y,
                  (q.z - v.origin.z) / v.spacing.z};
    int cnt[3] = {v.counts.x, v.counts.y, v.counts.z};
    int base[3];
    float al[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int hi = max(cnt[a] - 2, 0);
        float f = floorf(g[a]);
        int b = f < 0.f ? 0 : (f > (float)hi ? hi : (int)f);
        base[a] = b;
        al[a] = cnt[a] > 1 ? fminf(fmaxf(g[a] - (float)b, 0.f), 1.f) : 0.f;
    }
    const int qi = (v.irr_n + 1) * (v.irr_n + 1), qd = (v.depth_n + 1) * (v.depth_n + 1);
    // the irradiance taps depend on n only: one set for the 8 probes
    const Taps tn = oct_taps(n, v.irr_n);
    const float n00 = (1.f - tn.ax) * (1.f - tn.ay), n10 = tn.ax * (1.f - tn.ay);
    const float n01 = (1.f - tn.ax) * tn.ay, n11 = tn.ax * tn.ay;
    float sw = 0.f;
    f3 se = {0.f, 0.f, 0.f};
#pragma unroll U
    for (int c = 0; c < 8; ++c) {
        int ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
        int gi = min(base[0] + ox, cnt[0] - 1);
        int gj = min(base[1] + oy, cnt[1] - 1);
        int gk = min(base[2] + oz, cnt[2] - 1);
        float tri = (ox ? al[0] : 1.f - al[0]) * (oy ? al[1] : 1.f - al[1]) *
                    (oz ? al[2] : 1.f - al[2]);
        int p = gi + cnt[0] * (gj + cnt[1] * gk);
        f3 P = probe_pos(v, gi, gj, gk, p);
        f3 dir = P - q;
        float r = length(dir);
        dir = r > 0.f ? dir * (1.f / r) : n;
        float wrap = 0.5f * (dot(dir, n) + 1.f);
        float w = wrap * wrap + 0.2f;
        float2 mom = sample_depth_q(v.depth_q + (size_t)p * qd * 2, v.depth_n, -dir);
        if (r > mom.x) {
            float var = fabsf(mom.y - mom.x * mom.x);
            float dd = r - mom.x;
            float ch = var / (var + dd * dd);
            w *= ch * ch * ch;
        }
        w = fmaxf(w, 1e-6f);
        if (w < 0.2f) w = w * w * w * 25.f;
        w *= tri;
        const float4* blk = v.irr_q + ((size_t)p * qi + tn.q00) * 4;
        float4 a, b, cc, d;
        ld32(blk, a, b);
        ld32(blk + 2, cc, d);
        const f3 e = {n00 * a.x + n10 * b.x + n01 * cc.x + n11 * d.x, n00 * a.y + n10 * b.y + n01 * cc.y + n11 * d.y,
                      n00 * a.z + n10 * b.z + n01 * cc.z + n11 * d.z};
        se = se + e * w;
        sw += w;
    }
    return sw > 0.f ? se * (1.f / sw) : f3{0.f, 0.f, 0.f};
}

// view-path bias (Sec. 3.4): move from y toward the previous vertex `from`
template <int U = 1>
__device__ __forceinline__ f3 ddgi_irradiance_biased(const VolumeView& v, f3 y, f3 n, f3 from) {
    f3 d = from - y;
    float l = length(d);
    f3 q = y;
    if (l > 0.f) {
        float dv = fminf(0.2f * v.min_spacing, 0.5f * l);
        q = y + d * (dv / l);
    }
    return ddgi_irradiance<U>(v, q, n);
}

// outgoing radiance (Le + L_DDGI+)(y, y -> from) of a triangle point
template <int U = 1>
__device__ __forceinline__ f3 radiance_at(const SceneView& s, const VolumeView& v, f3 y,
                                          uint32_t tri, f3 from) {
    f3 n = xyz(__ldg(s.nrm + tri));
    if (dot(n, from - y) <= 0.f) return {0.f, 0.f, 0.f};
    f3 le = xyz(__ldg(s.emi + tri));
    f3 rho = xyz(__ldg(s.alb + tri));
    if (any_pos(rho)) {
        f3 E = ddgi_irradiance_biased<U>(v, y, n, from);
        le = le + mul(rho, E) * (1.f / DDGI_PI);
    }
    return le;
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

// ---------------------------------------------------------------------------
// glossy lobe (Sec. 3.3): per triangle a GGX microfacet lobe with reflectance
// k_s and roughness alpha, f_g = k_s D(h) G1(wo) G1(wi) / (4 |n.wo| |n.wi|)
// (separable Smith masking, no Fresnel term)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ggx_D(float nh, float a) {
    if (nh <= 0.f) return 0.f;
    const float a2 = a * a, den = nh * nh * (a2 - 1.f) + 1.f;
    return a2 / (DDGI_PI * den * den);
}

__device__ __forceinline__ float ggx_G1(float nw, float a) {
    if (nw <= 0.f) return 0.f;
    const float a2 = a * a;
    return 2.f * nw / (nw + sqrtf(a2 + (1.f - a2) * nw * nw));
}

// One direction wi of the glossy lobe around n seen from wo: the mirror of
// wo about a half vector drawn from D(h) (n.h).  Returns false when wi falls
// below the surface; else g = f_g (n.wi) / (k_s pdf) and the density pdf.
__device__ __forceinline__ bool glossy_sample(f3 n, f3 wo, float a, float u0, float u1, f3& wi, float& g,
                                              float& pdf) {
    const float c2 = (1.f - u0) / (1.f + (a * a - 1.f) * u0);
    const float c = sqrtf(c2), sn = sqrtf(fmaxf(0.f, 1.f - c2));
    float sp, cp;
    sincospif(2.f * u1, &sp, &cp);
    const f3 h = onb_to_world(n, sn * cp, sn * sp, c);
    const float oh = dot(wo, h);
    wi = h * (2.f * oh) - wo;
    const float ni = dot(n, wi), no = dot(n, wo), nh = dot(n, h);
    if (!(ni > 0.f && no > 0.f && nh > 0.f && oh > 0.f)) return false;
    pdf = ggx_D(nh, a) * nh / (4.f * oh);
    g = ggx_G1(no, a) * ggx_G1(ni, a) * oh / (no * nh);
    return true;
}

// view-path-biased query point (Sec. 3.4) of y seen from `from`
__device__ __forceinline__ f3 biased_point(const VolumeView& v, f3 y, f3 from) {
    f3 d = from - y;
    float l = length(d);
    if (!(l > 0.f)) return y;
    float dv = fminf(0.2f * v.min_spacing, 0.5f * l);
    return y + d * (dv / l);
}

// The glossy half of Eq. lddgiplus at query point q (normal n, seen from
// wo): one sample wi of the lobe, E(q, wi) read as cosine-prefiltered
// incident radiance around wi, (1 / pi) E(q, wi) f_g (n.wi) / pdf.  With E
// normalised so that uniform radiance L gives pi L, the factor 1 / pi
// reflects a uniform environment exactly.
template <int U = 1>
__device__ __forceinline__ f3 glossy_ddgi(const VolumeView& v, f3 q, f3 n, f3 wo, float4 spec, float u0, float u1) {
    f3 wi;
    float g, pdf;
    if (!glossy_sample(n, wo, spec.w, u0, u1, wi, g, pdf)) return {0.f, 0.f, 0.f};
    const f3 E = ddgi_irradiance<U>(v, q, wi);
    return mul(E, xyz(spec)) * (g * (1.f / DDGI_PI));
}

__device__ __forceinline__ bool is_glossy(float4 spec) { return spec.x > 0.f || spec.y > 0.f || spec.z > 0.f; }

// (Le + L_DDGI+)(y, y -> from) of a glossy scene: radiance_at plus the
// one-sample glossy half drawn with (u0, u1); the same value as radiance_at
// on a triangle without a glossy lobe
template <int U = 1>
__device__ __forceinline__ f3 radiance_at_glossy(const SceneView& s, const VolumeView& v, f3 y, uint32_t tri,
                                                 f3 from, float u0, float u1) {
    const float4 spec = __ldg(s.spec + tri);
    if (!is_glossy(spec)) return radiance_at<U>(s, v, y, tri, from);
    f3 n = xyz(__ldg(s.nrm + tri));
    const f3 back = from - y;
    if (dot(n, back) <= 0.f) return {0.f, 0.f, 0.f};
    f3 L = xyz(__ldg(s.emi + tri));
    const f3 rho = xyz(__ldg(s.alb + tri));
    const f3 q = biased_point(v, y, from);
    if (any_pos(rho)) L = L + mul(rho, ddgi_irradiance<U>(v, q, n)) * (1.f / DDGI_PI);
    return L + glossy_ddgi<U>(v, q, n, back * rsqrtf(dot(back, back)), spec, u0, u1);
}

// target function: luminance of rho_x / pi * L * min(G, 1) for a point y with
// unit normal ny (only |cos| at y enters)
__device__ __forceinline__ float target_at(f3 x, f3 nx, f3 rho, f3 y, f3 ny, f3 L) {
    f3 d = y - x;
    float d2 = dot(d, d);
    if (d2 <= 0.f) return 0.f;
    float inv = rsqrtf(d2);
    f3 w = d * inv;
    float cx = dot(nx, w);
    if (cx <= 0.f) return 0.f;
    float cy = fabsf(dot(ny, w));
    float G = cx * cy / d2;
    float Gb = fminf(G, 1.f);
    return luminance(mul(rho, L)) * (Gb * (1.f / DDGI_PI));
}

// ---------------------------------------------------------------------------
// emitter choice proportional to area, orthonormal basis
// ---------------------------------------------------------------------------
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

// the same search on tables staged in shared memory
__device__ __forceinline__ uint32_t sample_emitter_smem(const float* cdf, const uint32_t* guide, uint32_t E,
                                                        uint32_t G, float u) {
    const float target = u * cdf[E - 1];
    uint32_t j = min((uint32_t)(u * (float)G), G - 1);
    uint32_t i = guide[j];
    while (i < E - 1 && !(target < cdf[i])) ++i;
    return i;
}


// reservoir record: q0 = (y, W), q1 = (L, M), q2 = (owner normal, owner
// distance, > 0 exactly when the owner has a G-buffer hit), q3 = (triangle of
// y, tag, octahedral map of y's unit normal)
struct Rec {
    float4 q0, q1, q2, q3;
};

// words 12..15: triangle of y, tag, y's normal (octahedral, 0 0 without a sample)
__device__ __forceinline__ float4 rec_tail(uint32_t tri, uint32_t tag, float2 ny) {
    return make_float4(__uint_as_float(tri), __uint_as_float(tag), ny.x, ny.y);
}

__device__ __forceinline__ void store_rec(float4* p, float4 q0, float4 q1, float4 q2, float4 q3) {
    st32(p, q0, q1);
    st32(p + 2, q2, q3);
}

__device__ __forceinline__ void copy_rec(float4* p, const Rec& r) {
    st32(p, r.q0, r.q1);
    st32(p + 2, r.q2, r.q3);
}

__device__ __forceinline__ Rec load_rec(const float4* p) {
    Rec r;
    ld32(p, r.q0, r.q1);
    ld32(p + 2, r.q2, r.q3);
    return r;
}

__device__ __forceinline__ bool rec_owner_valid(const Rec& r) { return r.q2.w > 0.f; }

// target of a record's sample at x (the sample's normal travels in the record)
__device__ __forceinline__ float rec_target(f3 x, f3 nx, f3 rho, float4 q0, float4 q1, float4 q3) {
    if (__float_as_uint(q3.x) == DDGI_NONE) return 0.f;
    return target_at(x, nx, rho, xyz(q0), oct_decode(q3.z, q3.w), xyz(q1));
}

