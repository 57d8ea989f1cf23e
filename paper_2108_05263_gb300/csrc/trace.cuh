// Software ray traversal of the 4-wide BVH (the ray-casting operation h of
// Sec. 3.2; the paper uses DXR hardware, here it is plain SM code).
//
// Node layout (128 B = 8 float4, 128-byte aligned):
//   [0] lo.x of children 0..3   [1] hi.x   [2] lo.y   [3] hi.y
//   [4] lo.z                    [5] hi.z
//   [6] slot entry (int bits): > 0 inner node index, < 0 a leaf of count
//       triangle slots from first, coded -1 - (first * 8 + count - 1);
//       0 an empty slot   [7] unused
// Empty slots have an inverted box (lo = FLT_MAX, hi = -FLT_MAX) and entry 0:
// a slab test that takes each axis's near and far plane by the ray's sign
// never enters them; the symmetric min / max form tests the entry.
// Triangles are stored in leaf order as 3 float4: (v0, original index
// bits), (e1 = v1 - v0, 0), (e2 = v2 - v0, 0).
#pragma once
#include "common.cuh"

#define TRAV_STACK 64

struct Ray {
    f3 o, d;
    float tmin, tmax;
};

struct Hit {
    float t;
    uint32_t tri;   // original triangle index, DDGI_NONE on miss
};

__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// Moller-Trumbore, two-sided; returns t or +inf
__device__ __forceinline__ float tri_hit(const float4* tp, f3 o, f3 d, uint32_t* orig) {
    float4 a = ldg4(tp), b = ldg4(tp + 1), c = ldg4(tp + 2);
    f3 v0 = xyz(a), e1 = xyz(b), e2 = xyz(c);
    *orig = __float_as_uint(a.w);
    f3 p = cross(d, e2);
    float det = dot(e1, p);
    if (det == 0.f) return INFINITY;
    float inv = 1.f / det;
    f3 tv = o - v0;
    float b1 = dot(tv, p) * inv;
    if (b1 < 0.f || b1 > 1.f) return INFINITY;
    f3 q = cross(tv, e1);
    float b2 = dot(d, q) * inv;
    if (b2 < 0.f || b1 + b2 > 1.f) return INFINITY;
    return dot(e2, q) * inv;
}

__device__ __forceinline__ float safe_inv(float x) {
    return 1.f / (fabsf(x) > 1e-20f ? x : copysignf(1e-20f, x));
}

// any_hit = true: return as soon as something is hit in (tmin, tmax)
template <bool ANY_HIT>
__device__ __forceinline__ Hit trace_bvh(const SceneView& s, const Ray& ray) {
    Hit h;
    h.t = ray.tmax;
    h.tri = DDGI_NONE;
    const f3 inv = {safe_inv(ray.d.x), safe_inv(ray.d.y), safe_inv(ray.d.z)};
    const f3 oi = {ray.o.x * inv.x, ray.o.y * inv.y, ray.o.z * inv.z};
    int2 stack[TRAV_STACK];   // (node, entry distance bits): one 8-byte access
    int sp = 0;
    int node = 0;
    int visits = 0;
    const float widen = 1.0000004f;   // robust slab test (a few ulp of slack)
    while (true) {
        if (++visits > s.max_visits) {
            atomicOr(s.err, ERRBIT_TRAVERSAL);
            h.tri = DDGI_NONE;
            h.t = ray.tmax;
            return h;
        }
        const float4* np = s.nodes + (size_t)node * 8;
        // a node is three 32-byte box loads and the 16-byte entry row
        float4 lx, hx, ly, hy, lz, hz;
        ld32(np, lx, hx);
        ld32(np + 2, ly, hy);
        ld32(np + 4, lz, hz);
        const float4 ef = ldg4(np + 6);
        const float blo[4][3] = {{lx.x, ly.x, lz.x}, {lx.y, ly.y, lz.y}, {lx.z, ly.z, lz.z}, {lx.w, ly.w, lz.w}};
        const float bhi[4][3] = {{hx.x, hy.x, hz.x}, {hx.y, hy.y, hz.y}, {hx.z, hy.z, hz.z}, {hx.w, hy.w, hz.w}};
        const int entry[4] = {__float_as_int(ef.x), __float_as_int(ef.y), __float_as_int(ef.z),
                              __float_as_int(ef.w)};
        float tnear[4];
        int order[4];
        int ninner = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float tx0 = fmaf(blo[c][0], inv.x, -oi.x), tx1 = fmaf(bhi[c][0], inv.x, -oi.x);
            float ty0 = fmaf(blo[c][1], inv.y, -oi.y), ty1 = fmaf(bhi[c][1], inv.y, -oi.y);
            float tz0 = fmaf(blo[c][2], inv.z, -oi.z), tz1 = fmaf(bhi[c][2], inv.z, -oi.z);
            float t0 = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), ray.tmin));
            float t1 = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), h.t)) * widen;
            bool hit = t0 <= t1;
            if (hit && entry[c] < 0) {
                // leaf: intersect its triangles now
                const int v = -1 - entry[c], first = v >> 3, count = (v & 7) + 1;
                for (int k = 0; k < count; ++k) {
                    uint32_t orig;
                    float t = tri_hit(s.tris + (size_t)(first + k) * 3, ray.o, ray.d, &orig);
                    if (t > ray.tmin && t < ray.tmax) {
                        if (ANY_HIT) {
                            h.t = t;
                            h.tri = orig;
                            return h;
                        }
                        if (t < h.t || (t == h.t && orig < h.tri)) {
                            h.t = t;
                            h.tri = orig;
                        }
                    }
                }
            } else if (hit && entry[c] > 0) {
                tnear[ninner] = t0;
                order[ninner] = entry[c];
                ++ninner;
            }
        }
        // sort the (at most 4) inner children by entry distance, nearest last
        for (int i = 1; i < ninner; ++i) {
            float tk = tnear[i];
            int ok = order[i];
            int j = i - 1;
            while (j >= 0 && tnear[j] < tk) {
                tnear[j + 1] = tnear[j];
                order[j + 1] = order[j];
                --j;
            }
            tnear[j + 1] = tk;
            order[j + 1] = ok;
        }
        if (ninner > 0) {
            if (sp + ninner - 1 > TRAV_STACK) {
                atomicOr(s.err, ERRBIT_STACK);
                h.tri = DDGI_NONE;
                h.t = ray.tmax;
                return h;
            }
            for (int i = 0; i < ninner - 1; ++i) stack[sp++] = make_int2(order[i], __float_as_int(tnear[i]));
            node = order[ninner - 1];
            continue;
        }
        // pop the next node that can still hold a closer hit
        bool found = false;
        while (sp > 0) {
            const int2 e = stack[--sp];
            if (__int_as_float(e.y) <= h.t * widen) {
                node = e.x;
                found = true;
                break;
            }
        }
        if (!found) break;
    }
    return h;
}
