// Scene dynamics (the method targets fully dynamic scenes, Sec. 1, Sec. 4):
// rigid instance motion written into the BVH-ordered triangles, a bottom-up
// refit of the BVH4 boxes over the nodes whose subtrees hold instanced
// triangles (the topology of the first build is kept), and new emitter
// radiance.
#include "internal.h"

namespace {

__device__ __forceinline__ f3 apply(const float4* m, f3 p) {
    const float4 r0 = __ldg(m), r1 = __ldg(m + 1), r2 = __ldg(m + 2);
    return {r0.x * p.x + r0.y * p.y + r0.z * p.z + r0.w, r1.x * p.x + r1.y * p.y + r1.z * p.z + r1.w,
            r2.x * p.x + r2.y * p.y + r2.z * p.z + r2.w};
}

// one thread per instanced triangle: world vertices M p0, the BVH record
// (v0 + original index, e1, e2) and the unit winding normal (fp64 cross
// product of the float edges, as at build time)
__global__ void __launch_bounds__(128) k_instance_tris(const float4* __restrict__ obj, const uint4* __restrict__ map,
                                                       const float4* __restrict__ xf, float4* __restrict__ tris,
                                                       float4* __restrict__ nrm, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 m = __ldg(map + i);   // slot, triangle, instance
    const float4* M = xf + 3 * (size_t)m.z;
    const f3 v0 = apply(M, xyz(__ldg(obj + 3 * (size_t)i)));
    const f3 v1 = apply(M, xyz(__ldg(obj + 3 * (size_t)i + 1)));
    const f3 v2 = apply(M, xyz(__ldg(obj + 3 * (size_t)i + 2)));
    const double e1[3] = {(double)v1.x - v0.x, (double)v1.y - v0.y, (double)v1.z - v0.z};
    const double e2[3] = {(double)v2.x - v0.x, (double)v2.y - v0.y, (double)v2.z - v0.z};
    float4* t = tris + 3 * (size_t)m.x;
    t[0] = make_float4(v0.x, v0.y, v0.z, __uint_as_float(m.y));
    t[1] = make_float4(v1.x - v0.x, v1.y - v0.y, v1.z - v0.z, 0.f);
    t[2] = make_float4(v2.x - v0.x, v2.y - v0.y, v2.z - v0.z, 0.f);
    const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                         e1[0] * e2[1] - e1[1] * e2[0]};
    const double l = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    nrm[m.y] = l > 0.0 ? make_float4((float)(c[0] / l), (float)(c[1] / l), (float)(c[2] / l), 0.f)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
}

// one thread per listed node of one depth: each occupied slot's box is the
// union of its child node's slot boxes, or for a leaf slot the box of its
// unmoved references as built (static, clipped where the build split their
// triangles) and its moving triangles' corners (v0, v0 + e1, v0 + e2, the
// points the intersection test spans)
__global__ void __launch_bounds__(128) k_refit(float4* __restrict__ nodes, const float4* __restrict__ tris,
                                               const uint32_t* __restrict__ list, const float* __restrict__ stat,
                                               const int32_t* __restrict__ tri_inst, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float* nd = reinterpret_cast<float*>(nodes + 8 * (size_t)list[i]);
    for (int c = 0; c < 4; ++c) {
        // slot entry: 0 empty, > 0 inner node, < 0 leaf (-1 - (first * 8 + count - 1))
        const int entry = __float_as_int(nd[24 + c]);
        if (entry == 0) continue;
        f3 lo = {FLT_MAX, FLT_MAX, FLT_MAX}, hi = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
        if (entry < 0) {
            const float* sb = stat + 24 * (size_t)i + 6 * c;
            lo = {sb[0], sb[1], sb[2]};
            hi = {sb[3], sb[4], sb[5]};
            const int v = -1 - entry, first = v >> 3, cnt = (v & 7) + 1;
            for (int k = first; k < first + cnt; ++k) {
                if (tri_inst[__float_as_uint(tris[3 * (size_t)k].w)] < 0) continue;   // unmoved: in the static box
                const f3 v0 = xyz(tris[3 * (size_t)k]);
                const f3 p1 = v0 + xyz(tris[3 * (size_t)k + 1]), p2 = v0 + xyz(tris[3 * (size_t)k + 2]);
                lo = {fminf(lo.x, fminf(v0.x, fminf(p1.x, p2.x))), fminf(lo.y, fminf(v0.y, fminf(p1.y, p2.y))),
                      fminf(lo.z, fminf(v0.z, fminf(p1.z, p2.z)))};
                hi = {fmaxf(hi.x, fmaxf(v0.x, fmaxf(p1.x, p2.x))), fmaxf(hi.y, fmaxf(v0.y, fmaxf(p1.y, p2.y))),
                      fmaxf(hi.z, fmaxf(v0.z, fmaxf(p1.z, p2.z)))};
            }
        } else {
            const float* cn = reinterpret_cast<const float*>(nodes + 8 * (size_t)entry);
            for (int cc = 0; cc < 4; ++cc) {
                if (__float_as_int(cn[24 + cc]) == 0) continue;
                lo = {fminf(lo.x, cn[0 + cc]), fminf(lo.y, cn[8 + cc]), fminf(lo.z, cn[16 + cc])};
                hi = {fmaxf(hi.x, cn[4 + cc]), fmaxf(hi.y, cn[12 + cc]), fmaxf(hi.z, cn[20 + cc])};
            }
        }
        // (a slot whose subtree holds no occupied slot keeps the inverted box: never entered)
        nd[0 + c] = lo.x;
        nd[4 + c] = hi.x;
        nd[8 + c] = lo.y;
        nd[12 + c] = hi.y;
        nd[16 + c] = lo.z;
        nd[20 + c] = hi.z;
    }
}

// new radiance of emitter e (emitter-list order): the triangle table and the
// emitter record
__global__ void k_emitter_radiance(const float* __restrict__ le, const uint32_t* __restrict__ etri,
                                   float4* __restrict__ emi, float4* __restrict__ evert, float4* __restrict__ evert3,
                                   uint32_t E) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const float r = le[3 * (size_t)e], g = le[3 * (size_t)e + 1], b = le[3 * (size_t)e + 2];
    const uint32_t t = etri[e];
    emi[t] = make_float4(r, g, b, 1.f);   // w: member of the emitter list
    evert[4 * (size_t)e + 1].w = r;
    evert[4 * (size_t)e + 2].w = g;
    evert[4 * (size_t)e + 3].w = b;
    evert3[3 * (size_t)e].w = b;
    evert3[3 * (size_t)e + 1].w = r;
    evert3[3 * (size_t)e + 2].w = g;
}

}  // namespace

cudaError_t launch_instance_update(const float4* obj, const uint4* map, uint32_t n, const float4* xf, float4* tris,
                                   float4* nrm, float4* nodes, const uint32_t* refit_list, const float* refit_static,
                                   const int32_t* tri_inst, const std::vector<uint32_t>& level_offsets,
                                   cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_instance_tris<<<(n + 127) / 128, 128, 0, st>>>(obj, map, xf, tris, nrm, n);
    cudaError_t e = cudaGetLastError();
    // level_offsets[d]..[d+1] lists the nodes of one depth, deepest depth first
    for (size_t d = 0; e == cudaSuccess && d + 1 < level_offsets.size(); ++d) {
        const uint32_t a = level_offsets[d], b = level_offsets[d + 1];
        if (b == a) continue;
        k_refit<<<(b - a + 127) / 128, 128, 0, st>>>(nodes, tris, refit_list + a, refit_static + 24 * (size_t)a,
                                                      tri_inst, b - a);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_emitter_radiance(const float* le, const uint32_t* etri, float4* emi, float4* evert,
                                    float4* evert3, uint32_t E, cudaStream_t st) {
    if (E == 0) return cudaSuccess;
    k_emitter_radiance<<<(E + 127) / 128, 128, 0, st>>>(le, etri, emi, evert, evert3, E);
    return cudaGetLastError();
}
