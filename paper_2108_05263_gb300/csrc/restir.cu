// Reservoir resampling of Sec. 3.1 step 2 with candidates of step 1: the
// initial candidates on all surfaces (emitter points + BSDF rays, Sec. 3.5
// residual), temporal reuse and spatial reuse with the cached probe query of
// Sec. 3.6.  One thread per pixel; SoA planes read and written as 16-byte
// records.
#include <algorithm>

#include "internal.h"
#include "trace_engine.cuh"

namespace {

struct Sel {
    f3 y, L;
    uint32_t tri, tag;
    float p;   // target at the owning pixel
};

// cosine-distributed direction of BSDF candidate c at pixel pix (Sec. 3.1 step 1)
__device__ __forceinline__ f3 bsdf_dir(const RestirParams& rp, uint32_t pix, uint32_t frame,
                                       uint32_t c, f3 nx) {
    const uint32_t cp = rng_cand(rng_prefix(rp.seed, pix, frame, PASS_INITIAL), c);
    float u0 = u01(rng_u32_dim(cp, 0)), u1 = u01(rng_u32_dim(cp, 1));
    float r = sqrtf(u0);
    float sn, cs;
    sincospif(2.f * u1, &sn, &cs);
    return onb_to_world(nx, r * cs, r * sn, sqrtf(fmaxf(0.f, 1.f - u0)));
}

// Sec. 5 subsampling: does pixel pix generate candidates in this frame?
__device__ __forceinline__ bool generates(const RestirParams& rp, int width, uint32_t pix, uint32_t frame) {
    if (rp.stride <= 1u) return true;
    const uint32_t x = pix % (uint32_t)width, y = pix / (uint32_t)width;
    return (x + y + frame) % rp.stride == 0u;
}

// BSDF candidate rays: work item i = pixel * n_bsdf + b
struct BsdfGen {
    GBufView g;
    RestirParams rp;
    uint32_t frame, nl, nb;
    __device__ __forceinline__ bool ray(uint32_t i, Ray& r) const {
        const uint32_t pix = i / nb, b = i - pix * nb;
        r.tmax = DDGI_MISS_T;
        float4 g1 = g.g1[pix];
        if (__float_as_uint(g1.w) == DDGI_NONE || !generates(rp, g.width, pix, frame)) return false;
        r.o = xyz(g.g0[pix]);
        r.d = bsdf_dir(rp, pix, frame, nl + b, xyz(g1));
        r.tmin = DDGI_T_EPS;
        return true;
    }
};

// network query at each BSDF hit (learned target form): rho(y) max(f(y), 0)
struct BsdfHitQuery {
    SceneView s;
    GBufView g;
    RestirParams rp;
    uint32_t frame, nl, nb;
    const float2* hits;
    float4* ind;
    __device__ bool query(uint32_t i, f3& p, f3& n) const {
        const uint32_t pix = i / nb, b = i - pix * nb;
        float4 g1 = g.g1[pix];
        if (__float_as_uint(g1.w) == DDGI_NONE) return false;
        float2 hv = hits[i];
        uint32_t tri = __float_as_uint(hv.y);
        if (tri == DDGI_NONE) return false;
        f3 w = bsdf_dir(rp, pix, frame, nl + b, xyz(g1));
        f3 ny = xyz(__ldg(s.nrm + tri));
        if (!(dot(ny, w) < 0.f) || !any_pos(xyz(__ldg(s.alb + tri)))) return false;
        p = xyz(g.g0[pix]) + w * hv.x;
        n = ny;
        return true;
    }
    __device__ void store(uint32_t i, bool valid, f3 f) const {
        if (!valid) {
            ind[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            return;
        }
        f3 rho = xyz(__ldg(s.alb + __float_as_uint(hits[i].y)));
        ind[i] = make_float4(rho.x * fmaxf(f.x, 0.f), rho.y * fmaxf(f.y, 0.f), rho.z * fmaxf(f.z, 0.f), 1.f);
    }
};

// streaming weighted reservoir sampling over one pixel's candidates in order
// (emitter points first, then BSDF rays): balance-heuristic mixture density in
// area measure, bounded geometry term in the target
struct CandidateStream {
    f3 rho;
    uint32_t pix, NL, NB;
    float invM;
    float wsum;
    Sel sel;
    // returns whether the candidate was taken
    __device__ __forceinline__ bool add(uint32_t c, uint32_t cp, f3 y, f3 L, uint32_t tri, float d2, float cx, float cy,
                                        float pL) {
        if (cx <= 0.f) return false;
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
            return true;
        }
        return false;
    }
};

// Emitter candidate c of pixel x (key prefix cp): the emitter drawn by area,
// the point y on it, its triangle, the unit direction's cosines and the
// radiance toward x.  The emitter kernel runs it for every candidate, the
// BSDF kernel once more for the candidate the emitter part selected (the
// same code and random numbers: the same values).
struct EmitterCand {
    f3 y, L;
    uint32_t tri, e;
    float d2, cx, cy;
};

// the point of emitter candidate cp on emitter record (q0..q3) and what it
// sends toward x
template <bool REFLECT>
__device__ __forceinline__ bool emitter_point(const SceneView& s, const VolumeView& v, f3 x, f3 nx, uint32_t cp,
                                              float4 q0, float4 q1, float4 q2, float4 q3, EmitterCand& ec) {
    float u1 = u01(rng_u32_dim(cp, 1)), u2 = u01(rng_u32_dim(cp, 2));
    ec.tri = __float_as_uint(q0.w);
    float sq = sqrtf(u1);
    float b1 = sq * (1.f - u2), b2 = sq * u2;
    ec.y = xyz(q0) + xyz(q1) * b1 + xyz(q2) * b2;
    f3 d = ec.y - x;
    ec.d2 = dot(d, d);
    if (ec.d2 <= 0.f) return false;
    f3 w = d * rsqrtf(ec.d2);
    ec.cx = dot(nx, w);
    const float cyn = dot(xyz(q3), w);
    ec.cy = fabsf(cyn);
    if (REFLECT) {
        ec.L = radiance_at(s, v, ec.y, ec.tri, x);
    } else {
        // pure emitter: one-sided Le toward x
        ec.L = cyn < 0.f ? f3{q1.w, q2.w, q3.w} : f3{0.f, 0.f, 0.f};
    }
    return true;
}

template <bool REFLECT, bool SMEM>
__device__ __forceinline__ bool emitter_candidate(const SceneView& s, const VolumeView& v, f3 x, f3 nx, uint32_t cp,
                                                  const float4* e_vert, const float* e_cdf, const uint32_t* e_guide,
                                                  EmitterCand& ec) {
    const float u0 = u01(rng_u32_dim(cp, 0));
    float4 q0, q1, q2, q3;
    if (SMEM) {
        // four planes of E records each (SoA: consecutive emitters on
        // consecutive 16-byte bank groups)
        const uint32_t E = s.num_emitters;
        ec.e = sample_emitter_smem(e_cdf, e_guide, E, s.guide_size, u0);
        q0 = e_vert[ec.e];
        q1 = e_vert[E + ec.e];
        q2 = e_vert[2 * E + ec.e];
        q3 = e_vert[3 * E + ec.e];
    } else {
        ec.e = sample_emitter(s, u0);
        const float4* er = s.evert + 4 * (size_t)ec.e;
        ld32(er, q0, q1);
        ld32(er + 2, q2, q3);
    }
    return emitter_point<REFLECT>(s, v, x, nx, cp, q0, q1, q2, q3, ec);
}

// Candidates of step 1, emitter part, for one pixel: points uniform in
// emitter area.  The stream's state after them -- running weight sum, the
// selected candidate's target and index -- is left in the pixel's 16-byte
// residual slot (state) for k_restir_initial, which recomputes that one
// candidate's point and radiance and continues the stream with the BSDF rays
// (it overwrites the slot with the residual); the split keeps this loop free
// of the probe query's registers (REFLECT: some emitter also reflects, so its
// candidates need the query too).  MODE 0: every emitter table from global
// memory; 1: the records, cumulative areas and guide table from shared
// memory (e_vert, e_cdf, e_guide); 2: the cumulative areas and guide table
// from shared memory and the records from global memory, each candidate's
// record requested before the candidate ahead of it is evaluated (tables
// too large for shared memory: the record loads are L2 round trips); without
// reflecting emitters the 48-byte records, the normal rebuilt from the edges
// (a quarter fewer bytes: 4K building 8.93 -> 8.70 ms for restir_initial).
template <bool REFLECT, int MODE>
__device__ __forceinline__ void emitter_candidates(const SceneView& s, const VolumeView& v, const RestirParams& rp,
                                                   const GBufView& g, float4* __restrict__ state, uint32_t frame,
                                                   uint32_t pix, const float4* e_vert, const float* e_cdf,
                                                   const uint32_t* e_guide) {
    const float4 g1 = g.g1[pix];
    if (__float_as_uint(g1.w) == DDGI_NONE || !generates(rp, g.width, pix, frame)) return;
    const float4 g0 = g.g0[pix], g2 = g.g2[pix];
    const f3 x = xyz(g0), nx = xyz(g1);
    CandidateStream cs;
    cs.rho = xyz(g2);
    cs.pix = pix;
    cs.NL = rp.n_light;
    cs.NB = rp.n_bsdf;
    cs.invM = 1.f / (float)(cs.NL + cs.NB);
    cs.wsum = 0.f;
    cs.sel.tri = DDGI_NONE;
    cs.sel.tag = 0u;
    cs.sel.p = 0.f;
    cs.sel.y = cs.sel.L = f3{0.f, 0.f, 0.f};
    const uint32_t prefix = rng_prefix(rp.seed, pix, frame, PASS_INITIAL);
    const float inv_area = 1.f / s.area_total;
    uint32_t esel = 0u;
    if (MODE == 2) {
        // candidate c + 1's emitter and record, requested a candidate ahead
        const uint32_t E = s.num_emitters;
        uint32_t cp_n = 0u, e_n = 0u;
        float4 n0, n1, n2, n3 = make_float4(0.f, 0.f, 0.f, 0.f);
        auto fetch = [&](uint32_t c) {
            cp_n = rng_cand(prefix, c);
            e_n = sample_emitter_smem(e_cdf, e_guide, E, s.guide_size, u01(rng_u32_dim(cp_n, 0)));
            if (REFLECT) {   // the query at the point needs the record's triangle
                const float4* er = s.evert + 4 * (size_t)e_n;
                ld32_issue(er, n0, n1);
                ld32_issue(er + 2, n2, n3);
            } else {
                // (a 32-byte load on the record's aligned half and a 16-byte
                // one, chosen by the parity of e, measured 9% slower)
                const float4* er = s.evert3 + 3 * (size_t)e_n;
                ld16_issue(er, n0);
                ld16_issue(er + 1, n1);
                ld16_issue(er + 2, n2);
            }
        };
        if (cs.NL > 0) fetch(0);
        for (uint32_t c = 0; c < cs.NL; ++c) {
            const uint32_t cp = cp_n;
            EmitterCand ec;
            ec.e = e_n;
            float4 q0 = n0, q1 = n1, q2 = n2, q3 = n3;
            if (!REFLECT) {
                // (n, Le.b) of the full record.  q0.w holds Le.b, so ec.tri
                // below is no triangle: this pass only tests the selected
                // one against DDGI_NONE, which no finite radiance matches
                const f3 cr = cross(xyz(q1), xyz(q2));
                const f3 nn = cr * rsqrtf(dot(cr, cr));
                q3 = make_float4(nn.x, nn.y, nn.z, q0.w);
            }
            if (c + 1 < cs.NL) fetch(c + 1);
            if (!emitter_point<REFLECT>(s, v, x, nx, cp, q0, q1, q2, q3, ec)) continue;
            if (cs.add(c, cp, ec.y, ec.L, ec.tri, ec.d2, ec.cx, ec.cy, inv_area)) esel = ec.e;
        }
    } else {
        for (uint32_t c = 0; c < cs.NL; ++c) {
            const uint32_t cp = rng_cand(prefix, c);
            EmitterCand ec;
            if (!emitter_candidate<REFLECT, MODE == 1>(s, v, x, nx, cp, e_vert, e_cdf, e_guide, ec)) continue;
            if (cs.add(c, cp, ec.y, ec.L, ec.tri, ec.d2, ec.cx, ec.cy, inv_area)) esel = ec.e;
        }
    }
    // the selected candidate's index (tag = pixel * 64 + candidate) or none,
    // and its emitter
    const uint32_t csel = cs.sel.tri == DDGI_NONE ? DDGI_NONE : cs.sel.tag - pix * 64u;
    state[pix] = make_float4(cs.wsum, cs.sel.p, __uint_as_float(csel), __uint_as_float(esel));
}

// one thread per pixel, emitter tables from global memory (L1); rows run
// bottom-up, so that k_restir_initial, top-down, starts on rows still in L2
template <bool REFLECT>
__global__ void __launch_bounds__(128) k_restir_emitters(SceneView s, VolumeView v, RestirParams rp, GBufView g,
                                                         float4* __restrict__ state, uint32_t frame) {
    int px = blockIdx.x * blockDim.x + threadIdx.x;
    int py = (gridDim.y - 1 - blockIdx.y) * blockDim.y + threadIdx.y;
    if (px >= g.width || py >= g.height) return;
    emitter_candidates<REFLECT, 0>(s, v, rp, g, state, frame, (uint32_t)py * g.width + px, nullptr, nullptr,
                                   nullptr);
}

// Persistent variant for emitter tables that fit in shared memory: each CTA
// copies the records, cumulative areas and guide table once, then walks
// 64 x 8 pixel tiles (bottom row of tiles first); the 32-byte record reads
// of the candidates then come from shared memory instead of the L1 that the
// per-pixel kernel saturates.  RECORDS false: the records are too many for
// shared memory and only the search tables are staged (MODE 2 above; 72
// registers, one CTA per SM: caps at two CTAs spill and ran 2-4% slower).
constexpr int kEmitTileW = 64, kEmitTileH = 8;   // measured best (32 x 16, 128 x 4, 16 x 32 slower)
template <bool REFLECT, bool RECORDS>
__global__ void __launch_bounds__(512, 1) k_restir_emitters_smem(SceneView s, VolumeView v, RestirParams rp, GBufView g,
                                                              float4* __restrict__ state, uint32_t frame) {
    extern __shared__ float4 e_smem[];
    const uint32_t E = s.num_emitters, G = s.guide_size;
    float4* e_vert = e_smem;
    float* e_cdf = reinterpret_cast<float*>(e_smem + (RECORDS ? 4 * (size_t)E : 0));
    uint32_t* e_guide = reinterpret_cast<uint32_t*>(e_cdf + E);
    if (RECORDS)
        for (uint32_t i = threadIdx.x; i < 4 * E; i += blockDim.x) e_vert[(i & 3u) * E + (i >> 2)] = __ldg(s.evert + i);
    for (uint32_t i = threadIdx.x; i < E; i += blockDim.x) e_cdf[i] = __ldg(s.cdf + i);
    for (uint32_t i = threadIdx.x; i < G; i += blockDim.x) e_guide[i] = __ldg(s.guide + i);
    __syncthreads();
    const int tiles_x = (g.width + kEmitTileW - 1) / kEmitTileW;
    const int tiles_y = (g.height + kEmitTileH - 1) / kEmitTileH;
    const int tx = threadIdx.x % kEmitTileW, ty = threadIdx.x / kEmitTileW;
    for (int t = blockIdx.x; t < tiles_x * tiles_y; t += gridDim.x) {
        const int bx = t % tiles_x, by = tiles_y - 1 - t / tiles_x;
        const int px = bx * kEmitTileW + tx, py = by * kEmitTileH + ty;
        if (px >= g.width || py >= g.height) continue;
        emitter_candidates<REFLECT, RECORDS ? 1 : 2>(s, v, rp, g, state, frame, (uint32_t)py * g.width + px, e_vert,
                                                     e_cdf, e_guide);
    }
}

// Temporal reuse of pixel pix (Sec. 3.1 step 2, Sec. 3.6): merge its current
// record c with the previous frame's record at the reprojected pixel (cached
// radiance, normal and depth rejection, M capped relative to the current M)
// and store the result at o.
__device__ __forceinline__ void temporal_merge(const SceneView& s, const RestirParams& rp, const GBufView& g,
                                               float3 cam_prev, const ResView& prev, uint32_t frame, uint32_t pix,
                                               const Rec& c, float4 g2, float4* o) {
    int pq = __float_as_int(g2.w);
    const bool moving = pq >= 0 && (pq & DDGI_PREV_MOVING);
    pq &= ~DDGI_PREV_MOVING;
    // the owner validity of the current record is this pixel's G-buffer validity
    bool merge = rec_owner_valid(c) && pq >= 0 && (uint32_t)pq < prev.n;
    Rec p;
    float4 g0;
    if (merge) {
        p = load_rec(prev.rec + 4 * (size_t)pq);
        g0 = g.g0[pix];
        merge = rec_owner_valid(p) && dot(xyz(c.q2), xyz(p.q2)) > rp.normal_reject_cos;
        if (merge) {
            // a surface on a moving instance is compared at its previous position
            f3 xp = xyz(g0);
            if (moving) {
                bool mv;
                xp = prev_position(s, __float_as_uint(__ldg(&g.g1[pix].w)), xp, &mv);
            }
            float de = length(xp - f3{cam_prev.x, cam_prev.y, cam_prev.z});
            merge = fabsf(de - p.q2.w) <= rp.depth_reject_frac * de;
        }
    }
    if (!merge) {
        store_rec(o, c.q0, c.q1, c.q2, c.q3);
        return;
    }
    const f3 x = xyz(g0), nx = xyz(c.q2), rho = xyz(g2);
    float Mc = c.q1.w;
    // the cap is relative to the current M, or to the nominal candidate count
    // for a pixel that generated none (subsampling)
    const float Mref = Mc > 0.f ? Mc : (float)((s.num_emitters > 0 ? rp.n_light : 0u) + rp.n_bsdf);
    float Mp = fminf(p.q1.w, rp.temporal_mcap * Mref);
    float pc = rec_target(x, nx, rho, c.q0, c.q1, c.q3);
    float wsum = pc * c.q0.w * Mc;
    float pp = rec_target(x, nx, rho, p.q0, p.q1, p.q3);
    float wp = pp * p.q0.w * Mp;
    wsum += wp;
    uint32_t h = rng_u32_dim(rng_cand(rng_prefix(rp.seed, pix, frame, PASS_TEMPORAL), 0u), 0u);
    float u = u01(h);
    float4 q0 = c.q0, q1 = c.q1, q3 = c.q3;
    float psel = pc;
    if (wp > 0.f && u * wsum < wp) {
        q0 = p.q0;
        q1 = p.q1;
        q3 = p.q3;
        psel = pp;
    }
    float Mo = Mc + Mp;
    q0.w = psel > 0.f ? wsum / (Mo * psel) : 0.f;
    q1.w = Mo;
    store_rec(o, q0, q1, c.q2, q3);
}

// Candidates of step 1, BSDF part, and the reservoir of step 2: continues the
// stream k_restir_emitters left in the record (when there are emitter
// candidates) with the cosine-distributed rays traced before this kernel;
// their residual transport (Sec. 3.5) on the side.
// FUSE: the pixel's initial record goes straight into temporal reuse with
// the previous frame's records (prev) and only the merged record is stored
// (in fin); the arithmetic is that of the two separate passes, up to the
// compiler's multiply-add contraction in each kernel (a few ulp).
// GLOSSY: the radiance at a BSDF hit includes the one-sample glossy half of
// L_DDGI+ (Sec. 3.3), drawn with dimensions 4 and 5 of the candidate's keys.
// Diffuse: at most 96 registers (five CTAs per SM, 24 bytes of spill) with
// the probe query's loop not unrolled: 1.183 -> 1.171 ms for the fused pass
// against 128 registers (four CTAs) with the loop unrolled 2x or not; the
// glossy form, whose second query would spill 200 bytes there, keeps 128
// (four CTAs).
template <bool FUSE, bool GLOSSY>
__global__ void __launch_bounds__(128, GLOSSY ? 4 : 5) k_restir_initial(SceneView s, VolumeView v, RestirParams rp,
                                                        GBufView g, ResView out,
                                                        float4* __restrict__ resid, uint32_t frame,
                                                        const float2* __restrict__ bsdf_hits,
                                                        const float4* __restrict__ ind,
                                                        const MLPState* __restrict__ mst, uint32_t nl,
                                                        float3 cam_prev, ResView prev, ResView fin) {
    int px = blockIdx.x * blockDim.x + threadIdx.x;
    int py = blockIdx.y * blockDim.y + threadIdx.y;
    if (px >= g.width || py >= g.height) return;
    uint32_t pix = (uint32_t)py * g.width + px;
    float4 g1 = g.g1[pix];
    uint32_t xtri = __float_as_uint(g1.w);
    const uint32_t NL = nl;
    const uint32_t NB = rp.n_bsdf;
    const uint32_t M = NL + NB;
    float4* rec = out.rec + 4 * (size_t)pix;
    const auto emit = [&](float4 q0, float4 q1, float4 q2, float4 q3, float4 g2v) {
        if (FUSE) {
            Rec c;
            c.q0 = q0;
            c.q1 = q1;
            c.q2 = q2;
            c.q3 = q3;
            temporal_merge(s, rp, g, cam_prev, prev, frame, pix, c, g2v, fin.rec + 4 * (size_t)pix);
        } else {
            store_rec(rec, q0, q1, q2, q3);
        }
    };
    if (xtri == DDGI_NONE) {   // no owner: temporal reuse keeps the empty record
        emit(make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f),
             rec_tail(DDGI_NONE, 0u, make_float2(0.f, 0.f)), make_float4(0.f, 0.f, 0.f, __int_as_float(-1)));
        resid[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float4 g0 = g.g0[pix], g2 = g.g2[pix];
    const float4 geo = make_float4(g1.x, g1.y, g1.z, g0.w);
    if (!generates(rp, g.width, pix, frame)) {   // subsampling: an empty reservoir that only reuses
        emit(make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f), geo,
             rec_tail(DDGI_NONE, 0u, make_float2(0.f, 0.f)), g2);
        resid[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const f3 x = xyz(g0), nx = xyz(g1);
    CandidateStream cs;
    cs.rho = xyz(g2);
    cs.pix = pix;
    cs.NL = NL;
    cs.NB = NB;
    cs.invM = 1.f / (float)M;
    const uint32_t prefix = rng_prefix(rp.seed, pix, frame, PASS_INITIAL);
    // the emitter part's state: weight sum, selected target, candidate index
    // and emitter; the stream needs only the first two until its end, so the
    // selected emitter candidate is rebuilt after the BSDF candidates, and
    // only if none of them displaced it
    uint32_t csel = DDGI_NONE, esel = 0u;
    if (NL > 0) {
        const float4 st = resid[pix];
        csel = __float_as_uint(st.z);
        esel = __float_as_uint(st.w);
        cs.wsum = st.x;
        cs.sel.p = st.y;
        cs.sel.tri = csel != DDGI_NONE ? 0u : DDGI_NONE;   // 0: the emitter candidate, rebuilt below
        cs.sel.tag = 0u;
        cs.sel.y = cs.sel.L = f3{0.f, 0.f, 0.f};
    } else {
        cs.wsum = 0.f;
        cs.sel.tri = DDGI_NONE;
        cs.sel.tag = 0u;
        cs.sel.p = 0.f;
        cs.sel.y = cs.sel.L = f3{0.f, 0.f, 0.f};
    }
    const float inv_area = 1.f / s.area_total;
    f3 res = {0.f, 0.f, 0.f};
    for (uint32_t c = NL; c < M; ++c) {
        const uint32_t cp = rng_cand(prefix, c);
        f3 w = bsdf_dir(rp, pix, frame, c, nx);
        float2 hb = __ldg(bsdf_hits + (size_t)pix * NB + (c - NL));
        const uint32_t tri = __float_as_uint(hb.y);
        if (tri == DDGI_NONE) continue;
        const float pL = __ldg(s.emi + tri).w > 0.f ? inv_area : 0.f;
        const f3 y = x + w * hb.x;
        const float d2 = hb.x * hb.x;
        const float cx = dot(nx, w);
        const float cyn = dot(xyz(__ldg(s.nrm + tri)), w);
        f3 L;
        if (mst != nullptr && mst->use_mlp) {
            // learned target: Le + the network's rho max(f, 0), front faces only
            const uint32_t qi = pix * NB + (c - NL);
            L = cyn < 0.f ? xyz(__ldg(s.emi + tri)) + xyz(__ldg(ind + qi)) : f3{0.f, 0.f, 0.f};
        } else if constexpr (GLOSSY) {
            L = radiance_at_glossy<2>(s, v, y, tri, x, u01(rng_u32_dim(cp, 4)), u01(rng_u32_dim(cp, 5)));
        } else {
            L = radiance_at<1>(s, v, y, tri, x);
        }
        if (cx > 0.f) {
            float G = cx * fabsf(cyn) / d2;
            if (G > 1.f) res = res + mul(cs.rho, L) * ((1.f - 1.f / G) / (float)NB);
        }
        cs.add(c, cp, y, L, tri, d2, cx, fabsf(cyn), pL);
    }
    // (the residual is stored last: a store before them would keep the loads
    // below -- emitter record, previous frame's record -- from overlapping)
    if (csel != DDGI_NONE && cs.sel.tag == 0u && cs.sel.tri == 0u) {
        // still the emitter part's selection (a BSDF candidate sets a tag >=
        // pixel * 64 + NL > 0): its record only, no emitter search
        const float4* er = s.evert + 4 * (size_t)esel;
        float4 q0, q1, q2, q3;
        ld32(er, q0, q1);
        ld32(er + 2, q2, q3);
        EmitterCand ec;
        if (s.emitters_reflect)
            emitter_point<true>(s, v, x, nx, rng_cand(prefix, csel), q0, q1, q2, q3, ec);
        else
            emitter_point<false>(s, v, x, nx, rng_cand(prefix, csel), q0, q1, q2, q3, ec);
        cs.sel.y = ec.y;
        cs.sel.L = ec.L;
        cs.sel.tri = ec.tri;
        cs.sel.tag = pix * 64u + csel;
    }
    const Sel& sel = cs.sel;
    if (sel.tri == DDGI_NONE) {
        emit(make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, (float)M), geo,
             rec_tail(DDGI_NONE, 0u, make_float2(0.f, 0.f)), g2);
    } else {
        float W = sel.p > 0.f ? cs.wsum / ((float)M * sel.p) : 0.f;
        emit(make_float4(sel.y.x, sel.y.y, sel.y.z, W), make_float4(sel.L.x, sel.L.y, sel.L.z, (float)M), geo,
             rec_tail(sel.tri, sel.tag, oct_encode(xyz(__ldg(s.nrm + sel.tri)))), g2);
    }
    resid[pix] = make_float4(res.x, res.y, res.z, 0.f);
}

__global__ void __launch_bounds__(256) k_restir_temporal(SceneView s, RestirParams rp, GBufView g,
                                                         float3 cam_prev, ResView cur, ResView prev,
                                                         ResView out, uint32_t frame) {
    // rows bottom-up: the candidate pass wrote the current records top-down,
    // so its last rows are still in L2 when this pass starts
    int px = blockIdx.x * blockDim.x + threadIdx.x;
    int py = (gridDim.y - 1 - blockIdx.y) * blockDim.y + threadIdx.y;
    if (px >= g.width || py >= g.height) return;
    uint32_t pix = (uint32_t)py * g.width + px;
    const Rec c = load_rec(cur.rec + 4 * (size_t)pix);
    temporal_merge(s, rp, g, cam_prev, prev, frame, pix, c, g.g2[pix], out.rec + 4 * (size_t)pix);
}

// x mod span for x < 2^16 via a multiply-high reciprocal (exact in that range)
__device__ __forceinline__ uint32_t mod_span(uint32_t x, uint32_t span, uint32_t magic) {
    return x - __umulhi(x, magic) * span;
}

// the j-th neighbour of pixel (px, py): integer offsets drawn by rejection
// from hashed lattice points of the disk of radius R (at most 8 tries);
// -1 when the tries run out or the point leaves the image
__device__ __forceinline__ int spatial_neighbour(const RestirParams& rp, const GBufView& g, uint32_t cp, int px,
                                                 int py) {
    const int R = (int)rp.spatial_radius;
    const uint32_t span = 2u * rp.spatial_radius + 1u;
    for (uint32_t a = 0; a < 8u; ++a) {
        uint32_t h = rng_u32_dim(cp, a);
        int ox = (int)mod_span(h & 0xFFFFu, span, rp.span_magic) - R;
        int oy = (int)mod_span(h >> 16, span, rp.span_magic) - R;
        if ((ox != 0 || oy != 0) && ox * ox + oy * oy <= R * R) {
            int qx = px + ox, qy = py + oy;
            return qx >= 0 && qy >= 0 && qx < g.width && qy < g.height ? qy * g.width + qx : -1;
        }
    }
    return -1;
}

// The neighbour gathers are L2 hits whose latency bounds this kernel: both
// halves of a neighbour record are requested together (the sample's normal
// rides in the record, so nothing else is gathered), and the next neighbour's
// pixel is drawn while they are in flight.  At most 56 registers keep nine
// CTAs per SM.
// UP: rows bottom-up (odd passes), so that each pass starts on the rows the
// pass before it wrote last, still in L2; a compile-time direction keeps the
// register count.
template <bool UP>
__global__ void __launch_bounds__(128, 9) k_restir_spatial(SceneView s, RestirParams rp, GBufView g,
                                                           ResView in, ResView out, uint32_t frame,
                                                           uint32_t pass) {
    int px = blockIdx.x * blockDim.x + threadIdx.x;
    int py = (UP ? gridDim.y - 1 - blockIdx.y : blockIdx.y) * blockDim.y + threadIdx.y;
    if (px >= g.width || py >= g.height) return;
    uint32_t pix = (uint32_t)py * g.width + px;
    Rec c = load_rec(in.rec + 4 * (size_t)pix);
    float4* o = out.rec + 4 * (size_t)pix;
    if (!rec_owner_valid(c)) {
        copy_rec(o, c);
        return;
    }
    float4 g0 = g.g0[pix], g2 = g.g2[pix];
    const f3 x = xyz(g0), nx = xyz(c.q2), rho = xyz(g2);
    const float dist = c.q2.w;
    float psel = rec_target(x, nx, rho, c.q0, c.q1, c.q3);
    float wsum = psel * c.q0.w * c.q1.w;
    float M = c.q1.w;
    float4 q0 = c.q0, q1 = c.q1, q3 = c.q3;
    const uint32_t prefix = rng_prefix(rp.seed, pix, frame, PASS_SPATIAL0 + pass);
    uint32_t cp_next = rng_cand(prefix, 0u);
    int nq_next = rp.spatial_neighbours > 0 ? spatial_neighbour(rp, g, cp_next, px, py) : -1;
    for (uint32_t j = 0; j < rp.spatial_neighbours; ++j) {
        const uint32_t cp = cp_next;
        const int nq = nq_next;
        // without a neighbour the pixel's own record stands in (read, not used)
        const float4* nr = in.rec + 4 * (size_t)(nq >= 0 ? (uint32_t)nq : pix);
        float4 n0, n1, n2, n3;
        ld32_l2(nr, n0, n1);
        ld32_l2(nr + 2, n2, n3);
        if (j + 1 < rp.spatial_neighbours) {
            cp_next = rng_cand(prefix, j + 1);
            nq_next = spatial_neighbour(rp, g, cp_next, px, py);
        }
        if (nq < 0) continue;
        if (!(n2.w > 0.f)) continue;
        if (dot(nx, xyz(n2)) <= rp.normal_reject_cos) continue;
        if (fabsf(dist - n2.w) > rp.depth_reject_frac * dist) continue;
        float pn = rec_target(x, nx, rho, n0, n1, n3);
        float wn = pn * n0.w * n1.w;
        wsum += wn;
        M += n1.w;
        float u = u01(rng_u32_dim(cp, 8u));
        if (wn > 0.f && u * wsum < wn) {
            q0 = n0;
            q1 = n1;
            q3 = n3;
            psel = pn;
        }
    }
    q0.w = psel > 0.f ? wsum / (M * psel) : 0.f;
    q1.w = M;
    store_rec(o, q0, q1, c.q2, q3);
}

// words 14..15 of caller-written records: the octahedral map of the normal of
// the sample's triangle
__global__ void k_attach_normals(const float4* __restrict__ nrm, uint32_t num_tris, float4* __restrict__ rec,
                                 uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4* q3 = rec + 4 * (size_t)i + 3;
    const uint32_t tri = __float_as_uint(q3->x);
    float2 o = make_float2(0.f, 0.f);
    if (tri < num_tris) o = oct_encode(xyz(__ldg(nrm + tri)));
    q3->z = o.x;
    q3->w = o.y;
}

inline dim3 tile_grid(int w, int h, dim3 b) { return dim3((w + b.x - 1) / b.x, (h + b.y - 1) / b.y); }

}  // namespace

// the emitter-candidate pass: the shared-memory kernel when the emitter
// tables fit beside enough resident threads (all of them, else the search
// tables alone), else the per-pixel kernel
cudaError_t launch_emitter_candidates(const SceneView& s, const VolumeView& v, const RestirParams& rp,
                                      const GBufView& g, float4* state, uint32_t frame, cudaStream_t st) {
    const size_t tables = sizeof(float) * (size_t)s.num_emitters + sizeof(uint32_t) * (size_t)s.guide_size;
    const size_t full = sizeof(float4) * 4 * (size_t)s.num_emitters + tables;
    static int dev_sms = 0, max_smem = 0;
    if (dev_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    const bool records = full <= 96 * 1024 && (int)full <= max_smem;
    const size_t smem = records ? full : tables;
    if (smem <= 96 * 1024 && (int)smem <= max_smem) {
        auto kern = records ? (s.emitters_reflect ? k_restir_emitters_smem<true, true>
                                                  : k_restir_emitters_smem<false, true>)
                            : (s.emitters_reflect ? k_restir_emitters_smem<true, false>
                                                  : k_restir_emitters_smem<false, false>);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, smem);
        if (e != cudaSuccess) return e;
        if (per_sm > 0) {
            const int tiles = ((g.width + kEmitTileW - 1) / kEmitTileW) * ((g.height + kEmitTileH - 1) / kEmitTileH);
            const int grid = std::min(tiles, dev_sms * per_sm);
            kern<<<grid, 512, smem, st>>>(s, v, rp, g, state, frame);
            return cudaGetLastError();
        }
    }
    dim3 b(16, 8);
    if (s.emitters_reflect)
        k_restir_emitters<true><<<tile_grid(g.width, g.height, b), b, 0, st>>>(s, v, rp, g, state, frame);
    else
        k_restir_emitters<false><<<tile_grid(g.width, g.height, b), b, 0, st>>>(s, v, rp, g, state, frame);
    return cudaGetLastError();
}

cudaError_t launch_restir_initial(const SceneView& s, const VolumeView& v, const RestirParams& rp,
                                  const GBufView& g, const ResView& out, float4* resid,
                                  uint32_t frame, float2* hits, uint32_t* counter, const MLPView* mlp,
                                  MLPState* mst, float4* ind, cudaStream_t st, cudaStream_t side,
                                  cudaEvent_t ev_fork, cudaEvent_t ev_join, const ResView* fuse_prev,
                                  const ResView* fuse_out, float3 cam_prev) {
    if (g.width == 0 || g.height == 0) return cudaSuccess;
    const uint32_t nl = s.num_emitters > 0 ? rp.n_light : 0u;
    BsdfGen gen{g, rp, frame, nl, rp.n_bsdf};
    // The emitter candidates and the BSDF rays read only the G-buffer and
    // write disjoint buffers (the records' stream state / the hits): with a
    // side stream they run concurrently, each at full occupancy, so that one
    // kernel's tail on the SMs overlaps the other; k_restir_initial waits for
    // both.
    const bool fork = nl > 0 && side && ev_fork && ev_join;
    cudaError_t e;
    if (fork) {
        if ((e = cudaEventRecord(ev_fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, ev_fork, 0)) != cudaSuccess) return e;
    }
    e = launch_trace<BsdfGen, false>(s, gen, (uint32_t)g.width * g.height * rp.n_bsdf, counter, hits, st);
    if (e != cudaSuccess) return e;
    if (fork) {
        if ((e = launch_emitter_candidates(s, v, rp, g, resid, frame, side)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(ev_join, side)) != cudaSuccess) return e;
    }
    if (mlp) {
        e = launch_mlp_infer(*mlp, BsdfHitQuery{s, g, rp, frame, nl, rp.n_bsdf, hits, ind},
                             (uint32_t)g.width * g.height * rp.n_bsdf, st);
        if (e != cudaSuccess) return e;
    }
    dim3 b(32, 4);   // measured best for this kernel (16 x 8, 8 x 16, 64 x 2 slower)
    if (fork) {
        if ((e = cudaStreamWaitEvent(st, ev_join, 0)) != cudaSuccess) return e;
    } else if (nl > 0) {
        e = launch_emitter_candidates(s, v, rp, g, resid, frame, st);
        if (e != cudaSuccess) return e;
    }
    const dim3 grid = tile_grid(g.width, g.height, b);
    const MLPState* ms = mlp ? mst : nullptr;
    const bool fuse = fuse_prev && fuse_out;
    const ResView& fp = fuse ? *fuse_prev : out;
    const ResView& fo = fuse ? *fuse_out : out;
    if (s.spec) {   // a glossy scene (no network: the two are exclusive)
        if (fuse)
            k_restir_initial<true, true><<<grid, b, 0, st>>>(s, v, rp, g, out, resid, frame, hits, ind, ms, nl,
                                                             cam_prev, fp, fo);
        else
            k_restir_initial<false, true><<<grid, b, 0, st>>>(s, v, rp, g, out, resid, frame, hits, ind, ms, nl,
                                                              cam_prev, fp, fo);
    } else if (fuse) {
        k_restir_initial<true, false><<<grid, b, 0, st>>>(s, v, rp, g, out, resid, frame, hits, ind, ms, nl,
                                                          cam_prev, fp, fo);
    } else {
        k_restir_initial<false, false><<<grid, b, 0, st>>>(s, v, rp, g, out, resid, frame, hits, ind, ms, nl,
                                                           cam_prev, fp, fo);
    }
    return cudaGetLastError();
}

cudaError_t launch_restir_temporal(const SceneView& s, const RestirParams& rp, const GBufView& g,
                                   float3 prev_cam, const ResView& cur, const ResView& prev,
                                   const ResView& out, uint32_t frame, cudaStream_t st) {
    if (g.width == 0 || g.height == 0) return cudaSuccess;
    dim3 b(32, 8);
    k_restir_temporal<<<tile_grid(g.width, g.height, b), b, 0, st>>>(s, rp, g, prev_cam, cur, prev,
                                                                      out, frame);
    return cudaGetLastError();
}

cudaError_t launch_restir_spatial(const SceneView& s, const RestirParams& rp, const GBufView& g,
                                  const ResView& in, const ResView& out, uint32_t frame,
                                  uint32_t pass, cudaStream_t st) {
    if (g.width == 0 || g.height == 0) return cudaSuccess;
    dim3 b(16, 8);
    if (pass & 1u)
        k_restir_spatial<true><<<tile_grid(g.width, g.height, b), b, 0, st>>>(s, rp, g, in, out, frame, pass);
    else
        k_restir_spatial<false><<<tile_grid(g.width, g.height, b), b, 0, st>>>(s, rp, g, in, out, frame, pass);
    return cudaGetLastError();
}

cudaError_t launch_attach_normals(const SceneView& s, const ResView& r, cudaStream_t st) {
    if (r.n == 0) return cudaSuccess;
    k_attach_normals<<<(r.n + 255) / 256, 256, 0, st>>>(s.nrm, s.num_tris, r.rec, r.n);
    return cudaGetLastError();
}
