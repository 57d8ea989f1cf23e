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
// 9 CTAs per SM: 56 registers, 12 bytes of spill (probe trace 0.182 -> 0.180 ms)
template <bool GLOSSY>
__global__ void __launch_bounds__(128, 9) k_probe_trace(SceneView s, VolumeView v, ProbeParams pp,
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
                const int qd = (v.depth_n + 1) * (v.depth_n + 1);
                float mu = sample_depth_q(v.depth_q + (size_t)p * qd * 2, v.depth_n, -w).x;
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

// The blend's weights depend on the texel and the frame's ray directions
// only, not on the probe: irradiance texel t weighs ray k by c = max(0,
// dir_t . w_k), distance texel t by c^sharpness.  They are written once per
// frame, ray-major (W[k][t] over the padded texel list: irradiance texels,
// padded to a multiple of 4, then distance texels, padded likewise; pads
// weigh 0), with partial weight sums over groups of 8 rays after them.  A
// distance texel's weights are taken relative to its largest cosine,
// (c / c_max)^sharpness: the normalised mean is the same, and the largest
// weight is 1, so no weight that matters underflows however few rays there
// are.  The blend is then, for each probe, a product of these fixed matrices
// with the probe's ray radiance and distances.
struct BlendShape {
    int G;          // probes per CTA (even)
    int nip, ndp;   // irradiance / distance texels, padded to multiples of 4
    int ci;         // irradiance columns per ray row: 3G padded to a multiple of 4
    int rg_d, cg_d, rg_i, cg_i;   // warps of each product: groups of 8 row tiles x 4 column tiles
    int warps;      // warps per CTA (one slice of the products' warps, <= 32)
    int slices;     // CTAs per probe group
    int kc;         // rays per staged chunk of weights
};

// CTA of 8 texels x 128 ray lanes: the distance texels' largest cosine
// first, then the weights (stores of W[k][t] in 32-byte runs) and the
// partial sum of each group of 8 rays, added in ray order
#define BW_T 8     // texels per CTA
#define BW_K 128   // ray lanes per CTA
__global__ void __launch_bounds__(BW_T * BW_K) k_blend_weights(VolumeView v, ProbeParams pp, BlendShape bs,
                                                               const float4* __restrict__ sf, float* __restrict__ w) {
    __shared__ float s_c[BW_K][BW_T + 1];
    __shared__ float s_max[BW_T];
    const int ntp = bs.nip + bs.ndp, R = (int)pp.rays;
    const int tx = threadIdx.x % BW_T, ky = threadIdx.x / BW_T;
    const int t = blockIdx.x * BW_T + tx;
    const bool irr = t < bs.nip;
    const int tt = irr ? t : t - bs.nip;
    const int n = irr ? v.irr_n : v.depth_n;
    const bool real = t < ntp && tt < n * n;
    const f3 dt = real ? texel_dir(tt % n, tt / n, n) : f3{0.f, 0.f, 0.f};
    float cmax = 0.f;
    if (real && !irr)
        for (int k = ky; k < R; k += BW_K) {
            const f3 d = rotate(pp, __ldg(sf + k));
            cmax = fmaxf(cmax, dt.x * d.x + dt.y * d.y + dt.z * d.z);
        }
    s_c[ky][tx] = cmax;
    __syncthreads();
    if (ky == 0) {
        float m = 0.f;
        for (int j = 0; j < BW_K; ++j) m = fmaxf(m, s_c[j][tx]);
        s_max[tx] = m;
    }
    __syncthreads();
    cmax = s_max[tx];
    float* part = w + (size_t)R * ntp;
    for (int k0 = 0; k0 < R; k0 += BW_K) {
        const int k = k0 + ky;
        float wk = 0.f;
        if (real && k < R) {
            const f3 d = rotate(pp, __ldg(sf + k));
            const float c = dt.x * d.x + dt.y * d.y + dt.z * d.z;
            if (c > 0.f) wk = irr ? c : __powf(c / cmax, pp.depth_sharpness);
        }
        if (t < ntp && k < R) w[(size_t)k * ntp + t] = wk;
        s_c[ky][tx] = wk;
        __syncthreads();
        const int g = k0 / 8 + ky;
        if (ky < BW_K / 8 && t < ntp && 8 * g < R) {
            float sum = 0.f;
            for (int j = 0; j < 8; ++j) sum += s_c[8 * ky + j][tx];
            part[(size_t)g * ntp + t] = sum;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Blend of G probes per CTA, one slice (blockIdx.y) of the products' warps
// per CTA.  The probes' ray data sit in shared memory, one row per ray
// (distance: d, d^2 of each probe, d = min(|t|, tmax); irradiance: L.rgb of
// each probe, padded); the weights stream through shared memory in chunks of
// bs.kc rays (cp.async, double-buffered), and each texel's weight sum adds
// the partial sums in ray order.  Each thread owns one 4 x 4 output tile (4
// texels x 4 columns: distance columns are (probe, moment), irradiance
// columns (probe, channel)) and sums it over the rays in order; a warp holds
// 8 row tiles x 4 column tiles, so one ray costs it one shared-memory
// wavefront of weights and one of ray data for 512 FMAs.  Epilogue: normalise by the texel's weight sum
// and mix with the old value by the hysteresis (texels whose weights sum to 0
// keep it).  With one slice per probe group the padded tiles are staged over
// the operands and written with their border texels; with several, the
// interior texels go straight to memory and k_probe_gutter refreshes the
// borders.
__global__ void __launch_bounds__(1024) k_probe_blend(VolumeView v, ProbeParams pp, BlendShape bs,
                                                      const float* __restrict__ w, const float4* __restrict__ rays,
                                                      int P) {
    extern __shared__ float4 smem4[];
    const int R = (int)pp.rays, G = bs.G;
    const int ni = v.irr_n, nd = v.depth_n, ni2 = ni * ni, nd2 = nd * nd;
    const int ti = ni + 2, td = nd + 2, ntp = bs.nip + bs.ndp;
    float* s_sum = reinterpret_cast<float*>(smem4);  // [ntp] weight sums
    float* s_bd = s_sum + ntp;                       // [R][2G]
    float* s_bi = s_bd + (size_t)R * 2 * G;          // [R][ci]
    float* s_w = s_bi + (size_t)R * bs.ci;           // [2][kc][ntp]
    const int p0 = blockIdx.x * G;
    const int tid = threadIdx.x;
    auto stage = [&](int c) {
        const int k0 = c * bs.kc, kc = min(bs.kc, R - k0);
        const float4* src = reinterpret_cast<const float4*>(w + (size_t)k0 * ntp);
        float4* dst = reinterpret_cast<float4*>(s_w + (size_t)(c & 1) * bs.kc * ntp);
        for (int i = tid; i < kc * ntp / 4; i += blockDim.x) cp_async16(dst + i, src + i);
        cp_async_commit();
    };
    stage(0);
    {
        const float* part = w + (size_t)R * ntp;
        const int nparts = (R + 7) / 8;
        for (int t = tid; t < ntp; t += blockDim.x) {
            float sum = 0.f;
            for (int j = 0; j < nparts; ++j) sum += __ldg(part + (size_t)j * ntp + t);
            s_sum[t] = sum;
        }
    }
    for (int i = tid; i < R * G; i += blockDim.x) {
        const int g = i / R, k = i - g * R;
        float4 ray = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p0 + g < P) ray = __ldg(rays + (size_t)(p0 + g) * R + k);
        const float d = fminf(fabsf(ray.w), pp.depth_tmax);
        s_bd[k * 2 * G + 2 * g] = d;
        s_bd[k * 2 * G + 2 * g + 1] = d * d;
        s_bi[k * bs.ci + 3 * g] = ray.x;
        s_bi[k * bs.ci + 3 * g + 1] = ray.y;
        s_bi[k * bs.ci + 3 * g + 2] = ray.z;
    }
    for (int i = tid; i < R * (bs.ci - 3 * G); i += blockDim.x) {   // pad columns
        const int k = i / (bs.ci - 3 * G), c = i - k * (bs.ci - 3 * G);
        s_bi[k * bs.ci + 3 * G + c] = 0.f;
    }
    // this thread's tile
    const int wg = blockIdx.y * bs.warps + (tid >> 5), lane = tid & 31;
    const int nwd = bs.rg_d * bs.cg_d, nwi = bs.rg_i * bs.cg_i;
    const bool is_d = wg < nwd, is_i = !is_d && wg < nwd + nwi;
    int rt = 0, ct = 0, nrt = 1, nct = 1;
    if (is_d) {
        rt = (wg % bs.rg_d) * 8 + (lane & 7);
        ct = (wg / bs.rg_d) * 4 + (lane >> 3);
        nrt = bs.ndp / 4;
        nct = 2 * G / 4;
    } else if (is_i) {
        const int wi = wg - nwd;
        rt = (wi % bs.rg_i) * 8 + (lane & 7);
        ct = (wi / bs.rg_i) * 4 + (lane >> 3);
        nrt = bs.nip / 4;
        nct = bs.ci / 4;
    }
    const bool live = (is_d || is_i) && rt < nrt && ct < nct;
    // clamped tile for lanes past the edge (their sums are not stored)
    const int wrow = (is_d ? bs.nip : 0) + 4 * min(rt, nrt - 1);
    const int col = 4 * min(ct, nct - 1);
    const float* bbase = is_d ? s_bd : s_bi;
    const int bstride = is_d ? 2 * G : bs.ci;
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.f;
    const int nchunk = (R + bs.kc - 1) / bs.kc;
    for (int c = 0; c < nchunk; ++c) {
        if (c + 1 < nchunk) {
            stage(c + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (is_d || is_i) {
            const float* wr = s_w + (size_t)(c & 1) * bs.kc * ntp + wrow;
            const int k0 = c * bs.kc, kc = min(bs.kc, R - k0);
            const float* br = bbase + (size_t)k0 * bstride + col;
#pragma unroll 4
            for (int kk = 0; kk < kc; ++kk) {
                const float4 wv = *reinterpret_cast<const float4*>(wr + kk * ntp);
                const float4 bv = *reinterpret_cast<const float4*>(br + kk * bstride);
                const float wa[4] = {wv.x, wv.y, wv.z, wv.w}, ba[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[4 * r + q] = fmaf(wa[r], ba[q], acc[4 * r + q]);
            }
        }
        __syncthreads();   // the buffer is refilled two chunks on
    }
    const float a = pp.hysteresis;
    const bool staged = bs.slices == 1;
    // padded tiles staged over the operands (after s_sum): [G][ti*ti] float4, [G][td*td] float2
    float4* s_irr = reinterpret_cast<float4*>(s_sum + (ntp + 3) / 4 * 4);
    float2* s_dep = reinterpret_cast<float2*>(s_irr + (size_t)G * ti * ti);
    if (live && is_d) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int t = wrow - bs.nip + r;
            if (t >= nd2) break;
            const float sw = s_sum[wrow + r];
            const int idx = (t / nd + 1) * td + (t % nd + 1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int g = col / 2 + h;
                if (g >= G || p0 + g >= P) break;
                float2* o = v.depth + (size_t)(p0 + g) * td * td + idx;
                float2 old = *o;
                if (sw > 0.f) {
                    old.x = a * old.x + (1.f - a) * (acc[4 * r + 2 * h] / sw);
                    old.y = a * old.y + (1.f - a) * (acc[4 * r + 2 * h + 1] / sw);
                }
                if (staged)
                    s_dep[g * td * td + idx] = old;
                else
                    *o = old;
            }
        }
    } else if (live) {
        const float* g_irr_f = reinterpret_cast<const float*>(v.irr);
        float* s_irr_f = reinterpret_cast<float*>(s_irr);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int t = wrow + r;
            if (t >= ni2) break;
            const float sw = s_sum[t];
            const int idx = (t / ni + 1) * ti + (t % ni + 1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int cc = col + q, g = cc / 3, ch = cc - 3 * g;
                if (g >= G || p0 + g >= P) break;
                const size_t o = ((size_t)(p0 + g) * ti * ti + idx) * 4;
                float old = g_irr_f[o + ch];
                if (sw > 0.f) old = a * old + (1.f - a) * (acc[4 * r + q] * (DDGI_PI / sw));
                if (staged) {
                    s_irr_f[((size_t)g * ti * ti + idx) * 4 + ch] = old;
                    if (ch == 0) s_irr_f[((size_t)g * ti * ti + idx) * 4 + 3] = g_irr_f[o + 3];
                } else {
                    reinterpret_cast<float*>(v.irr)[o + ch] = old;
                }
            }
        }
    }
    if (!staged) return;
    __syncthreads();
    // the padded tiles, border texels repeating their fold partner
    const int gn = min(G, P - p0);
    for (int i = tid; i < gn * ti * ti; i += blockDim.x) {
        const int g = i / (ti * ti), k = i - g * ti * ti;
        v.irr[(size_t)(p0 + g) * ti * ti + k] = s_irr[g * ti * ti + border_source(k % ti, k / ti, ni)];
    }
    for (int i = tid; i < gn * td * td; i += blockDim.x) {
        const int g = i / (td * td), k = i - g * td * td;
        v.depth[(size_t)(p0 + g) * td * td + k] = s_dep[g * td * td + border_source(k % td, k / td, nd)];
    }
    // the query's 2x2 tap blocks of the same tiles
    const int qi = (ni + 1) * (ni + 1), qd = (nd + 1) * (nd + 1);
    for (int i = tid; i < gn * qi; i += blockDim.x) {
        const int g = i / qi, j = i - g * qi, x0 = j % (ni + 1), y0 = j / (ni + 1);
        const float4* t = s_irr + (size_t)g * ti * ti;
        float4* o = v.irr_q + ((size_t)p0 * qi + i) * 4;
        st32(o, t[border_source(x0, y0, ni)], t[border_source(x0 + 1, y0, ni)]);
        st32(o + 2, t[border_source(x0, y0 + 1, ni)], t[border_source(x0 + 1, y0 + 1, ni)]);
    }
    for (int i = tid; i < gn * qd; i += blockDim.x) {
        const int g = i / qd, j = i - g * qd, x0 = j % (nd + 1), y0 = j / (nd + 1);
        const float2* t = s_dep + (size_t)g * td * td;
        const float2 a = t[border_source(x0, y0, nd)], b = t[border_source(x0 + 1, y0, nd)];
        const float2 c = t[border_source(x0, y0 + 1, nd)], e = t[border_source(x0 + 1, y0 + 1, nd)];
        st32(v.depth_q + ((size_t)p0 * qd + i) * 2, make_float4(a.x, a.y, b.x, b.y), make_float4(c.x, c.y, e.x, e.y));
    }
}

// border texels of every probe's padded tiles repeat their fold partner
// (after a blend whose CTAs each covered part of a probe's texels)
__global__ void __launch_bounds__(256) k_probe_gutter(VolumeView v, int P) {
    const int ni = v.irr_n, nd = v.depth_n, ti = ni + 2, td = nd + 2;
    const int bi = 4 * (ti - 1), bd = 4 * (td - 1);   // border texels per tile
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * (bi + bd)) return;
    const int p = i / (bi + bd), j = i - p * (bi + bd);
    const bool irr = j < bi;
    const int jj = irr ? j : j - bi, w = irr ? ti : td, n = irr ? ni : nd;
    // border walk: top row, bottom row, then the left and right columns
    int X, Y;
    if (jj < w) {
        X = jj, Y = 0;
    } else if (jj < 2 * w) {
        X = jj - w, Y = w - 1;
    } else {
        const int m = jj - 2 * w;
        X = (m & 1) ? w - 1 : 0;
        Y = 1 + (m >> 1);
    }
    const int src = border_source(X, Y, n);
    if (irr) {
        float4* tile = v.irr + (size_t)p * ti * ti;
        tile[Y * ti + X] = tile[src];
    } else {
        float2* tile = v.depth + (size_t)p * td * td;
        tile[Y * td + X] = tile[src];
    }
}

// the query's 2x2 tap blocks (VolumeView::irr_q / depth_q) of every probe,
// read from the padded tiles (borders included); one thread per block
__global__ void __launch_bounds__(256) k_probe_quads(VolumeView v, int P) {
    const int ni = v.irr_n, nd = v.depth_n, ti = ni + 2, td = nd + 2;
    const int qi = (ni + 1) * (ni + 1), qd = (nd + 1) * (nd + 1);
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t ni_all = (size_t)P * qi;
    if (i >= (size_t)P * (qi + qd)) return;
    if (i < ni_all) {
        const size_t p = i / qi;
        const int j = (int)(i - p * qi), x0 = j % (ni + 1), y0 = j / (ni + 1);
        const float4* t = v.irr + p * ti * ti + y0 * ti + x0;
        st32(v.irr_q + i * 4, t[0], t[1]);
        st32(v.irr_q + i * 4 + 2, t[ti], t[ti + 1]);
    } else {
        const size_t k = i - ni_all, p = k / qd;
        const int j = (int)(k - p * qd), x0 = j % (nd + 1), y0 = j / (nd + 1);
        const float2* t = v.depth + p * td * td + y0 * td + x0;
        st32(v.depth_q + k * 2, make_float4(t[0].x, t[0].y, t[1].x, t[1].y),
             make_float4(t[td].x, t[td].y, t[td + 1].x, t[td + 1].y));
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

namespace {

BlendShape blend_shape(const VolumeView& v, int G) {
    BlendShape b;
    b.G = G;
    b.nip = (v.irr_n * v.irr_n + 3) / 4 * 4;
    b.ndp = (v.depth_n * v.depth_n + 3) / 4 * 4;
    b.ci = (3 * G + 3) / 4 * 4;
    b.rg_d = (b.ndp / 4 + 7) / 8;
    b.cg_d = (2 * G / 4 + 3) / 4;
    b.rg_i = (b.nip / 4 + 7) / 8;
    b.cg_i = (b.ci / 4 + 3) / 4;
    const int total = b.rg_d * b.cg_d + b.rg_i * b.cg_i;
    b.slices = (total + 31) / 32;   // <= 32 warps per CTA
    b.warps = (total + b.slices - 1) / b.slices;
    b.kc = std::max(1, std::min(16, 8192 / (b.nip + b.ndp)));
    return b;
}

// shared memory of the blend: weight sums, the probes' ray rows and two
// weight chunks; with one slice, also room for the padded tiles staged
// after the sums
size_t blend_smem(const VolumeView& v, uint32_t rays, const BlendShape& b) {
    const size_t ntp = b.nip + b.ndp, ti = v.irr_n + 2, td = v.depth_n + 2;
    const size_t ops = sizeof(float) * (ntp + (size_t)rays * (2 * b.G + b.ci) + 2ull * b.kc * ntp);
    const size_t tiles = sizeof(float) * ((ntp + 3) / 4 * 4) +
                         b.G * (sizeof(float4) * ti * ti + sizeof(float2) * td * td);
    return b.slices == 1 && tiles > ops ? tiles : ops;
}

// probes per CTA: even, at most 16, the CTAs no more than the SMs where
// possible, <= 160 KB of shared memory
BlendShape pick_blend(const VolumeView& v, uint32_t rays, int P) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int G = (P + sms - 1) / sms;
    G = std::max(2, std::min(16, (G + 1) / 2 * 2));
    for (; G > 2; G -= 2)
        if (blend_smem(v, rays, blend_shape(v, G)) <= 160 * 1024) break;
    return blend_shape(v, G);
}

}  // namespace

size_t probe_blend_weights_size(const VolumeView& v, uint32_t rays) {
    const BlendShape b = blend_shape(v, 2);
    return (size_t)(b.nip + b.ndp) * (rays + (rays + 7) / 8);
}

size_t probe_blend_smem(const VolumeView& v, uint32_t rays) {
    const int P = v.counts.x * v.counts.y * v.counts.z;
    return blend_smem(v, rays, pick_blend(v, rays, P));
}

cudaError_t launch_probe_blend(const VolumeView& v, const ProbeParams& p, const float4* rays, float* weights,
                               cudaStream_t st) {
    const int P = v.counts.x * v.counts.y * v.counts.z;
    if (P == 0) return cudaSuccess;
    const BlendShape b = pick_blend(v, p.rays, P);
    k_blend_weights<<<(b.nip + b.ndp + BW_T - 1) / BW_T, BW_T * BW_K, 0, st>>>(v, p, b, p.sf, weights);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = blend_smem(v, p.rays, b);
    static size_t attr = 0;
    if (smem > 48 * 1024 && smem > attr) {
        e = cudaFuncSetAttribute(k_probe_blend, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    k_probe_blend<<<dim3((P + b.G - 1) / b.G, b.slices), 32 * b.warps, smem, st>>>(v, p, b, weights, rays, P);
    e = cudaGetLastError();
    if (e != cudaSuccess || b.slices == 1) return e;
    const int borders = P * (4 * (v.irr_n + 1) + 4 * (v.depth_n + 1));
    k_probe_gutter<<<(borders + 255) / 256, 256, 0, st>>>(v, P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_probe_quads(v, st);
}

cudaError_t launch_probe_quads(const VolumeView& v, cudaStream_t st) {
    const int P = v.counts.x * v.counts.y * v.counts.z;
    if (P == 0) return cudaSuccess;
    const size_t n = (size_t)P * ((v.irr_n + 1) * (v.irr_n + 1) + (v.depth_n + 1) * (v.depth_n + 1));
    k_probe_quads<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, P);
    return cudaGetLastError();
}
