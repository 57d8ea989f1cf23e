/* CPU oracle for DDGI resampling (arXiv 2108.05263).  TEST INFRASTRUCTURE:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file's library.  Plain C99, fp64 arithmetic, brute force everywhere,
 * one thread.  Decisions that turn a floating-point value into an integer
 * (emitter choice, reservoir selection) are taken in float32, the precision of
 * the CUDA kernels, as the method fixes no precision of its own.
 *
 * Sections cited are those of the paper; the readings taken where it is
 * silent (probe texel counts, Chebyshev form, attenuation units, candidate
 * split, random-number keys) are listed in the design notes. */
#include "ddgi_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846
#define T_EPS 1e-4          /* ray offset (m) */
#define MISS_T 1e30

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static void sub3(const double a[3], const double b[3], double c[3]) { c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2]; }
static double len3(const double a[3]) { return sqrt(dot3(a, a)); }
static double lum(const double c[3]) { return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2]; }
static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* ------------------------------------------------------------------------ */
/* scene                                                                    */
/* ------------------------------------------------------------------------ */

static void tri_geometry(or_scene* s, int32_t i) {
    const double* v = s->verts + 9 * i;
    double e1[3], e2[3], c[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    cross3(e1, e2, c);
    double l = len3(c);
    s->area[i] = 0.5 * l;
    for (int k = 0; k < 3; ++k) s->normal[3 * i + k] = l > 0 ? c[k] / l : 0.0;
}

static void identity34(double* m) {
    for (int k = 0; k < 12; ++k) m[k] = (k == 0 || k == 5 || k == 10) ? 1.0 : 0.0;
}

int or_scene_init(or_scene* s) {
    int32_t T = s->num_tris, I = s->tri_instance ? s->num_instances : 0;
    s->normal = (double*)malloc(sizeof(double) * 3 * (T > 0 ? T : 1));
    s->area = (double*)malloc(sizeof(double) * (T > 0 ? T : 1));
    s->emitter_tri = (int32_t*)malloc(sizeof(int32_t) * (T > 0 ? T : 1));
    s->emitter_of = (int32_t*)malloc(sizeof(int32_t) * (T > 0 ? T : 1));
    s->emitter_cdf = (float*)malloc(sizeof(float) * (T > 0 ? T : 1));
    s->inst_cur = (double*)malloc(sizeof(double) * 12 * (I > 0 ? I : 1));
    s->inst_prev = (double*)malloc(sizeof(double) * 12 * (I > 0 ? I : 1));
    if (!s->normal || !s->area || !s->emitter_tri || !s->emitter_of || !s->emitter_cdf || !s->inst_cur ||
        !s->inst_prev)
        return -1;
    for (int32_t k = 0; k < I; ++k) {
        identity34(s->inst_cur + 12 * k);
        identity34(s->inst_prev + 12 * k);
    }
    s->num_emitters = 0;
    double acc = 0.0;
    for (int32_t i = 0; i < T; ++i) {
        tri_geometry(s, i);
        s->emitter_of[i] = -1;
        const double* e = s->emission + 3 * i;
        if (e[0] > 0 || e[1] > 0 || e[2] > 0) {
            acc += s->area[i];
            s->emitter_of[i] = s->num_emitters;
            s->emitter_tri[s->num_emitters] = i;
            s->emitter_cdf[s->num_emitters] = (float)acc;
            s->num_emitters++;
        }
    }
    s->area_total = acc;
    return 0;
}

void or_scene_free(or_scene* s) {
    free(s->normal); free(s->area); free(s->emitter_tri); free(s->emitter_of); free(s->emitter_cdf);
    free(s->inst_cur); free(s->inst_prev);
    s->normal = NULL; s->area = NULL; s->emitter_tri = NULL; s->emitter_of = NULL; s->emitter_cdf = NULL;
    s->inst_cur = NULL; s->inst_prev = NULL;
}

/* y = M x for a row-major 3x4 affine transform */
static void xform(const double* m, const double x[3], double y[3]) {
    for (int r = 0; r < 3; ++r) y[r] = m[4 * r] * x[0] + m[4 * r + 1] * x[1] + m[4 * r + 2] * x[2] + m[4 * r + 3];
}

/* Scene dynamics (the dynamic scenes the method is built for, Sec. 1 and
 * Sec. 4): instanced triangles take positions M_i p0 from their identity-pose
 * positions p0 (xf: [n][12] row-major 3x4, n = num_instances; the old
 * transforms are kept for reprojection), and the emitters take new radiance
 * (emitter_radiance: [E][3] in emitter-list order).  Either may be NULL.  The
 * emitter list and its area distribution stay those of the first scene. */
int or_scene_update(or_scene* s, const double* xf, int32_t n, const double* emitter_radiance) {
    if (xf) {
        if (!s->tri_instance || n != s->num_instances) return -1;
        memcpy(s->inst_prev, s->inst_cur, sizeof(double) * 12 * (size_t)n);
        memcpy(s->inst_cur, xf, sizeof(double) * 12 * (size_t)n);
        for (int32_t i = 0; i < s->num_tris; ++i) {
            int32_t k = s->tri_instance[i];
            if (k < 0) continue;
            for (int c = 0; c < 3; ++c) xform(s->inst_cur + 12 * k, s->object_verts + 9 * i + 3 * c, s->verts + 9 * i + 3 * c);
            tri_geometry(s, i);
        }
    }
    if (emitter_radiance)
        for (int32_t e = 0; e < s->num_emitters; ++e)
            for (int c = 0; c < 3; ++c) s->emission[3 * s->emitter_tri[e] + c] = emitter_radiance[3 * e + c];
    return 0;
}

/* Where a point x on triangle tri was one update earlier: an instanced
 * triangle moved with its instance, x_prev = M_prev M_cur^-1 x (the 3x3 part
 * inverted by cofactors); a static one stayed. */
void or_prev_position(const or_scene* s, int32_t tri, const double x[3], double xp[3]) {
    int32_t k = (s->tri_instance && tri >= 0) ? s->tri_instance[tri] : -1;
    if (k < 0) {
        for (int a = 0; a < 3; ++a) xp[a] = x[a];
        return;
    }
    const double* m = s->inst_cur + 12 * k;
    double A[9] = {m[0], m[1], m[2], m[4], m[5], m[6], m[8], m[9], m[10]};
    double C[9] = {A[4] * A[8] - A[5] * A[7], A[2] * A[7] - A[1] * A[8], A[1] * A[5] - A[2] * A[4],
                   A[5] * A[6] - A[3] * A[8], A[0] * A[8] - A[2] * A[6], A[2] * A[3] - A[0] * A[5],
                   A[3] * A[7] - A[4] * A[6], A[1] * A[6] - A[0] * A[7], A[0] * A[4] - A[1] * A[3]};
    double det = A[0] * C[0] + A[1] * C[3] + A[2] * C[6];
    double d[3] = {x[0] - m[3], x[1] - m[7], x[2] - m[11]}, p0[3];
    for (int r = 0; r < 3; ++r) p0[r] = (C[3 * r] * d[0] + C[3 * r + 1] * d[1] + C[3 * r + 2] * d[2]) / det;
    xform(s->inst_prev + 12 * k, p0, xp);
}

/* ------------------------------------------------------------------------ */
/* counter-based random numbers: the PCG hash of Jarzynski and Olano,       */
/* "Hash Functions for GPU Rendering" (JCGT 2020), chained over the key     */
/* (seed, pixel, frame, pass, candidate, dimension).                         */
/* ------------------------------------------------------------------------ */

uint32_t or_pcg(uint32_t v) {
    uint32_t state = v * 747796405u + 2891336453u;
    uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}

uint32_t or_rng_u32(uint32_t seed, uint32_t pixel, uint32_t frame, uint32_t pass,
                    uint32_t cand, uint32_t dim) {
    uint32_t h = or_pcg(seed);
    h = or_pcg(h + pixel);
    h = or_pcg(h + frame);
    h = or_pcg(h + pass);
    h = or_pcg(h + cand);
    h = or_pcg(h + dim);
    return h;
}

double or_rng(uint32_t seed, uint32_t pixel, uint32_t frame, uint32_t pass,
              uint32_t cand, uint32_t dim) {
    /* the top 24 bits as a float in [0, 1) */
    return (double)(or_rng_u32(seed, pixel, frame, pass, cand, dim) >> 8) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------------ */
/* ray casting: brute force over every triangle (the hardware ray tracing   */
/* operation h of Sec. 3.2).  Moller-Trumbore, two-sided; the closest t in  */
/* (tmin, tmax) wins, equal t goes to the lower triangle index.              */
/* ------------------------------------------------------------------------ */

static int hit_tri(const double* v, const double o[3], const double d[3], double* t) {
    double e1[3], e2[3], p[3], tv[3], q[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    sub3(o, v, tv);
    double b1 = dot3(tv, p) * inv;
    if (b1 < 0.0 || b1 > 1.0) return 0;
    cross3(tv, e1, q);
    double b2 = dot3(d, q) * inv;
    if (b2 < 0.0 || b1 + b2 > 1.0) return 0;
    *t = dot3(e2, q) * inv;
    return 1;
}

int or_intersect(const or_scene* s, const double o[3], const double d[3],
                 double tmin, double tmax, int32_t* tri, double* t) {
    int32_t best = -1;
    double bt = tmax;
    for (int32_t i = 0; i < s->num_tris; ++i) {
        double ti;
        if (hit_tri(s->verts + 9 * i, o, d, &ti) && ti > tmin && ti < tmax) {
            if (best < 0 || ti < bt) { best = i; bt = ti; }
        }
    }
    *tri = best;
    *t = best >= 0 ? bt : MISS_T;
    return best >= 0;
}

void or_trace_batch(const or_scene* s, int32_t n, const double* o, const double* d,
                    double tmin, double tmax, int32_t* tri, double* t) {
    for (int32_t i = 0; i < n; ++i) or_intersect(s, o + 3 * i, d + 3 * i, tmin, tmax, tri + i, t + i);
}

static int occluded(const or_scene* s, const double o[3], const double d[3], double tmin, double tmax) {
    for (int32_t i = 0; i < s->num_tris; ++i) {
        double ti;
        if (hit_tri(s->verts + 9 * i, o, d, &ti) && ti > tmin && ti < tmax) return 1;
    }
    return 0;
}

/* Emitters are chosen with probability proportional to area: the first
 * emitter whose cumulative area exceeds u times the total (decided in float). */
int32_t or_sample_emitter(const or_scene* s, double u) {
    int32_t E = s->num_emitters;
    float target = (float)u * s->emitter_cdf[E - 1];
    for (int32_t i = 0; i < E; ++i)
        if (target < s->emitter_cdf[i]) return s->emitter_tri[i];
    return s->emitter_tri[E - 1];
}

/* ------------------------------------------------------------------------ */
/* probe representation (DDGI volume cited in Sec. 2 and Sec. 3.2): octa-   */
/* hedral maps of irradiance and of mean / mean-square distance, each with a */
/* one-texel border that repeats the texel across the octahedral fold.       */
/* ------------------------------------------------------------------------ */

static double sgn(double x) { return x >= 0.0 ? 1.0 : -1.0; }

void or_oct_encode(const double d[3], double uv[2]) {
    double s = fabs(d[0]) + fabs(d[1]) + fabs(d[2]);
    double u = d[0] / s, v = d[1] / s;
    if (d[2] < 0.0) {
        double fu = (1.0 - fabs(v)) * sgn(u);
        double fv = (1.0 - fabs(u)) * sgn(v);
        u = fu; v = fv;
    }
    uv[0] = u; uv[1] = v;
}

void or_oct_decode(const double uv[2], double d[3]) {
    double u = uv[0], v = uv[1];
    double z = 1.0 - fabs(u) - fabs(v);
    double x = u, y = v;
    if (z < 0.0) {
        x = (1.0 - fabs(v)) * sgn(u);
        y = (1.0 - fabs(u)) * sgn(v);
    }
    double l = sqrt(x * x + y * y + z * z);
    d[0] = x / l; d[1] = y / l; d[2] = z / l;
}

/* direction at the centre of interior texel (column i, row j) of an n x n map */
void or_texel_dir(int32_t i, int32_t j, int32_t n, double d[3]) {
    double uv[2] = {2.0 * (i + 0.5) / n - 1.0, 2.0 * (j + 0.5) / n - 1.0};
    or_oct_decode(uv, d);
}

/* Border texels copy the interior texel that lies across the fold: an edge
 * texel mirrors along that edge, a corner takes the opposite corner. */
void or_gutter(double* tile, int32_t n, int32_t ch) {
    int32_t w = n + 2;
#define TX(X, Y) (tile + ((Y) * w + (X)) * ch)
    for (int32_t X = 1; X <= n; ++X) {
        memcpy(TX(X, 0), TX(n + 1 - X, 1), sizeof(double) * ch);
        memcpy(TX(X, n + 1), TX(n + 1 - X, n), sizeof(double) * ch);
    }
    for (int32_t Y = 1; Y <= n; ++Y) {
        memcpy(TX(0, Y), TX(1, n + 1 - Y), sizeof(double) * ch);
        memcpy(TX(n + 1, Y), TX(n, n + 1 - Y), sizeof(double) * ch);
    }
    memcpy(TX(0, 0), TX(n, n), sizeof(double) * ch);
    memcpy(TX(n + 1, 0), TX(1, n), sizeof(double) * ch);
    memcpy(TX(0, n + 1), TX(n, 1), sizeof(double) * ch);
    memcpy(TX(n + 1, n + 1), TX(1, 1), sizeof(double) * ch);
#undef TX
}

void or_fill_gutters(or_volume* v) {
    int32_t P = v->counts[0] * v->counts[1] * v->counts[2];
    int32_t wi = v->irr_n + 2, wd = v->depth_n + 2;
    for (int32_t p = 0; p < P; ++p) {
        or_gutter(v->irr + (size_t)p * wi * wi * 3, v->irr_n, 3);
        or_gutter(v->depth + (size_t)p * wd * wd * 2, v->depth_n, 2);
    }
}

/* Bilinear lookup of a padded (n+2)^2 tile in direction d. */
void or_bilinear(const double* tile, int32_t n, int32_t ch, const double d[3], double* out) {
    double uv[2];
    or_oct_encode(d, uv);
    int32_t w = n + 2;
    double fx = (uv[0] + 1.0) * 0.5 * n + 1.0 - 0.5;
    double fy = (uv[1] + 1.0) * 0.5 * n + 1.0 - 0.5;
    double x0f = floor(fx), y0f = floor(fy);
    double ax = fx - x0f, ay = fy - y0f;
    int32_t x0 = (int32_t)x0f, y0 = (int32_t)y0f;
    if (x0 < 0) { x0 = 0; ax = 0.0; }
    if (y0 < 0) { y0 = 0; ay = 0.0; }
    if (x0 > n) { x0 = n; ax = 1.0; }
    if (y0 > n) { y0 = n; ay = 1.0; }
    for (int32_t c = 0; c < ch; ++c) {
        double t00 = tile[(y0 * w + x0) * ch + c], t10 = tile[(y0 * w + x0 + 1) * ch + c];
        double t01 = tile[((y0 + 1) * w + x0) * ch + c], t11 = tile[((y0 + 1) * w + x0 + 1) * ch + c];
        out[c] = (1 - ay) * ((1 - ax) * t00 + ax * t10) + ay * ((1 - ax) * t01 + ax * t11);
    }
}

void or_probe_pos(const or_volume* v, int32_t p, double P[3]) {
    int32_t i = p % v->counts[0];
    int32_t j = (p / v->counts[0]) % v->counts[1];
    int32_t k = p / (v->counts[0] * v->counts[1]);
    int32_t g[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) P[a] = v->origin[a] + v->spacing[a] * g[a] + v->offset[3 * p + a];
}

static double min_spacing(const or_volume* v) {
    double m = v->spacing[0];
    if (v->spacing[1] < m) m = v->spacing[1];
    if (v->spacing[2] < m) m = v->spacing[2];
    return m;
}
static double max_spacing(const or_volume* v) {
    double m = v->spacing[0];
    if (v->spacing[1] > m) m = v->spacing[1];
    if (v->spacing[2] > m) m = v->spacing[2];
    return m;
}

/* Irradiance E(q, n) from the 8 probes around q: trilinear weights times a
 * wrap-shading term times the cubed Chebyshev visibility bound from the
 * probe's distance moments, with weights below 0.2 crushed, then normalised. */
double or_ddgi_query(const or_volume* v, const double q[3], const double n[3], double E[3]) {
    int32_t base[3];
    double alpha[3];
    for (int a = 0; a < 3; ++a) {
        double g = (q[a] - v->origin[a]) / v->spacing[a];
        int32_t hi = v->counts[a] - 2;
        if (hi < 0) hi = 0;
        double f = floor(g);
        int32_t b = f < 0 ? 0 : (f > hi ? hi : (int32_t)f);
        base[a] = b;
        alpha[a] = v->counts[a] > 1 ? clampd(g - b, 0.0, 1.0) : 0.0;
    }
    int32_t wi = v->irr_n + 2, wd = v->depth_n + 2;
    double sw = 0.0, se[3] = {0, 0, 0};
    for (int c = 0; c < 8; ++c) {
        int32_t off[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        int32_t gi[3];
        double tri = 1.0;
        for (int a = 0; a < 3; ++a) {
            gi[a] = base[a] + off[a];
            if (gi[a] > v->counts[a] - 1) gi[a] = v->counts[a] - 1;
            tri *= off[a] ? alpha[a] : 1.0 - alpha[a];
        }
        int32_t p = gi[0] + v->counts[0] * (gi[1] + v->counts[1] * gi[2]);
        double P[3], dir[3];
        or_probe_pos(v, p, P);
        sub3(P, q, dir);
        double r = len3(dir);
        if (r > 0.0) { dir[0] /= r; dir[1] /= r; dir[2] /= r; }
        else { dir[0] = n[0]; dir[1] = n[1]; dir[2] = n[2]; }
        double wrap = 0.5 * (dot3(dir, n) + 1.0);
        double w = wrap * wrap + 0.2;
        double back[3] = {-dir[0], -dir[1], -dir[2]};
        double mom[2];
        or_bilinear(v->depth + (size_t)p * wd * wd * 2, v->depth_n, 2, back, mom);
        if (r > mom[0]) {
            double var = fabs(mom[1] - mom[0] * mom[0]);
            double dd = r - mom[0];
            double ch = var / (var + dd * dd);
            w *= ch * ch * ch;
        }
        if (w < 1e-6) w = 1e-6;
        if (w < 0.2) w = w * w * w / (0.2 * 0.2);
        w *= tri;
        double irr[3];
        or_bilinear(v->irr + (size_t)p * wi * wi * 3, v->irr_n, 3, n, irr);
        for (int k = 0; k < 3; ++k) se[k] += w * irr[k];
        sw += w;
    }
    for (int k = 0; k < 3; ++k) E[k] = sw > 0.0 ? se[k] / sw : 0.0;
    return sw;
}

/* View-path bias (Sec. 3.4): the query point moves from y back toward the
 * previous path vertex by d = min(0.2 * min probe spacing, half the segment). */
static void biased_point(const or_volume* v, const double y[3], const double from[3], double q[3]) {
    double d[3];
    sub3(from, y, d);
    double l = len3(d);
    q[0] = y[0]; q[1] = y[1]; q[2] = y[2];
    if (l > 0.0) {
        double dv = 0.2 * min_spacing(v);
        if (0.5 * l < dv) dv = 0.5 * l;
        for (int a = 0; a < 3; ++a) q[a] = y[a] + dv * d[a] / l;
    }
}

void or_biased_query(const or_volume* v, const double y[3], const double n_y[3],
                     const double from[3], double E[3]) {
    double q[3];
    biased_point(v, y, from, q);
    or_ddgi_query(v, q, n_y, E);
}

/* ------------------------------------------------------------------------ */
/* glossy lobe (Sec. 3.3): a GGX microfacet lobe per triangle, reflectance   */
/* k_s and roughness alpha, f_g = k_s D(h) G1(wo) G1(wi) / (4 |n.wo| |n.wi|) */
/* (separable Smith masking, no Fresnel term)                               */
/* ------------------------------------------------------------------------ */

/* GGX (Trowbridge-Reitz) distribution of normals */
double or_ggx_D(double nh, double a) {
    if (nh <= 0.0) return 0.0;
    double a2 = a * a;
    double den = nh * nh * (a2 - 1.0) + 1.0;
    return a2 / (PI * den * den);
}

/* Smith masking of one direction for GGX */
double or_ggx_G1(double nw, double a) {
    if (nw <= 0.0) return 0.0;
    double a2 = a * a;
    return 2.0 * nw / (nw + sqrt(a2 + (1.0 - a2) * nw * nw));
}

/* half vector with density D(h) (n.h): cos^2 theta = (1 - u0) / (1 + (a^2 - 1) u0),
 * azimuth 2 pi u1 in the basis around n */
void or_ggx_sample_h(const double n[3], double a, double u0, double u1, double h[3]) {
    double c2 = (1.0 - u0) / (1.0 + (a * a - 1.0) * u0);
    double c = sqrt(c2), sn = sqrt(fmax(0.0, 1.0 - c2)), ph = 2.0 * PI * u1;
    double l[3] = {sn * cos(ph), sn * sin(ph), c};
    or_onb_local_to_world(n, l, h);
}

/* One direction wi drawn proportionally to the glossy lobe (the mirror of wo
 * about a half vector drawn by or_ggx_sample_h), its density
 * pdf = D (n.h) / (4 |wo.h|) and the weight f_g (n.wi) / pdf per channel.
 * Returns 0 (weight 0) when wi falls below the surface. */
int or_glossy_sample(const double n[3], const double wo[3], const double ks[3], double a, double u0,
                     double u1, double wi[3], double wgt[3], double* pdf) {
    double h[3];
    or_ggx_sample_h(n, a, u0, u1, h);
    double oh = dot3(wo, h);
    for (int k = 0; k < 3; ++k) wi[k] = 2.0 * oh * h[k] - wo[k];
    wgt[0] = wgt[1] = wgt[2] = 0.0;
    *pdf = 0.0;
    double ni = dot3(n, wi), no = dot3(n, wo), nh = dot3(n, h);
    if (ni <= 0.0 || no <= 0.0 || nh <= 0.0 || oh <= 0.0) return 0;
    *pdf = or_ggx_D(nh, a) * nh / (4.0 * oh);
    double g = or_ggx_G1(no, a) * or_ggx_G1(ni, a) * oh / (no * nh);
    for (int k = 0; k < 3; ++k) wgt[k] = ks[k] * g;
    return 1;
}

/* The glossy half of Eq. lddgiplus at a point with normal n seen from wo:
 * one sample wi of the glossy lobe, E(q, wi) read as cosine-prefiltered
 * incident radiance around wi, (1 / pi) E(q, wi) f_g (n.wi) / pdf.  (With E
 * normalised so that uniform radiance L gives pi L, 1 / pi reflects a uniform
 * environment exactly; the paper prints 1 / (2 pi) for its own
 * normalisation of E.) */
static void glossy_ddgi(const or_volume* v, const double q[3], const double n[3], const double wo[3],
                        const double* spec, double u0, double u1, double out[3]) {
    double wi[3], wgt[3], pdf;
    out[0] = out[1] = out[2] = 0.0;
    if (!or_glossy_sample(n, wo, spec, spec[3], u0, u1, wi, wgt, &pdf)) return;
    double E[3];
    or_ddgi_query(v, q, wi, E);
    for (int k = 0; k < 3; ++k) out[k] = E[k] / PI * wgt[k];
}

static int has_glossy(const or_scene* s, int32_t tri) {
    if (!s->glossy) return 0;
    const double* g = s->glossy + 4 * tri;
    return g[0] > 0 || g[1] > 0 || g[2] > 0;
}

/* ------------------------------------------------------------------------ */
/* probe update (Sec. 3.2, Eq. probeUpdate)                                 */
/* ------------------------------------------------------------------------ */

/* spherical Fibonacci point i of n */
void or_sf_dir(int32_t i, int32_t n, double d[3]) {
    double z = 1.0 - (2.0 * i + 1.0) / n;
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    double ph = i * 0.6180339887498949;    /* (sqrt(5) - 1) / 2 */
    ph = 2.0 * PI * (ph - floor(ph));
    d[0] = r * cos(ph); d[1] = r * sin(ph); d[2] = z;
}

/* per-frame random rotation from a uniform random unit quaternion
 * (Shoemake, "Uniform random rotations", Graphics Gems III) */
void or_probe_rotation(uint32_t seed, uint32_t frame, double R[9]) {
    double u0 = or_rng(seed, 0, frame, OR_PASS_PROBE_ROT, 0, 0);
    double u1 = or_rng(seed, 0, frame, OR_PASS_PROBE_ROT, 0, 1);
    double u2 = or_rng(seed, 0, frame, OR_PASS_PROBE_ROT, 0, 2);
    double a = sqrt(1.0 - u0), b = sqrt(u0);
    double x = a * sin(2 * PI * u1), y = a * cos(2 * PI * u1);
    double z = b * sin(2 * PI * u2), w = b * cos(2 * PI * u2);
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
    R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
    R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}

void or_probe_ray_dir(const double R[9], int32_t r, int32_t n, double d[3]) {
    double s[3];
    or_sf_dir(r, n, s);
    for (int a = 0; a < 3; ++a) d[a] = R[3 * a] * s[0] + R[3 * a + 1] * s[1] + R[3 * a + 2] * s[2];
}

/* distance from the probe to the boundary of its own cell along d */
static double cell_exit(const or_volume* v, const double d[3]) {
    double t = MISS_T;
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0) {
            double ta = 0.5 * v->spacing[a] / fabs(d[a]);
            if (ta < t) t = ta;
        }
    }
    return t;
}

/* For probe p and ray r: the radiance (L_DDGI+ + Le)(h(x, w), -w) of
 * Eq. probeUpdate.  Le is attenuated by (t / (t + s * d_back))^2 where d_back
 * is the probe's mean distance in the backward direction clipped to its cell
 * (Sec. 3.2); L_DDGI+ = rho / pi * E at the view-path-biased hit.  Back faces
 * and misses carry no radiance; the distance slot is +t (front), -t (back) or
 * 1e30 (miss). */
int or_probe_trace(const or_scene* s, const or_volume* v, const or_settings* st,
                   uint32_t frame, const int32_t* probes, int32_t nprobes, double* rays) {
    int32_t R = st->rays_per_probe;
    double Rf[9];
    or_probe_rotation(st->seed, frame, Rf);
    int32_t wd = v->depth_n + 2;
    for (int32_t k = 0; k < nprobes; ++k) {
        int32_t p = probes ? probes[k] : k;
        double P[3];
        or_probe_pos(v, p, P);
        for (int32_t r = 0; r < R; ++r) {
            double* out = rays + ((size_t)k * R + r) * 4;
            double w[3];
            or_probe_ray_dir(Rf, r, R, w);
            int32_t tri;
            double t;
            out[0] = out[1] = out[2] = 0.0;
            if (!or_intersect(s, P, w, T_EPS, MISS_T, &tri, &t)) { out[3] = MISS_T; continue; }
            const double* n_y = s->normal + 3 * tri;
            if (dot3(n_y, w) > 0.0) { out[3] = -t; continue; }
            out[3] = t;
            double att = 1.0;
            if (st->le_attenuation > 0.0) {
                double back[3] = {-w[0], -w[1], -w[2]};
                double mom[2];
                or_bilinear(v->depth + (size_t)p * wd * wd * 2, v->depth_n, 2, back, mom);
                double db = mom[0];
                double ce = cell_exit(v, back);
                if (ce < db) db = ce;
                double f = t / (t + st->le_attenuation * db);
                att = f * f;
            }
            const double* le = s->emission + 3 * tri;
            const double* rho = s->albedo + 3 * tri;
            double y[3] = {P[0] + t * w[0], P[1] + t * w[1], P[2] + t * w[2]};
            double q[3], E[3] = {0, 0, 0};
            biased_point(v, y, P, q);
            if (rho[0] > 0 || rho[1] > 0 || rho[2] > 0) or_ddgi_query(v, q, n_y, E);
            for (int c = 0; c < 3; ++c) out[c] = le[c] * att + rho[c] / PI * E[c];
            if (has_glossy(s, tri)) {   /* the glossy half of L_DDGI+ toward the probe */
                double wo[3] = {-w[0], -w[1], -w[2]}, G[3];
                double u0 = or_rng(st->seed, (uint32_t)p, frame, OR_PASS_PROBE_GLOSSY, (uint32_t)r, 0);
                double u1 = or_rng(st->seed, (uint32_t)p, frame, OR_PASS_PROBE_GLOSSY, (uint32_t)r, 1);
                glossy_ddgi(v, q, n_y, wo, s->glossy + 4 * tri, u0, u1, G);
                for (int c = 0; c < 3; ++c) out[c] += G[c];
            }
        }
    }
    return 0;
}

/* Monte Carlo estimate of the integral of Eq. probeUpdate per texel
 * direction (irradiance, normalised so that uniform radiance L gives pi L),
 * cosine-power-weighted distance moments, blended with hysteresis (weight 0
 * on the first update), then the border refresh. */
int or_probe_blend(or_volume* v, const or_settings* st, uint32_t frame,
                   const int32_t* probes, int32_t nprobes, const double* rays) {
    int32_t R = st->rays_per_probe;
    double Rf[9];
    or_probe_rotation(st->seed, frame, Rf);
    double* dirs = (double*)malloc(sizeof(double) * 3 * R);
    if (!dirs) return -1;
    for (int32_t r = 0; r < R; ++r) or_probe_ray_dir(Rf, r, R, dirs + 3 * r);
    double alpha = v->updates == 0 ? 0.0 : st->hysteresis;
    double tmax = 1.5 * max_spacing(v);
    int32_t ni = v->irr_n, nd = v->depth_n, wi = ni + 2, wd = nd + 2;
    for (int32_t k = 0; k < nprobes; ++k) {
        int32_t p = probes ? probes[k] : k;
        const double* ray = rays + (size_t)k * R * 4;
        double* irr = v->irr + (size_t)p * wi * wi * 3;
        double* dep = v->depth + (size_t)p * wd * wd * 2;
        for (int32_t j = 0; j < ni; ++j)
            for (int32_t i = 0; i < ni; ++i) {
                double dt[3];
                or_texel_dir(i, j, ni, dt);
                double sw = 0.0, sl[3] = {0, 0, 0};
                for (int32_t r = 0; r < R; ++r) {
                    double c = dot3(dt, dirs + 3 * r);
                    if (c <= 0.0) continue;
                    sw += c;
                    for (int a = 0; a < 3; ++a) sl[a] += c * ray[4 * r + a];
                }
                if (sw <= 0.0) continue;
                double* tx = irr + ((j + 1) * wi + (i + 1)) * 3;
                for (int a = 0; a < 3; ++a) tx[a] = alpha * tx[a] + (1.0 - alpha) * (PI * sl[a] / sw);
            }
        for (int32_t j = 0; j < nd; ++j)
            for (int32_t i = 0; i < nd; ++i) {
                double dt[3];
                or_texel_dir(i, j, nd, dt);
                double sw = 0.0, s1 = 0.0, s2 = 0.0;
                for (int32_t r = 0; r < R; ++r) {
                    double c = dot3(dt, dirs + 3 * r);
                    if (c <= 0.0) continue;
                    double wr = pow(c, st->depth_sharpness);
                    double td = fabs(ray[4 * r + 3]);
                    if (td > tmax) td = tmax;
                    sw += wr; s1 += wr * td; s2 += wr * td * td;
                }
                if (sw <= 0.0) continue;
                double* tx = dep + ((j + 1) * wd + (i + 1)) * 2;
                tx[0] = alpha * tx[0] + (1.0 - alpha) * (s1 / sw);
                tx[1] = alpha * tx[1] + (1.0 - alpha) * (s2 / sw);
            }
        or_gutter(irr, ni, 3);
        or_gutter(dep, nd, 2);
    }
    free(dirs);
    return 0;
}

/* Probe relocation (the paper cites it for its probe volume, Sec. 2; the
 * method is that of Majercik et al. 2021): from this frame's rays of a probe,
 * with delta = 0.1 * min spacing the smallest distance a probe keeps from a
 * front face:
 *   - more than a quarter of the rays hit back faces (the probe sits inside
 *     geometry): move along the direction of the closest back-face hit by its
 *     distance + delta / 2, through that face;
 *   - else if the closest front-face hit is nearer than delta: move away from
 *     it by the shortfall;
 * then clamp every axis of the offset to +-0.45 of the grid spacing, so a
 * probe never leaves its cell's inner region.  Misses count as neither. */
int or_probe_relocate(or_volume* v, const or_settings* st, uint32_t frame,
                      const int32_t* probes, int32_t nprobes, const double* rays) {
    int32_t R = st->rays_per_probe;
    double Rf[9];
    or_probe_rotation(st->seed, frame, Rf);
    double delta = v->spacing[0];
    for (int a = 1; a < 3; ++a)
        if (v->spacing[a] < delta) delta = v->spacing[a];
    delta *= 0.1;
    for (int32_t k = 0; k < nprobes; ++k) {
        int32_t p = probes ? probes[k] : k;
        const double* ray = rays + (size_t)k * R * 4;
        int32_t nback = 0, rb = -1, rf = -1;
        double tb = MISS_T, tf = MISS_T;
        for (int32_t r = 0; r < R; ++r) {
            double t = ray[4 * r + 3];
            if (t >= MISS_T) continue;
            if (t < 0.0) {
                ++nback;
                if (-t < tb) { tb = -t; rb = r; }
            } else if (t < tf) {
                tf = t;
                rf = r;
            }
        }
        double* off = v->offset + 3 * (size_t)p;
        double d[3];
        if (4 * nback > R && rb >= 0) {
            or_probe_ray_dir(Rf, rb, R, d);
            for (int a = 0; a < 3; ++a) off[a] += d[a] * (tb + 0.5 * delta);
        } else if (rf >= 0 && tf < delta) {
            or_probe_ray_dir(Rf, rf, R, d);
            for (int a = 0; a < 3; ++a) off[a] -= d[a] * (delta - tf);
        }
        for (int a = 0; a < 3; ++a) {
            double lim = 0.45 * v->spacing[a];
            if (off[a] > lim) off[a] = lim;
            if (off[a] < -lim) off[a] = -lim;
        }
    }
    return 0;
}

/* one full update: trace every probe against the previous maps, blend, and
 * (when enabled) relocate */
int or_probe_update(const or_scene* s, or_volume* v, const or_settings* st, uint32_t frame) {
    int32_t P = v->counts[0] * v->counts[1] * v->counts[2];
    double* rays = (double*)malloc(sizeof(double) * 4 * (size_t)P * st->rays_per_probe);
    if (!rays) return -1;
    or_probe_trace(s, v, st, frame, NULL, P, rays);
    int rc = or_probe_blend(v, st, frame, NULL, P, rays);
    if (rc == 0 && st->relocate) rc = or_probe_relocate(v, st, frame, NULL, P, rays);
    v->updates++;
    free(rays);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* primary visibility (support pass): pinhole rays through pixel centres     */
/* ------------------------------------------------------------------------ */

int or_gbuffer(const or_scene* s, const or_camera* cam, const or_camera* pc,
               const int32_t* pix, int32_t npix, or_gbuf* g) {
    int32_t W = cam->width, H = cam->height;
    double aspect = (double)W / H;
    for (int32_t k = 0; k < npix; ++k) {
        int32_t q = pix ? pix[k] : k;
        int32_t i = q % W, j = q / W;
        double sx = (2.0 * (i + 0.5) / W - 1.0) * cam->tan_half_fovy * aspect;
        double sy = (1.0 - 2.0 * (j + 0.5) / H) * cam->tan_half_fovy;
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = cam->fwd[a] + sx * cam->right[a] + sy * cam->up[a];
        double l = len3(d);
        for (int a = 0; a < 3; ++a) d[a] /= l;
        int32_t tri;
        double t;
        g->tri[k] = -1;
        g->prev[k] = -1;
        g->dist[k] = 0.0;
        for (int a = 0; a < 3; ++a) g->pos[3 * k + a] = g->nrm[3 * k + a] = g->alb[3 * k + a] = 0.0;
        if (!or_intersect(s, cam->pos, d, T_EPS, MISS_T, &tri, &t)) continue;
        const double* n = s->normal + 3 * tri;
        if (dot3(n, d) > 0.0) continue;
        g->tri[k] = tri;
        g->dist[k] = t;
        for (int a = 0; a < 3; ++a) {
            g->pos[3 * k + a] = cam->pos[a] + t * d[a];
            g->nrm[3 * k + a] = n[a];
            g->alb[3 * k + a] = s->albedo[3 * tri + a];
        }
        if (pc) {
            double vv[3], xp[3];
            or_prev_position(s, tri, g->pos + 3 * k, xp);
            sub3(xp, pc->pos, vv);
            double z = dot3(vv, pc->fwd);
            if (z > 0.0) {
                double px = dot3(vv, pc->right) / z / (pc->tan_half_fovy * aspect);
                double py = dot3(vv, pc->up) / z / pc->tan_half_fovy;
                double fx = (px + 1.0) * 0.5 * W, fy = (1.0 - py) * 0.5 * H;
                if (fx >= 0.0 && fy >= 0.0 && fx < W && fy < H)
                    g->prev[k] = (int32_t)floor(fy) * W + (int32_t)floor(fx);
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* resampling (Sec. 3.1 steps 1-2, Sec. 3.5, Sec. 3.6)                       */
/* ------------------------------------------------------------------------ */

/* Target function at shading point x for a sample y on triangle tri with
 * outgoing radiance L (Sec. 3.1 step 2, bounded geometry term of Sec. 3.5):
 * luminance of rho_x / pi * L * min(G, 1); no visibility. */
/* target of a point y with unit normal ny (only |cos| at y enters) */
static double target_with_normal(const double x[3], const double nx[3], const double rho[3], const double y[3],
                                 const double ny[3], const double L[3]) {
    double d[3];
    sub3(y, x, d);
    double d2 = dot3(d, d);
    if (d2 <= 0.0) return 0.0;
    double l = sqrt(d2);
    double w[3] = {d[0] / l, d[1] / l, d[2] / l};
    double cx = dot3(nx, w);
    if (cx <= 0.0) return 0.0;
    double cy = fabs(dot3(ny, w));
    double G = cx * cy / d2;
    double Gb = G < 1.0 ? G : 1.0;
    double f[3] = {rho[0] / PI * L[0] * Gb, rho[1] / PI * L[1] * Gb, rho[2] / PI * L[2] * Gb};
    return lum(f);
}

double or_target(const or_scene* s, const double x[3], const double nx[3],
                 const double rho[3], const double y[3], int32_t tri, const double L[3]) {
    if (tri < 0) return 0.0;
    return target_with_normal(x, nx, rho, y, s->normal + 3 * tri, L);
}

/* Orthonormal basis around n (Duff et al., "Building an Orthonormal Basis,
 * Revisited", JCGT 2017); l is (tangent, bitangent, normal) coordinates. */
void or_onb_local_to_world(const double n[3], const double l[3], double w[3]) {
    double sign = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    double t[3] = {1.0 + sign * n[0] * n[0] * a, sign * b, -sign * n[0]};
    double bt[3] = {b, sign + n[1] * n[1] * a, -n[1]};
    for (int k = 0; k < 3; ++k) w[k] = l[0] * t[k] + l[1] * bt[k] + l[2] * n[k];
}

/* Network of the learned target form: frequency-encoded position (12
 * frequencies, 3 axes, sin and cos), normal, 5 zeros; 4 ReLU layers of 64; a
 * linear 3-channel output.  Parameters in the library's documented layout. */
void or_mlp_eval(const or_volume* v, const double p[3], const double n[3], double out[3]) {
    static const int off_w[5] = {0, 5120, 9216, 13312, 17408};
    double x[80], h[64], g[64];
    for (int a = 0; a < 3; ++a) {
        double q = (p[a] - v->mlp_lo[a]) * v->mlp_scale;
        for (int k = 0; k < 12; ++k) {
            double arg = ldexp(1.0, k) * PI * q;
            x[24 * a + 2 * k] = sin(arg);
            x[24 * a + 2 * k + 1] = cos(arg);
        }
    }
    x[72] = n[0]; x[73] = n[1]; x[74] = n[2];
    for (int i = 75; i < 80; ++i) x[i] = 0.0;
    const double* w = v->mlp;
    for (int o = 0; o < 64; ++o) {
        double acc = w[17920 + o];
        for (int i = 0; i < 80; ++i) acc += w[off_w[0] + o * 80 + i] * x[i];
        h[o] = acc > 0.0 ? acc : 0.0;
    }
    for (int l = 1; l < 4; ++l) {
        for (int o = 0; o < 64; ++o) {
            double acc = w[17920 + 64 * l + o];
            for (int i = 0; i < 64; ++i) acc += w[off_w[l] + o * 64 + i] * h[i];
            g[o] = acc > 0.0 ? acc : 0.0;
        }
        memcpy(h, g, sizeof(h));
    }
    for (int o = 0; o < 3; ++o) {
        double acc = w[17920 + 256 + o];
        for (int i = 0; i < 64; ++i) acc += w[off_w[4] + o * 64 + i] * h[i];
        out[o] = acc;
    }
}

/* outgoing radiance (Le + L_DDGI+)(y, y -> x): emission is one-sided, back
 * faces carry nothing, the probe term is queried with the view-path bias (or
 * the network is evaluated at y in the learned target form); a glossy
 * triangle adds the one-sample glossy half of Eq. lddgiplus, drawn with the
 * random numbers (u0, u1) */
static void radiance_at(const or_scene* s, const or_volume* v, const double y[3], int32_t tri,
                        const double x[3], double u0, double u1, double L[3]) {
    const double* n = s->normal + 3 * tri;
    double d[3];
    sub3(x, y, d);
    L[0] = L[1] = L[2] = 0.0;
    if (dot3(n, d) <= 0.0) return;
    const double* le = s->emission + 3 * tri;
    const double* rho = s->albedo + 3 * tri;
    const int glossy = has_glossy(s, tri) && !(v->use_mlp && v->mlp);
    if (!(rho[0] > 0 || rho[1] > 0 || rho[2] > 0) && !glossy) {
        for (int c = 0; c < 3; ++c) L[c] = le[c];
        return;
    }
    if (v->use_mlp && v->mlp) {
        double f[3];
        or_mlp_eval(v, y, n, f);
        for (int c = 0; c < 3; ++c) L[c] = le[c] + rho[c] * (f[c] > 0.0 ? f[c] : 0.0);
        return;
    }
    double q[3], E[3] = {0, 0, 0};
    biased_point(v, y, x, q);
    or_ddgi_query(v, q, n, E);
    for (int c = 0; c < 3; ++c) L[c] = le[c] + rho[c] / PI * E[c];
    if (glossy) {
        double l = len3(d), wo[3] = {d[0] / l, d[1] / l, d[2] / l}, G[3];
        glossy_ddgi(v, q, n, wo, s->glossy + 4 * tri, u0, u1, G);
        for (int c = 0; c < 3; ++c) L[c] += G[c];
    }
}

/* batch form of the outgoing radiance, for estimator tests; u: [n][2]
 * random numbers of the glossy sample (NULL: 0.5, 0.5) */
void or_radiance_batch(const or_scene* s, const or_volume* v, int32_t n, const double* y,
                       const int32_t* tri, const double* from, const double* u, double* L) {
    for (int32_t k = 0; k < n; ++k) {
        L[3 * k] = L[3 * k + 1] = L[3 * k + 2] = 0.0;
        if (tri[k] >= 0)
            radiance_at(s, v, y + 3 * k, tri[k], from + 3 * k, u ? u[2 * k] : 0.5, u ? u[2 * k + 1] : 0.5,
                        L + 3 * k);
    }
}

/* Outgoing radiance at the selected sample y toward the shaded point x1
 * (normal n1, seen from the camera at eye), for shading (Sec. 3.3, specular
 * recursion): at each path vertex x_n (n >= 2) the emission and the diffuse
 * half rho / pi E(x_n, n_n) are added; the glossy half is either estimated
 * by the one-sample glossy term of Eq. lddgiplus -- once the path footprint
 * a(x_1 .. x_n) exceeds c a_0, or at the last of OR_MAX_SHADE_VERTS vertices
 * -- or continued by tracing the sampled glossy direction to x_{n+1}.  The
 * footprint (Bekaert et al., as the paper adopts it) is
 * a = (sum_i sqrt(|x_i - x_{i+1}|^2 / (p_i <n_{i+1}, -w_i>)))^2 with p_1 the
 * density of sampling w_1 at the (Lambertian) primary vertex, cos / pi, and
 * p_i the glossy sampling density beyond it; a_0 = |x_0 - x_1|^2 /
 * (4 pi <n_1, -w_0>).  Random numbers: (seed, pixel, frame, OR_PASS_SHADE,
 * vertex n, dimension 0 / 1).  verts (optional) receives the vertices used. */
void or_shade_radiance(const or_scene* s, const or_volume* v, const or_settings* st, const double eye[3],
                       const double x1[3], const double n1[3], const double y[3], int32_t tri, uint32_t pix,
                       uint32_t frame, double L[3], int32_t* verts) {
    L[0] = L[1] = L[2] = 0.0;
    double e0[3], d1[3];
    sub3(eye, x1, e0);
    sub3(y, x1, d1);
    double l0 = len3(e0), l1 = len3(d1);
    double c0 = dot3(n1, e0) / l0;
    double a0 = l0 * l0 / (4.0 * PI * c0);
    double alim = st->footprint_c * a0;
    double w1[3] = {d1[0] / l1, d1[1] / l1, d1[2] / l1};
    double p1 = dot3(n1, w1) / PI;
    double c2 = fabs(dot3(s->normal + 3 * tri, w1));
    double sa = sqrt(l1 * l1 / (p1 * c2));
    double thr[3] = {1.0, 1.0, 1.0};
    double prev[3] = {x1[0], x1[1], x1[2]}, cur[3] = {y[0], y[1], y[2]};
    int32_t t = tri, n = 2;
    for (;;) {
        const double* nrm = s->normal + 3 * t;
        double back[3];
        sub3(prev, cur, back);
        if (dot3(nrm, back) <= 0.0) break;
        const double* le = s->emission + 3 * t;
        const double* rho = s->albedo + 3 * t;
        for (int c = 0; c < 3; ++c) L[c] += thr[c] * le[c];
        const int glossy = has_glossy(s, t);
        if (!(rho[0] > 0 || rho[1] > 0 || rho[2] > 0) && !glossy) break;
        double q[3], E[3];
        biased_point(v, cur, prev, q);
        or_ddgi_query(v, q, nrm, E);
        for (int c = 0; c < 3; ++c) L[c] += thr[c] * rho[c] / PI * E[c];
        if (!glossy) break;
        double lb = len3(back), wo[3] = {back[0] / lb, back[1] / lb, back[2] / lb};
        double u0 = or_rng(st->seed, pix, frame, OR_PASS_SHADE, (uint32_t)n, 0);
        double u1 = or_rng(st->seed, pix, frame, OR_PASS_SHADE, (uint32_t)n, 1);
        const double* spec = s->glossy + 4 * t;
        double wi[3], wgt[3], pdf;
        if (!or_glossy_sample(nrm, wo, spec, spec[3], u0, u1, wi, wgt, &pdf)) break;
        if (st->footprint_c < 0.0 || sa * sa > alim || n >= OR_MAX_SHADE_VERTS) {
            or_ddgi_query(v, q, wi, E);
            for (int c = 0; c < 3; ++c) L[c] += thr[c] * wgt[c] * E[c] / PI;
            break;
        }
        int32_t hit;
        double th;
        if (!or_intersect(s, cur, wi, T_EPS, MISS_T, &hit, &th)) break;
        double c3 = -dot3(s->normal + 3 * hit, wi);
        if (c3 <= 0.0) break;
        sa += sqrt(th * th / (pdf * c3));
        for (int c = 0; c < 3; ++c) {
            thr[c] *= wgt[c];
            prev[c] = cur[c];
            cur[c] += th * wi[c];
        }
        t = hit;
        ++n;
    }
    if (verts) *verts = n;
}

static void res_set_empty(or_res* r, int32_t k, double M) {
    r->y[3 * k] = r->y[3 * k + 1] = r->y[3 * k + 2] = 0.0;
    r->L[3 * k] = r->L[3 * k + 1] = r->L[3 * k + 2] = 0.0;
    r->ny[3 * k] = r->ny[3 * k + 1] = r->ny[3 * k + 2] = 0.0;
    r->W[k] = 0.0; r->M[k] = M; r->tri[k] = -1; r->tag[k] = 0u;
}

static void res_copy(or_res* dst, int32_t k, const or_res* src, int32_t q) {
    for (int a = 0; a < 3; ++a) {
        dst->y[3 * k + a] = src->y[3 * q + a];
        dst->L[3 * k + a] = src->L[3 * q + a];
        dst->ny[3 * k + a] = src->ny[3 * q + a];
    }
    dst->W[k] = src->W[q]; dst->M[k] = src->M[q]; dst->tri[k] = src->tri[q]; dst->tag[k] = src->tag[q];
}

/* streaming weighted reservoir sampling step, decided in float */
static int wrs_take(double u, double wsum, double w) {
    return (float)u * (float)wsum < (float)w;
}

/* Sec. 3.1 step 1: candidates on all surfaces -- n_light points uniform in
 * area on the emitters plus n_bsdf cosine-distributed rays from x -- each
 * weighted by target / mixture density (balance heuristic, area measure);
 * Sec. 3.1 step 2: one is kept by weighted reservoir sampling with
 * W = w_sum / (M target(y)).  The BSDF rays also estimate the residual
 * transport of Sec. 3.5: rho_x L(y) max(0, 1 - 1/G) per ray. */
/* Sec. 5 (subsampling): with a candidate stride n >= 2 only every n-th
 * pixel, on diagonals that move by one pixel per frame, generates new
 * candidates; the others start from an empty reservoir and only reuse. */
static int generates_candidates(const or_settings* st, const or_gbuf* g, int32_t q, uint32_t frame) {
    if (st->candidate_stride <= 1) return 1;
    const uint32_t x = (uint32_t)(q % g->width), y = (uint32_t)(q / g->width);
    return (x + y + frame) % (uint32_t)st->candidate_stride == 0u;
}

int or_restir_initial(const or_scene* s, const or_volume* v, const or_settings* st,
                      const or_gbuf* g, uint32_t frame, const int32_t* pix, int32_t npix,
                      or_res* out, double* resid) {
    int32_t NL = s->num_emitters > 0 ? st->n_light : 0;
    int32_t NB = st->n_bsdf;
    int32_t M = NL + NB;
    for (int32_t k = 0; k < npix; ++k) {
        int32_t q = pix ? pix[k] : k;
        resid[3 * k] = resid[3 * k + 1] = resid[3 * k + 2] = 0.0;
        if (g->tri[q] < 0) { res_set_empty(out, k, 0.0); continue; }
        if (!generates_candidates(st, g, q, frame)) { res_set_empty(out, k, 0.0); continue; }
        const double* x = g->pos + 3 * q;
        const double* nx = g->nrm + 3 * q;
        const double* rho = g->alb + 3 * q;
        double wsum = 0.0, sel_p = 0.0, sel_y[3] = {0, 0, 0}, sel_L[3] = {0, 0, 0};
        int32_t sel_tri = -1, sel_c = -1;
        for (int32_t c = 0; c < M; ++c) {
            double y[3], L[3], dist2, cx, cy, pB, pL;
            int32_t tri;
            if (c < NL) {
                double u0 = or_rng(st->seed, q, frame, OR_PASS_INITIAL, c, 0);
                double u1 = or_rng(st->seed, q, frame, OR_PASS_INITIAL, c, 1);
                double u2 = or_rng(st->seed, q, frame, OR_PASS_INITIAL, c, 2);
                tri = or_sample_emitter(s, u0);
                const double* tv = s->verts + 9 * tri;
                double sq = sqrt(u1), b1 = sq * (1.0 - u2), b2 = sq * u2;
                for (int a = 0; a < 3; ++a) y[a] = tv[a] + b1 * (tv[3 + a] - tv[a]) + b2 * (tv[6 + a] - tv[a]);
                double d[3];
                sub3(y, x, d);
                dist2 = dot3(d, d);
                if (dist2 <= 0.0) continue;
                double l = sqrt(dist2);
                double w[3] = {d[0] / l, d[1] / l, d[2] / l};
                cx = dot3(nx, w);
                cy = fabs(dot3(s->normal + 3 * tri, w));
                radiance_at(s, v, y, tri, x, 0.5, 0.5, L);   /* an emitter: no glossy lobe */
            } else {
                double u0 = or_rng(st->seed, q, frame, OR_PASS_INITIAL, c, 0);
                double u1 = or_rng(st->seed, q, frame, OR_PASS_INITIAL, c, 1);
                double r = sqrt(u0), ph = 2.0 * PI * u1;
                double lc[3] = {r * cos(ph), r * sin(ph), sqrt(fmax(0.0, 1.0 - u0))};
                double w[3];
                or_onb_local_to_world(nx, lc, w);
                double t;
                if (!or_intersect(s, x, w, T_EPS, MISS_T, &tri, &t)) continue;
                for (int a = 0; a < 3; ++a) y[a] = x[a] + t * w[a];
                dist2 = t * t;
                cx = dot3(nx, w);
                cy = fabs(dot3(s->normal + 3 * tri, w));
                radiance_at(s, v, y, tri, x, or_rng(st->seed, q, frame, OR_PASS_INITIAL, c, 4),
                            or_rng(st->seed, q, frame, OR_PASS_INITIAL, c, 5), L);
                if (cx > 0.0) {
                    double G = cx * cy / dist2;
                    if (G > 1.0)
                        for (int a = 0; a < 3; ++a) resid[3 * k + a] += rho[a] * L[a] * (1.0 - 1.0 / G) / NB;
                }
            }
            if (cx <= 0.0) continue;
            pB = cx / PI * cy / dist2;
            const double* le = s->emission + 3 * tri;
            pL = s->emitter_of[tri] >= 0 ? 1.0 / s->area_total : 0.0;
            double pmix = (NL * pL + NB * pB) / M;
            double ph = or_target(s, x, nx, rho, y, tri, L);
            double wc = pmix > 0.0 ? ph / pmix : 0.0;
            wsum += wc;
            double u3 = or_rng(st->seed, q, frame, OR_PASS_INITIAL, c, 3);
            if (wc > 0.0 && wrs_take(u3, wsum, wc)) {
                sel_c = c; sel_tri = tri; sel_p = ph;
                for (int a = 0; a < 3; ++a) { sel_y[a] = y[a]; sel_L[a] = L[a]; }
            }
        }
        if (sel_c < 0) { res_set_empty(out, k, (double)M); continue; }
        for (int a = 0; a < 3; ++a) {
            out->y[3 * k + a] = sel_y[a];
            out->L[3 * k + a] = sel_L[a];
            out->ny[3 * k + a] = s->normal[3 * sel_tri + a];
        }
        out->W[k] = sel_p > 0.0 ? wsum / (M * sel_p) : 0.0;
        out->M[k] = M;
        out->tri[k] = sel_tri;
        out->tag[k] = (uint32_t)q * 64u + (uint32_t)sel_c;
    }
    return 0;
}

/* target at pixel q of a reused sample: its cached point, normal and
 * radiance (Sec. 3.6 caches the query with the sample; the point and normal
 * stay those of the frame the sample was found in, as the radiance does).
 * With rq != NULL caching is off (a test setting, to check Sec. 3.6's claim
 * that caching adds no bias): the radiance leaving y toward this pixel is
 * queried afresh from the volume rq instead of read from the reservoir. */
static double target_of(const or_scene* s, const or_gbuf* g, int32_t q, const or_res* r, int32_t k,
                        const or_volume* rq) {
    if (r->tri[k] < 0) return 0.0;
    const double* L = r->L + 3 * k;
    double Lf[3];
    if (rq) {
        radiance_at(s, rq, r->y + 3 * k, r->tri[k], g->pos + 3 * q, 0.5, 0.5, Lf);
        L = Lf;
    }
    return target_with_normal(g->pos + 3 * q, g->nrm + 3 * q, g->alb + 3 * q, r->y + 3 * k, r->ny + 3 * k, L);
}

/* Sec. 3.1 step 2 (temporal reuse, mechanics of the cited ReSTIR): the
 * reservoir of the reprojected pixel joins the current one if the normals
 * agree (cos > threshold) and the depths agree within a fraction; its M is
 * capped at mcap times the current M; its target is re-evaluated at x with the
 * cached radiance of Sec. 3.6. */
int or_restir_temporal(const or_scene* s, const or_settings* st, const or_gbuf* g,
                       const or_gbuf* gp, const double cpos[3], const or_res* cur,
                       const or_res* prev, uint32_t frame, const int32_t* pix, int32_t npix,
                       or_res* out) {
    return or_restir_temporal_rq(s, st, g, gp, cpos, cur, prev, frame, pix, npix, NULL, out);
}

int or_restir_temporal_rq(const or_scene* s, const or_settings* st, const or_gbuf* g,
                          const or_gbuf* gp, const double cpos[3], const or_res* cur,
                          const or_res* prev, uint32_t frame, const int32_t* pix, int32_t npix,
                          const or_volume* rq, or_res* out) {
    for (int32_t k = 0; k < npix; ++k) {
        int32_t q = pix ? pix[k] : k;
        res_copy(out, k, cur, q);
        if (g->tri[q] < 0) continue;
        int32_t pq = g->prev[q];
        if (pq < 0 || gp->tri[pq] < 0) continue;
        if (dot3(g->nrm + 3 * q, gp->nrm + 3 * pq) <= st->normal_reject_cos) continue;
        double dv[3], xp[3];
        or_prev_position(s, g->tri[q], g->pos + 3 * q, xp);
        sub3(xp, cpos, dv);
        double de = len3(dv);
        if (fabs(de - gp->dist[pq]) > st->depth_reject_frac * de) continue;
        double Mc = cur->M[q];
        double Mp = prev->M[pq];
        /* the cap is relative to the current M, or to the nominal candidate
         * count for a pixel that generated none (subsampling) */
        const double Mnom = (double)((s->num_emitters > 0 ? st->n_light : 0) + st->n_bsdf);
        const double Mref = Mc > 0.0 ? Mc : Mnom;
        if (Mp > st->temporal_mcap * Mref) Mp = st->temporal_mcap * Mref;
        double pc = target_of(s, g, q, cur, q, rq);
        double wsum = pc * cur->W[q] * Mc;
        double pp = target_of(s, g, q, prev, pq, rq);
        double wp = pp * prev->W[pq] * Mp;
        wsum += wp;
        double u = or_rng(st->seed, q, frame, OR_PASS_TEMPORAL, 0, 0);
        double psel = pc;
        if (wp > 0.0 && wrs_take(u, wsum, wp)) { res_copy(out, k, prev, pq); psel = pp; }
        out->M[k] = Mc + Mp;
        out->W[k] = psel > 0.0 ? wsum / (out->M[k] * psel) : 0.0;
    }
    return 0;
}

/* integer neighbour offset in the disk of the given radius, drawn by
 * rejection from hashed lattice points (at most 8 tries) */
static int spatial_offset(uint32_t seed, int32_t q, uint32_t frame, uint32_t pass, int32_t j,
                          int32_t radius, int32_t* dx, int32_t* dy) {
    uint32_t span = 2u * (uint32_t)radius + 1u;
    for (uint32_t a = 0; a < 8u; ++a) {
        uint32_t h = or_rng_u32(seed, (uint32_t)q, frame, pass, (uint32_t)j, a);
        int32_t x = (int32_t)((h & 0xFFFFu) % span) - radius;
        int32_t y = (int32_t)((h >> 16) % span) - radius;
        if ((x != 0 || y != 0) && x * x + y * y <= radius * radius) { *dx = x; *dy = y; return 1; }
    }
    return 0;
}

/* Sec. 3.1 step 2 (spatial reuse): k neighbours in a disk, normal / depth
 * rejection, combined with the cached radiance (Sec. 3.6), 1/M weights. */
int or_restir_spatial(const or_scene* s, const or_settings* st, const or_gbuf* g,
                      const or_res* in, uint32_t frame, uint32_t pass_idx,
                      const int32_t* pix, int32_t npix, or_res* out) {
    return or_restir_spatial_rq(s, st, g, in, frame, pass_idx, pix, npix, NULL, out);
}

int or_restir_spatial_rq(const or_scene* s, const or_settings* st, const or_gbuf* g,
                         const or_res* in, uint32_t frame, uint32_t pass_idx,
                         const int32_t* pix, int32_t npix, const or_volume* rq, or_res* out) {
    uint32_t pass = OR_PASS_SPATIAL0 + pass_idx;
    int32_t W = g->width, H = g->height;
    for (int32_t k = 0; k < npix; ++k) {
        int32_t q = pix ? pix[k] : k;
        res_copy(out, k, in, q);
        if (g->tri[q] < 0) continue;
        int32_t px = q % W, py = q / W;
        double psel = target_of(s, g, q, in, q, rq);
        double wsum = psel * in->W[q] * in->M[q];
        double M = in->M[q];
        for (int32_t j = 0; j < st->spatial_neighbours; ++j) {
            int32_t dx, dy;
            if (!spatial_offset(st->seed, q, frame, pass, j, st->spatial_radius, &dx, &dy)) continue;
            int32_t nxp = px + dx, nyp = py + dy;
            if (nxp < 0 || nyp < 0 || nxp >= W || nyp >= H) continue;
            int32_t nq = nyp * W + nxp;
            if (g->tri[nq] < 0) continue;
            if (dot3(g->nrm + 3 * q, g->nrm + 3 * nq) <= st->normal_reject_cos) continue;
            if (fabs(g->dist[q] - g->dist[nq]) > st->depth_reject_frac * g->dist[q]) continue;
            double pn = target_of(s, g, q, in, nq, rq);
            double wn = pn * in->W[nq] * in->M[nq];
            wsum += wn;
            M += in->M[nq];
            double u = or_rng(st->seed, q, frame, pass, j, 8);
            if (wn > 0.0 && wrs_take(u, wsum, wn)) { res_copy(out, k, in, nq); psel = pn; }
        }
        out->M[k] = M;
        out->W[k] = psel > 0.0 ? wsum / (M * psel) : 0.0;
    }
    return 0;
}

/* Sec. 3.1 steps 3-4 and Eq. Algorithm: Le at x, plus one shadow ray to the
 * selected y and, if visible, rho_x / pi * (Le + L_DDGI+)(y) * min(G, 1) * W
 * with a fresh probe query at y, plus the residual estimated by the BSDF
 * ray.  In a scene with glossy triangles the radiance at y comes from the
 * specular recursion of Sec. 3.3 (or_shade_radiance). */
int or_shade(const or_scene* s, const or_volume* v, const or_settings* st, const or_gbuf* g, const or_res* r,
             const double* resid, uint32_t frame, const int32_t* pix, int32_t npix, double* rad) {
    for (int32_t k = 0; k < npix; ++k) {
        int32_t q = pix ? pix[k] : k;
        rad[3 * k] = rad[3 * k + 1] = rad[3 * k + 2] = 0.0;
        int32_t tx = g->tri[q];
        if (tx < 0) continue;
        const double* x = g->pos + 3 * q;
        const double* nx = g->nrm + 3 * q;
        const double* rho = g->alb + 3 * q;
        for (int a = 0; a < 3; ++a) rad[3 * k + a] = s->emission[3 * tx + a] + resid[3 * q + a];
        int32_t ty = r->tri[q];
        if (ty < 0 || r->W[q] <= 0.0) continue;
        const double* y = r->y + 3 * q;
        double d[3];
        sub3(y, x, d);
        double d2 = dot3(d, d);
        if (d2 <= 0.0) continue;
        double l = sqrt(d2);
        double w[3] = {d[0] / l, d[1] / l, d[2] / l};
        double cx = dot3(nx, w);
        if (cx <= 0.0) continue;
        if (occluded(s, x, w, T_EPS, (1.0 - 1e-4) * l)) continue;
        double L[3];
        if (s->glossy)
            or_shade_radiance(s, v, st, g->eye, x, nx, y, ty, (uint32_t)q, frame, L, NULL);
        else
            radiance_at(s, v, y, ty, x, 0.5, 0.5, L);
        double cy = fabs(dot3(s->normal + 3 * ty, w));
        double G = cx * cy / d2;
        double Gb = G < 1.0 ? G : 1.0;
        for (int a = 0; a < 3; ++a) rad[3 * k + a] += rho[a] / PI * L[a] * Gb * r->W[q];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* path-traced reference (Sec. 4): next-event estimation toward an emitter  */
/* point uniform in area, cosine continuation, Russian roulette from the    */
/* 4th vertex, at most 64 vertices; keys (seed, pixel, sample, pass 8,      */
/* vertex, dimension)                                                       */
/* ------------------------------------------------------------------------ */

void or_pt_pixel(const or_scene* s, const or_camera* cam, int32_t pix, uint32_t seed, uint32_t sample0,
                 uint32_t spp, double out[3]) {
    int32_t W = cam->width, H = cam->height;
    int32_t i = pix % W, j = pix / W;
    double aspect = (double)W / H;
    double sx = (2.0 * (i + 0.5) / W - 1.0) * cam->tan_half_fovy * aspect;
    double sy = (1.0 - 2.0 * (j + 0.5) / H) * cam->tan_half_fovy;
    double d0[3];
    for (int a = 0; a < 3; ++a) d0[a] = cam->fwd[a] + sx * cam->right[a] + sy * cam->up[a];
    double l0 = len3(d0);
    for (int a = 0; a < 3; ++a) d0[a] /= l0;
    out[0] = out[1] = out[2] = 0.0;
    for (uint32_t k = 0; k < spp; ++k) {
        uint32_t smp = sample0 + k;
        double o[3] = {cam->pos[0], cam->pos[1], cam->pos[2]}, d[3] = {d0[0], d0[1], d0[2]};
        double beta[3] = {1, 1, 1}, L[3] = {0, 0, 0};
        int32_t tri;
        double t;
        int hit = or_intersect(s, o, d, T_EPS, MISS_T, &tri, &t);
        for (uint32_t depth = 1; depth <= 64; ++depth) {
            if (!hit) break;
            const double* n = s->normal + 3 * tri;
            if (!(dot3(n, d) < 0.0)) break;
            double x[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
            if (depth == 1)
                for (int c = 0; c < 3; ++c) L[c] += s->emission[3 * tri + c];
            const double* rho = s->albedo + 3 * tri;
            if (!(rho[0] > 0 || rho[1] > 0 || rho[2] > 0)) break;
            if (s->num_emitters > 0) {
                double u0 = or_rng(seed, pix, smp, 8, depth, 0);
                double u1 = or_rng(seed, pix, smp, 8, depth, 1);
                double u2 = or_rng(seed, pix, smp, 8, depth, 2);
                int32_t et = or_sample_emitter(s, u0);
                const double* tv = s->verts + 9 * et;
                double sq = sqrt(u1), b1 = sq * (1.0 - u2), b2 = sq * u2, y[3], dv[3];
                for (int a = 0; a < 3; ++a) y[a] = tv[a] + b1 * (tv[3 + a] - tv[a]) + b2 * (tv[6 + a] - tv[a]);
                sub3(y, x, dv);
                double d2 = dot3(dv, dv);
                if (d2 > 0.0) {
                    double l = sqrt(d2), w[3] = {dv[0] / l, dv[1] / l, dv[2] / l};
                    double cx = dot3(n, w), cy = -dot3(s->normal + 3 * et, w);
                    if (cx > 0.0 && cy > 0.0 && !occluded(s, x, w, T_EPS, (1.0 - 1e-4) * l)) {
                        double gf = cx * cy / d2 * s->area_total / PI;
                        for (int c = 0; c < 3; ++c) L[c] += beta[c] * rho[c] * s->emission[3 * et + c] * gf;
                    }
                }
            }
            double u3 = or_rng(seed, pix, smp, 8, depth, 3), u4 = or_rng(seed, pix, smp, 8, depth, 4);
            double r = sqrt(u3), ph = 2.0 * PI * u4;
            double lc[3] = {r * cos(ph), r * sin(ph), sqrt(fmax(0.0, 1.0 - u3))}, w[3];
            or_onb_local_to_world(n, lc, w);
            for (int c = 0; c < 3; ++c) beta[c] *= rho[c];
            if (depth >= 4) {
                double q = beta[0] > beta[1] ? beta[0] : beta[1];
                if (beta[2] > q) q = beta[2];
                if (q > 0.95) q = 0.95;
                if ((float)or_rng(seed, pix, smp, 8, depth, 5) >= (float)q) break;
                for (int c = 0; c < 3; ++c) beta[c] /= q;
            }
            for (int a = 0; a < 3; ++a) { o[a] = x[a]; d[a] = w[a]; }
            hit = or_intersect(s, o, d, T_EPS, MISS_T, &tri, &t);
        }
        for (int c = 0; c < 3; ++c) out[c] += L[c];
    }
}
