/* CPU oracle for DDGI resampling (Majercik et al., "Dynamic Diffuse Global
 * Illumination Resampling", arXiv 2108.05263).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded, fp64
 * restatement of what the method computes: brute-force ray-triangle
 * intersection over every triangle, the probe update of Sec. 3.2
 * (Eq. probeUpdate with the Le attenuation of Sec. 3.2), the probe query with
 * the view-path bias of Sec. 3.4, the unified candidate generation and
 * reservoir resampling of Sec. 3.1, the bounded geometry term and residual of
 * Sec. 3.5, the cached-query reuse of Sec. 3.6 and the final estimator
 * (Eq. Algorithm).  It is used by the tests, by the smoke check and by the
 * benchmark's CPU-baseline leg, never by the product path, and it shares no
 * code with the CUDA library.
 *
 * Conventions: all buffers are host memory owned by the caller; input and
 * output per-pixel buffers are "full" (indexed by pixel) except the outputs of
 * the pass functions, which are "compact" (entry k belongs to pix[k]; when
 * pix is NULL, entry k is pixel k).  Triangle index -1 marks an empty slot.
 */
#ifndef DDGI_ORACLE_H
#define DDGI_ORACLE_H
#include <stdint.h>

typedef struct {
    int32_t num_tris;
    double* verts;           /* [T][3][3] current positions (or_scene_update moves instances) */
    const double* albedo;    /* [T][3] */
    double* emission;        /* [T][3] (or_scene_update sets the emitters' radiance) */
    /* scene dynamics (tri_instance NULL: a static scene) */
    const int32_t* tri_instance;  /* [T] rigid instance of each triangle, -1 = static */
    int32_t num_instances;
    const double* object_verts;   /* [T][3][3] positions at the identity pose */
    /* derived by or_scene_init */
    double* normal;          /* [T][3] winding normal cross(v1-v0, v2-v0), unit */
    double* area;            /* [T] */
    int32_t num_emitters;
    int32_t* emitter_tri;    /* [E] emissive triangles in increasing index */
    int32_t* emitter_of;     /* [T] position in the emitter list, -1 = not an emitter */
    float* emitter_cdf;      /* [E] cumulative emitter area, rounded to float */
    double area_total;       /* total emissive area (fp64) */
    double* inst_cur;        /* [I][12] current instance transforms (row-major 3x4) */
    double* inst_prev;       /* [I][12] the transforms of the previous update */
    /* glossy lobe of every triangle (NULL: a diffuse scene): [T][4] =
     * reflectance k_s.rgb and GGX roughness alpha (Sec. 3.3) */
    const double* glossy;
} or_scene;

typedef struct {
    int32_t rays_per_probe, irr_n, depth_n;
    double hysteresis, le_attenuation, depth_sharpness;
    int32_t n_light, n_bsdf;
    double temporal_mcap;
    int32_t spatial_neighbours, spatial_radius;
    double normal_reject_cos, depth_reject_frac;
    uint32_t seed;
    int32_t relocate;        /* probe relocation after each blend (1) or not */
    int32_t candidate_stride;   /* >= 2: pixel (x, y) generates candidates in frame f only when
                                 * (x + y + f) mod stride == 0 (Sec. 5, subsampling); 0, 1: every pixel */
    double footprint_c;      /* threshold c of the shading recursion (Sec. 3.3); < 0: never recurse */
} or_settings;

typedef struct {
    double origin[3], spacing[3];
    int32_t counts[3];
    int32_t irr_n, depth_n;
    double* irr;     /* [P][irr_n+2][irr_n+2][3] (row, column) incl. gutter */
    double* depth;   /* [P][depth_n+2][depth_n+2][2] (mean, mean square) */
    double* offset;  /* [P][3] relocation offsets */
    int32_t updates; /* number of completed probe updates */
    /* learned target form: when use_mlp, (Le + L_DDGI+)(y) uses the network
     * rho(y) max(f(y), 0) in place of the probe query */
    const double* mlp;   /* [18184] parameters in the library's layout */
    double mlp_lo[3], mlp_scale;
    int32_t use_mlp;
} or_volume;

typedef struct {
    double pos[3], fwd[3], right[3], up[3];
    double tan_half_fovy;
    int32_t width, height;
} or_camera;

typedef struct {          /* full per-pixel G-buffer */
    double* pos;          /* [N][3] */
    double* dist;         /* [N]   distance from the camera */
    double* nrm;          /* [N][3] */
    double* alb;          /* [N][3] */
    int32_t* tri;         /* [N]   -1: no valid front-facing hit */
    int32_t* prev;        /* [N]   previous-frame pixel or -1 */
    int32_t width, height;
    double eye[3];        /* the camera position the G-buffer was rendered from */
} or_gbuf;

typedef struct {          /* reservoirs (full or compact) */
    double* y;            /* [N][3] selected point */
    double* W;            /* [N]   unbiased contribution weight */
    double* L;            /* [N][3] cached radiance leaving y toward its pixel */
    double* M;            /* [N]   candidate count */
    int32_t* tri;         /* [N]   triangle of y, -1 = empty */
    uint32_t* tag;        /* [N]   origin id: pixel * 64 + candidate */
    double* ny;           /* [N][3] unit normal at y when the sample was found */
} or_res;

/* pass identifiers used in the random-number keys */
#define OR_PASS_INITIAL 0u
#define OR_PASS_SPATIAL0 1u
#define OR_PASS_TEMPORAL 5u
#define OR_PASS_PROBE_ROT 7u
#define OR_PASS_SHADE 12u          /* glossy directions of the shading recursion (cand = vertex) */
#define OR_PASS_PROBE_GLOSSY 13u   /* glossy direction at a probe ray's hit (pixel = probe, cand = ray) */
#define OR_MAX_SHADE_VERTS 8       /* path vertices of the shading recursion, x1 included */

#ifdef __cplusplus
extern "C" {
#endif
int or_scene_init(or_scene* s);
void or_scene_free(or_scene* s);
int or_scene_update(or_scene* s, const double* xf, int32_t n, const double* emitter_radiance);
void or_prev_position(const or_scene* s, int32_t tri, const double x[3], double xp[3]);

uint32_t or_pcg(uint32_t v);
uint32_t or_rng_u32(uint32_t seed, uint32_t pixel, uint32_t frame, uint32_t pass,
                    uint32_t cand, uint32_t dim);
double or_rng(uint32_t seed, uint32_t pixel, uint32_t frame, uint32_t pass,
              uint32_t cand, uint32_t dim);

int or_intersect(const or_scene* s, const double o[3], const double d[3],
                 double tmin, double tmax, int32_t* tri, double* t);
void or_trace_batch(const or_scene* s, int32_t n, const double* o, const double* d,
                    double tmin, double tmax, int32_t* tri, double* t);
int32_t or_sample_emitter(const or_scene* s, double u);

void or_oct_encode(const double d[3], double uv[2]);
void or_oct_decode(const double uv[2], double d[3]);
void or_texel_dir(int32_t i, int32_t j, int32_t n, double d[3]);
void or_sf_dir(int32_t i, int32_t n, double d[3]);
void or_probe_rotation(uint32_t seed, uint32_t frame, double R[9]);
void or_probe_ray_dir(const double R[9], int32_t r, int32_t n, double d[3]);
void or_onb_local_to_world(const double n[3], const double l[3], double w[3]);
void or_gutter(double* tile, int32_t n, int32_t ch);
void or_fill_gutters(or_volume* v);
void or_bilinear(const double* tile, int32_t n, int32_t ch, const double d[3], double* out);
void or_probe_pos(const or_volume* v, int32_t p, double P[3]);

double or_ddgi_query(const or_volume* v, const double q[3], const double n[3], double E[3]);
void or_biased_query(const or_volume* v, const double y[3], const double n_y[3],
                     const double from[3], double E[3]);

int or_probe_trace(const or_scene* s, const or_volume* v, const or_settings* st,
                   uint32_t frame, const int32_t* probes, int32_t nprobes, double* rays);
int or_probe_blend(or_volume* v, const or_settings* st, uint32_t frame,
                   const int32_t* probes, int32_t nprobes, const double* rays);
int or_probe_relocate(or_volume* v, const or_settings* st, uint32_t frame,
                      const int32_t* probes, int32_t nprobes, const double* rays);
int or_probe_update(const or_scene* s, or_volume* v, const or_settings* st, uint32_t frame);

int or_gbuffer(const or_scene* s, const or_camera* cam, const or_camera* prev_cam,
               const int32_t* pix, int32_t npix, or_gbuf* out);
int or_restir_initial(const or_scene* s, const or_volume* v, const or_settings* st,
                      const or_gbuf* g, uint32_t frame, const int32_t* pix, int32_t npix,
                      or_res* out, double* resid);
int or_restir_temporal(const or_scene* s, const or_settings* st, const or_gbuf* g,
                       const or_gbuf* gp, const double prev_cam_pos[3], const or_res* cur,
                       const or_res* prev, uint32_t frame, const int32_t* pix, int32_t npix,
                       or_res* out);
int or_restir_spatial(const or_scene* s, const or_settings* st, const or_gbuf* g,
                      const or_res* in, uint32_t frame, uint32_t pass,
                      const int32_t* pix, int32_t npix, or_res* out);
/* the same two passes with caching off when rq != NULL (a test setting): the
 * target of a reused sample queries its radiance afresh from the volume rq,
 * from the current pixel, instead of the radiance cached with it (Sec. 3.6) */
int or_restir_temporal_rq(const or_scene* s, const or_settings* st, const or_gbuf* g,
                          const or_gbuf* gp, const double prev_cam_pos[3], const or_res* cur,
                          const or_res* prev, uint32_t frame, const int32_t* pix, int32_t npix,
                          const or_volume* rq, or_res* out);
int or_restir_spatial_rq(const or_scene* s, const or_settings* st, const or_gbuf* g,
                         const or_res* in, uint32_t frame, uint32_t pass,
                         const int32_t* pix, int32_t npix, const or_volume* rq, or_res* out);
int or_shade(const or_scene* s, const or_volume* v, const or_settings* st, const or_gbuf* g, const or_res* r,
             const double* resid, uint32_t frame, const int32_t* pix, int32_t npix, double* radiance);
void or_radiance_batch(const or_scene* s, const or_volume* v, int32_t n, const double* y,
                       const int32_t* tri, const double* from, const double* u, double* L);
double or_ggx_D(double nh, double alpha);
double or_ggx_G1(double nw, double alpha);
void or_ggx_sample_h(const double n[3], double alpha, double u0, double u1, double h[3]);
int or_glossy_sample(const double n[3], const double wo[3], const double ks[3], double alpha, double u0,
                     double u1, double wi[3], double wgt[3], double* pdf);
void or_shade_radiance(const or_scene* s, const or_volume* v, const or_settings* st, const double eye[3],
                       const double x1[3], const double n1[3], const double y[3], int32_t tri, uint32_t pix,
                       uint32_t frame, double L[3], int32_t* verts);
void or_pt_pixel(const or_scene* s, const or_camera* cam, int32_t pix, uint32_t seed, uint32_t sample0,
                 uint32_t spp, double out[3]);
void or_mlp_eval(const or_volume* v, const double p[3], const double n[3], double out[3]);
double or_target(const or_scene* s, const double x[3], const double nx[3],
                 const double rho[3], const double y[3], int32_t tri, const double L[3]);
#ifdef __cplusplus
}
#endif
#endif
