/* ddgi.h -- C ABI of the GB300 DDGI-resampling library (libddgi.so).
 *
 * The library implements, as CUDA kernels for sm_103a, the per-frame path of
 * "Dynamic Diffuse Global Illumination Resampling" (Majercik et al., arXiv
 * 2108.05263): the augmented probe update of Sec. 3.2, the unified candidate
 * generation and reservoir resampling of Sec. 3.1 (with the bounded geometry
 * term and residual of Sec. 3.5 and the cached probe queries of Sec. 3.6),
 * and the shading estimator of Eq. Algorithm.
 *
 * General rules
 *  - Every function returns a ddgi_status (0 = success, negative = error).
 *  - Pointers marked "device" must be CUDA device (or managed) memory owned by
 *    the caller; "host" pointers are ordinary host memory.  The library never
 *    frees caller memory.
 *  - Per-pixel planes are arrays of 4-float (16-byte) records, one per pixel
 *    in row-major order (pixel = y * width + x), 16-byte aligned; reservoirs
 *    are 64-byte records, 64-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work and return without synchronising, except
 *    ddgi_get_status and the *_get functions, which synchronise `stream`.
 *    restir_initial forks part of its work to a stream the context owns and
 *    joins it back into `stream` (events; also under graph capture), so
 *    every effect is still ordered on `stream`.
 *  - Argument errors (NULL, misalignment, size mismatch, out-of-range
 *    configuration) are detected on the host before anything is enqueued and
 *    return DDGI_ERR_INVALID_ARG.  Launch failures return DDGI_ERR_CUDA with
 *    the CUDA message available from ddgi_last_error.  Device-side limits
 *    (traversal iteration cap, traversal stack overflow) set an error word
 *    that ddgi_get_status reports; a kernel that hits one returns "no hit"
 *    for that ray and the frame continues.
 *  - A context is not thread-safe, and calls on one context share its scratch
 *    buffers: issue them on one stream (or order the streams).
 */
#ifndef DDGI_H
#define DDGI_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ddgi_status;
#define DDGI_OK 0
#define DDGI_ERR_INVALID_ARG (-1)
#define DDGI_ERR_CUDA (-2)
#define DDGI_ERR_NOT_READY (-3)
#define DDGI_ERR_TRAVERSAL_LIMIT (-4)
#define DDGI_ERR_BOUNDS (-5)
#define DDGI_ERR_OOM (-6)
#define DDGI_ERR_DEVICE_WAIT (-7)   /* a device-side wait hit its iteration bound */

typedef struct ddgi_ctx ddgi_ctx;

/* Scene: a triangle soup (host memory, copied at ddgi_create).  The facing
 * side of triangle i is the side its winding normal cross(v1-v0, v2-v0)
 * points to; emission is one-sided (Sec. 3.1 treats every surface as a light
 * source; emitters here are pure emitters with albedo 0). */
typedef struct {
    uint32_t num_tris;
    const float* vertices;   /* host [num_tris][3][3] */
    const float* albedo;     /* host [num_tris][3]  diffuse albedo rho */
    const float* emission;   /* host [num_tris][3]  emitted radiance Le */
    /* dynamics (NULL / 0: a static scene): the rigid instance of each
     * triangle, -1 = static; instance ids < num_instances; the vertices above
     * are the instances' identity pose; instanced triangles may not emit */
    const int32_t* tri_instance;   /* host [num_tris] or NULL */
    uint32_t num_instances;        /* <= 2^20 */
    /* glossy materials (Sec. 3.3; NULL: every triangle is Lambertian):
     * host [num_tris][4] = reflectance k_s.rgb (>= 0) and GGX roughness
     * alpha in [1e-3, 1] of a microfacet lobe f_g = k_s D(h) G1(wo) G1(wi) /
     * (4 |n.wo| |n.wi|) (GGX distribution, separable Smith masking, no
     * Fresnel term) added to the diffuse lobe rho / pi.  It enters L_DDGI+
     * (Eq. lddgiplus) wherever the probes are queried -- the probe update,
     * the radiance of BSDF candidates, shading -- and shading follows it by
     * specular recursion (ddgi_shade).  The primary vertex (the G-buffer
     * surface) is shaded with its diffuse lobe.  Emitters may not be glossy,
     * and a glossy scene may not use the learned target. */
    const float* glossy;
} ddgi_scene;

/* Method parameters.  Probe volume: a counts[0] x counts[1] x counts[2] grid,
 * probe (i,j,k) at origin + spacing * (i,j,k) + its relocation offset. */
typedef struct {
    float origin[3];
    float spacing[3];
    int32_t counts[3];
    uint32_t rays_per_probe;      /* 1..1024 (Sec. 3.2 update rays) */
    uint32_t irr_texels;          /* octahedral irradiance map side, 2..32 */
    uint32_t depth_texels;        /* octahedral distance-moment map side, 2..32 */
    float hysteresis;             /* blend weight of the old value, [0, 1) */
    float le_attenuation;         /* slider s of Sec. 3.2; 0 disables */
    float depth_sharpness;        /* cosine exponent of the distance blend */
    uint32_t num_light_candidates;/* emitter candidates per pixel (Sec. 3.1) */
    uint32_t num_bsdf_candidates; /* BSDF candidates per pixel; sum <= 64 */
    float temporal_mcap;          /* temporal M cap, multiple of current M */
    uint32_t spatial_neighbours;  /* neighbours per spatial pass, <= 32 */
    uint32_t spatial_radius;      /* pixels, 1..255 */
    float normal_reject_cos;      /* reuse only if dot(n, n') > this */
    float depth_reject_frac;      /* ... and |d - d'| <= this * d */
    uint32_t seed;
    /* learned target form: a network stands in for the probe lookup (the
     * paper names neural radiance caches as interchangeable with the probes,
     * Sec. 2 and Sec. 5) */
    uint32_t learned_target;      /* 1: resampling and shading query the network while
                                   * its held-out error is not above the probes' */
    uint32_t train_samples;       /* self-training samples per ddgi_mlp_train call; a
                                   * multiple of 16 and of the probe count (0 = none) */
    float train_lr;               /* Adam learning rate */
    uint32_t mlp_seed;            /* seed of the weight initialisation */
    float train_ema;              /* the network that serves queries is an exponential
                                   * moving average of the trained weights, blended
                                   * once per ddgi_mlp_train call with this weight on
                                   * the old average (the probes' hysteresis 0.97 is
                                   * the default); 0 serves the trained weights */
    uint32_t probe_relocation;    /* 1: ddgi_probe_update ends with ddgi_probe_relocate */
    uint32_t mlp_bf16;            /* network weights and activations in bf16 (1) or fp16 (0),
                                   * fp32 accumulation either way */
    uint32_t candidate_stride;    /* Sec. 5 subsampling: 0 or 1, every pixel generates
                                   * candidates; n >= 2 (at most 64), only pixels with
                                   * (x + y + frame) % n == 0 do, the others start from an
                                   * empty reservoir (M = 0, no residual) and only reuse;
                                   * temporal reuse then caps the previous M at
                                   * temporal_mcap x the nominal candidate count */
    float footprint_c;            /* threshold c of the shading recursion in glossy scenes
                                   * (Sec. 3.3): a glossy path stops when its footprint
                                   * exceeds c x the pixel's; 0 = the paper's 0.2,
                                   * < 0 = never recurse (one glossy sample per query) */
    uint32_t mlp_fp32;            /* 1: a debug form of the network for gradient checks --
                                   * every network evaluation and gradient runs in fp32 on
                                   * the CUDA cores (fp32 weights, activations and
                                   * accumulation, one thread per query or sample); 0: the
                                   * tensor-core kernels (mlp_bf16 selects their format) */
    uint32_t traversal_visit_cap; /* BVH nodes one ray may visit before its traversal
                                   * gives up (the ray then reports no hit and
                                   * ddgi_get_status returns DDGI_ERR_TRAVERSAL_LIMIT);
                                   * 0 = the default 65536 */
} ddgi_config;

/* Pinhole camera: orthonormal right/up/fwd, vertical half-angle tangent. */
typedef struct {
    float pos[3], fwd[3], right[3], up[3];
    float tan_half_fovy;
    uint32_t width, height;
} ddgi_camera;

/* G-buffer planes (device): g0 = position.xyz, distance to camera (> 0 at
 * a hit: reservoir records take the owner's validity from it);
 * g1 = normal.xyz, triangle index (uint32 bits, 0xFFFFFFFF = no valid
 * front-facing hit); g2 = albedo.rgb, previous-frame pixel (int32 bits, -1 =
 * none; bit 30 set: the surface belongs to a rigid instance, whose motion
 * restir_temporal undoes before its distance test). */
typedef struct {
    float* g0;
    float* g1;
    float* g2;
    uint32_t width, height;
    float eye[3];   /* the camera position the planes were rendered from; read
                     * only by ddgi_shade in glossy scenes (the pixel footprint
                     * of the shading recursion) */
} ddgi_gbuf;

/* Reservoirs (device): one 64-byte record per pixel, 64-byte aligned, as
 * 16 floats:
 *   [0..3]   y.xyz (selected point), W (unbiased contribution weight; 0 for
 *            an empty reservoir)
 *   [4..7]   cached radiance L(y).rgb leaving y toward its pixel, M
 *   [8..11]  the owning pixel's normal.xyz and distance to the camera
 *            (0 when the owning pixel has no valid G-buffer hit: the owner
 *            is valid exactly when this distance is > 0)
 *   [12..13] uint32 bits: triangle of y (0xFFFFFFFF = empty), tag (origin
 *            pixel * 64 + candidate index)
 *   [14..15] y's unit normal, octahedral map (u, v) in [-1, 1]^2 as floats
 *            (0, 0 for an empty reservoir); ddgi_reservoirs_attach_normals
 *            fills them for records written by the caller.
 * Words 8..11 repeat the owning pixel's G-buffer and words 14..15 the normal
 * of y's triangle, so that neighbour and previous-frame reuse read one record
 * (two 32-byte sectors) per candidate and gather nothing else. */
typedef struct {
    float* rec;
    uint32_t num_pixels;
} ddgi_reservoirs;

typedef struct {
    uint32_t num_tris, num_emitters, num_probes, rays_per_probe;
    uint32_t irr_tile, depth_tile;   /* padded map side (texels + 2) */
    uint32_t bvh_nodes, bvh_depth;
    uint32_t updates;                /* completed probe updates */
    uint64_t device_bytes;           /* device memory held by the context */
} ddgi_info;

/* Build the context: copies the scene, builds a 4-wide BVH on the host
 * (binned SAH) and uploads it, builds the emitter area table, allocates the
 * probe maps (zero) and the probe ray buffer.  Synchronous. */
ddgi_status ddgi_create(const ddgi_scene* scene, const ddgi_config* cfg, ddgi_ctx** out);
ddgi_status ddgi_destroy(ddgi_ctx* ctx);
ddgi_status ddgi_get_info(ddgi_ctx* ctx, ddgi_info* out);

/* Sec. 3.2, Eq. probeUpdate: trace rays_per_probe rays from every probe
 * (spherical Fibonacci set under a per-frame random rotation), radiance at the
 * hit = Le attenuated by (t / (t + s d_back))^2 + rho / pi * E at the
 * view-path-biased hit point (previous maps); then blend irradiance and
 * distance moments per texel with hysteresis and refresh the map borders.
 * ddgi_probe_update = ddgi_probe_trace + ddgi_probe_blend. */
ddgi_status ddgi_probe_update(ddgi_ctx* ctx, uint32_t frame, void* stream);
ddgi_status ddgi_probe_trace(ddgi_ctx* ctx, uint32_t frame, void* stream);
ddgi_status ddgi_probe_blend(ddgi_ctx* ctx, uint32_t frame, void* stream);

/* Scene dynamics, enqueued on `stream` (the paper's scenes are fully
 * dynamic, Sec. 1, Sec. 4).  xf (host [n][12], n = num_instances, or NULL):
 * row-major 3x4 transforms [R | t] of the instances relative to their
 * identity pose; the instanced triangles move there, and the BVH boxes over
 * them are refitted (the topology of ddgi_create is kept, so large motions
 * cost traversal time, not correctness).  The transforms of the previous call
 * are kept: ddgi_gbuffer reprojects a surface on an instance through
 * M_prev M_cur^-1 and marks it (bit 30 of the previous-pixel word).
 * emitter_radiance (host [E][3] in increasing triangle order of the emissive
 * triangles of ddgi_create, or NULL): new radiance, 0 switches an emitter
 * off; the emitter list and its area distribution do not change.  Host
 * buffers may be reused when the call returns: they are copied into a
 * page-locked staging buffer of the context, from which the device copies
 * run asynchronously; a call first waits (on the host) until the copies of
 * the previous call have run.  Both arguments are validated before anything
 * is enqueued.  Calls on other streams must be ordered with this one by the
 * caller. */
ddgi_status ddgi_scene_update(ddgi_ctx* ctx, const float* xf, uint32_t n, const float* emitter_radiance,
                              void* stream);

/* Snapshot of the context's evolving state, for checkpoint / resume: probe
 * maps, offsets and update count, instance poses (current and previous),
 * emitter radiance, and for a learned-target context the network (master,
 * Adam moments, served average, fp16 copies, optimiser / judge state, step
 * count, serving mode).  Scene geometry, configuration and the caller's
 * per-pixel buffers are not included.  ddgi_state_save with host_buf NULL
 * sets *bytes to the size needed; otherwise *bytes must be at least that and
 * is set to the bytes written.  ddgi_state_load accepts only a snapshot of a
 * context created from the same scene and configuration (probe count, map
 * sizes, instance and emitter counts, learned target; else
 * DDGI_ERR_INVALID_ARG).  Both synchronise `stream`. */
ddgi_status ddgi_state_save(ddgi_ctx* ctx, void* host_buf, size_t* bytes, void* stream);
ddgi_status ddgi_state_load(ddgi_ctx* ctx, const void* host_buf, size_t bytes, void* stream);

/* Probe relocation from the rays of the last ddgi_probe_trace of `frame`
 * (the paper's probe volume, Sec. 2, cites it; the rule is that of Majercik
 * et al. 2021).  delta = 0.1 x the smallest grid spacing.  A probe with more
 * than a quarter of its rays on back faces moves along its closest back-face
 * ray by that distance + delta / 2 (out of the geometry it sits in); else a
 * front face nearer than delta pushes it back along that ray by the
 * shortfall.  Each offset axis is clamped to +-0.45 x its spacing.  Offsets
 * persist and move the probe for every later trace and query. */
ddgi_status ddgi_probe_relocate(ddgi_ctx* ctx, uint32_t frame, void* stream);

/* Probe state transfer (host or device pointers; synchronises the stream):
 * irr [P][irr_tile^2][4] floats (rgb, 0), depth [P][depth_tile^2][2],
 * offsets [P][4] (xyz, 0), rays [P][rays_per_probe][4] (L.rgb, signed
 * distance: +t front hit, -t back hit, 1e30 miss).  NULL skips a buffer. */
ddgi_status ddgi_probe_state_get(ddgi_ctx* ctx, float* irr, float* depth, float* offsets,
                                 uint32_t* updates, void* stream);
ddgi_status ddgi_probe_state_set(ddgi_ctx* ctx, const float* irr, const float* depth,
                                 const float* offsets, uint32_t updates, void* stream);
ddgi_status ddgi_probe_rays_get(ddgi_ctx* ctx, float* rays, void* stream);
ddgi_status ddgi_probe_rays_set(ddgi_ctx* ctx, const float* rays, void* stream);

/* Primary visibility (support pass, the paper rasterises it): one pinhole
 * ray per pixel centre; prev_cam (nullable) gives the previous-frame pixel of
 * each hit.  out->width/height must equal cam->width/height. */
ddgi_status ddgi_gbuffer(ddgi_ctx* ctx, const ddgi_camera* cam, const ddgi_camera* prev_cam,
                         const ddgi_gbuf* out, void* stream);

/* Sec. 3.1 steps 1-2 and Sec. 3.5: per valid pixel x, num_light_candidates
 * area-uniform emitter points and num_bsdf_candidates cosine-distributed rays
 * (the BSDF hit's radiance (Le + L_DDGI+) is queried once and cached in the
 * reservoir), weighted by target / mixture density in area measure; one is
 * kept by weighted reservoir sampling, W = w_sum / (M target(y)).  residual
 * (device [N][4]) receives the BSDF-ray estimate rho_x L(y) max(0, 1 - 1/G)
 * of the residual transport (on the way it carries the emitter candidates'
 * state between the pass's kernels). */
ddgi_status restir_initial(ddgi_ctx* ctx, const ddgi_gbuf* g, const ddgi_reservoirs* out,
                           float* residual, uint32_t frame, void* stream);

/* Sec. 3.1 step 2 (temporal): merge each pixel's reservoir with that of its
 * previous-frame pixel if the normals (cos > normal_reject_cos) and the
 * distances (within depth_reject_frac) agree; the previous M is capped at
 * temporal_mcap times the current M; targets use the cached radiance
 * (Sec. 3.6).  The previous pixel's normal, distance and validity come from
 * its reservoir record (words 8..11); prev may hold a different number of
 * pixels than cur.  prev_cam_pos: host float[3], the previous camera
 * position.  out must not alias cur or prev. */
ddgi_status restir_temporal(ddgi_ctx* ctx, const ddgi_gbuf* g,
                            const float* prev_cam_pos, const ddgi_reservoirs* cur,
                            const ddgi_reservoirs* prev, const ddgi_reservoirs* out,
                            uint32_t frame, void* stream);

/* restir_initial followed by restir_temporal in one pass over the pixels
 * (Sec. 3.1 step 2 fused into step 1): each pixel's initial reservoir is
 * merged with its previous-frame pixel's reservoir before it is stored, so
 * only the merged reservoir reaches memory.  out and residual are those of
 * restir_initial into some buffer c followed by restir_temporal(c, prev)
 * into out: the same arithmetic, up to a few ulp where the compiler fuses a
 * multiply and an add differently in the one kernel (a selection can
 * differ where two weights tie that closely).  scratch (N records) is not
 * written (the emitter candidates hand their state to the BSDF candidates
 * through `residual`); it is validated and kept for compatibility.  out,
 * scratch and prev must be distinct; prev may hold a different number of
 * pixels; prev_cam_pos: host float[3]. */
ddgi_status restir_initial_temporal(ddgi_ctx* ctx, const ddgi_gbuf* g, const float* prev_cam_pos,
                                    const ddgi_reservoirs* scratch, const ddgi_reservoirs* prev,
                                    const ddgi_reservoirs* out, float* residual, uint32_t frame,
                                    void* stream);

/* Sec. 3.1 step 2 (spatial): merge with spatial_neighbours reservoirs drawn in
 * a disk of spatial_radius pixels, with the same rejection and cached
 * radiance.  `pass` (0-based) keys the random numbers.  out must not alias
 * in. */
ddgi_status restir_spatial(ddgi_ctx* ctx, const ddgi_gbuf* g, const ddgi_reservoirs* in,
                           const ddgi_reservoirs* out, uint32_t frame, uint32_t pass,
                           void* stream);

/* Words 14..15 of n caller-written records (triangle of y in word 12): the
 * octahedral map of that triangle's unit normal, as restir_initial writes it
 * (0, 0 where word 12 is not a triangle of the scene).  For reservoirs built
 * outside the library before they enter restir_temporal, restir_spatial or
 * ddgi_shade. */
ddgi_status ddgi_reservoirs_attach_normals(ddgi_ctx* ctx, const ddgi_reservoirs* r, void* stream);

/* Sec. 3.1 steps 3-4, Eq. Algorithm: radiance (device [N][4], rgb, 1) = Le(x)
 * + residual + (if the shadow ray to y is clear) rho_x / pi (Le +
 * L_DDGI+)(y) min(G, 1) W, with a fresh probe query at y.  In a glossy scene
 * the radiance at y follows the specular recursion of Sec. 3.3: at each path
 * vertex the emission and the diffuse half rho / pi E are added; the glossy
 * half is traced on (one sampled direction of the lobe) while the path
 * footprint a(x1..xn) stays within footprint_c x the pixel footprint a0 (g's
 * eye and the G-buffer give a0), else estimated by one glossy sample of
 * Eq. lddgiplus; at most 8 path vertices.  `frame` keys the random numbers
 * of that recursion. */
ddgi_status ddgi_shade(ddgi_ctx* ctx, const ddgi_gbuf* g, const ddgi_reservoirs* r,
                       const float* residual, float* radiance, uint32_t frame, void* stream);

/* Path-traced reference of Sec. 4 ("Reference" images for MAPE): unbiased
 * path tracing with next-event estimation toward area-sampled emitters,
 * cosine continuation, Russian roulette from the 4th vertex, at most 64
 * vertices, one path per pixel centre and sample.  Adds samples sample0 ..
 * sample0 + spp - 1 to accum (device [N][4] doubles: rgb sums, sample count;
 * zero it before the first call) and, if mean (device [N][4] floats) is not
 * NULL, writes the running mean there. */
ddgi_status ddgi_reference_accumulate(ddgi_ctx* ctx, const ddgi_camera* cam, uint32_t sample0, uint32_t spp,
                                      double* accum, float* mean, void* stream);

/* Error metrics of Sec. 4 between a rendered image and a reference: out[0] =
 * mean squared error, out[1] = mean absolute percentage error
 * mean(|v - ref| / (ref + 0.01)), both over the 3 colour values of every
 * pixel, accumulated in fp64 (0 for n = 0).  img, ref: device [n][4] floats
 * (rgb, ignored), 16-byte aligned; out: device double[2]; scratch: device
 * memory of at least scratch_doubles doubles for per-block partial sums
 * (2048 always suffice), 8-byte aligned, owned by the caller and overwritten.
 * n may be any uint32 value (the kernels index with 64 bits).  Does not
 * depend on a context. */
ddgi_status ddgi_image_metrics(const float* img, const float* ref, uint32_t n, double* scratch,
                               uint32_t scratch_doubles, double* out, void* stream);

/* Allocation-free form of ddgi_image_metrics (the paper has no counterpart:
 * this exists for callers that must not call cudaMalloc, e.g. a plug-in whose
 * host application owns all device memory, or a real-time thread where an
 * allocation and its implicit device synchronisation are not allowed).
 * Same inputs, output and result as ddgi_image_metrics, but the partial sums
 * live in a 16 KiB array inside the library that every GPU which loads the
 * library keeps until the process exits; nothing is allocated.
 *  - n must be <= 2^26 pixels; larger n returns DDGI_ERR_INVALID_ARG.
 *  - The first call on each device looks up that array's device address (with
 *    the device current) and caches it; make that first call before any
 *    stream capture.  The cached address belongs to the device's current
 *    primary context: after cudaDeviceReset (or anything else that tears
 *    that context down) the array may sit elsewhere, so do not call this
 *    entry point again in that process.
 *  - All calls share the one array: calls that overlap on the GPU (different
 *    streams, or different host threads) race and may return wrong values;
 *    serialise them.  Each call writes every partial sum it reads, so what an
 *    earlier call left behind does not matter. */
ddgi_status ddgi_image_metrics_static(const float* img, const float* ref, uint32_t n,
                                      double* out, void* stream);

/* ---- learned target form ------------------------------------------------
 * Network: input = sin / cos(2^k pi p'_a) for k = 0..11 and the 3 axes of the
 * position normalised to the scene box (p' = (p - box_lo) / max box extent),
 * the normal, 5 zeros (80 values); 4 hidden layers of 64 ReLU units; linear
 * 3-channel output f ~ E / pi, so the reflected indirect radiance at y is
 * rho(y) max(f, 0).  Weights and activations fp16, tensor-core accumulation
 * fp32, fp32 master weights, Adam (beta 0.9 / 0.99, eps 1e-8), relative-L2
 * loss with dynamic loss scaling.  Parameters: MLP_NPARAM = 18184 floats:
 * W1 [64][80] at 0, W2..W4 [64][64] at 5120 / 9216 / 13312, W5 [8][64] at
 * 17408 (rows 3..7 zero), b1..b4 [64] at 17920 + 64 l, b5 [8] at 18176. */
#define DDGI_MLP_NPARAM 18184

/* One self-training step: train_samples rays from the probe centres
 * (spherical Fibonacci set per probe, per-frame random rotation) hit y; a
 * cosine-distributed bounce from y hits z; target = Le(z) + rho(z) max(f(z),
 * 0), f the served network.  The samples train in minibatches of 16,384,
 * one Adam step each; then the served network is blended toward the trained
 * weights (train_ema).  Samples 16 j + 15 are held out and judge the served
 * network against the probe lookup (squared error relative to the mean of
 * the two predictions squared plus 0.01, so that the target's noise weighs
 * both equally); the decision holds for the following resampling / shading
 * calls whether the network or the probes serve the queries.  Requires
 * train_samples > 0. */
ddgi_status ddgi_mlp_train(ddgi_ctx* ctx, uint32_t frame, void* stream);

/* Evaluate the served network: queries (device [n][8] floats: p.xyz,
 * valid, n.xyz, 0), out (device [n][4]: f.rgb, valid). */
ddgi_status ddgi_mlp_infer(ddgi_ctx* ctx, const float* queries, float* out, uint32_t n, void* stream);

/* Gradient of the mean relative-L2 loss over caller samples (host or device
 * [n][12] floats: y.xyz, _, n.xyz, _, target.rgb, weight; weight 0 excludes
 * a sample) at the current weights, without updating them; grad: host or
 * device [DDGI_MLP_NPARAM].  Synchronises the stream. */
ddgi_status ddgi_mlp_grad(ddgi_ctx* ctx, const float* samples, uint32_t n, float* grad, void* stream);

/* One Adam step on caller samples (same layout as ddgi_mlp_grad). */
ddgi_status ddgi_mlp_step(ddgi_ctx* ctx, const float* samples, uint32_t n, void* stream);

/* fp32 master parameters (host or device [DDGI_MLP_NPARAM]); set also resets
 * the Adam moments and step count and makes the served network equal to
 * the given one.  Both synchronise the stream. */
ddgi_status ddgi_mlp_params_get(ddgi_ctx* ctx, float* params, void* stream);

/* fp32 parameters of the served network (the moving average of the trained
 * weights; host or device [DDGI_MLP_NPARAM]).  Its weights serve queries
 * rounded to fp16.  Synchronises the stream. */
ddgi_status ddgi_mlp_params_served_get(ddgi_ctx* ctx, float* params, void* stream);
ddgi_status ddgi_mlp_params_set(ddgi_ctx* ctx, const float* params, void* stream);

/* Who serves the queries of a learned-target context: 0 = the judge of the
 * last ddgi_mlp_train call (default), 1 = always the network, 2 = always the
 * probes.  Takes effect for the calls enqueued after it. */
ddgi_status ddgi_mlp_serve(ddgi_ctx* ctx, int32_t mode, void* stream);

/* The last ddgi_mlp_train call's samples (host or device [train_samples][12]
 * floats: y.xyz, valid, n.xyz, 0, target.rgb, weight).  Synchronises. */
ddgi_status ddgi_mlp_samples_get(ddgi_ctx* ctx, float* out, void* stream);

/* Optimiser / judge state (host double[8]): loss scale, last step overflowed,
 * training samples of the last step, held-out error of the network, of the
 * probes, held-out count, network serving (1/0), Adam steps.  Synchronises. */
ddgi_status ddgi_mlp_status(ddgi_ctx* ctx, double* out, void* stream);

/* Synchronise `stream`, return (and clear) the device error word:
 * DDGI_ERR_DEVICE_WAIT if a network kernel's wait for its tensor-core
 * results ran past its iteration bound (the kernel then waited once more,
 * bounded, for the products it had issued, skipped its remaining work and
 * released its tensor memory), DDGI_ERR_TRAVERSAL_LIMIT if a ray exceeded
 * the node-visit cap (traversal_visit_cap) or the traversal stack, else
 * DDGI_OK.  DDGI_ERR_DEVICE_WAIT is fatal for the context: the network
 * state is undefined from then on, every later ddgi_get_status returns it
 * again, and the context should be destroyed.  A traversal limit is not:
 * the frame finished with "no hit" for the rays concerned, and the error
 * word is clear again for the next frame. */
ddgi_status ddgi_get_status(ddgi_ctx* ctx, void* stream);
const char* ddgi_last_error(ddgi_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
