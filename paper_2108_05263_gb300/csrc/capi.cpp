// C ABI of libddgi.so: context lifetime, argument validation and kernel
// launches.  Every call validates on the host, enqueues on the caller's
// stream and returns without synchronising (except the documented getters).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

struct ddgi_ctx {
    ddgi_config cfg{};
    uint32_t T = 0, E = 0, P = 0;
    float4* nodes = nullptr;
    float4* tris = nullptr;
    float4* nrm = nullptr;
    float4* alb = nullptr;
    float4* emi = nullptr;
    float4* spec = nullptr;        // glossy lobe per triangle (k_s.rgb, alpha); null: a diffuse scene
    float4* evert = nullptr;
    float4* evert3 = nullptr;      // 48-byte emitter records: (v0, Le.b), (e1, Le.r), (e2, Le.g)
    float* cdf = nullptr;
    uint32_t* etri = nullptr;
    uint32_t* guide = nullptr;
    uint32_t G = 0;
    uint32_t emitters_reflect = 0;
    float area_total = 0.f;
    float4* irr = nullptr;
    float2* depth = nullptr;
    float4* irr_q = nullptr;       // the query's 2x2 tap blocks of irr / depth (VolumeView)
    float4* depth_q = nullptr;
    float4* offset = nullptr;
    float4* rays = nullptr;
    float* blend_w = nullptr;      // the probe blend's per-frame weight tables
    float4* sf = nullptr;
    uint32_t* sf_order = nullptr;  // probe rays in an order that keeps a warp's directions together
    uint32_t* err = nullptr;
    uint32_t* counter = nullptr;   // work counter of the persistent trace kernel
    float2* hits = nullptr;        // per-ray hit records (t, triangle), grown on demand
    size_t hits_cap = 0;
    float4* ind = nullptr;         // per-query network radiance, grown on demand
    size_t ind_cap = 0;
    // learned target form
    float* mlp_params = nullptr;   // fp32 master [MLP_NPARAM]
    float* mlp_grad = nullptr;
    float* mlp_m = nullptr;
    float* mlp_v = nullptr;
    uint16_t* mlp_w16 = nullptr;   // 16-bit weights (fp16 or bf16 bits) [MLP_NW]
    float* mlp_ema = nullptr;      // served network: moving average of the master weights
    uint16_t* mlp_w16s = nullptr;  // its 16-bit weights
    MLPState* mlp_state = nullptr;
    float4* train_smp = nullptr;   // [train_samples][3]
    float4* train_sf = nullptr;    // [train_per]
    uint32_t train_per = 0;
    uint32_t mlp_step = 0;
    int serve = 0;                 // 0 judge, 1 network, 2 probes
    bool wait_failed = false;      // a tensor-core wait gave up: the context is unusable
    float mlp_lo[3] = {0.f, 0.f, 0.f};
    float mlp_scale = 1.f;
    float4* tmp_smp = nullptr;     // caller samples staged on the device
    size_t tmp_cap = 0;
    float* tmp_grad = nullptr;
    uint32_t updates = 0;
    uint32_t bvh_nodes = 0, bvh_depth = 0;
    // scene dynamics
    uint32_t I = 0, NI = 0;          // instances, instanced triangles
    int32_t* tri_inst = nullptr;     // [T] instance or -1
    uint4* inst_map = nullptr;       // [NI] BVH slot, triangle, instance
    float4* inst_obj = nullptr;      // [3 NI] identity-pose vertices
    float4* inst_xf = nullptr;       // [3 I] current transform rows
    float4* inst_delta = nullptr;    // [3 I] rows of M_prev M_cur^-1
    uint32_t* refit_list = nullptr;  // nodes over instanced triangles, deepest depth first
    std::vector<uint32_t> refit_levels;
    float* refit_static = nullptr;   // per listed node and slot: the box of the slot's unmoved references
    std::vector<double> xf_cur, xf_prev;   // [12 I] host copies
    float* le_stage = nullptr;       // [3 E] staged emitter radiance
    // page-locked host staging of ddgi_scene_update ([12 I] transforms,
    // [12 I] reprojection rows, [3 E] radiance), so that its copies are
    // asynchronous; the event marks the end of the last copies out of it
    float* pin = nullptr;
    cudaEvent_t pin_ev = nullptr;
    bool pin_pending = false;
    // second stream of restir_initial: the emitter candidates run there while
    // the BSDF rays are traced on the caller's stream (fork / join events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool offsets_used = false;       // some probe offset may be non-zero (relocation ran or offsets were set)
    uint64_t device_bytes = 0;
    std::vector<void*> allocs;
    std::string last_error;
};

namespace {

ddgi_status fail(ddgi_ctx* c, ddgi_status code, const std::string& msg) {
    if (c) c->last_error = msg;
    return code;
}

ddgi_status cuda_fail(ddgi_ctx* c, cudaError_t e, const char* where) {
    return fail(c, DDGI_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                            \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

template <class T>
cudaError_t dalloc(ddgi_ctx* ctx, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    size_t bytes = sizeof(T) * count;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e == cudaSuccess) {
        ctx->allocs.push_back(*p);
        ctx->device_bytes += bytes;
    }
    return e;
}

// PCG hash (Jarzynski & Olano 2020), host copy for the per-frame rotation
uint32_t pcg_h(uint32_t v) {
    uint32_t state = v * 747796405u + 2891336453u;
    uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}
double rng_h(uint32_t seed, uint32_t pixel, uint32_t frame, uint32_t pass, uint32_t cand, uint32_t dim) {
    uint32_t h = pcg_h(seed);
    h = pcg_h(h + pixel);
    h = pcg_h(h + frame);
    h = pcg_h(h + pass);
    h = pcg_h(h + cand);
    h = pcg_h(h + dim);
    return (double)(h >> 8) * (1.0 / 16777216.0);
}

// uniform random rotation from a unit quaternion (Shoemake's method)
void frame_rotation(uint32_t seed, uint32_t frame, float R[9], uint32_t pass = PASS_PROBE_ROT) {
    const double PI = 3.14159265358979323846;
    double u0 = rng_h(seed, 0, frame, pass, 0, 0);
    double u1 = rng_h(seed, 0, frame, pass, 0, 1);
    double u2 = rng_h(seed, 0, frame, pass, 0, 2);
    double a = std::sqrt(1.0 - u0), b = std::sqrt(u0);
    double x = a * std::sin(2 * PI * u1), y = a * std::cos(2 * PI * u1);
    double z = b * std::sin(2 * PI * u2), w = b * std::cos(2 * PI * u2);
    double M[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
                   2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
                   2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)};
    for (int i = 0; i < 9; ++i) R[i] = (float)M[i];
}

SceneView scene_view(ddgi_ctx* c) {
    SceneView s;
    s.nodes = c->nodes;
    s.tris = c->tris;
    s.nrm = c->nrm;
    s.alb = c->alb;
    s.emi = c->emi;
    s.cdf = c->cdf;
    s.etri = c->etri;
    s.evert = c->evert;
    s.evert3 = c->evert3;
    s.guide = c->guide;
    s.guide_size = c->G;
    s.emitters_reflect = c->emitters_reflect;
    s.num_emitters = c->E;
    s.area_total = c->area_total;
    s.err = c->err;
    s.tri_inst = c->I ? c->tri_inst : nullptr;
    s.num_tris = c->T;
    s.inst_delta = c->inst_delta;
    s.max_visits = c->cfg.traversal_visit_cap ? (int)c->cfg.traversal_visit_cap : TRAV_MAX_VISITS;
    s.spec = c->spec;
    return s;
}

VolumeView volume_view(ddgi_ctx* c) {
    VolumeView v;
    v.irr = c->irr;
    v.depth = c->depth;
    v.irr_q = c->irr_q;
    v.depth_q = c->depth_q;
    v.offset = c->offset;
    v.has_offset = c->offsets_used ? 1 : 0;
    v.origin = make_float3(c->cfg.origin[0], c->cfg.origin[1], c->cfg.origin[2]);
    v.spacing = make_float3(c->cfg.spacing[0], c->cfg.spacing[1], c->cfg.spacing[2]);
    v.counts = make_int3(c->cfg.counts[0], c->cfg.counts[1], c->cfg.counts[2]);
    v.irr_n = (int)c->cfg.irr_texels;
    v.depth_n = (int)c->cfg.depth_texels;
    v.min_spacing = std::fmin(std::fmin(c->cfg.spacing[0], c->cfg.spacing[1]), c->cfg.spacing[2]);
    v.max_spacing = std::fmax(std::fmax(c->cfg.spacing[0], c->cfg.spacing[1]), c->cfg.spacing[2]);
    return v;
}

RestirParams restir_params(ddgi_ctx* c) {
    RestirParams r;
    r.seed = c->cfg.seed;
    r.n_light = c->cfg.num_light_candidates;
    r.n_bsdf = c->cfg.num_bsdf_candidates;
    r.temporal_mcap = c->cfg.temporal_mcap;
    r.spatial_neighbours = c->cfg.spatial_neighbours;
    r.spatial_radius = c->cfg.spatial_radius;
    r.normal_reject_cos = c->cfg.normal_reject_cos;
    r.depth_reject_frac = c->cfg.depth_reject_frac;
    const uint64_t span = 2ull * c->cfg.spatial_radius + 1ull;
    r.span_magic = (uint32_t)(((1ull << 32) + span - 1) / span);
    r.stride = c->cfg.candidate_stride > 1 ? c->cfg.candidate_stride : 1u;
    return r;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

const uint32_t kMaxPixels = 1u << 26;   // tag = pixel * 64 + candidate fits 32 bits

ddgi_status check_gbuf(ddgi_ctx* ctx, const ddgi_gbuf* g, GBufView* out) {
    if (!g) return fail(ctx, DDGI_ERR_INVALID_ARG, "gbuffer is NULL");
    uint64_t n = (uint64_t)g->width * g->height;
    if (n > kMaxPixels) return fail(ctx, DDGI_ERR_INVALID_ARG, "gbuffer larger than 2^26 pixels");
    if (n > 0 && (!g->g0 || !g->g1 || !g->g2))
        return fail(ctx, DDGI_ERR_INVALID_ARG, "gbuffer plane is NULL");
    if (!aligned(g->g0, 16) || !aligned(g->g1, 16) || !aligned(g->g2, 16))
        return fail(ctx, DDGI_ERR_INVALID_ARG, "gbuffer plane not 16-byte aligned");
    out->g0 = reinterpret_cast<float4*>(g->g0);
    out->g1 = reinterpret_cast<float4*>(g->g1);
    out->g2 = reinterpret_cast<float4*>(g->g2);
    out->width = (int)g->width;
    out->height = (int)g->height;
    out->eye = make_float3(g->eye[0], g->eye[1], g->eye[2]);
    return DDGI_OK;
}

ddgi_status check_res(ddgi_ctx* ctx, const ddgi_reservoirs* r, uint64_t npix, ResView* out) {
    if (!r) return fail(ctx, DDGI_ERR_INVALID_ARG, "reservoirs is NULL");
    if (npix != UINT64_MAX && r->num_pixels != npix)
        return fail(ctx, DDGI_ERR_INVALID_ARG, "reservoir size != gbuffer size");
    if (npix == UINT64_MAX) npix = r->num_pixels;
    if (npix > 0 && !r->rec) return fail(ctx, DDGI_ERR_INVALID_ARG, "reservoir records are NULL");
    if (!aligned(r->rec, 64)) return fail(ctx, DDGI_ERR_INVALID_ARG, "reservoir records not 64-byte aligned");
    out->rec = reinterpret_cast<float4*>(r->rec);
    out->n = (uint32_t)npix;
    return DDGI_OK;
}

bool finite3(const float* p) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }

ddgi_status check_config(const ddgi_config* c, std::string* why) {
    for (int a = 0; a < 3; ++a) {
        if (c->counts[a] < 1 || c->counts[a] > 4096) { *why = "probe counts out of range"; return DDGI_ERR_INVALID_ARG; }
        if (!(c->spacing[a] > 0.f) || !std::isfinite(c->spacing[a])) { *why = "probe spacing must be > 0"; return DDGI_ERR_INVALID_ARG; }
    }
    if (!finite3(c->origin)) { *why = "probe origin not finite"; return DDGI_ERR_INVALID_ARG; }
    if ((uint64_t)c->counts[0] * c->counts[1] * c->counts[2] > (1u << 22)) { *why = "too many probes"; return DDGI_ERR_INVALID_ARG; }
    if (c->rays_per_probe < 1 || c->rays_per_probe > 1024) { *why = "rays_per_probe must be 1..1024"; return DDGI_ERR_INVALID_ARG; }
    if (c->irr_texels < 2 || c->irr_texels > 32 || c->depth_texels < 2 || c->depth_texels > 32) {
        *why = "texel counts must be 2..32"; return DDGI_ERR_INVALID_ARG;
    }
    if (!(c->hysteresis >= 0.f && c->hysteresis < 1.f)) { *why = "hysteresis must be in [0,1)"; return DDGI_ERR_INVALID_ARG; }
    if (!(c->le_attenuation >= 0.f) || !std::isfinite(c->le_attenuation)) { *why = "le_attenuation must be >= 0"; return DDGI_ERR_INVALID_ARG; }
    if (!(c->depth_sharpness > 0.f) || !std::isfinite(c->depth_sharpness)) { *why = "depth_sharpness must be > 0"; return DDGI_ERR_INVALID_ARG; }
    uint32_t M = c->num_light_candidates + c->num_bsdf_candidates;
    if (c->num_bsdf_candidates < 1 || M > 64) { *why = "need 1..64 candidates with at least one BSDF candidate"; return DDGI_ERR_INVALID_ARG; }
    if (!(c->temporal_mcap >= 0.f) || !std::isfinite(c->temporal_mcap)) { *why = "temporal_mcap must be >= 0"; return DDGI_ERR_INVALID_ARG; }
    if (c->spatial_neighbours > 32) { *why = "spatial_neighbours must be <= 32"; return DDGI_ERR_INVALID_ARG; }
    if (c->candidate_stride > 64) { *why = "candidate_stride must be <= 64"; return DDGI_ERR_INVALID_ARG; }
    if (c->traversal_visit_cap > (1u << 30)) { *why = "traversal_visit_cap must be <= 2^30"; return DDGI_ERR_INVALID_ARG; }
    if (!std::isfinite(c->footprint_c)) { *why = "footprint_c must be finite"; return DDGI_ERR_INVALID_ARG; }
    if (c->spatial_radius < 1 || c->spatial_radius > 255) { *why = "spatial_radius must be 1..255"; return DDGI_ERR_INVALID_ARG; }
    if (!std::isfinite(c->normal_reject_cos) || !(c->depth_reject_frac >= 0.f)) { *why = "bad rejection thresholds"; return DDGI_ERR_INVALID_ARG; }
    const uint64_t P = (uint64_t)c->counts[0] * c->counts[1] * c->counts[2];
    if (c->train_samples > 0 && (c->train_samples % 16 != 0 || c->train_samples % P != 0 ||
                                 c->train_samples / P > 65536 || c->train_samples > (1u << 24))) {
        *why = "train_samples must be a multiple of 16 and of the probe count"; return DDGI_ERR_INVALID_ARG;
    }
    if (c->learned_target && c->train_samples == 0) { *why = "learned target needs train_samples"; return DDGI_ERR_INVALID_ARG; }
    if (c->train_samples > 0 && !(c->train_lr > 0.f && c->train_lr < 1.f)) { *why = "train_lr must be in (0, 1)"; return DDGI_ERR_INVALID_ARG; }
    if (!(c->train_ema >= 0.f && c->train_ema < 1.f)) { *why = "train_ema must be in [0, 1)"; return DDGI_ERR_INVALID_ARG; }
    return DDGI_OK;
}

CamView cam_view(const ddgi_camera* c) {
    CamView v;
    v.pos = make_float3(c->pos[0], c->pos[1], c->pos[2]);
    v.fwd = make_float3(c->fwd[0], c->fwd[1], c->fwd[2]);
    v.right = make_float3(c->right[0], c->right[1], c->right[2]);
    v.up = make_float3(c->up[0], c->up[1], c->up[2]);
    v.tan_half_fovy = c->tan_half_fovy;
    v.width = (int)c->width;
    v.height = (int)c->height;
    return v;
}

ddgi_status probe_params(ddgi_ctx* c, uint32_t frame, ProbeParams* p) {
    p->sf = c->sf;
    p->order = c->sf_order;
    p->rays = c->cfg.rays_per_probe;
    frame_rotation(c->cfg.seed, frame, p->R);
    p->hysteresis = c->updates == 0 ? 0.f : c->cfg.hysteresis;
    p->le_attenuation = c->cfg.le_attenuation;
    p->depth_sharpness = c->cfg.depth_sharpness;
    p->depth_tmax = 1.5f * std::fmax(std::fmax(c->cfg.spacing[0], c->cfg.spacing[1]), c->cfg.spacing[2]);
    p->seed = c->cfg.seed;
    p->frame = frame;
    return DDGI_OK;
}

void release(ddgi_ctx* c) {
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    if (c->hits) cudaFree(c->hits);
    c->hits = nullptr;
    c->hits_cap = 0;
    if (c->ind) cudaFree(c->ind);
    c->ind = nullptr;
    c->ind_cap = 0;
    if (c->tmp_smp) cudaFree(c->tmp_smp);
    c->tmp_smp = nullptr;
    c->tmp_cap = 0;
    if (c->pin_ev) {
        cudaEventSynchronize(c->pin_ev);
        cudaEventDestroy(c->pin_ev);
    }
    c->pin_ev = nullptr;
    c->pin_pending = false;
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    c->side = nullptr;
    c->ev_fork = c->ev_join = nullptr;
    if (c->pin) cudaFreeHost(c->pin);
    c->pin = nullptr;
}

// stream-ordered growth of a scratch buffer of T
template <class T>
cudaError_t grow(ddgi_ctx* c, T** buf, size_t* cap, size_t n, cudaStream_t st) {
    if (n <= *cap) return cudaSuccess;
    size_t nc = n + n / 4;
    T* p = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&p), nc * sizeof(T), st);
    if (e != cudaSuccess) return e;
    if (*buf) {
        e = cudaFreeAsync(*buf, st);
        c->device_bytes -= *cap * sizeof(T);
    }
    *buf = p;
    *cap = nc;
    c->device_bytes += nc * sizeof(T);
    return e;
}

// served: the moving-average network that answers queries; else the
// network being trained
MLPView mlp_view(ddgi_ctx* c, bool served = true) {
    MLPView m;
    m.w16 = served ? c->mlp_w16s : c->mlp_w16;
    m.params = served ? c->mlp_ema : c->mlp_params;
    for (int a = 0; a < 3; ++a) m.lo[a] = c->mlp_lo[a];
    m.scale = c->mlp_scale;
    m.err = c->err;
    m.bf16 = c->cfg.mlp_bf16 ? 1 : 0;
    m.fp32 = c->cfg.mlp_fp32 ? 1 : 0;
    return m;
}

// He-uniform initialisation from the PCG hash: w = (2u - 1) sqrt(6 / fan_in)
void mlp_init(uint32_t seed, std::vector<float>& p) {
    p.assign(MLP_NPARAM, 0.f);
    for (int l = 0; l < 5; ++l) {
        const int in = mlp_in(l), out = l == 4 ? 3 : 64;
        const double bound = std::sqrt(6.0 / in);
        for (int o = 0; o < out; ++o)
            for (int i = 0; i < in; ++i) {
                const uint32_t idx = (uint32_t)(mlp_off_w(l) + o * in + i);
                const double u = rng_h(seed, idx, 0, 11, 0, 0);
                p[idx] = (float)((2.0 * u - 1.0) * bound);
            }
    }
}

cudaError_t mlp_upload(ddgi_ctx* c, const float* host_params) {
    std::vector<uint16_t> h(MLP_NW);
    for (int i = 0; i < MLP_NW; ++i)
        h[i] = c->cfg.mlp_bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(host_params[i]))
                               : __half_as_ushort(__float2half_rn(host_params[i]));
    cudaError_t e = cudaMemcpy(c->mlp_params, host_params, MLP_NPARAM * sizeof(float), cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(c->mlp_w16, h.data(), MLP_NW * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->mlp_ema, host_params, MLP_NPARAM * sizeof(float), cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(c->mlp_w16s, h.data(), MLP_NW * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->mlp_m, 0, MLP_NPARAM * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->mlp_v, 0, MLP_NPARAM * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->mlp_grad, 0, 2 * MLP_NPARAM * sizeof(float));
    if (e == cudaSuccess && c->mlp_state)   // Adam restarts: no step applied yet
        e = cudaMemset(reinterpret_cast<char*>(c->mlp_state) + offsetof(MLPState, adam_t), 0, sizeof(uint32_t));
    c->mlp_step = 0;
    return e;
}

// Hit-record scratch for n rays; grows stream-ordered (no device sync).
cudaError_t ensure_hits(ddgi_ctx* c, size_t n, cudaStream_t st) {
    if (n <= c->hits_cap) return cudaSuccess;
    size_t cap = n + n / 4;
    float2* p = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&p), cap * sizeof(float2), st);
    if (e != cudaSuccess) return e;
    if (c->hits) {
        e = cudaFreeAsync(c->hits, st);
        c->device_bytes -= c->hits_cap * sizeof(float2);
    }
    c->hits = p;
    c->hits_cap = cap;
    c->device_bytes += cap * sizeof(float2);
    return e;
}

// Tables of the rigid instances: BVH slots of the instanced triangles with
// their identity-pose vertices, and the BVH4 nodes whose subtrees hold any of
// them, grouped by depth (deepest first) for the bottom-up refit.
cudaError_t setup_instances(ddgi_ctx* c, const ddgi_scene* scene, const Bvh4& bvh) {
    const uint32_t S = (uint32_t)(bvh.tris.size() / 12), I = scene->num_instances, N = bvh.num_nodes;
    std::vector<uint4> map;
    std::vector<float4> obj;
    std::vector<uint8_t> slot_moving(S, 0);
    for (uint32_t k = 0; k < S; ++k) {
        uint32_t orig;
        std::memcpy(&orig, &bvh.tris[12ull * k + 3], 4);
        const int32_t inst = scene->tri_instance[orig];
        if (inst < 0) continue;
        slot_moving[k] = 1;
        map.push_back(make_uint4(k, orig, (uint32_t)inst, 0u));
        const float* v = scene->vertices + 9ull * orig;
        for (int q = 0; q < 3; ++q) obj.push_back(make_float4(v[3 * q], v[3 * q + 1], v[3 * q + 2], 0.f));
    }
    // dirty nodes: children follow their parent in the node order, so one
    // backward sweep sees every child before its parent
    std::vector<uint8_t> dirty(N, 0);
    std::vector<uint32_t> depth(N, 0);
    for (uint32_t n = 0; n < N; ++n)
        for (int s = 0; s < 4; ++s) {
            int32_t en;
            std::memcpy(&en, &bvh.nodes[32ull * n + 24 + s], 4);
            if (en > 0) depth[en] = depth[n] + 1;
        }
    uint32_t maxd = 0;
    for (uint32_t n = N; n-- > 0;) {
        for (int s = 0; s < 4; ++s) {
            int32_t en, first, cnt;
            std::memcpy(&en, &bvh.nodes[32ull * n + 24 + s], 4);
            if (en > 0) {
                dirty[n] |= dirty[en];
            } else if (en < 0) {
                bvh_leaf_range(en, &first, &cnt);
                for (int k = first; k < first + cnt; ++k) dirty[n] |= slot_moving[k];
            }
        }
        if (dirty[n]) maxd = std::max(maxd, depth[n]);
    }
    std::vector<uint32_t> list;
    c->refit_levels.assign(1, 0u);
    for (uint32_t d = maxd + 1; d-- > 0;) {
        for (uint32_t n = 0; n < N; ++n)
            if (dirty[n] && depth[n] == d) list.push_back(n);
        c->refit_levels.push_back((uint32_t)list.size());
    }
    // the unmoved references of each listed node's leaf slots keep the boxes
    // they were built with (clipped where a spatial split cut their triangle);
    // the refit adds the moving triangles' current boxes to them
    std::vector<float> stat(24 * list.size());
    for (size_t i = 0; i < list.size(); ++i)
        for (int sl = 0; sl < 4; ++sl) {
            float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
            int32_t en, first, cnt;
            std::memcpy(&en, &bvh.nodes[32ull * list[i] + 24 + sl], 4);
            if (en < 0) {
                bvh_leaf_range(en, &first, &cnt);
                for (int k = first; k < first + cnt; ++k) {
                    if (slot_moving[k]) continue;
                    for (int a = 0; a < 3; ++a) {
                        lo[a] = std::min(lo[a], bvh.slot_box[6ull * k + a]);
                        hi[a] = std::max(hi[a], bvh.slot_box[6ull * k + 3 + a]);
                    }
                }
            }
            for (int a = 0; a < 3; ++a) {
                stat[24 * i + 6 * sl + a] = lo[a];
                stat[24 * i + 6 * sl + 3 + a] = hi[a];
            }
        }
    std::vector<int32_t> ti(scene->tri_instance, scene->tri_instance + c->T);
    c->I = I;
    c->NI = (uint32_t)map.size();
    c->xf_cur.assign(12ull * I, 0.0);
    for (uint32_t k = 0; k < I; ++k) c->xf_cur[12 * k] = c->xf_cur[12 * k + 5] = c->xf_cur[12 * k + 10] = 1.0;
    c->xf_prev = c->xf_cur;
    std::vector<float4> ident(3ull * I);
    for (uint32_t k = 0; k < I; ++k) {
        ident[3 * k] = make_float4(1.f, 0.f, 0.f, 0.f);
        ident[3 * k + 1] = make_float4(0.f, 1.f, 0.f, 0.f);
        ident[3 * k + 2] = make_float4(0.f, 0.f, 1.f, 0.f);
    }
    cudaError_t e = dalloc(c, &c->tri_inst, c->T);
    if (e == cudaSuccess) e = dalloc(c, &c->inst_map, map.size());
    if (e == cudaSuccess) e = dalloc(c, &c->inst_obj, obj.size());
    if (e == cudaSuccess) e = dalloc(c, &c->inst_xf, 3ull * I);
    if (e == cudaSuccess) e = dalloc(c, &c->inst_delta, 3ull * I);
    if (e == cudaSuccess) e = dalloc(c, &c->refit_list, list.size());
    if (e == cudaSuccess) e = dalloc(c, &c->refit_static, stat.size());
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up(c->tri_inst, ti.data(), c->T * sizeof(int32_t));
    up(c->inst_map, map.data(), map.size() * sizeof(uint4));
    up(c->inst_obj, obj.data(), obj.size() * sizeof(float4));
    up(c->inst_xf, ident.data(), ident.size() * sizeof(float4));
    up(c->inst_delta, ident.data(), ident.size() * sizeof(float4));
    up(c->refit_list, list.data(), list.size() * sizeof(uint32_t));
    up(c->refit_static, stat.data(), stat.size() * sizeof(float));
    return e;
}

// rows of A B for row-major 3x4 affine transforms
void compose34(const double* A, const double* B, double* out) {
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k)
            out[4 * r + k] = A[4 * r] * B[k] + A[4 * r + 1] * B[4 + k] + A[4 * r + 2] * B[8 + k];
        out[4 * r + 3] = A[4 * r] * B[3] + A[4 * r + 1] * B[7] + A[4 * r + 2] * B[11] + A[4 * r + 3];
    }
}

// inverse of a 3x4 affine transform (cofactors); false if singular
bool invert34(const double* M, double* out) {
    const double a = M[0], b = M[1], cc = M[2], d = M[4], e = M[5], f = M[6], g = M[8], h = M[9], i = M[10];
    const double C[9] = {e * i - f * h, cc * h - b * i, b * f - cc * e, f * g - d * i, a * i - cc * g,
                         cc * d - a * f, d * h - e * g, b * g - a * h, a * e - b * d};
    const double det = a * C[0] + b * C[3] + cc * C[6];
    if (!(std::fabs(det) > 1e-12) || !std::isfinite(det)) return false;
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) out[4 * r + k] = C[3 * r + k] / det;
        out[4 * r + 3] = -(out[4 * r] * M[3] + out[4 * r + 1] * M[7] + out[4 * r + 2] * M[11]);
    }
    return true;
}

// --- state snapshot --------------------------------------------------------
// Layout (host byte stream): a header of 16 uint32 (magic, version, P,
// irradiance tile, distance tile, instances, emitters, learned flag,
// probe updates, Adam steps, serve mode, 5 zero), then, in this order:
// irradiance [P][ti^2] float4, distance moments [P][td^2] float2, offsets
// [P] float4, current / previous instance transforms [I][12] double each,
// emitter radiance [E][3] float, and for a learned-target context the master
// parameters, Adam moments m and v, served (averaged) parameters [NPARAM]
// float each, their fp16 copies [NW] x 2, and the optimiser / judge state.
const uint32_t kStateMagic = 0x44444749u;   // "IGDD"
const uint32_t kStateVersion = 1u;

struct StateLayout {
    size_t irr, dep, off, xf, le, mlp32, mlp16, mst, total;
};

StateLayout state_layout(const ddgi_ctx* c) {
    StateLayout L;
    const size_t P = c->P, ti = c->cfg.irr_texels + 2, td = c->cfg.depth_texels + 2;
    size_t o = 16 * sizeof(uint32_t);
    L.irr = o; o += P * ti * ti * sizeof(float4);
    L.dep = o; o += P * td * td * sizeof(float2);
    L.off = o; o += P * sizeof(float4);
    L.xf = o; o += 2 * 12ull * c->I * sizeof(double);
    L.le = o; o += 3ull * c->E * sizeof(float);
    L.mlp32 = o;
    L.mlp16 = L.mst = o;
    if (c->cfg.learned_target) {
        o += 4ull * MLP_NPARAM * sizeof(float);
        L.mlp16 = o; o += 2ull * MLP_NW * sizeof(uint16_t);
        L.mst = o; o += sizeof(MLPState);
    }
    L.total = o;
    return L;
}
}  // namespace

extern "C" {

ddgi_status ddgi_create(const ddgi_scene* scene, const ddgi_config* cfg, ddgi_ctx** out) {
    if (!out) return DDGI_ERR_INVALID_ARG;
    *out = nullptr;
    if (!scene || !cfg) return DDGI_ERR_INVALID_ARG;
    if (scene->num_tris > 0 && (!scene->vertices || !scene->albedo || !scene->emission))
        return DDGI_ERR_INVALID_ARG;
    if (scene->num_tris > (1u << 28)) return DDGI_ERR_INVALID_ARG;
    std::string why;
    if (check_config(cfg, &why) != DDGI_OK) return DDGI_ERR_INVALID_ARG;
    for (uint64_t i = 0; i < 9ull * scene->num_tris; ++i)
        if (!std::isfinite(scene->vertices[i])) return DDGI_ERR_INVALID_ARG;
    for (uint64_t i = 0; i < 3ull * scene->num_tris; ++i)
        if (!(scene->albedo[i] >= 0.f && scene->albedo[i] <= 1.f) ||
            !(scene->emission[i] >= 0.f) || !std::isfinite(scene->emission[i]))
            return DDGI_ERR_INVALID_ARG;
    bool glossy = false;   // some triangle has a glossy lobe
    if (scene->glossy) {
        for (uint32_t i = 0; i < scene->num_tris; ++i) {
            const float* gl = scene->glossy + 4ull * i;
            const float* e = scene->emission + 3ull * i;
            for (int a = 0; a < 3; ++a)
                if (!(gl[a] >= 0.f && gl[a] <= 1.f)) return DDGI_ERR_INVALID_ARG;
            const bool has = gl[0] > 0.f || gl[1] > 0.f || gl[2] > 0.f;
            if (has && !(gl[3] >= 1e-3f && gl[3] <= 1.f)) return DDGI_ERR_INVALID_ARG;
            if (has && (e[0] > 0.f || e[1] > 0.f || e[2] > 0.f)) return DDGI_ERR_INVALID_ARG;   // emitters
            glossy = glossy || has;
        }
        if (glossy && cfg->learned_target) return DDGI_ERR_INVALID_ARG;
    }
    if (scene->tri_instance) {
        if (scene->num_instances == 0 || scene->num_instances > (1u << 20)) return DDGI_ERR_INVALID_ARG;
        for (uint32_t i = 0; i < scene->num_tris; ++i) {
            const int32_t k = scene->tri_instance[i];
            const float* e = scene->emission + 3ull * i;
            if (k < -1 || k >= (int32_t)scene->num_instances) return DDGI_ERR_INVALID_ARG;
            if (k >= 0 && (e[0] > 0.f || e[1] > 0.f || e[2] > 0.f)) return DDGI_ERR_INVALID_ARG;
        }
    }

    ddgi_ctx* ctx = new (std::nothrow) ddgi_ctx;
    if (!ctx) return DDGI_ERR_OOM;
    ctx->cfg = *cfg;
    const uint32_t T = scene->num_tris;
    ctx->T = T;
    ctx->P = (uint32_t)(cfg->counts[0] * cfg->counts[1] * cfg->counts[2]);

    // scene tables (host), fp64 geometry for normals / areas
    Bvh4 bvh;
    // instanced scenes refit slot boxes from whole triangles: no split references
    std::vector<uint8_t> fixed;
    if (scene->tri_instance) {   // moving triangles: never split (refitted from whole triangles)
        fixed.resize(T);
        for (uint32_t t = 0; t < T; ++t) fixed[t] = scene->tri_instance[t] >= 0 ? 1 : 0;
    }
    build_bvh4(scene->vertices, T, fixed.empty() ? nullptr : fixed.data(), &bvh);
    ctx->bvh_nodes = bvh.num_nodes;
    ctx->bvh_depth = bvh.depth;
    std::vector<float4> nrm(T), alb(T), emi(T);
    std::vector<float4> evert;
    std::vector<float> cdf;
    std::vector<uint32_t> etri;
    double acc = 0.0;
    for (uint32_t i = 0; i < T; ++i) {
        const float* v = scene->vertices + 9ull * i;
        double e1[3], e2[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = (double)v[3 + a] - (double)v[a];
            e2[a] = (double)v[6 + a] - (double)v[a];
        }
        double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                       e1[0] * e2[1] - e1[1] * e2[0]};
        double l = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        nrm[i] = l > 0 ? make_float4((float)(c[0] / l), (float)(c[1] / l), (float)(c[2] / l), 0.f)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        const float* a = scene->albedo + 3ull * i;
        const float* e = scene->emission + 3ull * i;
        bool emissive = e[0] > 0.f || e[1] > 0.f || e[2] > 0.f;
        alb[i] = make_float4(a[0], a[1], a[2], 0.f);
        emi[i] = make_float4(e[0], e[1], e[2], emissive ? 1.f : 0.f);
        if (emissive) {
            acc += 0.5 * l;
            cdf.push_back((float)acc);
            etri.push_back(i);
            // packed record: v0 + triangle id, e1 + Le.r, e2 + Le.g, normal + Le.b
            uint32_t tid = i;
            float tbits;
            std::memcpy(&tbits, &tid, 4);
            evert.push_back(make_float4(v[0], v[1], v[2], tbits));
            evert.push_back(make_float4(v[3] - v[0], v[4] - v[1], v[5] - v[2], e[0]));
            evert.push_back(make_float4(v[6] - v[0], v[7] - v[1], v[8] - v[2], e[1]));
            evert.push_back(make_float4(nrm[i].x, nrm[i].y, nrm[i].z, e[2]));
            if (a[0] > 0.f || a[1] > 0.f || a[2] > 0.f) ctx->emitters_reflect = 1;
        }
    }
    ctx->E = (uint32_t)etri.size();
    ctx->area_total = (float)acc;
    if (ctx->E > 0 && !(acc > 0.0)) {
        delete ctx;
        return DDGI_ERR_INVALID_ARG;   // emissive triangles of zero area
    }
    // guide table for the emitter search: guide[j] = first emitter whose
    // cumulative area exceeds (j / G) * total, evaluated in float exactly as
    // the kernel forms its search target, so a scan from guide[floor(u G)]
    // ends on the same emitter as a search over the whole table
    std::vector<uint32_t> guide;
    if (ctx->E > 0) {
        uint32_t G = 1;
        while (G < ctx->E && G < (1u << 16)) G <<= 1;
        guide.resize(G);
        const float total = cdf.back();
        uint32_t i = 0;
        for (uint32_t j = 0; j < G; ++j) {
            float Tj = ((float)j / (float)G) * total;
            while (i < ctx->E - 1 && !(Tj < cdf[i])) ++i;
            guide[j] = i;
        }
    }
    ctx->G = (uint32_t)guide.size();
    // spherical Fibonacci directions (fp64 on the host)
    const uint32_t R = cfg->rays_per_probe;
    std::vector<float4> sf(R);
    for (uint32_t i = 0; i < R; ++i) {
        double z = 1.0 - (2.0 * i + 1.0) / R;
        double r = std::sqrt(std::fmax(0.0, 1.0 - z * z));
        double ph = i * 0.6180339887498949;
        ph = 2.0 * 3.14159265358979323846 * (ph - std::floor(ph));
        sf[i] = make_float4((float)(r * std::cos(ph)), (float)(r * std::sin(ph)), (float)z, 0.f);
    }
    // the order in which a probe's threads take its rays: by the Morton code
    // of each direction's octahedral map, so that every 32 consecutive rays
    // form a compact patch of the sphere (the per-frame rotation moves all of
    // them rigidly and keeps the patches); a spherical Fibonacci index step
    // turns the azimuth by the golden angle, which scatters a warp's rays
    std::vector<uint32_t> sf_order(R);
    {
        std::vector<std::pair<uint64_t, uint32_t>> key(R);
        for (uint32_t i = 0; i < R; ++i) {
            double x = sf[i].x, y = sf[i].y, zz = sf[i].z;
            double s = std::fabs(x) + std::fabs(y) + std::fabs(zz);
            double u = x / s, w = y / s;
            if (zz < 0.0) {
                double fu = (1.0 - std::fabs(w)) * (u >= 0.0 ? 1.0 : -1.0);
                double fw = (1.0 - std::fabs(u)) * (w >= 0.0 ? 1.0 : -1.0);
                u = fu;
                w = fw;
            }
            uint32_t qu = (uint32_t)std::min(65535.0, std::floor((u + 1.0) * 32768.0));
            uint32_t qw = (uint32_t)std::min(65535.0, std::floor((w + 1.0) * 32768.0));
            uint64_t m = 0;
            for (int b = 0; b < 16; ++b) m |= (uint64_t)((qu >> b) & 1u) << (2 * b) | (uint64_t)((qw >> b) & 1u) << (2 * b + 1);
            key[i] = {m, i};
        }
        std::sort(key.begin(), key.end());
        for (uint32_t i = 0; i < R; ++i) sf_order[i] = key[i].second;
    }

    const size_t ti = cfg->irr_texels + 2, td = cfg->depth_texels + 2;
    const size_t P = ctx->P;
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, n)                                 \
    if (e == cudaSuccess) e = dalloc(ctx, &ctx->ptr, (n));
    ALLOC(nodes, 8ull * bvh.num_nodes)
    ALLOC(tris, bvh.tris.size() / 4)
    ALLOC(nrm, T)
    ALLOC(alb, T)
    ALLOC(emi, T)
    ALLOC(evert, 4ull * ctx->E)
    ALLOC(evert3, 3ull * ctx->E)
    ALLOC(guide, ctx->G)
    ALLOC(cdf, ctx->E)
    ALLOC(etri, ctx->E)
    ALLOC(irr, P * ti * ti)
    ALLOC(depth, P * td * td)
    ALLOC(irr_q, P * (ti - 1) * (ti - 1) * 4)
    ALLOC(depth_q, P * (td - 1) * (td - 1) * 2)
    ALLOC(offset, P)
    ALLOC(rays, P * R)
    ALLOC(blend_w, probe_blend_weights_size(volume_view(ctx), R))
    ALLOC(sf, R)
    ALLOC(sf_order, R)
    ALLOC(err, 4)
    ALLOC(counter, 4)
    ALLOC(mlp_params, MLP_NPARAM)
    ALLOC(mlp_grad, 2 * MLP_NPARAM)   // two buffers: Adam step t accumulates in buffer t & 1
    ALLOC(mlp_m, MLP_NPARAM)
    ALLOC(mlp_v, MLP_NPARAM)
    ALLOC(tmp_grad, MLP_NPARAM)
    ALLOC(mlp_w16, MLP_NW)
    ALLOC(mlp_ema, MLP_NPARAM)
    ALLOC(mlp_w16s, MLP_NW)
    ALLOC(mlp_state, 1)
    ALLOC(train_smp, 3ull * cfg->train_samples)
    ALLOC(le_stage, 3ull * ctx->E)
    ALLOC(train_sf, cfg->train_samples ? cfg->train_samples / P : 0)
    ALLOC(spec, glossy ? T : 0)
#undef ALLOC
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up(ctx->nodes, bvh.nodes.data(), bvh.nodes.size() * sizeof(float));
    up(ctx->tris, bvh.tris.data(), bvh.tris.size() * sizeof(float));
    up(ctx->nrm, nrm.data(), T * sizeof(float4));
    up(ctx->alb, alb.data(), T * sizeof(float4));
    up(ctx->emi, emi.data(), T * sizeof(float4));
    up(ctx->evert, evert.data(), evert.size() * sizeof(float4));
    {
        std::vector<float4> ev3(3ull * ctx->E);
        for (size_t k = 0; k < ctx->E; ++k) {
            ev3[3 * k] = evert[4 * k];
            ev3[3 * k].w = evert[4 * k + 3].w;
            ev3[3 * k + 1] = evert[4 * k + 1];
            ev3[3 * k + 2] = evert[4 * k + 2];
        }
        up(ctx->evert3, ev3.data(), ev3.size() * sizeof(float4));
    }
    up(ctx->cdf, cdf.data(), cdf.size() * sizeof(float));
    up(ctx->etri, etri.data(), etri.size() * sizeof(uint32_t));
    up(ctx->guide, guide.data(), guide.size() * sizeof(uint32_t));
    up(ctx->sf, sf.data(), R * sizeof(float4));
    up(ctx->sf_order, sf_order.data(), R * sizeof(uint32_t));
    if (glossy) up(ctx->spec, scene->glossy, T * sizeof(float4));
    if (e == cudaSuccess && scene->tri_instance) e = setup_instances(ctx, scene, bvh);
    if (e == cudaSuccess) e = cudaMemset(ctx->irr, 0, P * ti * ti * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemset(ctx->depth, 0, P * td * td * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(ctx->irr_q, 0, P * (ti - 1) * (ti - 1) * 4 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemset(ctx->depth_q, 0, P * (td - 1) * (td - 1) * 2 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemset(ctx->offset, 0, P * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemset(ctx->rays, 0, P * R * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemset(ctx->err, 0, 4 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->counter, 0, 4 * sizeof(uint32_t));
    if (e == cudaSuccess) e = ensure_hits(ctx, std::max<size_t>(P * R, cfg->train_samples), 0);
    if (e == cudaSuccess) {
        // network: scene box for the input normalisation, initial weights, state
        float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
        for (uint64_t i = 0; i < 3ull * T; ++i)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::fmin(lo[a], scene->vertices[3 * i + a]);
                hi[a] = std::fmax(hi[a], scene->vertices[3 * i + a]);
            }
        float ext = 0.f;
        for (int a = 0; a < 3; ++a) {
            ctx->mlp_lo[a] = T ? lo[a] : 0.f;
            ext = std::fmax(ext, hi[a] - lo[a]);
        }
        ctx->mlp_scale = ext > 0.f ? 1.f / ext : 1.f;
        std::vector<float> p0;
        mlp_init(cfg->mlp_seed, p0);
        e = mlp_upload(ctx, p0.data());
        MLPState st0{};
        st0.loss_scale = 1.f;
        if (e == cudaSuccess) e = cudaMemcpy(ctx->mlp_state, &st0, sizeof(st0), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && cfg->train_samples) {
            const uint32_t per = (uint32_t)(cfg->train_samples / P);
            ctx->train_per = per;
            std::vector<float4> tsf(per);
            for (uint32_t i = 0; i < per; ++i) {
                double z = 1.0 - (2.0 * i + 1.0) / per;
                double r = std::sqrt(std::fmax(0.0, 1.0 - z * z));
                double ph = i * 0.6180339887498949;
                ph = 2.0 * 3.14159265358979323846 * (ph - std::floor(ph));
                tsf[i] = make_float4((float)(r * std::cos(ph)), (float)(r * std::sin(ph)), (float)z, 0.f);
            }
            e = cudaMemcpy(ctx->train_sf, tsf.data(), per * sizeof(float4), cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
        VolumeView v = volume_view(ctx);
        if (probe_blend_smem(v, R) > 200 * 1024) e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) {
        release(ctx);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? DDGI_ERR_OOM : DDGI_ERR_CUDA;
    }
    *out = ctx;
    return DDGI_OK;
}

ddgi_status ddgi_destroy(ddgi_ctx* ctx) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    release(ctx);
    delete ctx;
    return DDGI_OK;
}

ddgi_status ddgi_get_info(ddgi_ctx* ctx, ddgi_info* out) {
    if (!ctx || !out) return DDGI_ERR_INVALID_ARG;
    out->num_tris = ctx->T;
    out->num_emitters = ctx->E;
    out->num_probes = ctx->P;
    out->rays_per_probe = ctx->cfg.rays_per_probe;
    out->irr_tile = ctx->cfg.irr_texels + 2;
    out->depth_tile = ctx->cfg.depth_texels + 2;
    out->bvh_nodes = ctx->bvh_nodes;
    out->bvh_depth = ctx->bvh_depth;
    out->updates = ctx->updates;
    out->device_bytes = ctx->device_bytes;
    return DDGI_OK;
}

ddgi_status ddgi_probe_trace(ddgi_ctx* ctx, uint32_t frame, void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    ProbeParams p;
    probe_params(ctx, frame, &p);
    CK(launch_probe_trace(scene_view(ctx), volume_view(ctx), p, ctx->rays, ctx->hits, ctx->counter,
                          (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_probe_blend(ddgi_ctx* ctx, uint32_t frame, void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    ProbeParams p;
    probe_params(ctx, frame, &p);
    CK(launch_probe_blend(volume_view(ctx), p, ctx->rays, ctx->blend_w, (cudaStream_t)stream));
    ctx->updates++;
    return DDGI_OK;
}

namespace {
// the staging buffer may be rewritten once the copies of the previous update
// out of it have run (allocated on first use)
cudaError_t stage_ready(ddgi_ctx* c) {
    if (!c->pin) {
        cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&c->pin), (24ull * c->I + 3ull * c->E) * sizeof(float));
        if (e != cudaSuccess) {
            c->pin = nullptr;
            return e;
        }
        e = cudaEventCreateWithFlags(&c->pin_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) c->pin_ev = nullptr;
        return e;
    }
    if (!c->pin_pending) return cudaSuccess;
    c->pin_pending = false;
    return cudaEventSynchronize(c->pin_ev);
}
}  // namespace

ddgi_status ddgi_scene_update(ddgi_ctx* ctx, const float* xf, uint32_t n, const float* emitter_radiance,
                              void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    bool staged = false;
    if (emitter_radiance) {   // both arguments are checked before anything is enqueued
        if (ctx->E == 0) return fail(ctx, DDGI_ERR_INVALID_ARG, "the scene has no emitters");
        for (size_t k = 0; k < 3ull * ctx->E; ++k)
            if (!(emitter_radiance[k] >= 0.f) || !std::isfinite(emitter_radiance[k]))
                return fail(ctx, DDGI_ERR_INVALID_ARG, "emitter radiance must be finite and >= 0");
    }
    if (xf) {
        if (ctx->I == 0 || n != ctx->I) return fail(ctx, DDGI_ERR_INVALID_ARG, "transform count != instance count");
        std::vector<double> cur(12ull * n), delta(12ull * n);
        for (size_t k = 0; k < 12ull * n; ++k) {
            if (!std::isfinite(xf[k])) return fail(ctx, DDGI_ERR_INVALID_ARG, "non-finite transform");
            cur[k] = xf[k];
        }
        for (uint32_t k = 0; k < n; ++k) {
            double inv[12];
            if (!invert34(&cur[12ull * k], inv)) return fail(ctx, DDGI_ERR_INVALID_ARG, "singular transform");
            compose34(&ctx->xf_cur[12ull * k], inv, &delta[12ull * k]);
        }
        CK(stage_ready(ctx));
        float* sx = ctx->pin;
        float* sd = ctx->pin + 12ull * ctx->I;
        std::memcpy(sx, xf, 12ull * n * sizeof(float));
        for (size_t k = 0; k < 12ull * n; ++k) sd[k] = (float)delta[k];
        CK(cudaMemcpyAsync(ctx->inst_xf, sx, 12ull * n * sizeof(float), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ctx->inst_delta, sd, 12ull * n * sizeof(float), cudaMemcpyHostToDevice, st));
        staged = true;
        CK(launch_instance_update(ctx->inst_obj, ctx->inst_map, ctx->NI, ctx->inst_xf, ctx->tris, ctx->nrm,
                                  ctx->nodes, ctx->refit_list, ctx->refit_static, ctx->tri_inst, ctx->refit_levels,
                                  st));
        ctx->xf_prev = ctx->xf_cur;
        ctx->xf_cur = cur;
    }
    if (emitter_radiance) {
        if (!staged) CK(stage_ready(ctx));
        float* sl = ctx->pin + 24ull * ctx->I;
        std::memcpy(sl, emitter_radiance, 3ull * ctx->E * sizeof(float));
        CK(cudaMemcpyAsync(ctx->le_stage, sl, 3ull * ctx->E * sizeof(float), cudaMemcpyHostToDevice, st));
        staged = true;
        CK(launch_emitter_radiance(ctx->le_stage, ctx->etri, ctx->emi, ctx->evert, ctx->evert3, ctx->E, st));
    }
    if (staged) {
        CK(cudaEventRecord(ctx->pin_ev, st));
        ctx->pin_pending = true;
    }
    return DDGI_OK;
}

ddgi_status ddgi_probe_relocate(ddgi_ctx* ctx, uint32_t frame, void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    ProbeParams p;
    probe_params(ctx, frame, &p);
    CK(launch_probe_relocate(volume_view(ctx), p, ctx->rays, ctx->offset, (cudaStream_t)stream));
    ctx->offsets_used = true;
    return DDGI_OK;
}

ddgi_status ddgi_probe_update(ddgi_ctx* ctx, uint32_t frame, void* stream) {
    ddgi_status s = ddgi_probe_trace(ctx, frame, stream);
    if (s != DDGI_OK) return s;
    s = ddgi_probe_blend(ctx, frame, stream);
    if (s != DDGI_OK || !ctx->cfg.probe_relocation) return s;
    return ddgi_probe_relocate(ctx, frame, stream);
}

ddgi_status ddgi_probe_state_get(ddgi_ctx* ctx, float* irr, float* depth, float* offsets,
                                 uint32_t* updates, void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t P = ctx->P, ti = ctx->cfg.irr_texels + 2, td = ctx->cfg.depth_texels + 2;
    if (irr) CK(cudaMemcpyAsync(irr, ctx->irr, P * ti * ti * sizeof(float4), cudaMemcpyDefault, st));
    if (depth) CK(cudaMemcpyAsync(depth, ctx->depth, P * td * td * sizeof(float2), cudaMemcpyDefault, st));
    if (offsets) CK(cudaMemcpyAsync(offsets, ctx->offset, P * sizeof(float4), cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    if (updates) *updates = ctx->updates;
    return DDGI_OK;
}

ddgi_status ddgi_probe_state_set(ddgi_ctx* ctx, const float* irr, const float* depth,
                                 const float* offsets, uint32_t updates, void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t P = ctx->P, ti = ctx->cfg.irr_texels + 2, td = ctx->cfg.depth_texels + 2;
    if (irr) CK(cudaMemcpyAsync(ctx->irr, irr, P * ti * ti * sizeof(float4), cudaMemcpyDefault, st));
    if (depth) CK(cudaMemcpyAsync(ctx->depth, depth, P * td * td * sizeof(float2), cudaMemcpyDefault, st));
    if (irr || depth) CK(launch_probe_quads(volume_view(ctx), st));
    if (offsets) {
        CK(cudaMemcpyAsync(ctx->offset, offsets, P * sizeof(float4), cudaMemcpyDefault, st));
        ctx->offsets_used = true;
    }
    CK(cudaStreamSynchronize(st));
    ctx->updates = updates;
    return DDGI_OK;
}

ddgi_status ddgi_state_save(ddgi_ctx* ctx, void* host_buf, size_t* bytes, void* stream) {
    if (!ctx || !bytes) return DDGI_ERR_INVALID_ARG;
    const StateLayout L = state_layout(ctx);
    if (!host_buf) {
        *bytes = L.total;
        return DDGI_OK;
    }
    if (*bytes < L.total) return fail(ctx, DDGI_ERR_INVALID_ARG, "state buffer too small");
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t* b = static_cast<uint8_t*>(host_buf);
    uint32_t h[16] = {kStateMagic, kStateVersion, ctx->P, ctx->cfg.irr_texels + 2, ctx->cfg.depth_texels + 2,
                      ctx->I, ctx->E, ctx->cfg.learned_target ? 1u : 0u, ctx->updates, ctx->mlp_step,
                      (uint32_t)ctx->serve, 0, 0, 0, 0, 0};
    std::memcpy(b, h, sizeof(h));
    CK(cudaMemcpyAsync(b + L.irr, ctx->irr, L.dep - L.irr, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(b + L.dep, ctx->depth, L.off - L.dep, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(b + L.off, ctx->offset, L.xf - L.off, cudaMemcpyDeviceToHost, st));
    if (ctx->I) {
        std::memcpy(b + L.xf, ctx->xf_cur.data(), 12ull * ctx->I * sizeof(double));
        std::memcpy(b + L.xf + 12ull * ctx->I * sizeof(double), ctx->xf_prev.data(), 12ull * ctx->I * sizeof(double));
    }
    float* le = reinterpret_cast<float*>(b + L.le);
    if (ctx->E) {   // the radiance words of the emitter records
        std::vector<float4> ev(4ull * ctx->E);
        CK(cudaMemcpyAsync(ev.data(), ctx->evert, ev.size() * sizeof(float4), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (uint32_t e = 0; e < ctx->E; ++e) {
            le[3 * e] = ev[4 * e + 1].w;
            le[3 * e + 1] = ev[4 * e + 2].w;
            le[3 * e + 2] = ev[4 * e + 3].w;
        }
    }
    if (ctx->cfg.learned_target) {
        float* const src32[4] = {ctx->mlp_params, ctx->mlp_m, ctx->mlp_v, ctx->mlp_ema};
        for (int k = 0; k < 4; ++k)
            CK(cudaMemcpyAsync(b + L.mlp32 + k * MLP_NPARAM * sizeof(float), src32[k], MLP_NPARAM * sizeof(float),
                               cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(b + L.mlp16, ctx->mlp_w16, MLP_NW * sizeof(uint16_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(b + L.mlp16 + MLP_NW * sizeof(uint16_t), ctx->mlp_w16s, MLP_NW * sizeof(uint16_t),
                           cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(b + L.mst, ctx->mlp_state, sizeof(MLPState), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    *bytes = L.total;
    return DDGI_OK;
}

ddgi_status ddgi_state_load(ddgi_ctx* ctx, const void* host_buf, size_t bytes, void* stream) {
    if (!ctx || !host_buf) return DDGI_ERR_INVALID_ARG;
    const StateLayout L = state_layout(ctx);
    const uint8_t* b = static_cast<const uint8_t*>(host_buf);
    uint32_t h[16];
    if (bytes < sizeof(h)) return fail(ctx, DDGI_ERR_INVALID_ARG, "state buffer too small");
    std::memcpy(h, b, sizeof(h));
    if (h[0] != kStateMagic || h[1] != kStateVersion) return fail(ctx, DDGI_ERR_INVALID_ARG, "not a state snapshot");
    if (h[2] != ctx->P || h[3] != ctx->cfg.irr_texels + 2 || h[4] != ctx->cfg.depth_texels + 2 || h[5] != ctx->I ||
        h[6] != ctx->E || h[7] != (ctx->cfg.learned_target ? 1u : 0u) || bytes != L.total)
        return fail(ctx, DDGI_ERR_INVALID_ARG, "snapshot of a different scene or configuration");
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->I) {
        // replay the last two poses: the triangles land on the current one and
        // the reprojection delta is that of the saved pair
        std::vector<double> cur(12ull * ctx->I), prev(12ull * ctx->I);
        std::memcpy(cur.data(), b + L.xf, cur.size() * sizeof(double));
        std::memcpy(prev.data(), b + L.xf + cur.size() * sizeof(double), prev.size() * sizeof(double));
        std::vector<float> pf(prev.begin(), prev.end()), cf(cur.begin(), cur.end());
        ddgi_status s = ddgi_scene_update(ctx, pf.data(), ctx->I, nullptr, stream);
        if (s == DDGI_OK) s = ddgi_scene_update(ctx, cf.data(), ctx->I, nullptr, stream);
        if (s != DDGI_OK) return s;
        ctx->xf_cur = cur;   // exact fp64 copies (the replay went through float)
        ctx->xf_prev = prev;
    }
    if (ctx->E) {
        ddgi_status s = ddgi_scene_update(ctx, nullptr, 0, reinterpret_cast<const float*>(b + L.le), stream);
        if (s != DDGI_OK) return s;
    }
    CK(cudaMemcpyAsync(ctx->irr, b + L.irr, L.dep - L.irr, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->depth, b + L.dep, L.off - L.dep, cudaMemcpyHostToDevice, st));
    CK(launch_probe_quads(volume_view(ctx), st));
    CK(cudaMemcpyAsync(ctx->offset, b + L.off, L.xf - L.off, cudaMemcpyHostToDevice, st));
    ctx->offsets_used = true;
    if (ctx->cfg.learned_target) {
        float* const dst32[4] = {ctx->mlp_params, ctx->mlp_m, ctx->mlp_v, ctx->mlp_ema};
        for (int k = 0; k < 4; ++k)
            CK(cudaMemcpyAsync(dst32[k], b + L.mlp32 + k * MLP_NPARAM * sizeof(float), MLP_NPARAM * sizeof(float),
                               cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ctx->mlp_w16, b + L.mlp16, MLP_NW * sizeof(uint16_t), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ctx->mlp_w16s, b + L.mlp16 + MLP_NW * sizeof(uint16_t), MLP_NW * sizeof(uint16_t),
                           cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ctx->mlp_state, b + L.mst, sizeof(MLPState), cudaMemcpyHostToDevice, st));
        // both gradient buffers zero, whichever the restored step uses next
        CK(cudaMemsetAsync(ctx->mlp_grad, 0, 2 * MLP_NPARAM * sizeof(float), st));
    }
    CK(cudaStreamSynchronize(st));
    ctx->updates = h[8];
    ctx->mlp_step = h[9];
    ctx->serve = (int)h[10];
    return DDGI_OK;
}

ddgi_status ddgi_probe_rays_get(ddgi_ctx* ctx, float* rays, void* stream) {
    if (!ctx || !rays) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(rays, ctx->rays, (size_t)ctx->P * ctx->cfg.rays_per_probe * sizeof(float4),
                       cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    return DDGI_OK;
}

ddgi_status ddgi_probe_rays_set(ddgi_ctx* ctx, const float* rays, void* stream) {
    if (!ctx || !rays) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(ctx->rays, rays, (size_t)ctx->P * ctx->cfg.rays_per_probe * sizeof(float4),
                       cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    return DDGI_OK;
}

ddgi_status ddgi_gbuffer(ddgi_ctx* ctx, const ddgi_camera* cam, const ddgi_camera* prev_cam,
                         const ddgi_gbuf* out, void* stream) {
    if (!ctx || !cam) return fail(ctx, DDGI_ERR_INVALID_ARG, "NULL argument");
    GBufView g;
    ddgi_status s = check_gbuf(ctx, out, &g);
    if (s != DDGI_OK) return s;
    if (cam->width != out->width || cam->height != out->height)
        return fail(ctx, DDGI_ERR_INVALID_ARG, "camera size != gbuffer size");
    if (!(cam->tan_half_fovy > 0.f) || (prev_cam && !(prev_cam->tan_half_fovy > 0.f)))
        return fail(ctx, DDGI_ERR_INVALID_ARG, "field of view must be > 0");
    if (prev_cam && (prev_cam->width != cam->width || prev_cam->height != cam->height))
        return fail(ctx, DDGI_ERR_INVALID_ARG, "previous camera size differs");
    CamView c = cam_view(cam), pc;
    if (prev_cam) pc = cam_view(prev_cam);
    CK(ensure_hits(ctx, (size_t)g.width * g.height, (cudaStream_t)stream));
    CK(launch_gbuffer(scene_view(ctx), c, prev_cam ? &pc : nullptr, g, ctx->hits, ctx->counter,
                      (cudaStream_t)stream));
    return DDGI_OK;
}

// restir_initial, and with fin / prev set the fused initial + temporal pass
static ddgi_status initial_impl(ddgi_ctx* ctx, const GBufView& g, const ResView& r, float* residual, uint32_t frame,
                                void* stream, const ResView* prev, const ResView* fin, float3 cam_prev) {
    const uint64_t n = (uint64_t)g.width * g.height;
    if (n > 0 && (!residual || !aligned(residual, 16)))
        return fail(ctx, DDGI_ERR_INVALID_ARG, "residual NULL or misaligned");
    CK(ensure_hits(ctx, (size_t)n * ctx->cfg.num_bsdf_candidates, (cudaStream_t)stream));
    MLPView mv = mlp_view(ctx);
    if (ctx->cfg.learned_target)
        CK(grow(ctx, &ctx->ind, &ctx->ind_cap, (size_t)n * ctx->cfg.num_bsdf_candidates, (cudaStream_t)stream));
    if (!ctx->side) {
        CK(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    }
    CK(launch_restir_initial(scene_view(ctx), volume_view(ctx), restir_params(ctx), g, r,
                             reinterpret_cast<float4*>(residual), frame, ctx->hits, ctx->counter,
                             ctx->cfg.learned_target ? &mv : nullptr, ctx->mlp_state, ctx->ind,
                             (cudaStream_t)stream, ctx->side, ctx->ev_fork, ctx->ev_join, prev, fin, cam_prev));
    return DDGI_OK;
}

ddgi_status restir_initial(ddgi_ctx* ctx, const ddgi_gbuf* gb, const ddgi_reservoirs* out,
                           float* residual, uint32_t frame, void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    GBufView g;
    ResView r;
    ddgi_status s = check_gbuf(ctx, gb, &g);
    if (s != DDGI_OK) return s;
    uint64_t n = (uint64_t)g.width * g.height;
    if ((s = check_res(ctx, out, n, &r)) != DDGI_OK) return s;
    return initial_impl(ctx, g, r, residual, frame, stream, nullptr, nullptr, make_float3(0.f, 0.f, 0.f));
}

ddgi_status restir_initial_temporal(ddgi_ctx* ctx, const ddgi_gbuf* gb, const float* prev_cam_pos,
                                    const ddgi_reservoirs* scratch, const ddgi_reservoirs* prev,
                                    const ddgi_reservoirs* out, float* residual, uint32_t frame, void* stream) {
    if (!ctx || !prev_cam_pos) return fail(ctx, DDGI_ERR_INVALID_ARG, "NULL argument");
    GBufView g;
    ResView rs, rpv, ro;
    ddgi_status s;
    if ((s = check_gbuf(ctx, gb, &g)) != DDGI_OK) return s;
    uint64_t n = (uint64_t)g.width * g.height;
    if ((s = check_res(ctx, scratch, n, &rs)) != DDGI_OK) return s;
    if ((s = check_res(ctx, prev, UINT64_MAX, &rpv)) != DDGI_OK) return s;
    if ((s = check_res(ctx, out, n, &ro)) != DDGI_OK) return s;
    if (n > 0 && (ro.rec == rs.rec || ro.rec == rpv.rec || rs.rec == rpv.rec))
        return fail(ctx, DDGI_ERR_INVALID_ARG, "reservoir buffers alias");
    if (!finite3(prev_cam_pos)) return fail(ctx, DDGI_ERR_INVALID_ARG, "camera position not finite");
    return initial_impl(ctx, g, rs, residual, frame, stream, &rpv, &ro,
                        make_float3(prev_cam_pos[0], prev_cam_pos[1], prev_cam_pos[2]));
}

ddgi_status restir_temporal(ddgi_ctx* ctx, const ddgi_gbuf* gb, const float* prev_cam_pos,
                            const ddgi_reservoirs* cur, const ddgi_reservoirs* prev,
                            const ddgi_reservoirs* out, uint32_t frame, void* stream) {
    if (!ctx || !prev_cam_pos) return fail(ctx, DDGI_ERR_INVALID_ARG, "NULL argument");
    GBufView g;
    ResView rc, rpv, ro;
    ddgi_status s;
    if ((s = check_gbuf(ctx, gb, &g)) != DDGI_OK) return s;
    uint64_t n = (uint64_t)g.width * g.height;
    if ((s = check_res(ctx, cur, n, &rc)) != DDGI_OK) return s;
    if ((s = check_res(ctx, prev, UINT64_MAX, &rpv)) != DDGI_OK) return s;
    if ((s = check_res(ctx, out, n, &ro)) != DDGI_OK) return s;
    if (n > 0 && (ro.rec == rc.rec || ro.rec == rpv.rec))
        return fail(ctx, DDGI_ERR_INVALID_ARG, "output reservoirs alias an input");
    if (!finite3(prev_cam_pos)) return fail(ctx, DDGI_ERR_INVALID_ARG, "camera position not finite");
    CK(launch_restir_temporal(scene_view(ctx), restir_params(ctx), g,
                              make_float3(prev_cam_pos[0], prev_cam_pos[1], prev_cam_pos[2]), rc, rpv,
                              ro, frame, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status restir_spatial(ddgi_ctx* ctx, const ddgi_gbuf* gb, const ddgi_reservoirs* in,
                           const ddgi_reservoirs* out, uint32_t frame, uint32_t pass,
                           void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    GBufView g;
    ResView ri, ro;
    ddgi_status s;
    if ((s = check_gbuf(ctx, gb, &g)) != DDGI_OK) return s;
    uint64_t n = (uint64_t)g.width * g.height;
    if ((s = check_res(ctx, in, n, &ri)) != DDGI_OK) return s;
    if ((s = check_res(ctx, out, n, &ro)) != DDGI_OK) return s;
    if (n > 0 && ro.rec == ri.rec)
        return fail(ctx, DDGI_ERR_INVALID_ARG, "output reservoirs alias the input");
    if (pass > 3) return fail(ctx, DDGI_ERR_INVALID_ARG, "spatial pass index must be 0..3");
    CK(launch_restir_spatial(scene_view(ctx), restir_params(ctx), g, ri, ro, frame, pass,
                             (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_reservoirs_attach_normals(ddgi_ctx* ctx, const ddgi_reservoirs* r, void* stream) {
    if (!ctx || !r) return DDGI_ERR_INVALID_ARG;
    ResView v;
    ddgi_status s;
    if ((s = check_res(ctx, r, r->num_pixels, &v)) != DDGI_OK) return s;
    CK(launch_attach_normals(scene_view(ctx), v, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_shade(ddgi_ctx* ctx, const ddgi_gbuf* gb, const ddgi_reservoirs* res,
                       const float* residual, float* radiance, uint32_t frame, void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    GBufView g;
    ResView r;
    ddgi_status s;
    if ((s = check_gbuf(ctx, gb, &g)) != DDGI_OK) return s;
    uint64_t n = (uint64_t)g.width * g.height;
    if ((s = check_res(ctx, res, n, &r)) != DDGI_OK) return s;
    if (n > 0 && (!residual || !radiance || !aligned(residual, 16) || !aligned(radiance, 16)))
        return fail(ctx, DDGI_ERR_INVALID_ARG, "residual / radiance NULL or misaligned");
    CK(ensure_hits(ctx, (size_t)n, (cudaStream_t)stream));
    MLPView mv = mlp_view(ctx);
    if (ctx->cfg.learned_target) CK(grow(ctx, &ctx->ind, &ctx->ind_cap, (size_t)n, (cudaStream_t)stream));
    ShadeParams sp;
    sp.seed = ctx->cfg.seed;
    sp.frame = frame;
    sp.footprint_c = ctx->cfg.footprint_c == 0.f ? 0.2f : ctx->cfg.footprint_c;   // the paper's c by default
    if (ctx->spec && n > 0 && !(std::isfinite(gb->eye[0]) && std::isfinite(gb->eye[1]) && std::isfinite(gb->eye[2])))
        return fail(ctx, DDGI_ERR_INVALID_ARG, "gbuffer eye not finite");
    CK(launch_shade(scene_view(ctx), volume_view(ctx), g, r, reinterpret_cast<const float4*>(residual),
                    reinterpret_cast<float4*>(radiance), ctx->hits, ctx->counter,
                    ctx->cfg.learned_target ? &mv : nullptr, ctx->mlp_state, ctx->ind, sp, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_reference_accumulate(ddgi_ctx* ctx, const ddgi_camera* cam, uint32_t sample0, uint32_t spp,
                                      double* accum, float* mean, void* stream) {
    if (!ctx || !cam) return DDGI_ERR_INVALID_ARG;
    uint64_t n = (uint64_t)cam->width * cam->height;
    if (n > kMaxPixels || (n > 0 && !accum) || !aligned(accum, 16) || (mean && !aligned(mean, 16)))
        return fail(ctx, DDGI_ERR_INVALID_ARG, "accum / mean NULL, misaligned or too large");
    if (!(cam->tan_half_fovy > 0.f)) return fail(ctx, DDGI_ERR_INVALID_ARG, "field of view must be > 0");
    CK(launch_reference(scene_view(ctx), cam_view(cam), ctx->cfg.seed, sample0, spp, 64, accum,
                        reinterpret_cast<float4*>(mean), (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_mlp_train(ddgi_ctx* ctx, uint32_t frame, void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    if (ctx->cfg.train_samples == 0) return fail(ctx, DDGI_ERR_INVALID_ARG, "train_samples is 0");
    TrainParams tp;
    frame_rotation(ctx->cfg.seed, frame, tp.R, PASS_TRAIN_ROT);
    tp.sf = ctx->train_sf;
    tp.per = ctx->train_per;
    tp.samples = ctx->cfg.train_samples;
    tp.seed = ctx->cfg.seed;
    tp.frame = frame;
    CK(launch_mlp_train_frame(scene_view(ctx), volume_view(ctx), mlp_view(ctx, false), mlp_view(ctx, true), tp,
                              ctx->train_smp, ctx->hits, ctx->counter, ctx->mlp_state, ctx->mlp_params,
                              ctx->mlp_grad, ctx->mlp_m, ctx->mlp_v, ctx->mlp_w16, ctx->mlp_ema, ctx->mlp_w16s,
                              ctx->cfg.train_ema, ctx->cfg.train_lr, ctx->mlp_step + 1, ctx->serve,
                              (cudaStream_t)stream));
    ctx->mlp_step += (ctx->cfg.train_samples + MLP_BATCH - 1) / MLP_BATCH;
    return DDGI_OK;
}

ddgi_status ddgi_mlp_infer(ddgi_ctx* ctx, const float* queries, float* out, uint32_t n, void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    if (n > 0 && (!queries || !out || !aligned(queries, 16) || !aligned(out, 16)))
        return fail(ctx, DDGI_ERR_INVALID_ARG, "queries / out NULL or misaligned");
    CK(launch_mlp_infer_buffer(mlp_view(ctx), queries, out, n, (cudaStream_t)stream));
    return DDGI_OK;
}

static ddgi_status stage_samples(ddgi_ctx* ctx, const float* samples, uint32_t n, cudaStream_t st) {
    if (n == 0 || !samples) return fail(ctx, DDGI_ERR_INVALID_ARG, "no samples");
    CK(grow(ctx, &ctx->tmp_smp, &ctx->tmp_cap, 3ull * n, st));
    CK(cudaMemcpyAsync(ctx->tmp_smp, samples, 3ull * n * sizeof(float4), cudaMemcpyDefault, st));
    return DDGI_OK;
}

ddgi_status ddgi_mlp_grad(ddgi_ctx* ctx, const float* samples, uint32_t n, float* grad, void* stream) {
    if (!ctx || !grad) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ddgi_status s = stage_samples(ctx, samples, n, st);
    if (s != DDGI_OK) return s;
    CK(launch_mlp_grad_only(mlp_view(ctx, false), ctx->tmp_smp, n, ctx->mlp_state, ctx->tmp_grad, st));
    CK(cudaMemcpyAsync(grad, ctx->tmp_grad, MLP_NPARAM * sizeof(float), cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    return DDGI_OK;
}

ddgi_status ddgi_mlp_step(ddgi_ctx* ctx, const float* samples, uint32_t n, void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ddgi_status s = stage_samples(ctx, samples, n, st);
    if (s != DDGI_OK) return s;
    CK(launch_mlp_step(mlp_view(ctx, false), ctx->tmp_smp, n, ctx->mlp_state, ctx->mlp_params, ctx->mlp_grad,
                       ctx->mlp_m, ctx->mlp_v, ctx->mlp_w16, ctx->cfg.train_lr > 0.f ? ctx->cfg.train_lr : 1e-3f,
                       ++ctx->mlp_step, st));
    return DDGI_OK;
}

ddgi_status ddgi_mlp_params_get(ddgi_ctx* ctx, float* params, void* stream) {
    if (!ctx || !params) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(params, ctx->mlp_params, MLP_NPARAM * sizeof(float), cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    return DDGI_OK;
}

ddgi_status ddgi_mlp_params_served_get(ddgi_ctx* ctx, float* params, void* stream) {
    if (!ctx || !params) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(params, ctx->mlp_ema, MLP_NPARAM * sizeof(float), cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    return DDGI_OK;
}

ddgi_status ddgi_mlp_params_set(ddgi_ctx* ctx, const float* params, void* stream) {
    if (!ctx || !params) return DDGI_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    std::vector<float> h(MLP_NPARAM);
    CK(cudaMemcpy(h.data(), params, MLP_NPARAM * sizeof(float), cudaMemcpyDefault));
    for (float v : h)
        if (!std::isfinite(v)) return fail(ctx, DDGI_ERR_INVALID_ARG, "non-finite parameter");
    CK(mlp_upload(ctx, h.data()));
    return DDGI_OK;
}

ddgi_status ddgi_mlp_serve(ddgi_ctx* ctx, int32_t mode, void* stream) {
    if (!ctx || mode < 0 || mode > 2) return DDGI_ERR_INVALID_ARG;
    ctx->serve = mode;
    CK(launch_mlp_serve(ctx->mlp_state, mode, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_mlp_samples_get(ddgi_ctx* ctx, float* out, void* stream) {
    if (!ctx || !out || ctx->cfg.train_samples == 0) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(out, ctx->train_smp, 3ull * ctx->cfg.train_samples * sizeof(float4), cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    return DDGI_OK;
}

ddgi_status ddgi_mlp_status(ddgi_ctx* ctx, double* out, void* stream) {
    if (!ctx || !out) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    MLPState h;
    CK(cudaMemcpyAsync(&h, ctx->mlp_state, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out[0] = h.loss_scale;
    out[1] = h.overflow;
    out[2] = h.count;
    out[3] = h.judge_mlp;
    out[4] = h.judge_probe;
    out[5] = h.judge_n;
    out[6] = h.use_mlp;
    out[7] = ctx->mlp_step;
    return DDGI_OK;
}

ddgi_status ddgi_get_status(ddgi_ctx* ctx, void* stream) {
    if (!ctx) return DDGI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t w[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(w, ctx->err, sizeof(w), cudaMemcpyDeviceToHost, st));
    CK(cudaMemsetAsync(ctx->err, 0, sizeof(w), st));
    CK(cudaStreamSynchronize(st));
    if ((w[0] & ERRBIT_MMA_WAIT) || ctx->wait_failed) {
        // fatal: tensor memory may have been freed under a running product
        ctx->wait_failed = true;
        ctx->last_error = "tensor-core completion wait ran past its bound";
        return DDGI_ERR_DEVICE_WAIT;
    }
    if (w[0] & (ERRBIT_TRAVERSAL | ERRBIT_STACK)) {
        ctx->last_error = (w[0] & ERRBIT_STACK) ? "traversal stack overflow" : "traversal visit limit";
        return DDGI_ERR_TRAVERSAL_LIMIT;
    }
    return DDGI_OK;
}

const char* ddgi_last_error(ddgi_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "NULL context"; }

}  // extern "C"
