// Internal host-side declarations shared by the C-ABI layer and the kernel
// translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ddgi.h"
#include "bvh.h"
#include "common.cuh"

// ---------------------------------------------------------------------------
// per-launch parameter blocks
// ---------------------------------------------------------------------------
struct GBufView {
    float4* g0;
    float4* g1;
    float4* g2;
    int width, height;
    float3 eye;   // camera position (the pixel footprint of glossy shading)
};

// shading parameters of glossy scenes (Sec. 3.3 recursion)
struct ShadeParams {
    uint32_t seed, frame;
    float footprint_c;   // < 0: never recurse
};

// reservoir records: 4 float4 per pixel (see ddgi_reservoirs)
struct ResView {
    float4* rec;
    uint32_t n;   // number of records
};

struct CamView {
    float3 pos, fwd, right, up;
    float tan_half_fovy;
    int width, height;
};

struct RestirParams {
    uint32_t seed;
    uint32_t n_light, n_bsdf;
    float temporal_mcap;
    uint32_t spatial_neighbours, spatial_radius;
    float normal_reject_cos, depth_reject_frac;
    uint32_t span_magic;   // ceil(2^32 / (2 radius + 1)): x / span = mulhi(x, magic) for x < 2^16
    uint32_t stride;       // candidate subsampling: 1 every pixel, n: (x + y + frame) % n == 0
};

struct ProbeParams {
    const float4* sf;    // spherical Fibonacci directions, [rays]
    const uint32_t* order;   // ray traced by each thread of a probe: directions of a warp lie together
    uint32_t rays;
    float R[9];          // per-frame rotation of the ray set
    float hysteresis;    // effective (0 on the first update)
    float le_attenuation;
    float depth_sharpness;
    float depth_tmax;
    uint32_t seed, frame;   // keys of the glossy samples at the rays' hits
};

// kernel launchers (return the launch error)
cudaError_t launch_probe_trace(const SceneView& s, const VolumeView& v, const ProbeParams& p,
                               float4* rays, float2* hits, uint32_t* counter, cudaStream_t st);
cudaError_t launch_instance_update(const float4* obj, const uint4* map, uint32_t n, const float4* xf, float4* tris,
                                   float4* nrm, float4* nodes, const uint32_t* refit_list, const float* refit_static,
                                   const int32_t* tri_inst, const std::vector<uint32_t>& level_offsets,
                                   cudaStream_t st);
cudaError_t launch_emitter_radiance(const float* le, const uint32_t* etri, float4* emi, float4* evert,
                                    float4* evert3, uint32_t E, cudaStream_t st);
cudaError_t launch_probe_relocate(const VolumeView& v, const ProbeParams& p, const float4* rays, float4* offset,
                                  cudaStream_t st);
size_t probe_blend_smem(const VolumeView& v, uint32_t rays);
// floats of the blend's per-frame weight tables (ray-major weights of every
// texel, then each texel's weight sum)
size_t probe_blend_weights_size(const VolumeView& v, uint32_t rays);
cudaError_t launch_probe_blend(const VolumeView& v, const ProbeParams& p, const float4* rays, float* weights,
                               cudaStream_t st);
// rebuilds the query's 2x2 tap blocks from the padded maps (after the maps
// were written other than by launch_probe_blend, which keeps them current)
cudaError_t launch_probe_quads(const VolumeView& v, cudaStream_t st);
cudaError_t launch_gbuffer(const SceneView& s, const CamView& cam, const CamView* prev,
                           const GBufView& g, float2* hits, uint32_t* counter, cudaStream_t st);
cudaError_t launch_restir_initial(const SceneView& s, const VolumeView& v, const RestirParams& rp,
                                  const GBufView& g, const ResView& out, float4* resid,
                                  uint32_t frame, float2* hits, uint32_t* counter, const struct MLPView* mlp,
                                  struct MLPState* mst, float4* ind, cudaStream_t st, cudaStream_t side,
                                  cudaEvent_t ev_fork, cudaEvent_t ev_join, const ResView* fuse_prev = nullptr,
                                  const ResView* fuse_out = nullptr, float3 cam_prev = float3{0.f, 0.f, 0.f});
cudaError_t launch_restir_temporal(const SceneView& s, const RestirParams& rp, const GBufView& g,
                                   float3 prev_cam, const ResView& cur,
                                   const ResView& prev, const ResView& out, uint32_t frame,
                                   cudaStream_t st);
cudaError_t launch_restir_spatial(const SceneView& s, const RestirParams& rp, const GBufView& g,
                                  const ResView& in, const ResView& out, uint32_t frame,
                                  uint32_t pass, cudaStream_t st);
cudaError_t launch_attach_normals(const SceneView& s, const ResView& r, cudaStream_t st);
// learned target form (mlp.cu)
#include "mlp.cuh"
#define PASS_TRAIN_ROT 9u
#define PASS_TRAIN_BOUNCE 10u
struct TrainParams {
    float R[9];           // per-frame rotation of the training ray set
    const float4* sf;     // spherical Fibonacci directions, [per]
    uint32_t per;         // training rays per probe
    uint32_t samples;     // probes * per
    uint32_t seed, frame;
};
cudaError_t launch_mlp_infer_buffer(const MLPView& m, const float* queries, float* out, uint32_t n,
                                    cudaStream_t st);
// m: the trained network (master weights), ms: the served network (moving
// average, blended with weight ema_a on the old average after the steps)
cudaError_t launch_mlp_train_frame(const SceneView& s, const VolumeView& v, const MLPView& m, const MLPView& ms,
                                   const TrainParams& tp, float4* smp, float2* hits, uint32_t* counter,
                                   MLPState* state, float* params, float* grad, float* mom, float* vel, uint16_t* w16,
                                   float* ema, uint16_t* w16s, float ema_a, float lr, uint32_t step, int serve,
                                   cudaStream_t st);
cudaError_t launch_mlp_serve(MLPState* state, int serve, cudaStream_t st);
cudaError_t launch_mlp_grad_only(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* out,
                                 cudaStream_t st);
cudaError_t launch_mlp_step(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* params,
                            float* grad, float* mom, float* vel, uint16_t* w16, float lr, uint32_t step,
                            cudaStream_t st);
cudaError_t launch_mlp_grad(const MLPView& m, const float4* smp, uint32_t n, MLPState* state, float* grad,
                            cudaStream_t st);
cudaError_t launch_mlp_adam(float* params, float* grad2, float* mom, float* vel, uint16_t* w16, int bf16,
                            MLPState* state, float lr, uint32_t step, cudaStream_t st, float* ema, uint16_t* w16s,
                            float ema_a);

cudaError_t launch_reference(const SceneView& s, const CamView& cam, uint32_t seed, uint32_t sample0,
                             uint32_t spp, uint32_t max_depth, double* accum, float4* mean, cudaStream_t st);

// image metrics: per-block fp64 partials in `scratch` (2 doubles per block)
constexpr uint32_t kMetricMaxBlocks = 1024;
uint32_t metric_blocks(uint32_t n);
cudaError_t launch_metrics(const float4* img, const float4* ref, uint32_t n, double* scratch,
                           double* out, cudaStream_t st);

cudaError_t launch_shade(const SceneView& s, const VolumeView& v, const GBufView& g,
                         const ResView& r, const float4* resid, float4* radiance, float2* hits,
                         uint32_t* counter, const struct MLPView* mlp, struct MLPState* mst, float4* ind,
                         const ShadeParams& sp, cudaStream_t st);
