// render.cuh -- launch parameters and helpers shared by the rendering,
// tensor-core and training translation units.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace nr {

constexpr int kModeRender = 0;   // input float4 (x, y, z, delta), output float4 (r, g, b, alpha)
constexpr int kModeQuery = 1;    // input float3 points, output NR_QUERY_STRIDE floats per point
constexpr int kModeDensity = 2;  // canonical cell centres: bit = sigma > occ_tau (FP32 tier only)
constexpr int kModePose = 3;     // posed cell centres: bit = canonical cell of x_final set (FP32 tier only)
constexpr int kCounters = 16;    // device counters per subject: live samples of each ray chunk

struct CamParams {
  float R[9], t[3];
  float fx, fy, cx, cy, t_near, t_far;
  uint32_t width, height, n_samples;
};

struct MarchParams {
  float bmin[3], bmax[3];
  int grid;
  const uint32_t *bits;          // posed occupancy bitfield, or NULL to keep every sample
  uint32_t ray0, ray_end;        // rays of this chunk
};

// Slab clip of the ray o + t d against [bmin, bmax] starting from
// [t_near, t_far], in explicitly rounded float32 (see render.cu).
__device__ __forceinline__ bool clip_box(const float o[3], const float d[3], const float bmin[3], const float bmax[3],
                                         float t_near, float t_far, float &lo, float &hi) {
  lo = t_near;
  hi = t_far;
  bool miss = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (d[k] == 0.f) {
      miss |= (o[k] < bmin[k]) || (o[k] > bmax[k]);
    } else {
      const float ta = __fdiv_rn(__fsub_rn(bmin[k], o[k]), d[k]);
      const float tb = __fdiv_rn(__fsub_rn(bmax[k], o[k]), d[k]);
      lo = fmaxf(lo, fminf(ta, tb));
      hi = fminf(hi, fmaxf(ta, tb));
    }
  }
  return !miss && lo < hi;
}

// --------------------------------------------------------------- ray setup
// Ray of pixel (u, v), clipped to [t_near, t_far] and the box (Sec. 4.4:
// samples lie inside the performer's bounding box).  Every operation is an
// explicitly rounded float32 operation (no FMA contraction): which rays hit
// the box and which cell a sample falls in are integer decisions, and they
// must come out the same on every platform.  Evaluation order:
//   o_k = -(((R0k t0) + (R1k t1)) + (R2k t2))
//   a = ((u + 0.5) - cx) / fx, b = ((v + 0.5) - cy) / fy
//   w_k = ((R0k a) + (R1k b)) + R2k,  n = sqrt(((w0 w0) + (w1 w1)) + (w2 w2)),  d_k = w_k / n
//   per axis with d_k != 0: ta = (bmin_k - o_k) / d_k, tb = (bmax_k - o_k) / d_k,
//     lo = max(lo, min(ta, tb)), hi = min(hi, max(ta, tb)); an axis with d_k == 0
//     misses when o_k lies outside its slab.
__device__ __forceinline__ void camera_origin(const CamParams &c, float o[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k)
    o[k] = -__fadd_rn(__fadd_rn(__fmul_rn(c.R[k], c.t[0]), __fmul_rn(c.R[3 + k], c.t[1])), __fmul_rn(c.R[6 + k], c.t[2]));
}

__device__ __forceinline__ bool ray_setup(const CamParams &c, const float o[3], const float bmin[3], const float bmax[3],
                                          uint32_t u, uint32_t v, float d[3], float &lo, float &hi) {
  const float a = __fdiv_rn(__fsub_rn(__fadd_rn((float)u, 0.5f), c.cx), c.fx);
  const float b = __fdiv_rn(__fsub_rn(__fadd_rn((float)v, 0.5f), c.cy), c.fy);
  float w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) w[k] = __fadd_rn(__fadd_rn(__fmul_rn(c.R[k], a), __fmul_rn(c.R[3 + k], b)), c.R[6 + k]);
  const float n = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(w[0], w[0]), __fmul_rn(w[1], w[1])), __fmul_rn(w[2], w[2])));
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = __fdiv_rn(w[k], n);
  return clip_box(o, d, bmin, bmax, c.t_near, c.t_far, lo, hi);
}

__global__ void march_kernel(CamParams cam, MarchParams mp, float4 *__restrict__ samp, uint2 *__restrict__ ray_range,
                             uint32_t *__restrict__ counter);
__global__ void composite_kernel(const uint2 *__restrict__ ray_range, const float4 *__restrict__ so, uint32_t n_rays,
                                 float t_min, float bg0, float bg1, float bg2, float4 *__restrict__ out);

// Explicit work buffers of one frame render (the serving loop gives each request its own).
struct FrameWork {
  float4 *samp, *samp_out;        // [cap_samples]
  uint2 *ray_range;               // [cap_rays]
  uint32_t *counter;              // [1] live samples of the current round
  uint32_t *total;                // [2] live samples over the frame (profiling), or NULL
  float4 *state;                  // [cap_rays] running (C, T) for round-based early termination
  uint32_t *next;                 // [cap_rays] next slot / retired flag
  size_t cap_samples, cap_rays;
};

// Start/end CUDA-event pairs recorded around each launch of a profiled render.
struct Prof {
  cudaEvent_t *ev;                // [cap] events, one per launch boundary
  int *stage;                     // [cap] the stage ending at each: 0 march, 1 field, 2 composite, -1 none
  int cap, used;
  bool overflow;
};

uint32_t round_samples(const nr_camera *cam, const nr_render_opts *opts);
nr_status render_rays(const nr_subject *s, const FieldParams &P, const uint32_t *bits, const nr_camera *cam,
                      const nr_render_opts *opts, const FrameWork &w, float4 *dst, cudaStream_t st, int mma_path,
                      Prof *prof);
// Renders `cam` for the pose whose transforms / folded bias are in P (P.G, P.bias1) and whose posed
// occupancy bitfield is `bits` into the device buffer dst[height * width], in ray chunks that fit w.
nr_status render_frame(const nr_subject *s, const FieldParams &P, const uint32_t *bits, const nr_camera *cam,
                       const nr_render_opts *opts, const FrameWork &w, float4 *dst, cudaStream_t st);

CamParams cam_params(const nr_camera *c);
int render_path(const nr_render_opts *o);                     // the launch_field path the options select
bool path_uses_tcgen05(const nr_render_opts *o, int path);    // needs prepare_t5, sets the error word
nr_status check_field_timeouts(nr_subject *s, cudaStream_t st);   // NR_ETIMEOUT if a bounded wait gave up
int num_sms(int device);
size_t field_f32_smem(const FieldParams &P);
// mma_path for the bf16/f16 tiers: 0 = the warp-specialised tcgen05 pipeline (field_ws.cu), 1 = tcgen05
// with one group per tile and activations through shared memory (field_t5.cu), 2 = warp-level mma.sync
// over two m-tiles per weight read (12 warps/SM), 4 = warp-level mma.sync over one 16-row m-tile per
// weight-fragment read (20 warps/SM, field_tc.cu); for the f32 tier: 3 = TF32 tensor-core layers at
// float32 accuracy (field_tf32.cu), else CUDA cores.  Paths 0 and 1 need prepare_t5 first.
nr_status launch_field(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                       const uint32_t *n_dev, float *out, int device, cudaStream_t st, int mma_path = 0);
nr_status launch_field_fp8(const FieldParams &P, int mode, const float4 *in, uint32_t n_fixed, const uint32_t *n_dev,
                           float *out, int device, cudaStream_t st);
nr_status launch_field_t5(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                          const uint32_t *n_dev, float *out, int device, cudaStream_t st);
nr_status launch_field_ws(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                          const uint32_t *n_dev, float *out, int device, cudaStream_t st);
nr_status launch_field_tc(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                          const uint32_t *n_dev, float *out, int device, cudaStream_t st, int mt);
nr_status fold_frame_biases(nr_subject *s, cudaStream_t st);
// the float32 tier on the tensor cores: threads per block and scratch rows per thread
constexpr int kTf32Threads = 512;
constexpr int kTf32Rows = kResGammaPad + 2 * kWidth + kMlpIn + 4;
nr_status launch_field_tf32(const FieldParams &P, int mode, const float4 *in, uint32_t n_fixed, const uint32_t *n_dev,
                            float *out, int device, cudaStream_t st);

}  // namespace nr
