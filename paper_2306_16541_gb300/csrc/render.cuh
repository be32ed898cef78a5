// render.cuh -- launch parameters and helpers shared by the rendering,
// tensor-core and training translation units.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace nr {

constexpr int kModeRender = 0;   // input float4 (x, y, z, delta), output float4 (r, g, b, alpha)
constexpr int kModeQuery = 1;    // input float3 points, output NR_QUERY_STRIDE floats per point
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

__global__ void march_kernel(CamParams cam, MarchParams mp, float4 *__restrict__ samp, uint2 *__restrict__ ray_range,
                             uint32_t *__restrict__ counter);
__global__ void composite_kernel(const uint2 *__restrict__ ray_range, const float4 *__restrict__ so, uint32_t n_rays,
                                 float t_min, float bg0, float bg1, float bg2, float4 *__restrict__ out);

CamParams cam_params(const nr_camera *c);
int num_sms(int device);
nr_status launch_field(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                       const uint32_t *n_dev, float *out, int device, cudaStream_t st);
nr_status launch_field_tc(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                          const uint32_t *n_dev, float *out, int device, cudaStream_t st);
nr_status fold_frame_biases(nr_subject *s, cudaStream_t st);

}  // namespace nr
