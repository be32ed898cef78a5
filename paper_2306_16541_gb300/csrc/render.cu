// render.cu -- forward rendering: ray generation and compacted ray marching
// through the posed occupancy bitfield, the per-sample field (float32 CUDA
// cores here; tensor-core tiers in field_tc.cu), front-to-back compositing
// with early ray termination, and point queries.
#include <math.h>
#include <string.h>

#include "field.cuh"
#include "render.cuh"

namespace nr {

// ------------------------------------------------------------ ray marching
// One thread per ray.  Pass 1 counts the live samples (midpoint of each of the
// S bins, kept when its occupancy cell is set); a warp-wide prefix sum and one
// atomic per warp reserve a contiguous run of the sample queue; pass 2 writes
// each live sample's position and spacing in ray order.
//   D = (hi - lo) / S,  t_i = lo + ((i + 0.5) D),  x_k = o_k + (t_i d_k)
//   h_k = (bmax_k - bmin_k) / G,  c_k = clamp(floor((x_k - bmin_k) / h_k), 0, G - 1)
__global__ void __launch_bounds__(256) march_kernel(CamParams cam, MarchParams mp, float4 *__restrict__ samp,
                                                    uint2 *__restrict__ ray_range, uint32_t *__restrict__ counter) {
  const uint32_t r = mp.ray0 + blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = r < mp.ray_end;
  const uint32_t lane = threadIdx.x & 31;
  float o[3], d[3], lo = 0.f, hi = 0.f;
  camera_origin(cam, o);
  bool hit = false;
  if (valid) {
    const uint32_t u = r % cam.width, v = r / cam.width;
    hit = ray_setup(cam, o, mp.bmin, mp.bmax, u, v, d, lo, hi);
  }
  const uint32_t S = cam.n_samples;
  const float D = __fdiv_rn(__fsub_rn(hi, lo), (float)S);
  const int G = mp.grid;
  float h[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) h[k] = __fdiv_rn(__fsub_rn(mp.bmax[k], mp.bmin[k]), (float)G);
  auto live = [&](uint32_t i, float x[3]) -> bool {
    const float t = __fadd_rn(lo, __fmul_rn(__fadd_rn((float)i, 0.5f), D));
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = __fadd_rn(o[k], __fmul_rn(t, d[k]));
    if (!mp.bits) return true;
    int c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int ck = (int)floorf(__fdiv_rn(__fsub_rn(x[k], mp.bmin[k]), h[k]));
      c[k] = min(max(ck, 0), G - 1);
    }
    const uint32_t cell = ((uint32_t)c[2] * G + (uint32_t)c[1]) * G + (uint32_t)c[0];
    return (__ldg(mp.bits + (cell >> 5)) >> (cell & 31)) & 1u;
  };
  uint32_t count = 0;
  if (hit) {
    for (uint32_t i = 0; i < S; ++i) {
      float x[3];
      count += live(i, x) ? 1u : 0u;
    }
  }
  // warp-level exclusive scan of counts, one atomic per warp
  uint32_t incl = count;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= (uint32_t)off) incl += y;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  uint32_t base = 0;
  if (lane == 31) base = atomicAdd(counter, total);
  base = __shfl_sync(0xffffffffu, base, 31);
  const uint32_t off = base + incl - count;
  if (valid) ray_range[r - mp.ray0] = make_uint2(off, count);
  if (count) {
    uint32_t w = off;
    for (uint32_t i = 0; i < S; ++i) {
      float x[3];
      if (live(i, x)) samp[w++] = make_float4(x[0], x[1], x[2], D);
    }
  }
}

// ------------------------------------------------------------- field (FP32)
// One thread per sample; both MLPs' weights in shared memory (float32,
// transposed), read as broadcast float4.  Writes (r, g, b, alpha) per sample
// with alpha = (1 - exp(-sigma delta)) * min(S, 1) (Sec. 4.4 likelihood
// augmentation), zero when the canonical point leaves the box.
constexpr int kF32Threads = 192;
constexpr int kF32ColRows = kWidth + kResGammaPad;   // per-thread activation column: h (64) then gamma (48)

template <int MODE>
__global__ void __launch_bounds__(kF32Threads, 1) field_f32_kernel(FieldParams P, const float4 *__restrict__ in,
                                                                   uint32_t n_fixed, const uint32_t *__restrict__ n_dev,
                                                                   float *__restrict__ out) {
  extern __shared__ float4 smem4[];
  float *sW = reinterpret_cast<float *>(smem4);
  float *sG = sW + P.lay.total;
  float *sB1 = sG + kBones * 12;
  float *sCol = sB1 + kWidth;
  for (int i = threadIdx.x; i < P.lay.total / 4; i += blockDim.x)
    reinterpret_cast<float4 *>(sW)[i] = __ldg(reinterpret_cast<const float4 *>(P.blob) + i);
  for (int i = threadIdx.x; i < kBones * 12; i += blockDim.x) sG[i] = P.G[i];
  for (int i = threadIdx.x; i < kWidth; i += blockDim.x) sB1[i] = P.bias1[i];
  __syncthreads();
  const int stride = blockDim.x;
  float *hcol = sCol + threadIdx.x;
  float *gcol = hcol + kWidth * stride;
  const uint32_t n = n_dev ? *n_dev : n_fixed;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    float x0, x1, x2, delta = 0.f;
    if (MODE == kModeRender) {
      const float4 s = in[j];
      x0 = s.x;
      x1 = s.y;
      x2 = s.z;
      delta = s.w;
    } else {
      const float *q = reinterpret_cast<const float *>(in) + 3 * (size_t)j;
      x0 = q[0];
      x1 = q[1];
      x2 = q[2];
    }
    float s0, s1, s2, S;
    lbs_warp(P, sG, x0, x1, x2, s0, s1, s2, S);
    float f0 = s0, f1 = s1, f2 = s2;
    if (P.res_enabled) {
      pos_enc(P, s0, s1, s2, gcol, stride);
      float r0, r1, r2;
      residual_f32(P, sW, sB1, gcol, hcol, stride, r0, r1, r2);
      f0 += r0;
      f1 += r1;
      f2 += r2;
    }
    const bool inside = hash_encode(P, f0, f1, f2, hcol, stride);
    float o[4];
    canonical_f32(P, sW, hcol, stride, o);
    const float cr = sigmoidf_(o[0]), cg = sigmoidf_(o[1]), cb = sigmoidf_(o[2]);
    const float sigma = softplusf_(o[3]);
    if (MODE == kModeRender) {
      const float a = inside ? (1.f - __expf(-sigma * delta)) * fminf(S, 1.f) : 0.f;
      reinterpret_cast<float4 *>(out)[j] = make_float4(cr, cg, cb, a);
    } else {
      float *q = out + (size_t)NR_QUERY_STRIDE * j;
      q[0] = s0; q[1] = s1; q[2] = s2; q[3] = S;
      q[4] = f0; q[5] = f1; q[6] = f2; q[7] = inside ? 1.f : 0.f;
      q[8] = cr; q[9] = cg; q[10] = cb; q[11] = sigma;
    }
  }
}

// --------------------------------------------------------------- composite
// Eq. 3 front to back: T_0 = 1, w_i = T_i alpha_i, C += w_i c_i,
// T_{i+1} = T_i (1 - alpha_i); stop once T < t_min (early ray termination,
// Sec. 2.3).  Pixel = (C + T bg, 1 - T).  One thread per ray.
__global__ void __launch_bounds__(256) composite_kernel(const uint2 *__restrict__ ray_range,
                                                        const float4 *__restrict__ so, uint32_t n_rays, float t_min,
                                                        float bg0, float bg1, float bg2, float4 *__restrict__ out) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rays) return;
  const uint2 rr = ray_range[r];
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  for (uint32_t i = 0; i < rr.y; ++i) {
    const float4 v = so[rr.x + i];
    const float w = T * v.w;
    c0 = fmaf(w, v.x, c0);
    c1 = fmaf(w, v.y, c1);
    c2 = fmaf(w, v.z, c2);
    T *= 1.f - v.w;
    if (T < t_min) break;
  }
  out[r] = make_float4(fmaf(T, bg0, c0), fmaf(T, bg1, c1), fmaf(T, bg2, c2), 1.f - T);
}

size_t field_f32_smem(const FieldParams &P) {
  return sizeof(float) * (P.lay.total + kBones * 12 + kWidth + (size_t)kF32ColRows * kF32Threads);
}

int num_sms(int device) {
  static int cached[64] = {0};
  if (device < 0 || device >= 64) return 148;
  if (!cached[device]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    cached[device] = v > 0 ? v : 148;
  }
  return cached[device];
}

nr_status launch_field(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                       const uint32_t *n_dev, float *out, int device, cudaStream_t st, int mma_path) {
  if ((mlp_dtype == NR_BF16 || mlp_dtype == NR_F16) && mma_path == 1)
    return launch_field_t5(P, mlp_dtype, mode, in, n_fixed, n_dev, out, device, st);
  if (mlp_dtype == NR_BF16 || mlp_dtype == NR_F16)
    return launch_field_tc(P, mlp_dtype, mode, in, n_fixed, n_dev, out, device, st, mma_path == 2 ? 2 : 1);
  if (mlp_dtype == NR_FP8E4M3) return launch_field_fp8(P, mode, in, n_fixed, n_dev, out, device, st);
  if (mlp_dtype != NR_F32) {
    set_error("mlp_dtype %d is not implemented", (int)mlp_dtype);
    return NR_EUNSUPPORTED;
  }
  const size_t smem = field_f32_smem(P);
  const int blocks = num_sms(device);
  if (mode == kModeRender) {
    NR_CHECK_CUDA(cudaFuncSetAttribute(field_f32_kernel<kModeRender>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    field_f32_kernel<kModeRender><<<blocks, kF32Threads, smem, st>>>(P, in, n_fixed, n_dev, out);
  } else {
    NR_CHECK_CUDA(cudaFuncSetAttribute(field_f32_kernel<kModeQuery>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    field_f32_kernel<kModeQuery><<<blocks, kF32Threads, smem, st>>>(P, in, n_fixed, n_dev, out);
  }
  NR_CHECK_CUDA(cudaGetLastError());
  return NR_OK;
}

static nr_status check_opts(const nr_render_opts *o) {
  NR_REQUIRE(o, "NULL options");
  NR_REQUIRE(o->mlp_dtype == NR_F32 || o->mlp_dtype == NR_BF16 || o->mlp_dtype == NR_F16 ||
                 o->mlp_dtype == NR_FP8E4M3,
             "unknown mlp_dtype %d", (int)o->mlp_dtype);
  NR_REQUIRE(o->feat_dtype == NR_F32 || o->feat_dtype == NR_F16, "feat_dtype must be NR_F32 or NR_F16");
  NR_REQUIRE(o->t_min >= 0.f && o->t_min < 1.f, "t_min must be in [0, 1)");
  return NR_OK;
}

CamParams cam_params(const nr_camera *c) {
  CamParams p{};
  memcpy(p.R, c->R, sizeof(p.R));
  memcpy(p.t, c->t, sizeof(p.t));
  p.fx = c->fx;
  p.fy = c->fy;
  p.cx = c->cx;
  p.cy = c->cy;
  p.t_near = c->t_near;
  p.t_far = c->t_far;
  p.width = c->width;
  p.height = c->height;
  p.n_samples = c->n_samples;
  return p;
}

nr_status grow_workspace(nr_subject *s, size_t rays, size_t samples) {
  if (rays > s->ws_rays) {
    if (s->ray_range) cudaFree(s->ray_range);
    s->ray_range = nullptr;
    s->ws_rays = 0;
    NR_CHECK_CUDA(cudaMalloc(&s->ray_range, rays * sizeof(uint2)));
    s->ws_rays = rays;
  }
  if (samples > s->ws_samples) {
    if (s->samp) cudaFree(s->samp);
    if (s->samp_out) cudaFree(s->samp_out);
    s->samp = s->samp_out = nullptr;
    s->ws_samples = 0;
    NR_CHECK_CUDA(cudaMalloc(&s->samp, samples * sizeof(float4)));
    NR_CHECK_CUDA(cudaMalloc(&s->samp_out, samples * sizeof(float4)));
    s->ws_samples = samples;
  }
  return NR_OK;
}

nr_status render_frame(const nr_subject *s, const FieldParams &P, const uint32_t *bits, const nr_camera *cam,
                       const nr_render_opts *opts, const FrameWork &w, float4 *dst, cudaStream_t st) {
  const CamParams C = cam_params(cam);
  const uint32_t n_rays = cam->width * cam->height;
  const uint32_t chunk = (uint32_t)std::min<uint64_t>(
      std::min<uint64_t>(n_rays, w.cap_rays), std::max<uint64_t>(1, w.cap_samples / cam->n_samples));
  if (chunk == 0) {
    set_error("render_frame: workspace too small for one ray");
    return NR_EINVAL;
  }
  MarchParams mp{};
  for (int k = 0; k < 3; ++k) {
    mp.bmin[k] = s->bmin[k];
    mp.bmax[k] = s->bmax[k];
  }
  mp.grid = (int)s->occ_grid;
  mp.bits = opts->use_occupancy ? bits : nullptr;
  nr_status r;
  for (uint32_t r0 = 0; r0 < n_rays; r0 += chunk) {
    const uint32_t nr_ = std::min(chunk, n_rays - r0);
    mp.ray0 = r0;
    mp.ray_end = r0 + nr_;
    NR_CHECK_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(uint32_t), st));
    march_kernel<<<(nr_ + 255) / 256, 256, 0, st>>>(C, mp, w.samp, w.ray_range, w.counter);
    NR_CHECK_CUDA(cudaGetLastError());
    if ((r = launch_field(P, opts->mlp_dtype, kModeRender, w.samp, 0, w.counter, (float *)w.samp_out, s->device,
                          st)) != NR_OK)
      return r;
    composite_kernel<<<(nr_ + 255) / 256, 256, 0, st>>>(w.ray_range, w.samp_out, nr_, opts->t_min, cam->bg[0],
                                                        cam->bg[1], cam->bg[2], dst + r0);
    NR_CHECK_CUDA(cudaGetLastError());
    count_launches(3);
  }
  return NR_OK;
}

}  // namespace nr

using namespace nr;

extern "C" nr_status nr_render(nr_subject *s, const nr_camera *cam, const nr_render_opts *opts, float *out_rgba,
                               void *stream) {
  NR_REQUIRE(subject_ok(s), "nr_render: invalid handle");
  NR_REQUIRE(cam && out_rgba, "nr_render: NULL argument");
  nr_status r = check_opts(opts);
  if (r != NR_OK) return r;
  NR_REQUIRE(cam->width >= 1 && cam->height >= 1 && (uint64_t)cam->width * cam->height <= (1ull << 26),
             "nr_render: image size out of range");
  NR_REQUIRE(cam->n_samples >= 1 && cam->n_samples <= 1024, "nr_render: n_samples must be 1..1024");
  NR_REQUIRE(cam->fx != 0.f && cam->fy != 0.f, "nr_render: zero focal length");
  NR_REQUIRE(!opts->use_occupancy || s->has_ellipsoids, "nr_render: occupancy requested but the subject has none");
  if (!s->pose_set) {
    set_error("nr_render: call nr_set_pose first");
    return NR_ESTATE;
  }
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  cudaStream_t st = (cudaStream_t)stream;
  if ((r = prepare_params(s, st)) != NR_OK) return r;
  if ((r = ensure_bias(s, st)) != NR_OK) return r;
  if (opts->mlp_dtype == NR_FP8E4M3 && (r = prepare_fp8(s, st)) != NR_OK) return r;
  const int path = (opts->flags & NR_RENDER_TCGEN05) ? 1 : ((opts->flags & NR_RENDER_MMA2) ? 2 : 0);
  if (path == 1 && (r = prepare_t5(s, st)) != NR_OK) return r;
  const FieldParams P = field_params(s, opts);
  const CamParams C = cam_params(cam);
  const uint32_t n_rays = cam->width * cam->height;
  // chunk the rays so that the worst-case sample queue stays below 2^26 entries
  const uint64_t max_samples = 1ull << 26;
  uint32_t chunk = (uint32_t)std::min<uint64_t>(n_rays, std::max<uint64_t>(256, max_samples / cam->n_samples));
  if ((r = grow_workspace(s, chunk, (size_t)chunk * cam->n_samples)) != NR_OK) return r;
  cudaPointerAttributes attr{};
  const bool dev_out = cudaPointerGetAttributes(&attr, out_rgba) == cudaSuccess && attr.type == cudaMemoryTypeDevice;
  cudaGetLastError();
  float *dst = out_rgba;
  if (!dev_out) {
    if (s->stage_cap < (size_t)n_rays) {
      if (s->out_stage) cudaFree(s->out_stage);
      s->out_stage = nullptr;
      s->stage_cap = 0;
      NR_CHECK_CUDA(cudaMalloc(&s->out_stage, (size_t)n_rays * 16));
      s->stage_cap = n_rays;
    }
    dst = s->out_stage;
  }
  MarchParams mp{};
  for (int k = 0; k < 3; ++k) {
    mp.bmin[k] = s->bmin[k];
    mp.bmax[k] = s->bmax[k];
  }
  mp.grid = (int)s->occ_grid;
  mp.bits = opts->use_occupancy ? s->bits : nullptr;
  const bool prof = (opts->flags & NR_RENDER_PROFILE) != 0;
  const uint32_t n_chunks = (n_rays + chunk - 1) / chunk;
  if (prof) {
    NR_REQUIRE(4 * n_chunks <= (uint32_t)nr_subject::kProfEvents && n_chunks <= (uint32_t)kCounters,
               "nr_render: too many ray chunks to profile");
    for (uint32_t i = 0; i < 4 * n_chunks; ++i)
      if (!s->prof_ev[i]) NR_CHECK_CUDA(cudaEventCreate(&s->prof_ev[i]));
    s->prof_used = 0;
    s->prof_chunks = (int)n_chunks;
  }
  auto mark = [&](int i) -> cudaError_t { return prof ? cudaEventRecord(s->prof_ev[i], st) : cudaSuccess; };
  for (uint32_t ci = 0, r0 = 0; r0 < n_rays; ++ci, r0 += chunk) {
    const uint32_t nr_ = std::min(chunk, n_rays - r0);
    mp.ray0 = r0;
    mp.ray_end = r0 + nr_;
    uint32_t *cnt = s->counter + (ci % kCounters);
    NR_CHECK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t), st));
    NR_CHECK_CUDA(mark(4 * ci));
    march_kernel<<<(nr_ + 255) / 256, 256, 0, st>>>(C, mp, s->samp, s->ray_range, cnt);
    NR_CHECK_CUDA(cudaGetLastError());
    NR_CHECK_CUDA(mark(4 * ci + 1));
    if ((r = launch_field(P, opts->mlp_dtype, kModeRender, s->samp, 0, cnt, (float *)s->samp_out, s->device,
                          st, path)) != NR_OK)
      return r;
    NR_CHECK_CUDA(mark(4 * ci + 2));
    composite_kernel<<<(nr_ + 255) / 256, 256, 0, st>>>(s->ray_range, s->samp_out, nr_, opts->t_min, cam->bg[0],
                                                        cam->bg[1], cam->bg[2],
                                                        reinterpret_cast<float4 *>(dst) + r0);
    NR_CHECK_CUDA(cudaGetLastError());
    NR_CHECK_CUDA(mark(4 * ci + 3));
    count_launches(3);
  }
  if (prof) s->prof_used = 4 * (int)n_chunks;
  if (!dev_out) {
    NR_CHECK_CUDA(cudaMemcpyAsync(out_rgba, dst, (size_t)n_rays * 16, cudaMemcpyDeviceToHost, st));
    NR_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  return NR_OK;
}

extern "C" nr_status nr_stage_times(nr_subject *s, float *ms) {
  NR_REQUIRE(subject_ok(s) && ms, "nr_stage_times: bad argument");
  if (s->prof_used == 0) {
    set_error("nr_stage_times: no profiled render yet");
    return NR_ESTATE;
  }
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  NR_CHECK_CUDA(cudaEventSynchronize(s->prof_ev[s->prof_used - 1]));
  float acc[3] = {0.f, 0.f, 0.f};
  for (int c = 0; c < s->prof_chunks; ++c)
    for (int k = 0; k < 3; ++k) {
      float t = 0.f;
      NR_CHECK_CUDA(cudaEventElapsedTime(&t, s->prof_ev[4 * c + k], s->prof_ev[4 * c + k + 1]));
      acc[k] += t;
    }
  uint32_t live[kCounters];
  const int nc = std::min(s->prof_chunks, kCounters);
  NR_CHECK_CUDA(cudaMemcpy(live, s->counter, sizeof(uint32_t) * nc, cudaMemcpyDeviceToHost));
  double total = 0;
  for (int c = 0; c < nc; ++c) total += live[c];
  ms[0] = acc[0];
  ms[1] = acc[1];
  ms[2] = acc[2];
  ms[3] = (float)s->prof_chunks;
  ms[4] = (float)total;
  return NR_OK;
}

extern "C" nr_status nr_query(nr_subject *s, uint32_t n, const float *x_obs, const nr_render_opts *opts, float *out,
                              void *stream) {
  NR_REQUIRE(subject_ok(s), "nr_query: invalid handle");
  NR_REQUIRE(x_obs && out, "nr_query: NULL argument");
  nr_status r = check_opts(opts);
  if (r != NR_OK) return r;
  if (!s->pose_set) {
    set_error("nr_query: call nr_set_pose first");
    return NR_ESTATE;
  }
  if (n == 0) return NR_OK;
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  cudaStream_t st = (cudaStream_t)stream;
  if ((r = prepare_params(s, st)) != NR_OK) return r;
  if ((r = ensure_bias(s, st)) != NR_OK) return r;
  if (opts->mlp_dtype == NR_FP8E4M3 && (r = prepare_fp8(s, st)) != NR_OK) return r;
  const int path = (opts->flags & NR_RENDER_TCGEN05) ? 1 : ((opts->flags & NR_RENDER_MMA2) ? 2 : 0);
  if (path == 1 && (r = prepare_t5(s, st)) != NR_OK) return r;
  const FieldParams P = field_params(s, opts);
  count_launches(1);
  return launch_field(P, opts->mlp_dtype, kModeQuery, reinterpret_cast<const float4 *>(x_obs), n, nullptr, out,
                      s->device, st, path);
}
