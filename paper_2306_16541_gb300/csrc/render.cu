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
//
// Two more modes build occupancy bitfields from the field itself (empty-space
// skipping for subjects without ellipsoids, Sec. 2.3), one thread per cell of
// an occ_grid^3 grid over the box, cell centre y_k = bmin_k + ((j_k + 0.5) h_k):
//   kModeDensity: y is canonical; bit = softplus(o_3(enc(y))) > occ_tau.
//   kModePose:    y is observed; bit = S(y) >= occ_smin and canon_bits holds the
//                 canonical cell clamp(floor((x_final(y) - bmin) / h), 0, G - 1)
//                 (x_final: Eq. lbs then MLP_res, as for a sample).  The clamp
//                 keeps a cell whose centre maps just outside the box while
//                 other points of the cell map inside.
// Cells are word-aligned per warp (occ_grid^3 is a multiple of 32 and so are
// the block and the grid stride), so a warp ballot writes whole words.
constexpr int kF32Threads = 192;
constexpr int kF32ColRows = kWidth + kResGammaPad;   // per-thread activation column: h (64) then gamma (48)

template <int MODE>
__global__ void __launch_bounds__(kF32Threads, 1) field_f32_kernel(FieldParams P, const float4 *__restrict__ in,
                                                                   uint32_t n_fixed, const uint32_t *__restrict__ n_dev,
                                                                   float *__restrict__ out) {
  extern __shared__ float4 smem4[];
  float *sW = reinterpret_cast<float *>(smem4);
  float *sG = sW + P.lay.total;
  float *sB1 = sG + kPoseSmem;
  float *sCol = sB1 + kWidth;
  for (int i = threadIdx.x; i < P.lay.total / 4; i += blockDim.x)
    reinterpret_cast<float4 *>(sW)[i] = __ldg(reinterpret_cast<const float4 *>(P.blob) + i);
  const float *sBox = stage_pose(P, sG, threadIdx.x, blockDim.x);
  for (int i = threadIdx.x; i < kWidth; i += blockDim.x) sB1[i] = P.bias1[i];
  __syncthreads();
  const int stride = blockDim.x;
  float *hcol = sCol + threadIdx.x;
  float *gcol = hcol + kWidth * stride;
  constexpr bool kCells = MODE == kModeDensity || MODE == kModePose;
  float h[3] = {0.f, 0.f, 0.f};
  if (kCells) {
#pragma unroll
    for (int k = 0; k < 3; ++k) h[k] = __fdiv_rn(__fsub_rn(P.bmax[k], P.bmin[k]), (float)P.occ_grid);
  }
  const uint32_t n = kCells ? (uint32_t)P.occ_grid * P.occ_grid * P.occ_grid : (n_dev ? *n_dev : n_fixed);
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    float x0, x1, x2, delta = 0.f;
    if (MODE == kModeRender) {
      const float4 s = in[j];
      x0 = s.x;
      x1 = s.y;
      x2 = s.z;
      delta = s.w;
    } else if (MODE == kModeQuery) {
      const float *q = reinterpret_cast<const float *>(in) + 3 * (size_t)j;
      x0 = q[0];
      x1 = q[1];
      x2 = q[2];
    } else {
      const uint32_t g = (uint32_t)P.occ_grid;
      x0 = __fadd_rn(P.bmin[0], __fmul_rn(__fadd_rn((float)(j % g), 0.5f), h[0]));
      x1 = __fadd_rn(P.bmin[1], __fmul_rn(__fadd_rn((float)((j / g) % g), 0.5f), h[1]));
      x2 = __fadd_rn(P.bmin[2], __fmul_rn(__fadd_rn((float)(j / (g * g)), 0.5f), h[2]));
    }
    if (MODE == kModeDensity) {
      hash_encode(P, x0, x1, x2, hcol, stride);
      float o[4];
      canonical_f32(P, sW, hcol, stride, o);
      const unsigned word = __ballot_sync(0xffffffffu, softplusf_(o[3]) > P.occ_tau);
      if ((threadIdx.x & 31) == 0) reinterpret_cast<uint32_t *>(out)[j >> 5] = word;
      continue;
    }
    float s0, s1, s2, S;
    lbs_warp(P, sG, x0, x1, x2, s0, s1, s2, S, sBox);
    float f0 = s0, f1 = s1, f2 = s2;
    if (MODE == kModePose) {
      bool occ = false;
      if (S >= P.occ_smin) {
        if (P.res_enabled) {
          pos_enc(P, s0, s1, s2, gcol, stride);
          float r0, r1, r2;
          residual_f32(P, sW, sB1, gcol, hcol, stride, r0, r1, r2);
          f0 += r0;
          f1 += r1;
          f2 += r2;
        }
        // clamped to the grid as floats before the conversion (fmaxf maps NaN to 0)
        const float top = (float)(P.occ_grid - 1);
        const float c0 = fminf(fmaxf(floorf(__fdiv_rn(__fsub_rn(f0, P.bmin[0]), h[0])), 0.f), top);
        const float c1 = fminf(fmaxf(floorf(__fdiv_rn(__fsub_rn(f1, P.bmin[1]), h[1])), 0.f), top);
        const float c2 = fminf(fmaxf(floorf(__fdiv_rn(__fsub_rn(f2, P.bmin[2]), h[2])), 0.f), top);
        const uint32_t g = (uint32_t)P.occ_grid;
        const uint32_t cell = ((uint32_t)c2 * g + (uint32_t)c1) * g + (uint32_t)c0;
        occ = (__ldg(P.canon_bits + (cell >> 5)) >> (cell & 31)) & 1u;
      }
      const unsigned word = __ballot_sync(0xffffffffu, occ);
      if ((threadIdx.x & 31) == 0) reinterpret_cast<uint32_t *>(out)[j >> 5] = word;
      continue;
    }
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
      const float a = inside ? -expm1f(-sigma * delta) * fminf(S, 1.f) : 0.f;
      reinterpret_cast<float4 *>(out)[j] = make_float4(cr, cg, cb, a);
    } else {
      float *q = out + (size_t)NR_QUERY_STRIDE * j;
      q[0] = s0; q[1] = s1; q[2] = s2; q[3] = S;
      q[4] = f0; q[5] = f1; q[6] = f2; q[7] = inside ? 1.f : 0.f;
      q[8] = cr; q[9] = cg; q[10] = cb; q[11] = sigma;
    }
  }
}

// Launches the FP32 kernel in kModeDensity or kModePose over P.occ_grid^3 cells,
// writing occ_grid^3 / 32 words to bits.
nr_status launch_occupancy_field(const FieldParams &P, int mode, uint32_t *bits, int device, cudaStream_t st) {
  const size_t smem = field_f32_smem(P);
  const uint32_t cells = (uint32_t)P.occ_grid * P.occ_grid * P.occ_grid;
  const int blocks = std::min<int>(num_sms(device), (int)((cells + kF32Threads - 1) / kF32Threads));
  if (mode == kModeDensity) {
    NR_CHECK_CUDA(cudaFuncSetAttribute(field_f32_kernel<kModeDensity>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    field_f32_kernel<kModeDensity><<<blocks, kF32Threads, smem, st>>>(P, nullptr, 0, nullptr,
                                                                       reinterpret_cast<float *>(bits));
  } else {
    NR_CHECK_CUDA(cudaFuncSetAttribute(field_f32_kernel<kModePose>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    field_f32_kernel<kModePose><<<blocks, kF32Threads, smem, st>>>(P, nullptr, 0, nullptr,
                                                                    reinterpret_cast<float *>(bits));
  }
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(1);
  return NR_OK;
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

// ------------------------------------------------------- round-based ERT
// With early ray termination on, a frame is rendered in rounds so that a ray
// stops costing field evaluations once it is opaque: each round every active
// ray appends up to k more live samples (from the slot where the last round
// stopped), the field runs on that round's queue, and compositing folds them
// into the ray's running (C, T) and retires the ray when T < t_min or when its
// slots are exhausted.  The per-ray sequence of compositing operations is the
// single pass's, so the image is identical.
constexpr uint32_t kRayDone = 0x80000000u;

// Also clears the live-sample counter for the first round (the round's composite clears it for
// the next), so that no memset sits between the launches of a frame.
__global__ void init_rays_kernel(uint32_t n, float4 *__restrict__ state, uint32_t *__restrict__ next,
                                 uint32_t *__restrict__ counter) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r == 0) *counter = 0u;
  if (r < n) {
    state[r] = make_float4(0.f, 0.f, 0.f, 1.f);
    next[r] = 0u;
  }
}

// next[r]: the ray's next slot, kRayDone once retired.  The march writes the slot after this
// round's last sample into next[r] (the composite may then mark the ray done).
__global__ void __launch_bounds__(256) march_round_kernel(CamParams cam, MarchParams mp, uint32_t k,
                                                          float4 *__restrict__ samp, uint2 *__restrict__ ray_range,
                                                          uint32_t *__restrict__ counter, uint32_t *__restrict__ total,
                                                          uint32_t *__restrict__ next) {
  const uint32_t r = mp.ray0 + blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = r < mp.ray_end;
  const uint32_t lane = threadIdx.x & 31;
  float o[3], d[3], lo = 0.f, hi = 0.f;
  camera_origin(cam, o);
  const uint32_t st0 = valid ? next[r - mp.ray0] : kRayDone;
  bool active = !(st0 & kRayDone);
  if (active) {
    const uint32_t u = r % cam.width, v = r / cam.width;
    active = ray_setup(cam, o, mp.bmin, mp.bmax, u, v, d, lo, hi);
  }
  const uint32_t S = cam.n_samples;
  const float D = __fdiv_rn(__fsub_rn(hi, lo), (float)S);
  const int G = mp.grid;
  float h[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) h[q] = __fdiv_rn(__fsub_rn(mp.bmax[q], mp.bmin[q]), (float)G);
  auto pos = [&](uint32_t i, float x[3]) {
    const float t = __fadd_rn(lo, __fmul_rn(__fadd_rn((float)i, 0.5f), D));
#pragma unroll
    for (int q = 0; q < 3; ++q) x[q] = __fadd_rn(o[q], __fmul_rn(t, d[q]));
  };
  auto live = [&](uint32_t i, float x[3]) -> bool {
    pos(i, x);
    if (!mp.bits) return true;
    int c[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      int cq = (int)floorf(__fdiv_rn(__fsub_rn(x[q], mp.bmin[q]), h[q]));
      c[q] = min(max(cq, 0), G - 1);
    }
    const uint32_t cell = ((uint32_t)c[2] * G + (uint32_t)c[1]) * G + (uint32_t)c[0];
    return (__ldg(mp.bits + (cell >> 5)) >> (cell & 31)) & 1u;
  };
  const uint32_t i0 = st0 & ~kRayDone;
  uint32_t count = 0, i_end = S;                      // a ray that misses the box has no slots left
  uint64_t m0 = 0u, m1 = 0u;                          // live flags of slots i0 .. i0 + 63, i0 + 64 .. i0 + 127
  if (active) {
    float x[3];
    uint32_t i = i0;
    for (; i < S && count < k; ++i) {
      const bool lv = live(i, x);
      count += lv ? 1u : 0u;
      const uint32_t e = i - i0;
      if (lv && e < 64u) m0 |= 1ull << e;
      else if (lv && e < 128u) m1 |= 1ull << (e - 64u);
    }
    i_end = i;
  }
  uint32_t incl = count;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= (uint32_t)off) incl += y;
  }
  const uint32_t wtotal = __shfl_sync(0xffffffffu, incl, 31);
  uint32_t base = 0;
  if (lane == 31 && wtotal) {
    base = atomicAdd(counter, wtotal);
    if (total) atomicAdd(total, wtotal);
  }
  base = __shfl_sync(0xffffffffu, base, 31);
  const uint32_t off = base + incl - count;
  if (valid) {
    ray_range[r - mp.ray0] = make_uint2(off, count);
    if (!(st0 & kRayDone)) next[r - mp.ray0] = i_end;
  }
  if (count) {
    uint32_t w = off;
    if (i_end - i0 <= 128u) {   // the flags hold every slot tested: only positions are recomputed
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        uint64_t bits = q ? m1 : m0;
        while (bits) {
          const uint32_t e = 64u * q + (uint32_t)(__ffsll((long long)bits) - 1);
          bits &= bits - 1u;
          float x[3];
          pos(i0 + e, x);
          samp[w++] = make_float4(x[0], x[1], x[2], D);
        }
      }
    } else {
      for (uint32_t i = i0; w < off + count; ++i) {
        float x[3];
        if (live(i, x)) samp[w++] = make_float4(x[0], x[1], x[2], D);
      }
    }
  }
}

// Folds a round's samples into each active ray's (C, T); retires rays below t_min or out of slots.
__global__ void __launch_bounds__(256) composite_round_kernel(const uint2 *__restrict__ ray_range,
                                                              const float4 *__restrict__ so, uint32_t n_rays,
                                                              float t_min, uint32_t S, float4 *__restrict__ state,
                                                              uint32_t *__restrict__ next, uint32_t *__restrict__ counter) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r == 0) *counter = 0u;   // the round's field launch has read it: cleared for the next march
  if (r >= n_rays) return;
  const uint32_t nx = next[r];
  if (nx & kRayDone) return;
  float4 c = state[r];
  bool done = false;
  const uint2 rr = ray_range[r];
  for (uint32_t i = 0; i < rr.y; ++i) {
    const float4 v = so[rr.x + i];
    const float w = c.w * v.w;
    c.x = fmaf(w, v.x, c.x);
    c.y = fmaf(w, v.y, c.y);
    c.z = fmaf(w, v.z, c.z);
    c.w *= 1.f - v.w;
    if (c.w < t_min) {
      done = true;
      break;
    }
  }
  state[r] = c;
  if (done || nx >= S) next[r] = nx | kRayDone;
}

__global__ void add_u32_kernel(uint32_t *__restrict__ acc, const uint32_t *__restrict__ v) { *acc += *v; }

__global__ void finalize_rays_kernel(const float4 *__restrict__ state, uint32_t n_rays, float bg0, float bg1, float bg2,
                                     float4 *__restrict__ out) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rays) return;
  const float4 c = state[r];
  out[r] = make_float4(fmaf(c.w, bg0, c.x), fmaf(c.w, bg1, c.y), fmaf(c.w, bg2, c.z), 1.f - c.w);
}

size_t field_f32_smem(const FieldParams &P) {
  return sizeof(float) * (P.lay.total + kPoseSmem + kWidth + (size_t)kF32ColRows * kF32Threads);
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
  if (mlp_dtype == NR_BF16 || mlp_dtype == NR_F16) {
    if (mma_path == 1) return launch_field_t5(P, mlp_dtype, mode, in, n_fixed, n_dev, out, device, st);
    if (mma_path == 2 || mma_path == 4)
      return launch_field_tc(P, mlp_dtype, mode, in, n_fixed, n_dev, out, device, st, mma_path == 2 ? 2 : 1);
    return launch_field_ws(P, mlp_dtype, mode, in, n_fixed, n_dev, out, device, st);
  }
  if (mlp_dtype == NR_FP8E4M3)
    return mma_path == 4 ? launch_field_fp8(P, mode, in, n_fixed, n_dev, out, device, st)
                         : launch_field_ws(P, mlp_dtype, mode, in, n_fixed, n_dev, out, device, st);
  if (mlp_dtype != NR_F32) {
    set_error("mlp_dtype %d is not implemented", (int)mlp_dtype);
    return NR_EUNSUPPORTED;
  }
  if (mma_path == 3) return launch_field_tf32(P, mode, in, n_fixed, n_dev, out, device, st);
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

// The field kernel a render or query takes (launch_field's mma_path): for bf16/f16 MLPs 0 the
// warp-specialised tcgen05 pipeline (the default), 1 tcgen05 with one group per tile and the
// activations through shared memory, 2 warp-level mma.sync over two m-tiles per weight read,
// 4 warp-level mma.sync over one m-tile; for fp8 0 the tcgen05 pipeline, 4 warp-level mma.sync;
// for float32 3 the tensor-core tier, else CUDA cores.
int render_path(const nr_render_opts *o) {
  if (o->mlp_dtype == NR_F32) return (o->flags & NR_RENDER_F32_TC) ? 3 : 0;
  if (o->mlp_dtype == NR_FP8E4M3) return (o->flags & NR_RENDER_MMA_SYNC) ? 4 : 0;
  if (o->mlp_dtype != NR_BF16 && o->mlp_dtype != NR_F16) return 0;
  if (o->flags & NR_RENDER_TCGEN05) return 1;
  if (o->flags & NR_RENDER_MMA2) return 2;
  return (o->flags & NR_RENDER_MMA_SYNC) ? 4 : 0;
}

// Whether the path runs a tcgen05 kernel: it needs the swizzled weight blobs (prepare_t5) and
// keeps an error word for bounded waits that gave up.
bool path_uses_tcgen05(const nr_render_opts *o, int path) {
  if (o->mlp_dtype == NR_FP8E4M3) return path == 0;
  return (o->mlp_dtype == NR_BF16 || o->mlp_dtype == NR_F16) && (path == 0 || path == 1);
}

nr_status check_field_timeouts(nr_subject *s, cudaStream_t st) {
  if (!s->t5_err) return NR_OK;
  uint32_t word = 0;
  NR_CHECK_CUDA(cudaMemcpyAsync(&word, s->t5_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  NR_CHECK_CUDA(cudaStreamSynchronize(st));
  if (word == 0) return NR_OK;
  NR_CHECK_CUDA(cudaMemsetAsync(s->t5_err, 0, sizeof(uint32_t), st));
  set_error("field kernel: a bounded wait on the tensor-core pipeline gave up (code %u); the output is invalid",
            word);
  return NR_ETIMEOUT;
}

// One column of kTf32Rows floats per thread of one block per SM (allocated on first use).
static nr_status grow_tf32_scratch(nr_subject *s) {
  const size_t need = (size_t)num_sms(s->device) * kTf32Rows * kTf32Threads;
  if (need <= s->rw_scratch) return NR_OK;
  if (s->r_scratch) NR_CHECK_CUDA(cudaFree(s->r_scratch));
  s->r_scratch = nullptr;
  s->rw_scratch = 0;
  NR_CHECK_CUDA(cudaMalloc((void **)&s->r_scratch, need * sizeof(float)));
  s->rw_scratch = need;
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
    if (s->ray_state) cudaFree(s->ray_state);
    if (s->ray_next) cudaFree(s->ray_next);
    s->ray_range = nullptr;
    s->ray_state = nullptr;
    s->ray_next = nullptr;
    s->ws_rays = 0;
    NR_CHECK_CUDA(cudaMalloc(&s->ray_range, rays * sizeof(uint2)));
    NR_CHECK_CUDA(cudaMalloc(&s->ray_state, rays * sizeof(float4)));
    NR_CHECK_CUDA(cudaMalloc(&s->ray_next, rays * sizeof(uint32_t)));
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

// Samples per ray and round when early termination is on (the whole ray otherwise).
uint32_t round_samples(const nr_camera *cam, const nr_render_opts *opts) {
  if (opts->t_min <= 0.f) return cam->n_samples;
  return std::min<uint32_t>(cam->n_samples, std::max<uint32_t>(16u, (cam->n_samples + 3) / 4));
}

nr_status render_rays(const nr_subject *s, const FieldParams &P, const uint32_t *bits, const nr_camera *cam,
                      const nr_render_opts *opts, const FrameWork &w, float4 *dst, cudaStream_t st, int mma_path,
                      Prof *prof) {
  const CamParams C = cam_params(cam);
  const uint32_t n_rays = cam->width * cam->height;
  const uint32_t S = cam->n_samples;
  const uint32_t k = round_samples(cam, opts);
  const bool rounds = k < S || opts->t_min > 0.f;
  const uint32_t chunk = (uint32_t)std::min<uint64_t>(std::min<uint64_t>(n_rays, w.cap_rays),
                                                      std::max<uint64_t>(1, w.cap_samples / k));
  if (chunk == 0 || (rounds && (!w.state || !w.next))) {
    set_error("render: workspace too small");
    return NR_EINVAL;
  }
  MarchParams mp{};
  for (int q = 0; q < 3; ++q) {
    mp.bmin[q] = s->bmin[q];
    mp.bmax[q] = s->bmax[q];
  }
  mp.grid = (int)s->occ_grid;
  mp.bits = opts->use_occupancy ? bits : nullptr;
  // One event per launch boundary: mark(stage) closes the interval since the previous mark as
  // that stage's; mark(-1) opens a run of back-to-back launches (its interval is not counted).
  auto mark = [&](int stage) -> cudaError_t {
    if (!prof) return cudaSuccess;
    if (prof->used >= prof->cap) {
      prof->overflow = true;
      return cudaSuccess;
    }
    prof->stage[prof->used] = stage;
    return cudaEventRecord(prof->ev[prof->used++], st);
  };
  nr_status r;
  const uint32_t n_rounds = rounds ? (S + k - 1) / k : 1;
  for (uint32_t r0 = 0; r0 < n_rays; r0 += chunk) {
    const uint32_t nr_ = std::min(chunk, n_rays - r0);
    const unsigned nb = (nr_ + 255) / 256;
    mp.ray0 = r0;
    mp.ray_end = r0 + nr_;
    if (rounds) {
      init_rays_kernel<<<nb, 256, 0, st>>>(nr_, w.state, w.next, w.counter);
      count_launches(1);
    }
    for (uint32_t round = 0; round < n_rounds; ++round) {
      if (!rounds) NR_CHECK_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(uint32_t), st));
      if (round == 0 || !rounds) NR_CHECK_CUDA(mark(-1));
      if (rounds)
        march_round_kernel<<<nb, 256, 0, st>>>(C, mp, k, w.samp, w.ray_range, w.counter, w.total, w.next);
      else
        march_kernel<<<nb, 256, 0, st>>>(C, mp, w.samp, w.ray_range, w.counter);
      NR_CHECK_CUDA(cudaGetLastError());
      if (!rounds && w.total) {
        add_u32_kernel<<<1, 1, 0, st>>>(w.total, w.counter);
        count_launches(1);
      }
      NR_CHECK_CUDA(mark(0));
      if ((r = launch_field(P, opts->mlp_dtype, kModeRender, w.samp, 0, w.counter, (float *)w.samp_out, s->device, st,
                            mma_path)) != NR_OK)
        return r;
      NR_CHECK_CUDA(mark(1));
      if (rounds)
        composite_round_kernel<<<nb, 256, 0, st>>>(w.ray_range, w.samp_out, nr_, opts->t_min, S, w.state, w.next,
                                                   w.counter);
      else
        composite_kernel<<<nb, 256, 0, st>>>(w.ray_range, w.samp_out, nr_, opts->t_min, cam->bg[0], cam->bg[1],
                                             cam->bg[2], dst + r0);
      NR_CHECK_CUDA(cudaGetLastError());
      NR_CHECK_CUDA(mark(2));
      count_launches(3);
    }
    if (rounds) {
      finalize_rays_kernel<<<nb, 256, 0, st>>>(w.state, nr_, cam->bg[0], cam->bg[1], cam->bg[2], dst + r0);
      NR_CHECK_CUDA(cudaGetLastError());
      count_launches(1);
    }
  }
  return NR_OK;
}

nr_status render_frame(const nr_subject *s, const FieldParams &P, const uint32_t *bits, const nr_camera *cam,
                       const nr_render_opts *opts, const FrameWork &w, float4 *dst, cudaStream_t st) {
  const int path = render_path(opts);   // the float32 tensor-core tier needs a scratch buffer: CUDA cores
  return render_rays(s, P, bits, cam, opts, w, dst, st, path == 3 ? 0 : path, nullptr);
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
  NR_REQUIRE(!opts->use_occupancy || s->occ_source != kOccNone,
             "nr_render: occupancy requested but the subject has none");
  if (!s->pose_set) {
    set_error("nr_render: call nr_set_pose first");
    return NR_ESTATE;
  }
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  cudaStream_t st = (cudaStream_t)stream;
  if ((r = prepare_params(s, st)) != NR_OK) return r;
  if ((r = ensure_pose(s, st)) != NR_OK) return r;
  if ((r = ensure_bias(s, st)) != NR_OK) return r;
  if (opts->use_occupancy && (r = ensure_occupancy(s, st)) != NR_OK) return r;
  if (opts->mlp_dtype == NR_FP8E4M3 && (r = prepare_fp8(s, st)) != NR_OK) return r;
  const int path = render_path(opts);
  const bool t5 = path_uses_tcgen05(opts, path);
  if (t5 && (r = prepare_t5(s, st)) != NR_OK) return r;
  if (path == 3 && (r = grow_tf32_scratch(s)) != NR_OK) return r;
  FieldParams P = field_params(s, opts);
  const bool prof = (opts->flags & NR_RENDER_PROFILE) != 0;
  if (prof) P.kept_count = s->counter + 9;
  const uint32_t n_rays = cam->width * cam->height;
  // chunk the rays so that the worst-case sample queue of a round stays below 2^26 entries
  const uint64_t max_samples = 1ull << 26;
  const uint32_t k = round_samples(cam, opts);
  const uint32_t chunk = (uint32_t)std::min<uint64_t>(n_rays, std::max<uint64_t>(256, max_samples / k));
  if ((r = grow_workspace(s, chunk, (size_t)chunk * k)) != NR_OK) return r;
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
  Prof pr{};
  if (prof) {
    for (int i = 0; i < nr_subject::kProfEvents; ++i)
      if (!s->prof_ev[i]) NR_CHECK_CUDA(cudaEventCreate(&s->prof_ev[i]));
    pr.ev = s->prof_ev;
    pr.stage = s->prof_stage;
    pr.cap = nr_subject::kProfEvents;
    NR_CHECK_CUDA(cudaMemsetAsync(s->counter + 8, 0, 2 * sizeof(uint32_t), st));
  }
  FrameWork w{};
  w.samp = s->samp;
  w.samp_out = s->samp_out;
  w.ray_range = s->ray_range;
  w.counter = s->counter;
  w.total = prof ? s->counter + 8 : nullptr;
  w.state = s->ray_state;
  w.next = s->ray_next;
  w.cap_samples = s->ws_samples;
  w.cap_rays = s->ws_rays;
  s->prof_used = 0;
  if ((r = render_rays(s, P, s->bits, cam, opts, w, reinterpret_cast<float4 *>(dst), st, path, prof ? &pr : nullptr)) !=
      NR_OK)
    return r;
  if (prof) {
    s->prof_used = pr.used;
    s->prof_overflow = pr.overflow;
  }
  if (!dev_out) NR_CHECK_CUDA(cudaMemcpyAsync(out_rgba, dst, (size_t)n_rays * 16, cudaMemcpyDeviceToHost, st));
  if (t5) return check_field_timeouts(s, st);
  if (!dev_out) NR_CHECK_CUDA(cudaStreamSynchronize(st));
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
  int field_launches = 0;
  for (int i = 1; i < s->prof_used; ++i) {
    if (s->prof_stage[i] < 0) continue;
    float t = 0.f;
    NR_CHECK_CUDA(cudaEventElapsedTime(&t, s->prof_ev[i - 1], s->prof_ev[i]));
    acc[s->prof_stage[i]] += t;
    field_launches += s->prof_stage[i] == 1;
  }
  uint32_t cnt[2] = {0, 0};   // live samples, bone channels read
  NR_CHECK_CUDA(cudaMemcpy(cnt, s->counter + 8, sizeof(cnt), cudaMemcpyDeviceToHost));
  ms[0] = acc[0];
  ms[1] = acc[1];
  ms[2] = acc[2];
  ms[3] = (float)field_launches;
  ms[4] = (float)cnt[0];
  ms[5] = cnt[0] ? (float)((double)cnt[1] / (double)cnt[0]) : 0.f;
  if (s->prof_overflow) {
    set_error("nr_stage_times: more launches than profiling events; times are partial");
    return NR_EBUSY;
  }
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
  if ((r = ensure_pose(s, st)) != NR_OK) return r;
  if ((r = ensure_bias(s, st)) != NR_OK) return r;
  if (opts->mlp_dtype == NR_FP8E4M3 && (r = prepare_fp8(s, st)) != NR_OK) return r;
  const int path = render_path(opts);
  const bool t5 = path_uses_tcgen05(opts, path);
  if (t5 && (r = prepare_t5(s, st)) != NR_OK) return r;
  if (path == 3 && (r = grow_tf32_scratch(s)) != NR_OK) return r;
  const FieldParams P = field_params(s, opts);
  count_launches(1);
  if ((r = launch_field(P, opts->mlp_dtype, kModeQuery, reinterpret_cast<const float4 *>(x_obs), n, nullptr, out,
                        s->device, st, path)) != NR_OK)
    return r;
  return t5 ? check_field_timeouts(s, st) : NR_OK;
}
