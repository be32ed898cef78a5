// field.cuh -- device-side steps of the per-sample field (Sec. 4.2 - 4.4):
// inverse-LBS warp over the canonical weight volume, positional encoding with
// the truncated Hann window, multiresolution hash encoding, and the float32
// CUDA-core MLP layers.  Included by the forward and backward kernels.
#pragma once

#include "common.cuh"

namespace nr {

// ------------------------------------------------------------------ LBS warp
// Sec. 4.2: x_skel = sum_i w_i^c(G_i x) G_i(x) / sum_k w_k^c(G_k x), with the
// candidate p_i = G_i x = R_i x + t_i and w_i^c read trilinearly from channel
// i of the canonical weight volume (vertices on the box corners, a corner
// outside the grid contributes zero).  The denominator S is floored at kEpsW.

// Trilinear sample of one bone channel through its corner-block copy: entry
// (z, y, x), z in [-1, R], y and x in [-1, R-1], holds the float4
// (V[z][y][x], V[z][y][x+1], V[z][y+1][x], V[z][y+1][x+1]) with V = 0 outside the
// grid, so a point whose cell origin lies in [-1, R-1]^3 needs exactly two
// aligned 16-byte loads (z and z + 1); any other point is farther than one
// cell from the grid and reads zero.
__device__ __forceinline__ float trilinear_quad(const float4 *__restrict__ q, int R, float ux, float uy, float uz) {
  const float fx0 = floorf(ux), fy0 = floorf(uy), fz0 = floorf(uz);
  const int ix = (int)fx0, iy = (int)fy0, iz = (int)fz0;
  if (ix < -1 || iy < -1 || iz < -1 || ix >= R || iy >= R || iz >= R) return 0.f;
  const float fx = ux - fx0, fy = uy - fy0, fz = uz - fz0;
  const int R1 = R + 1;
  const int b = ((iz + 1) * R1 + (iy + 1)) * R1 + (ix + 1);
  const float4 a = __ldg(q + b), c = __ldg(q + b + R1 * R1);
  const float a0 = fmaf(fx, a.y - a.x, a.x), a1 = fmaf(fx, a.w - a.z, a.z);
  const float c0 = fmaf(fx, c.y - c.x, c.x), c1 = fmaf(fx, c.w - c.z, c.z);
  const float z0 = fmaf(fy, a1 - a0, a0), z1 = fmaf(fy, c1 - c0, c0);
  return fmaf(fz, z1 - z0, z0);
}

// The same trilinear sample and its gradient d/d(ux, uy, uz) inside the cell
// (one-sided on a cell face: the cell is the floor of u, as in the value).
__device__ __forceinline__ float trilinear_quad_grad(const float4 *__restrict__ q, int R, float ux, float uy, float uz,
                                                     float &gx, float &gy, float &gz) {
  gx = gy = gz = 0.f;
  const float fx0 = floorf(ux), fy0 = floorf(uy), fz0 = floorf(uz);
  const int ix = (int)fx0, iy = (int)fy0, iz = (int)fz0;
  if (ix < -1 || iy < -1 || iz < -1 || ix >= R || iy >= R || iz >= R) return 0.f;
  const float fx = ux - fx0, fy = uy - fy0, fz = uz - fz0;
  const int R1 = R + 1;
  const int b = ((iz + 1) * R1 + (iy + 1)) * R1 + (ix + 1);
  const float4 a = __ldg(q + b), c = __ldg(q + b + R1 * R1);
  const float a0 = fmaf(fx, a.y - a.x, a.x), a1 = fmaf(fx, a.w - a.z, a.z);
  const float c0 = fmaf(fx, c.y - c.x, c.x), c1 = fmaf(fx, c.w - c.z, c.z);
  const float z0 = fmaf(fy, a1 - a0, a0), z1 = fmaf(fy, c1 - c0, c0);
  const float ex0 = fmaf(fy, (a.w - a.z) - (a.y - a.x), a.y - a.x);   // d/dfx on the z0 face
  const float ex1 = fmaf(fy, (c.w - c.z) - (c.y - c.x), c.y - c.x);   // d/dfx on the z1 face
  gx = fmaf(fz, ex1 - ex0, ex0);
  gy = fmaf(fz, (c1 - c0) - (a1 - a0), a1 - a0);
  gz = z1 - z0;
  return fmaf(fz, z1 - z0, z0);
}

__host__ __device__ inline size_t quad_channel(int R) { return (size_t)(R + 2) * (R + 1) * (R + 1); }

// Stages the pose (and, when P.bone_box is set, the support boxes) into shared
// memory at sG [kPoseSmem]; returns the box pointer to pass to lbs_warp.
__device__ __forceinline__ const float *stage_pose(const FieldParams &P, float *sG, int tid, int nthreads) {
  for (int i = tid; i < kBones * 12; i += nthreads) sG[i] = P.G[i];
  if (!P.bone_box) return nullptr;
  for (int i = tid; i < kBones * 6; i += nthreads) sG[kBones * 12 + i] = P.bone_box[i];
  return sG + kBones * 12;
}

// sG: the 24 bone transforms [24][12] (rows [R | t]) in shared memory.
// sBox (render kernels, may be NULL): per bone (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z) in
// volume-index units such that every vertex of the channel above kBoneEps lies in
// [lo + 1, hi - 1]; a candidate with u outside [lo, hi) has all eight corners at or below
// kBoneEps and is skipped (its weight counts as 0).  Skipping changes S by at most
// 24 kBoneEps and x_skel by at most 24 kBoneEps |p_i - x_skel| / S.
__device__ __forceinline__ void lbs_warp(const FieldParams &P, const float *__restrict__ sG, float x0, float x1,
                                         float x2, float &s0, float &s1, float &s2, float &S,
                                         const float *__restrict__ sBox = nullptr) {
  const int R = P.wres;
  const size_t QC = quad_channel(R);
  float n0 = 0.f, n1 = 0.f, n2 = 0.f, sum = 0.f;
#pragma unroll 4
  for (int i = 0; i < kBones; ++i) {
    const float *g = sG + 12 * i;
    const float p0 = fmaf(g[0], x0, fmaf(g[1], x1, fmaf(g[2], x2, g[3])));
    const float p1 = fmaf(g[4], x0, fmaf(g[5], x1, fmaf(g[6], x2, g[7])));
    const float p2 = fmaf(g[8], x0, fmaf(g[9], x1, fmaf(g[10], x2, g[11])));
    const float ux = (p0 - P.bmin[0]) * P.vol_scale[0];
    const float uy = (p1 - P.bmin[1]) * P.vol_scale[1];
    const float uz = (p2 - P.bmin[2]) * P.vol_scale[2];
    if (sBox) {
      const float *b = sBox + 6 * i;
      if (ux < b[0] || uy < b[1] || uz < b[2] || ux >= b[3] || uy >= b[4] || uz >= b[5]) continue;
    }
    const float w = trilinear_quad(P.wquad + (size_t)i * QC, R, ux, uy, uz);
    sum += w;
    n0 = fmaf(w, p0, n0);
    n1 = fmaf(w, p1, n1);
    n2 = fmaf(w, p2, n2);
  }
  const float inv = 1.f / fmaxf(sum, kEpsW);
  s0 = n0 * inv;
  s1 = n1 * inv;
  s2 = n2 * inv;
  S = sum;
}

// ------------------------------------------------------- positional encoding
// Sec. 4.3: gamma(x) = [x^, w_k sin(2^k pi x^), w_k cos(2^k pi x^)]_{k<L} with
// x^ the point normalised to [-1, 1] over the box and w_k the truncated Hann
// weight of band k.  Writes kResGammaPad values (zero padded).
__device__ __forceinline__ void pos_enc(const FieldParams &P, float x0, float x1, float x2, float *__restrict__ g,
                                        int stride) {
  const float h0 = (x0 - P.box_c[0]) * P.box_ih[0];
  const float h1 = (x1 - P.box_c[1]) * P.box_ih[1];
  const float h2 = (x2 - P.box_c[2]) * P.box_ih[2];
  g[0] = h0;
  g[stride] = h1;
  g[2 * stride] = h2;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float sc = (float)(1 << k);
    float sa, ca, sb, cb, sd, cd;
    sincospif(sc * h0, &sa, &ca);
    sincospif(sc * h1, &sb, &cb);
    sincospif(sc * h2, &sd, &cd);
    const float w = (k < P.res_freqs) ? P.hann[k] : 0.f;
    float *q = g + (3 + 6 * k) * stride;
    q[0] = w * sa;
    q[stride] = w * sb;
    q[2 * stride] = w * sd;
    q[3 * stride] = w * ca;
    q[4 * stride] = w * cb;
    q[5 * stride] = w * cd;
  }
#pragma unroll
  for (int j = 39; j < kResGammaPad; ++j) g[j * stride] = 0.f;
}

// ------------------------------------------------------------- hash encoding
// Multiresolution hash encoding of the canonical point (the workloads' field):
// p = (x - box_min) / (box_max - box_min); on level l the point sits at p N_l
// among vertices 0..N_l; its cell is floor(p N_l) capped at N_l - 1; the 8
// corners are read trilinearly.  Dense levels ((N+1)^3 <= T) index row-major,
// the others by (x ^ y 2654435761 ^ z 805459861) mod T.  Outside the box the
// features are zero (and the sample gets no density).

constexpr uint32_t kPrimeY = 2654435761u;
constexpr uint32_t kPrimeZ = 805459861u;

struct HashCell {
  uint32_t idx[8];
  float w[8];
};

__device__ __forceinline__ void hash_cell(const FieldParams &P, int l, float p0, float p1, float p2, HashCell &c) {
  const uint32_t N = P.level_res[l];
  const float fn = (float)N;
  const float q0 = p0 * fn, q1 = p1 * fn, q2 = p2 * fn;
  const float a0 = fminf(floorf(q0), fn - 1.f), a1 = fminf(floorf(q1), fn - 1.f), a2 = fminf(floorf(q2), fn - 1.f);
  const float f0 = q0 - a0, f1 = q1 - a1, f2 = q2 - a2;
  const uint32_t i0 = (uint32_t)a0, i1 = (uint32_t)a1, i2 = (uint32_t)a2;
  const bool dense = (P.dense_mask >> l) & 1u;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t x = i0 + (k & 1), y = i1 + ((k >> 1) & 1), z = i2 + (k >> 2);
    uint32_t id;
    if (dense) {
      id = x + y * (N + 1) + z * (N + 1) * (N + 1);
    } else {
      id = (x ^ (y * kPrimeY) ^ (z * kPrimeZ)) & P.T_mask;
    }
    c.idx[k] = id;
    c.w[k] = ((k & 1) ? f0 : 1.f - f0) * (((k >> 1) & 1) ? f1 : 1.f - f1) * ((k >> 2) ? f2 : 1.f - f2);
  }
}

__device__ __forceinline__ float2 table_read(const FieldParams &P, int l, uint32_t id) {
  const size_t off = (size_t)l * (size_t)(P.T_mask + 1) + id;
  if (P.use_f16_table) {
    const __half2 h = P.table16[off];
    return __half22float2(h);
  }
  return __ldg(P.table32 + off);
}

// The two features of level l at the clamped box coordinate p: 8 corners read
// trilinearly from the f16 or f32 table (the dtype test sits outside the corners).
__device__ __forceinline__ void hash_level(const FieldParams &P, int l, float p0, float p1, float p2, float &fa,
                                           float &fb) {
  if (P.use_f16_table && P.dense_quad && ((P.dense_mask >> l) & 1u)) {
    // a dense level from its corner blocks: the same eight values, weights and order of
    // accumulation as the per-corner reads below, in two 16-byte loads
    const uint32_t N = P.level_res[l];
    const float fn = (float)N;
    const float q0 = p0 * fn, q1 = p1 * fn, q2 = p2 * fn;
    const float a0 = fminf(floorf(q0), fn - 1.f), a1 = fminf(floorf(q1), fn - 1.f), a2 = fminf(floorf(q2), fn - 1.f);
    const float f0 = q0 - a0, f1 = q1 - a1, f2 = q2 - a2;
    const uint4 *Q = P.dense_quad + P.dq_off[l] + ((size_t)a2 * N + (uint32_t)a1) * N + (uint32_t)a0;
    const uint4 lo = __ldg(Q), hi = __ldg(Q + (size_t)N * N);
    const uint32_t u[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    fa = 0.f;
    fb = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float w = ((k & 1) ? f0 : 1.f - f0) * (((k >> 1) & 1) ? f1 : 1.f - f1) * ((k >> 2) ? f2 : 1.f - f2);
      const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(&u[k]));
      fa = fmaf(w, v.x, fa);
      fb = fmaf(w, v.y, fb);
    }
    return;
  }
  HashCell c;
  hash_cell(P, l, p0, p1, p2, c);
  fa = 0.f;
  fb = 0.f;
  const size_t base = (size_t)l * (size_t)(P.T_mask + 1);
  if (P.use_f16_table) {
    const __half2 *tab = P.table16 + base;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float2 v = __half22float2(tab[c.idx[k]]);
      fa = fmaf(c.w[k], v.x, fa);
      fb = fmaf(c.w[k], v.y, fb);
    }
  } else {
    const float2 *tab = P.table32 + base;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float2 v = __ldg(tab + c.idx[k]);
      fa = fmaf(c.w[k], v.x, fa);
      fb = fmaf(c.w[k], v.y, fb);
    }
  }
}

// enc (a column with the given stride): 2 features per level, zero beyond 2L.  Returns whether x is inside the box.
__device__ __forceinline__ bool hash_encode(const FieldParams &P, float x0, float x1, float x2, float *__restrict__ enc,
                                            int stride) {
  float p0 = (x0 - P.bmin[0]) * P.inv_box[0];
  float p1 = (x1 - P.bmin[1]) * P.inv_box[1];
  float p2 = (x2 - P.bmin[2]) * P.inv_box[2];
  const bool inside = p0 >= 0.f && p0 <= 1.f && p1 >= 0.f && p1 <= 1.f && p2 >= 0.f && p2 <= 1.f;
  p0 = fminf(fmaxf(p0, 0.f), 1.f);
  p1 = fminf(fmaxf(p1, 0.f), 1.f);
  p2 = fminf(fmaxf(p2, 0.f), 1.f);
  // a runtime level loop: one copy of the level body keeps the kernels' code small
#pragma unroll 1
  for (int l = 0; l < P.L; ++l) {
    float a, b;
    hash_level(P, l, p0, p1, p2, a, b);
    enc[(2 * l) * stride] = inside ? a : 0.f;
    enc[(2 * l + 1) * stride] = inside ? b : 0.f;
  }
  for (int l = P.L; l < kMaxLevels; ++l) {
    enc[(2 * l) * stride] = 0.f;
    enc[(2 * l + 1) * stride] = 0.f;
  }
  return inside;
}

// -------------------------------------------------------- float32 MLP layers
// y = W x + b with W stored transposed ([in][out], out a multiple of 4) in
// shared memory and read as broadcast float4 (all threads of the block read
// the same weight).  Each thread keeps its activations in its own column of a
// shared-memory buffer, col[k * stride] (stride = threads per block), so the
// loop over inputs is a runtime loop; the 64 accumulators live in registers.
template <int OUT>
__device__ __forceinline__ void dense_acc_f32(const float *__restrict__ Wt, const float *__restrict__ col, int in,
                                              int stride, float (&y)[OUT]) {
#pragma unroll 2
  for (int k = 0; k < in; ++k) {
    const float xk = col[k * stride];
    const float4 *row = reinterpret_cast<const float4 *>(Wt + k * OUT);
#pragma unroll
    for (int j = 0; j < OUT / 4; ++j) {
      const float4 w = row[j];
      y[4 * j + 0] = fmaf(xk, w.x, y[4 * j + 0]);
      y[4 * j + 1] = fmaf(xk, w.y, y[4 * j + 1]);
      y[4 * j + 2] = fmaf(xk, w.z, y[4 * j + 2]);
      y[4 * j + 3] = fmaf(xk, w.w, y[4 * j + 3]);
    }
  }
}

template <int OUT>
__device__ __forceinline__ void dense_f32(const float *__restrict__ Wt, const float *__restrict__ b,
                                          const float *__restrict__ col, int in, int stride, float (&y)[OUT]) {
#pragma unroll
  for (int j = 0; j < OUT; ++j) y[j] = b[j];
  dense_acc_f32<OUT>(Wt, col, in, stride, y);
}

template <int N>
__device__ __forceinline__ void store_relu(const float (&y)[N], float *__restrict__ col, int stride) {
#pragma unroll
  for (int j = 0; j < N; ++j) col[j * stride] = fmaxf(y[j], 0.f);
}

// The output activations with the accurate expf / log1pf and an IEEE division: rgb =
// 1 / (1 + e^-o) (0 once e^-o overflows), sigma = max(o, 0) + log(1 + e^-|o|), which never
// overflows.  The opacity of a sample is formed as -expm1(-sigma delta) so that small
// sigma delta keep their significant bits.
__device__ __forceinline__ float sigmoidf_(float o) { return 1.f / (1.f + expf(-o)); }
__device__ __forceinline__ float softplusf_(float o) { return fmaxf(o, 0.f) + log1pf(expf(-fabsf(o))); }

// Residual MLP (Sec. 4.3, Fig. S3) in float32.  gcol holds gamma(x_skel)
// (kResGammaPad rows), hcol is the 64-row scratch column; returns x_res.
// bias1 holds b1 + W_Omega Omega (the pose folded into the first layer).
__device__ __forceinline__ void residual_f32(const FieldParams &P, const float *__restrict__ W,
                                             const float *__restrict__ bias1, const float *__restrict__ gcol,
                                             float *__restrict__ hcol, int stride, float &r0, float &r1, float &r2) {
  float y[kWidth];
  dense_f32<kWidth>(W + P.lay.r1, bias1, gcol, kResGammaPad, stride, y);
  store_relu(y, hcol, stride);
  dense_f32<kWidth>(W + P.lay.r2, W + P.lay.r2b, hcol, kWidth, stride, y);
  store_relu(y, hcol, stride);
  dense_f32<kWidth>(W + P.lay.r3, W + P.lay.r3b, hcol, kWidth, stride, y);
  store_relu(y, hcol, stride);
  // layer 4 sees [h3, gamma]: the transposed rows of h3, then those of gamma
  dense_f32<kWidth>(W + P.lay.r4, W + P.lay.r4b, hcol, kWidth, stride, y);
  dense_acc_f32<kWidth>(W + P.lay.r4 + kWidth * kWidth, gcol, kResGammaPad, stride, y);
  store_relu(y, hcol, stride);
  float o[4];
  dense_f32<4>(W + P.lay.r5, W + P.lay.r5b, hcol, kWidth, stride, o);
  r0 = o[0];
  r1 = o[1];
  r2 = o[2];
}

// Canonical MLP (MLP_nerf, Sec. 4.4) in float32 on the encoding held in hcol
// rows 0..31; returns the 4 raw outputs.
__device__ __forceinline__ void canonical_f32(const FieldParams &P, const float *__restrict__ W,
                                              float *__restrict__ hcol, int stride, float (&o)[4]) {
  float y[kWidth];
  dense_f32<kWidth>(W + P.lay.c0, W + P.lay.c0b, hcol, kMlpIn, stride, y);
  store_relu(y, hcol, stride);
  for (int l = 0; l < P.hidden - 1; ++l) {
    dense_f32<kWidth>(W + P.lay.ch[l], W + P.lay.chb[l], hcol, kWidth, stride, y);
    store_relu(y, hcol, stride);
  }
  dense_f32<4>(W + P.lay.cl, W + P.lay.clb, hcol, kWidth, stride, o);
}

}  // namespace nr
