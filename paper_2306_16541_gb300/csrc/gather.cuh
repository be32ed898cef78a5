// gather.cuh -- the per-sample gathers of the field (Sec. 4.2 inverse LBS, the
// multiresolution hash encoding of the canonical point) restructured so that
// each thread keeps many independent loads in flight: a kernel whose warps
// wait on other work (the tcgen05 pipeline of field_ws.cu) cannot hide one
// L2 round trip per bone and per level behind other warps.
//
//   - inverse LBS: the bones kept anywhere in the warp four at a time, their
//     kept corner blocks loaded together and folded into (sum, n) in
//     increasing bone order -- the arithmetic and order of lbs_warp in
//     field.cuh, so x_skel and S are bitwise the same;
//   - hash encoding (f16 table): the dense levels' corner blocks and the hashed
//     levels' corners read four levels at a time; each level's two features
//     interpolated as nested lerps on the packed f16 pairs (x, then y, then z),
//     whose rounding (2^-11 relative per step) stays below that of the bf16 /
//     f16 MLP operand the pair becomes.
#pragma once

#include "field.cuh"
#include "t5.cuh"

namespace nr {

// The two halves of a packed f16 pair as floats (low half first), without taking an address.
__device__ __forceinline__ float2 h2f2(uint32_t u) {
  return make_float2(__half2float(__ushort_as_half((unsigned short)(u & 0xFFFFu))),
                     __half2float(__ushort_as_half((unsigned short)(u >> 16))));
}

__device__ __forceinline__ float trilinear_from(const float4 a, const float4 c, float fx, float fy, float fz) {
  const float a0 = fmaf(fx, a.y - a.x, a.x), a1 = fmaf(fx, a.w - a.z, a.z);
  const float c0 = fmaf(fx, c.y - c.x, c.x), c1 = fmaf(fx, c.w - c.z, c.z);
  const float z0 = fmaf(fy, a1 - a0, a0), z1 = fmaf(fy, c1 - c0, c0);
  return fmaf(fz, z1 - z0, z0);
}

__device__ __forceinline__ void bone_point(const FieldParams &P, const float *__restrict__ g, float x0, float x1,
                                           float x2, float &p0, float &p1, float &p2, float &ux, float &uy,
                                           float &uz) {
  p0 = fmaf(g[0], x0, fmaf(g[1], x1, fmaf(g[2], x2, g[3])));
  p1 = fmaf(g[4], x0, fmaf(g[5], x1, fmaf(g[6], x2, g[7])));
  p2 = fmaf(g[8], x0, fmaf(g[9], x1, fmaf(g[10], x2, g[11])));
  ux = (p0 - P.bmin[0]) * P.vol_scale[0];
  uy = (p1 - P.bmin[1]) * P.vol_scale[1];
  uz = (p2 - P.bmin[2]) * P.vol_scale[2];
}

// lbs_warp with the corner blocks of four bones loaded together, as a resumable computation so
// that a kernel can spread it over waits for other work: lbs_begin takes the candidates'
// support-box tests (no loads); the bones kept by any lane of the warp are then visited four at a
// time by lbs_round -- the same bones in every lane, so the pose reads stay broadcasts -- with
// each lane's loads predicated on its own test, and folded into (sum, n) in increasing bone
// order; lbs_end forms x_skel and S.  A bone that no lane keeps is skipped by all (as lbs_warp
// skips it per lane).  Warp-collective: every lane of the warp calls each step.
struct LbsState {
  float x0, x1, x2;
  uint32_t mine;        // this lane's kept bones
  uint32_t todo;        // the warp's kept bones not visited yet
  float n0, n1, n2, sum;
};

// Margin, in voxels, of the warp-level candidate test below: far above the float32 rounding of
// the transformed points (about 1e-5 voxel).
constexpr float kCandMargin = 0.0625f;

// lbs_begin's support-box test, taken only for the bones whose box can meet one of the warp's
// samples.  The valid samples of the warp lie in an axis-aligned box of centre c and half
// extents e; its image under bone i's transform [R_i | t_i] lies in the box of centre G_i c and
// half extents |R_i| e (componentwise absolute values), so a bone whose support box misses that
// box, widened by kCandMargin, is kept by no lane: lane i < 24 takes bone i's test, and the
// exact per-sample tests run over the bones that pass (the same tests, so the kept bones are the
// same).  A lane without a sample (valid false) keeps no bone.  Warp-collective.
__device__ __forceinline__ void lbs_begin(const FieldParams &P, const float *__restrict__ sG,
                                          const float *__restrict__ sBox, LbsState &st, bool valid) {
  uint32_t mine = valid ? (1u << kBones) - 1u : 0u;
  if (sBox) {
    mine = 0u;
    float lo0 = valid ? st.x0 : INFINITY, lo1 = valid ? st.x1 : INFINITY, lo2 = valid ? st.x2 : INFINITY;
    float hi0 = valid ? st.x0 : -INFINITY, hi1 = valid ? st.x1 : -INFINITY, hi2 = valid ? st.x2 : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo0 = fminf(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
      lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
      lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
      hi0 = fmaxf(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
      hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
      hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
    }
    uint32_t cand = 0u;
    if (lo0 <= hi0) {   // some lane has a sample (warp-uniform)
      const int lane = threadIdx.x & 31;
      bool hit = false;
      if (lane < kBones) {
        const float c0 = 0.5f * (lo0 + hi0), c1 = 0.5f * (lo1 + hi1), c2 = 0.5f * (lo2 + hi2);
        const float e0 = 0.5f * (hi0 - lo0), e1 = 0.5f * (hi1 - lo1), e2 = 0.5f * (hi2 - lo2);
        const float *g = sG + 12 * lane;
        float p0, p1, p2, u0, u1, u2;
        bone_point(P, g, c0, c1, c2, p0, p1, p2, u0, u1, u2);
        const float r0 = (fabsf(g[0]) * e0 + fabsf(g[1]) * e1 + fabsf(g[2]) * e2) * P.vol_scale[0] + kCandMargin;
        const float r1 = (fabsf(g[4]) * e0 + fabsf(g[5]) * e1 + fabsf(g[6]) * e2) * P.vol_scale[1] + kCandMargin;
        const float r2 = (fabsf(g[8]) * e0 + fabsf(g[9]) * e1 + fabsf(g[10]) * e2) * P.vol_scale[2] + kCandMargin;
        const float *b = sBox + 6 * lane;
        hit = u0 + r0 >= b[0] && u1 + r1 >= b[1] && u2 + r2 >= b[2] && u0 - r0 < b[3] && u1 - r1 < b[4] &&
              u2 - r2 < b[5];
      }
      cand = __ballot_sync(0xffffffffu, hit);
    }
#pragma unroll 1
    while (cand) {
      const int i = __ffs(cand) - 1;
      cand &= cand - 1u;
      float p0, p1, p2, ux, uy, uz;
      bone_point(P, sG + 12 * i, st.x0, st.x1, st.x2, p0, p1, p2, ux, uy, uz);
      const float *b = sBox + 6 * i;
      const bool keep = valid && !(ux < b[0] || uy < b[1] || uz < b[2] || ux >= b[3] || uy >= b[4] || uz >= b[5]);
      mine |= (uint32_t)keep << i;
    }
  }
  st.mine = mine;
  st.todo = __reduce_or_sync(0xffffffffu, mine);
  st.n0 = st.n1 = st.n2 = st.sum = 0.f;
}

__device__ __forceinline__ void lbs_round(const FieldParams &P, const float *__restrict__ sG, LbsState &st) {
  if (!st.todo) return;
  const int R = P.wres;
  const size_t QC = quad_channel(R);
  const int R1 = R + 1;
  int bone[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    bone[k] = st.todo ? __ffs(st.todo) - 1 : -1;
    st.todo &= st.todo - 1u;
  }
  float4 qa[4], qc[4];
  float fx[4], fy[4], fz[4], pp[4][3];
  bool keep[4], inb[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = bone[k] < 0 ? 0 : bone[k];
    float ux, uy, uz;
    bone_point(P, sG + 12 * i, st.x0, st.x1, st.x2, pp[k][0], pp[k][1], pp[k][2], ux, uy, uz);
    keep[k] = bone[k] >= 0 && ((st.mine >> i) & 1u);
    const float fx0 = floorf(ux), fy0 = floorf(uy), fz0 = floorf(uz);
    const int ix = (int)fx0, iy = (int)fy0, iz = (int)fz0;
    inb[k] = keep[k] && !(ix < -1 || iy < -1 || iz < -1 || ix >= R || iy >= R || iz >= R);
    fx[k] = ux - fx0;
    fy[k] = uy - fy0;
    fz[k] = uz - fz0;
    const float4 *q = P.wquad + (size_t)i * QC + (inb[k] ? ((iz + 1) * R1 + (iy + 1)) * R1 + (ix + 1) : 0);
    qa[k] = inb[k] ? __ldg(q) : make_float4(0.f, 0.f, 0.f, 0.f);
    qc[k] = inb[k] ? __ldg(q + R1 * R1) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!keep[k]) continue;
    const float w = inb[k] ? trilinear_from(qa[k], qc[k], fx[k], fy[k], fz[k]) : 0.f;
    st.sum += w;
    st.n0 = fmaf(w, pp[k][0], st.n0);
    st.n1 = fmaf(w, pp[k][1], st.n1);
    st.n2 = fmaf(w, pp[k][2], st.n2);
  }
}

__device__ __forceinline__ void lbs_end(const FieldParams &P, const float *__restrict__ sG, LbsState &st, float &s0,
                                        float &s1, float &s2, float &S) {
  while (st.todo) lbs_round(P, sG, st);
  const float inv = 1.f / fmaxf(st.sum, kEpsW);
  s0 = st.n0 * inv;
  s1 = st.n1 * inv;
  s2 = st.n2 * inv;
  S = st.sum;
}

// Fractions of the point in level l's cell and the level's grid size (as in hash_cell).
struct LevelCell {
  uint32_t i0, i1, i2, N;
  float f0, f1, f2;
};

__device__ __forceinline__ LevelCell level_cell(const FieldParams &P, int l, float p0, float p1, float p2) {
  LevelCell c;
  c.N = P.level_res[l];
  const float fn = (float)c.N;
  const float q0 = p0 * fn, q1 = p1 * fn, q2 = p2 * fn;
  const float a0 = fminf(floorf(q0), fn - 1.f), a1 = fminf(floorf(q1), fn - 1.f), a2 = fminf(floorf(q2), fn - 1.f);
  c.f0 = q0 - a0;
  c.f1 = q1 - a1;
  c.f2 = q2 - a2;
  c.i0 = (uint32_t)a0;
  c.i1 = (uint32_t)a1;
  c.i2 = (uint32_t)a2;
  return c;
}

// The eight packed corners of a level: two 16-byte corner blocks (dense) or eight hashed slots.
template <bool DENSE>
__device__ __forceinline__ void level_load(const FieldParams &P, int l, const LevelCell &c, uint32_t (&v)[8]) {
  if (DENSE) {
    const uint4 *q = P.dense_quad + P.dq_off[l] + ((size_t)c.i2 * c.N + c.i1) * c.N + c.i0;
    const uint4 lo = __ldg(q), hi = __ldg(q + (size_t)c.N * c.N);
    v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
    v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
  } else {
    const uint32_t *t = reinterpret_cast<const uint32_t *>(P.table16) + (size_t)l * ((size_t)P.T_mask + 1);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t x = c.i0 + (k & 1), y = c.i1 + ((k >> 1) & 1), z = c.i2 + (k >> 2);
      v[k] = __ldg(t + ((x ^ (y * kPrimeY) ^ (z * kPrimeZ)) & P.T_mask));
    }
  }
}

// Packed f16 pair lerp a + f (b - a), both halves.
__device__ __forceinline__ uint32_t lerp_h2(uint32_t a, uint32_t b, uint32_t f) {
  uint32_t d;
  asm("{\n.reg .b32 t;\nsub.rn.f16x2 t, %2, %1;\nfma.rn.f16x2 %0, %3, t, %1;\n}\n" : "=r"(d) : "r"(a), "r"(b), "r"(f));
  return d;
}

__device__ __forceinline__ uint32_t f16x2_bcast(float f) {
  uint32_t d;
  asm("cvt.rn.f16x2.f32 %0, %1, %1;" : "=r"(d) : "f"(f));
  return d;
}

// A level's two features at the point: trilinear interpolation of the eight packed corners as
// seven packed lerps, then the pair in the MLP's operand type (0 outside the box).
template <typename T>
__device__ __forceinline__ uint32_t level_sum(const LevelCell &c, const uint32_t (&v)[8], bool inside) {
  const uint32_t fx = f16x2_bcast(c.f0), fy = f16x2_bcast(c.f1), fz = f16x2_bcast(c.f2);
  const uint32_t a = lerp_h2(v[0], v[1], fx), b = lerp_h2(v[2], v[3], fx);
  const uint32_t e = lerp_h2(v[4], v[5], fx), g = lerp_h2(v[6], v[7], fx);
  const uint32_t r = lerp_h2(lerp_h2(a, b, fy), lerp_h2(e, g, fy), fz);
  if (!inside) return 0u;
  if constexpr (TcFmt<T>::value == 0) return r;   // f16 operands (and the fp8 tier, which scales the pair)
  else {
    const float2 f = h2f2(r);
    return pack2<T>(f.x, f.y);
  }
}

// Levels l .. l + NL - 1 (each dense or hashed; the levels below n_dense are dense): every corner
// load is issued before any sum.
template <typename T, int NL, typename Emit>
__device__ __forceinline__ void level_group(const FieldParams &P, int l, int n_dense, float p0, float p1, float p2,
                                            bool inside, Emit &emit) {
  LevelCell c[NL];
  uint32_t v[NL][8];
#pragma unroll
  for (int q = 0; q < NL; ++q) {
    c[q] = level_cell(P, l + q, p0, p1, p2);
    if (l + q < n_dense)
      level_load<true>(P, l + q, c[q], v[q]);
    else
      level_load<false>(P, l + q, c[q], v[q]);
  }
#pragma unroll
  for (int q = 0; q < NL; ++q) emit(l + q, level_sum<T>(c[q], v[q], inside));
}

// Whether hash_encode_f16_grouped applies: the f16 table, and dense levels (if any) that form a
// prefix of the levels and have their corner blocks.
__device__ __forceinline__ bool grouped_apply(const FieldParams &P) {
  const uint32_t dm = P.dense_mask;
  return P.use_f16_table && (dm & (dm + 1u)) == 0u && (dm == 0u || P.dense_quad != nullptr);
}

// Hash encoding of the clamped box coordinate p with the f16 table and the dense levels'
// corner blocks (grouped_apply), four levels per step; emit(l, packed) receives each level's
// packed feature pair (0 outside the box) in increasing level order.
template <typename T, typename Emit>
__device__ __forceinline__ void hash_encode_f16_grouped(const FieldParams &P, float p0, float p1, float p2,
                                                        bool inside, Emit emit) {
  const int L = P.L;
  int n_dense = 0;
  while (n_dense < L && ((P.dense_mask >> n_dense) & 1u)) ++n_dense;
  int l = 0;
#pragma unroll 1
  for (; l + 4 <= L; l += 4) level_group<T, 4>(P, l, n_dense, p0, p1, p2, inside, emit);
  if (l + 2 <= L) {
    level_group<T, 2>(P, l, n_dense, p0, p1, p2, inside, emit);
    l += 2;
  }
  if (l < L) level_group<T, 1>(P, l, n_dense, p0, p1, p2, inside, emit);
}

}  // namespace nr
