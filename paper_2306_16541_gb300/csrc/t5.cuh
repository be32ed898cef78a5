// t5.cuh -- pieces shared by the tcgen05 field kernels (field_t5.cu, field_ws.cu):
// the layout of the swizzled K-major weight blob, shared-memory matrix and
// instruction descriptors of tcgen05.mma kind::f16, the commit to an mbarrier,
// and bf16/f16 packing.
#pragma once

#include "common.cuh"

namespace nr {

// Byte offsets of the swizzled weight blob (1024-byte aligned matrices of 128-byte rows).
struct T5Layout {
  int r1, r2, r3, r4h, r4g, r5, c0, ch[kMaxHidden], cl, total;
};

__host__ __device__ inline T5Layout t5_layout(int hidden) {
  T5Layout t{};
  int o = 0;
  t.r1 = o; o += 64 * 128;
  t.r2 = o; o += 64 * 128;
  t.r3 = o; o += 64 * 128;
  t.r4h = o; o += 64 * 128;
  t.r4g = o; o += 64 * 128;
  t.r5 = o; o += 16 * 128;
  t.c0 = o; o += 64 * 128;
  for (int l = 0; l < hidden - 1; ++l) { t.ch[l] = o; o += 64 * 128; }
  t.cl = o; o += 16 * 128;
  t.total = o;
  return t;
}

// Byte offset of element (row r, column k) of a 64-column 16-bit K-major tile, 128-byte swizzle.
__host__ __device__ inline int sw128(int r, int k) { return r * 128 + (((k >> 3) ^ (r & 7)) << 4) + ((k & 7) << 1); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: 128-byte swizzle, K-major, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t t5_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::f16: f32 accumulate, A/B bf16 (fmt 1) or f16 (fmt 0), K-major, M = 128.
__host__ __device__ inline uint32_t t5_idesc(int n, int fmt) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void t5_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

template <typename T>
struct TcFmt;
template <>
struct TcFmt<__nv_bfloat16> {
  static constexpr int value = 1;
};
template <>
struct TcFmt<__half> {
  static constexpr int value = 0;
};

template <typename T>
__device__ __forceinline__ uint32_t pack2(float a, float b);
template <>
__device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&v);
}
template <>
__device__ __forceinline__ uint32_t pack2<__half>(float a, float b) {
  __half2 v = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&v);
}

}  // namespace nr
