// mma.cuh -- warp-level tensor-core helpers (mma.sync, ldmatrix) shared by the
// bf16/f16 and fp8 field kernels.
#pragma once

#include <cuda_fp8.h>

#include "common.cuh"

namespace nr {

template <typename T>
struct TcOps;

template <>
struct TcOps<__nv_bfloat16> {
  static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
  }
  static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
  static __device__ __forceinline__ __nv_bfloat16 cvt(float v) { return __float2bfloat16_rn(v); }
};

template <>
struct TcOps<__half> {
  static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
  }
  static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
  static __device__ __forceinline__ __half cvt(float v) { return __float2half_rn(v); }
};

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldsm_x2(uint32_t &r0, uint32_t &r1, const void *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

// The MLP phase runs MT 16-row m-tiles of the warp's 32 samples per pass: with
// MT = 1 only one tile's accumulators (32 floats) and A fragments are live; with
// MT = 2 every weight fragment read from shared memory serves both tiles.

// A fragments of rows m0 + 16 mt .. of a row-major [32][lda] tile, K = 16 KT.
template <int KT, int MT, typename T>
__device__ __forceinline__ void load_a(const T *A, int lda, int m0, uint32_t (&a)[MT][KT][4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int kt = 0; kt < KT; ++kt)
      ldsm_x4(a[mt][kt], A + (m0 + 16 * mt + (lane & 15)) * lda + kt * 16 + (lane >> 4) * 8);
}

// acc[mt][nt] initialised with the bias of columns nt*8 + 2t, +1.
template <int NT, int MT>
__device__ __forceinline__ void init_bias(const float *bias, float (&acc)[MT][NT][4]) {
  const int t = threadIdx.x & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const float2 b = *reinterpret_cast<const float2 *>(bias + nt * 8 + 2 * t);
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      acc[mt][nt][0] = b.x;
      acc[mt][nt][1] = b.y;
      acc[mt][nt][2] = b.x;
      acc[mt][nt][3] = b.y;
    }
  }
}

// acc += A[16 MT x 16KT] * W^T, W row-major [8NT][ldw] (rows = outputs), columns k0 .. k0 + 16KT.
template <typename T, int KT, int NT, int MT>
__device__ __forceinline__ void mma_block(const uint32_t (&a)[MT][KT][4], const T *W, int ldw, int k0,
                                          float (&acc)[MT][NT][4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int kt = 0; kt < KT; ++kt) {
    if constexpr (NT == 1) {
      uint32_t b0, b1;
      ldsm_x2(b0, b1, W + (lane & 7) * ldw + k0 + kt * 16 + ((lane >> 3) & 1) * 8);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) TcOps<T>::mma(acc[mt][0], a[mt][kt], b0, b1);
    } else {
#pragma unroll
      for (int np = 0; np < NT / 2; ++np) {
        uint32_t b[4];
        const int m = lane >> 3, r = lane & 7;
        ldsm_x4(b, W + (np * 16 + (m >> 1) * 8 + r) * ldw + k0 + kt * 16 + (m & 1) * 8);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          TcOps<T>::mma(acc[mt][2 * np], a[mt][kt], b[0], b[1]);
          TcOps<T>::mma(acc[mt][2 * np + 1], a[mt][kt], b[2], b[3]);
        }
      }
    }
  }
}

// ReLU of a (16 MT) x 64 accumulator block, re-packed as the A operand (K = 64) of the next layer.
template <typename T, int MT>
__device__ __forceinline__ void relu_to_a(const float (&acc)[MT][8][4], uint32_t (&a)[MT][4][4]) {
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float *c0 = acc[mt][2 * j], *c1 = acc[mt][2 * j + 1];
      a[mt][j][0] = TcOps<T>::pack(fmaxf(c0[0], 0.f), fmaxf(c0[1], 0.f));
      a[mt][j][1] = TcOps<T>::pack(fmaxf(c0[2], 0.f), fmaxf(c0[3], 0.f));
      a[mt][j][2] = TcOps<T>::pack(fmaxf(c1[0], 0.f), fmaxf(c1[1], 0.f));
      a[mt][j][3] = TcOps<T>::pack(fmaxf(c1[2], 0.f), fmaxf(c1[3], 0.f));
    }
}

// Writes columns 0..3 of a (16 MT) x 8 accumulator block to rows m0.. of out[32][4] (float).
template <int MT>
__device__ __forceinline__ void store_out4(const float (&acc)[MT][1][4], int m0, float *out) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  if (t < 2) {
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const int r0 = m0 + 16 * mt + g;
      out[r0 * 4 + 2 * t] = acc[mt][0][0];
      out[r0 * 4 + 2 * t + 1] = acc[mt][0][1];
      out[(r0 + 8) * 4 + 2 * t] = acc[mt][0][2];
      out[(r0 + 8) * 4 + 2 * t + 1] = acc[mt][0][3];
    }
  }
}

// Float32 biases gathered from the float32 blob into one shared array.
struct TcBias {
  int r1, r2, r3, r4, r5, c0, ch[kMaxHidden], cl, total;
};

__host__ __device__ inline TcBias tc_bias_layout(int hidden) {
  TcBias b{};
  int o = 0;
  b.r1 = o; o += kWidth;
  b.r2 = o; o += kWidth;
  b.r3 = o; o += kWidth;
  b.r4 = o; o += kWidth;
  b.r5 = o; o += 8;
  b.c0 = o; o += kWidth;
  for (int l = 0; l < hidden - 1; ++l) { b.ch[l] = o; o += kWidth; }
  b.cl = o; o += 8;
  b.total = o;
  return b;
}

}  // namespace nr
