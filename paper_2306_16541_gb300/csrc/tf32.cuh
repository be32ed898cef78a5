// tf32.cuh -- float32-accurate warp-level layers on the tensor cores, shared by the
// training kernels and the float32 render tier on the tensor cores.
//
// Each float32 operand is split into two TF32 parts (x = hi + lo, both exact in TF32); a
// product x y is taken as hi_x hi_y + hi_x lo_y + lo_x hi_y (three m16n8k8 MMAs, the dropped
// lo_x lo_y term lies below float32 rounding), so the layers keep float32 accuracy.  Layer
// inputs and outputs live in per-thread columns of a scratch buffer (row r of sample s at
// wcol[r * stride + s]); weights come from a shared-memory copy whose 64-wide rows are
// padded against bank conflicts.
#pragma once

#include "common.cuh"

namespace nr {

// The shared-memory copy of the float32 blob used by the TF32 layers: each layer [in][out] with the
// rows of 64-output layers padded to kPadRow floats, so that the tensor-core fragments of
// W^T (8 rows x 4 columns per load) fall in distinct banks.
constexpr int kPadRow = 68;
constexpr int kMaxSeg = 2 * (6 + kMaxHidden);
struct PadSeg {
  int src, dst, rows, cols, dstride;
};
struct PadLay {
  int r1, r2, r3, r4, r5, c0, ch[kMaxHidden], cl;
  int r1b, r2b, r3b, r4b, r5b, c0b, chb[kMaxHidden], clb;
  int n_seg;
  PadSeg seg[kMaxSeg];
  int total;   // floats
};

inline PadLay pad_layout(const BlobLayout &b, int H) {
  PadLay p{};
  int o = 0;
  auto add = [&](int src, int rows, int cols) {
    PadSeg &g = p.seg[p.n_seg++];
    g.src = src;
    g.dst = o;
    g.rows = rows;
    g.cols = cols;
    g.dstride = cols == kWidth ? kPadRow : cols;
    o += (rows * g.dstride + 3) & ~3;
    return g.dst;
  };
  p.r1 = add(b.r1, kResGammaPad, kWidth);
  p.r1b = add(b.r1b, 1, kWidth);
  p.r2 = add(b.r2, kWidth, kWidth);
  p.r2b = add(b.r2b, 1, kWidth);
  p.r3 = add(b.r3, kWidth, kWidth);
  p.r3b = add(b.r3b, 1, kWidth);
  p.r4 = add(b.r4, kWidth + kResGammaPad, kWidth);
  p.r4b = add(b.r4b, 1, kWidth);
  p.r5 = add(b.r5, kWidth, 4);
  p.r5b = add(b.r5b, 1, 4);
  p.c0 = add(b.c0, kMlpIn, kWidth);
  p.c0b = add(b.c0b, 1, kWidth);
  for (int l = 0; l < H - 1; ++l) {
    p.ch[l] = add(b.ch[l], kWidth, kWidth);
    p.chb[l] = add(b.chb[l], 1, kWidth);
  }
  p.cl = add(b.cl, kWidth, 4);
  p.clb = add(b.clb, 1, 4);
  p.total = o;
  return p;
}

// TF32 with an error term: x = hi + lo, both exactly representable in tf32; a product
// x y = hi_x hi_y + hi_x lo_y + lo_x hi_y up to a term below float32's rounding, so three
// tensor-core products keep float32 accuracy ("3xTF32").
__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// The forward of one layer for the warp's 32 samples on the tensor cores:
//   out[s][o] = act(sum_i W[o][i] x[s][i] + bias)
// as C = W X^T with M = OUT (16-row tiles of outputs; rows past OUT are zero), N = the 32
// samples, K = IN + IN2 inputs (x rows r_in.. then r_in2.. for a second input segment, i.e.
// rows IN.. of W^T); m16n8k8 TF32 MMAs, three per step.  bias is b[o], or fb[frame][o] with
// each sample's frame taken from the lane that owns the sample (fr).  Outputs past OUT are not
// written.  Every lane of the warp must take part.
template <int OUT, int IN, int IN2>
__device__ __forceinline__ void warp_fwd(const float *__restrict__ Wt, int rs, float *wcol, int stride, int r_in,
                                         int r_in2, const float *__restrict__ b, const float *__restrict__ fb, int fr,
                                         bool relu, int r_out) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  constexpr int MT = (OUT + 15) / 16, KS = (IN + IN2) / 8;
  float acc[MT][4][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
#pragma unroll 1
  for (int ks = 0; ks < KS; ++ks) {
    const int i0 = 8 * ks + t, i1 = i0 + 4;
    const int x0 = i0 < IN ? r_in + i0 : r_in2 + (i0 - IN), x1 = i1 < IN ? r_in + i1 : r_in2 + (i1 - IN);
    uint32_t bh[4][2], bl[4][2];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      tf32_split(wcol[x0 * stride + 8 * n + g], bh[n][0], bl[n][0]);
      tf32_split(wcol[x1 * stride + 8 * n + g], bh[n][1], bl[n][1]);
    }
    const float *w0 = Wt + i0 * rs, *w1 = Wt + i1 * rs;
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const int o0 = 16 * m + g, o8 = o0 + 8;
      uint32_t ah[4], al[4];
      tf32_split(o0 < OUT ? w0[o0] : 0.f, ah[0], al[0]);
      tf32_split(o8 < OUT ? w0[o8] : 0.f, ah[1], al[1]);
      tf32_split(o0 < OUT ? w1[o0] : 0.f, ah[2], al[2]);
      tf32_split(o8 < OUT ? w1[o8] : 0.f, ah[3], al[3]);
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        mma_tf32(acc[m][n], al, bh[n]);
        mma_tf32(acc[m][n], ah, bl[n]);
        mma_tf32(acc[m][n], ah, bh[n]);
      }
    }
  }
  // acc[m][n] = C[16m + g][8n + 2t], C[16m + g][8n + 2t + 1], C[16m + g + 8][8n + 2t], C[16m + g + 8][8n + 2t + 1]
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const int s0 = 8 * n + 2 * t;
    const int f0 = __shfl_sync(0xffffffffu, fr, s0), f1 = __shfl_sync(0xffffffffu, fr, s0 + 1);
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = 16 * m + g + (q >= 2 ? 8 : 0), smp = s0 + (q & 1);
        if (o >= OUT) continue;
        float v = acc[m][n][q] + (fb ? fb[(size_t)((q & 1) ? f1 : f0) * kWidth + o] : b[o]);
        if (relu) v = fmaxf(v, 0.f);
        wcol[(r_out + o) * stride + smp] = v;
      }
  }
  __syncwarp();   // the next step reads these rows through other lanes
}

}  // namespace nr
