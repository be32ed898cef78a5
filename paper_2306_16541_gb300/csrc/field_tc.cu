// field_tc.cu -- the per-sample field with both MLPs on the tensor cores
// (bf16 or f16 operands, float32 accumulation).
//
// Work split: each warp owns a tile of 32 samples.  The gather-heavy steps
// (inverse-LBS warp, positional encoding, hash encoding) run one sample per
// lane in float32; their results are written as one bf16/f16 row per sample
// into the warp's shared-memory tile.  The MLP layers then run as warp-level
// m16n8k16 MMAs over the 32 x 64 activation block: the accumulator fragments
// of one layer are re-packed in registers as the next layer's A operand, so
// hidden activations never leave the register file; weights are staged once
// per block in shared memory ([out][in] rows padded for conflict-free
// ldmatrix) and biases stay float32.  The outputs (x_res, raw MLP outputs)
// return to their sample's lane through a small shared-memory buffer.
#include "field.cuh"
#include "render.cuh"

namespace nr {

constexpr int kTcThreads = 512;
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kGamRow = kResGammaPad + 8;   // 56: gamma tile row stride (elements)
constexpr int kEncRow = kMlpIn + 8;         // 40: encoding tile row stride (elements)

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

// The MLP phase runs one 16-row m-tile of the warp's 32 samples at a time, so
// only one tile's accumulators (32 floats) and A fragments (16 registers) are
// live; the two tiles reuse the same weight fragments from shared memory.

// A fragments of rows m0 .. m0+15 of a row-major [32][lda] tile, K = 16 KT.
template <int KT, typename T>
__device__ __forceinline__ void load_a(const T *A, int lda, int m0, uint32_t (&a)[KT][4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int kt = 0; kt < KT; ++kt) ldsm_x4(a[kt], A + (m0 + (lane & 15)) * lda + kt * 16 + (lane >> 4) * 8);
}

// acc[nt] initialised with the bias of columns nt*8 + 2t, +1.
template <int NT>
__device__ __forceinline__ void init_bias(const float *bias, float (&acc)[NT][4]) {
  const int t = threadIdx.x & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const float b0 = bias[nt * 8 + 2 * t], b1 = bias[nt * 8 + 2 * t + 1];
    acc[nt][0] = b0;
    acc[nt][1] = b1;
    acc[nt][2] = b0;
    acc[nt][3] = b1;
  }
}

// acc += A[16 x 16KT] * W^T, W row-major [8NT][ldw] (rows = outputs), columns k0 .. k0 + 16KT.
template <typename T, int KT, int NT>
__device__ __forceinline__ void mma_block(const uint32_t (&a)[KT][4], const T *W, int ldw, int k0,
                                          float (&acc)[NT][4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int kt = 0; kt < KT; ++kt) {
    if constexpr (NT == 1) {
      uint32_t b0, b1;
      ldsm_x2(b0, b1, W + (lane & 7) * ldw + k0 + kt * 16 + ((lane >> 3) & 1) * 8);
      TcOps<T>::mma(acc[0], a[kt], b0, b1);
    } else {
#pragma unroll
      for (int np = 0; np < NT / 2; ++np) {
        uint32_t b[4];
        const int m = lane >> 3, r = lane & 7;
        ldsm_x4(b, W + (np * 16 + (m >> 1) * 8 + r) * ldw + k0 + kt * 16 + (m & 1) * 8);
        TcOps<T>::mma(acc[2 * np], a[kt], b[0], b[1]);
        TcOps<T>::mma(acc[2 * np + 1], a[kt], b[2], b[3]);
      }
    }
  }
}

// ReLU of a 16 x 64 accumulator block, re-packed as the A operand (K = 64) of the next layer.
template <typename T>
__device__ __forceinline__ void relu_to_a(const float (&acc)[8][4], uint32_t (&a)[4][4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float *c0 = acc[2 * j], *c1 = acc[2 * j + 1];
    a[j][0] = TcOps<T>::pack(fmaxf(c0[0], 0.f), fmaxf(c0[1], 0.f));
    a[j][1] = TcOps<T>::pack(fmaxf(c0[2], 0.f), fmaxf(c0[3], 0.f));
    a[j][2] = TcOps<T>::pack(fmaxf(c1[0], 0.f), fmaxf(c1[1], 0.f));
    a[j][3] = TcOps<T>::pack(fmaxf(c1[2], 0.f), fmaxf(c1[3], 0.f));
  }
}

// Writes columns 0..3 of a 16 x 8 accumulator block to rows m0.. of out[32][4] (float).
__device__ __forceinline__ void store_out4(const float (&acc)[1][4], int m0, float *out) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  if (t < 2) {
    out[(m0 + g) * 4 + 2 * t] = acc[0][0];
    out[(m0 + g) * 4 + 2 * t + 1] = acc[0][1];
    out[(m0 + g + 8) * 4 + 2 * t] = acc[0][2];
    out[(m0 + g + 8) * 4 + 2 * t + 1] = acc[0][3];
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

template <typename T, int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) field_tc_kernel(FieldParams P, const float4 *__restrict__ in,
                                                                 uint32_t n_fixed, const uint32_t *__restrict__ n_dev,
                                                                 float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  T *sW = reinterpret_cast<T *>(smem);                                   // tensor-core weights
  float *sBias = reinterpret_cast<float *>(smem + ((P.tlay.total * sizeof(T) + 15) & ~size_t(15)));
  const TcBias bl = tc_bias_layout(P.hidden);
  float *sG = sBias + ((bl.total + 3) & ~3);
  // per warp: one [32][kGamRow] tile that holds gamma(x_skel) for the residual MLP and,
  // once that is done, the hash encoding (row stride kEncRow) for the canonical MLP
  T *sGam = reinterpret_cast<T *>(sG + kBones * 12);                     // [warps][32][kGamRow]
  float *sOut = reinterpret_cast<float *>(sGam + kTcWarps * 32 * kGamRow);  // [warps][32][4]

  {  // stage weights, biases and the pose's bone transforms
    const int4 *src = reinterpret_cast<const int4 *>(P.tc_blob);
    int4 *dst = reinterpret_cast<int4 *>(sW);
    const int n16 = (int)(P.tlay.total * sizeof(T) / 16);
    for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
    auto copyb = [&](int dsto, const float *s, int n, int npad) {
      for (int i = threadIdx.x; i < npad; i += blockDim.x) sBias[dsto + i] = i < n ? s[i] : 0.f;
    };
    copyb(bl.r1, P.bias1, kWidth, kWidth);
    copyb(bl.r2, P.blob + P.lay.r2b, kWidth, kWidth);
    copyb(bl.r3, P.blob + P.lay.r3b, kWidth, kWidth);
    copyb(bl.r4, P.blob + P.lay.r4b, kWidth, kWidth);
    copyb(bl.r5, P.blob + P.lay.r5b, 3, 8);
    copyb(bl.c0, P.blob + P.lay.c0b, kWidth, kWidth);
    for (int l = 0; l < P.hidden - 1; ++l) copyb(bl.c0 + kWidth * (l + 1), P.blob + P.lay.chb[l], kWidth, kWidth);
    copyb(bl.cl, P.blob + P.lay.clb, 4, 8);
    for (int i = threadIdx.x; i < kBones * 12; i += blockDim.x) sG[i] = P.G[i];
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T *gam = sGam + warp * 32 * kGamRow;
  T *enc = gam;
  float *o4 = sOut + warp * 32 * 4;
  const uint32_t n = n_dev ? *n_dev : n_fixed;
  const uint32_t n_tiles = (n + 31) / 32;
  for (uint32_t tile = blockIdx.x * kTcWarps + warp; tile < n_tiles; tile += gridDim.x * kTcWarps) {
    const uint32_t j = tile * 32 + lane;
    const bool valid = j < n;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, delta = 0.f;
    if (valid) {
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
    }
    float s0, s1, s2, S;
    lbs_warp(P, sG, x0, x1, x2, s0, s1, s2, S);
    float f0 = s0, f1 = s1, f2 = s2;
    if (P.res_enabled) {
      {  // gamma(x_skel) as one row of the warp's tile
        float g[kResGammaPad];
        const float h0 = (s0 - P.box_c[0]) * P.box_ih[0];
        const float h1 = (s1 - P.box_c[1]) * P.box_ih[1];
        const float h2 = (s2 - P.box_c[2]) * P.box_ih[2];
        g[0] = h0;
        g[1] = h1;
        g[2] = h2;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float sc = (float)(1 << k);
          float sa, ca, sb, cb, sd, cd;
          sincospif(sc * h0, &sa, &ca);
          sincospif(sc * h1, &sb, &cb);
          sincospif(sc * h2, &sd, &cd);
          const float w = (k < P.res_freqs) ? P.hann[k] : 0.f;
          g[3 + 6 * k + 0] = w * sa;
          g[3 + 6 * k + 1] = w * sb;
          g[3 + 6 * k + 2] = w * sd;
          g[3 + 6 * k + 3] = w * ca;
          g[3 + 6 * k + 4] = w * cb;
          g[3 + 6 * k + 5] = w * cd;
        }
#pragma unroll
        for (int k = 39; k < kResGammaPad; ++k) g[k] = 0.f;
        uint32_t *row = reinterpret_cast<uint32_t *>(gam + lane * kGamRow);
#pragma unroll
        for (int k = 0; k < kResGammaPad / 2; ++k) row[k] = TcOps<T>::pack(g[2 * k], g[2 * k + 1]);
      }
      __syncwarp();
#pragma unroll 1
      for (int m0 = 0; m0 < 32; m0 += 16) {
        uint32_t ag[3][4], a[4][4];
        float acc[8][4];
        load_a<3>(gam, kGamRow, m0, ag);
        init_bias(sBias + bl.r1, acc);
        mma_block<T, 3, 8>(ag, sW + P.tlay.r1, kTcRow, 0, acc);
        relu_to_a<T>(acc, a);
        init_bias(sBias + bl.r2, acc);
        mma_block<T, 4, 8>(a, sW + P.tlay.r2, kTcRow, 0, acc);
        relu_to_a<T>(acc, a);
        init_bias(sBias + bl.r3, acc);
        mma_block<T, 4, 8>(a, sW + P.tlay.r3, kTcRow, 0, acc);
        relu_to_a<T>(acc, a);
        init_bias(sBias + bl.r4, acc);                               // layer 4 sees [h3, gamma]
        mma_block<T, 4, 8>(a, sW + P.tlay.r4, kTcRowWide, 0, acc);
        mma_block<T, 3, 8>(ag, sW + P.tlay.r4, kTcRowWide, kWidth, acc);
        relu_to_a<T>(acc, a);
        float acc5[1][4];
        init_bias(sBias + bl.r5, acc5);
        mma_block<T, 4, 1>(a, sW + P.tlay.r5, kTcRow, 0, acc5);
        store_out4(acc5, m0, o4);
      }
      __syncwarp();
      f0 += o4[lane * 4 + 0];
      f1 += o4[lane * 4 + 1];
      f2 += o4[lane * 4 + 2];
      __syncwarp();
    }
    // canonical field: hash encoding (float32) -> one row of the encoding tile
    bool inside;
    {
      float p0 = (f0 - P.bmin[0]) * P.inv_box[0];
      float p1 = (f1 - P.bmin[1]) * P.inv_box[1];
      float p2 = (f2 - P.bmin[2]) * P.inv_box[2];
      inside = p0 >= 0.f && p0 <= 1.f && p1 >= 0.f && p1 <= 1.f && p2 >= 0.f && p2 <= 1.f;
      p0 = fminf(fmaxf(p0, 0.f), 1.f);
      p1 = fminf(fmaxf(p1, 0.f), 1.f);
      p2 = fminf(fmaxf(p2, 0.f), 1.f);
      uint32_t *row = reinterpret_cast<uint32_t *>(enc + lane * kEncRow);
#pragma unroll
      for (int l = 0; l < kMaxLevels; ++l) {
        float fa = 0.f, fb = 0.f;
        if (l < P.L) {
          HashCell c;
          hash_cell(P, l, p0, p1, p2, c);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float2 v = table_read(P, l, c.idx[k]);
            fa = fmaf(c.w[k], v.x, fa);
            fb = fmaf(c.w[k], v.y, fb);
          }
        }
        row[l] = inside ? TcOps<T>::pack(fa, fb) : 0u;
      }
    }
    __syncwarp();
#pragma unroll 1
    for (int m0 = 0; m0 < 32; m0 += 16) {
      uint32_t ae[2][4], a[4][4];
      float acc[8][4];
      load_a<2>(enc, kEncRow, m0, ae);
      init_bias(sBias + bl.c0, acc);
      mma_block<T, 2, 8>(ae, sW + P.tlay.c0, kTcRow, 0, acc);
      relu_to_a<T>(acc, a);
      for (int l = 0; l < P.hidden - 1; ++l) {
        init_bias(sBias + bl.c0 + kWidth * (l + 1), acc);
        mma_block<T, 4, 8>(a, sW + P.tlay.ch[l], kTcRow, 0, acc);
        relu_to_a<T>(acc, a);
      }
      float acco[1][4];
      init_bias(sBias + bl.cl, acco);
      mma_block<T, 4, 1>(a, sW + P.tlay.cl, kTcRow, 0, acco);
      store_out4(acco, m0, o4);
    }
    __syncwarp();
    if (valid) {
      const float cr = sigmoidf_(o4[lane * 4 + 0]), cg = sigmoidf_(o4[lane * 4 + 1]);
      const float cb = sigmoidf_(o4[lane * 4 + 2]), sigma = softplusf_(o4[lane * 4 + 3]);
      if (MODE == kModeRender) {
        const float al = inside ? (1.f - __expf(-sigma * delta)) * fminf(S, 1.f) : 0.f;
        reinterpret_cast<float4 *>(out)[j] = make_float4(cr, cg, cb, al);
      } else {
        float *q = out + (size_t)NR_QUERY_STRIDE * j;
        q[0] = s0; q[1] = s1; q[2] = s2; q[3] = S;
        q[4] = f0; q[5] = f1; q[6] = f2; q[7] = inside ? 1.f : 0.f;
        q[8] = cr; q[9] = cg; q[10] = cb; q[11] = sigma;
      }
    }
    __syncwarp();
  }
}

template <typename T>
static size_t tc_smem(const FieldParams &P) {
  const TcBias bl = tc_bias_layout(P.hidden);
  size_t b = ((P.tlay.total * sizeof(T) + 15) & ~size_t(15));
  b += sizeof(float) * (((bl.total + 3) & ~3) + kBones * 12);
  b += sizeof(T) * (size_t)kTcWarps * 32 * kGamRow;
  b += sizeof(float) * (size_t)kTcWarps * 32 * 4;
  return b;
}

template <typename T, int MODE>
static nr_status launch_tc(const FieldParams &P, const float4 *in, uint32_t n_fixed, const uint32_t *n_dev, float *out,
                           int device, cudaStream_t st) {
  const size_t smem = tc_smem<T>(P);
  NR_CHECK_CUDA(cudaFuncSetAttribute(field_tc_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  field_tc_kernel<T, MODE><<<num_sms(device), kTcThreads, smem, st>>>(P, in, n_fixed, n_dev, out);
  NR_CHECK_CUDA(cudaGetLastError());
  return NR_OK;
}

nr_status launch_field_tc(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                          const uint32_t *n_dev, float *out, int device, cudaStream_t st) {
  if (mlp_dtype == NR_BF16)
    return mode == kModeRender ? launch_tc<__nv_bfloat16, kModeRender>(P, in, n_fixed, n_dev, out, device, st)
                               : launch_tc<__nv_bfloat16, kModeQuery>(P, in, n_fixed, n_dev, out, device, st);
  return mode == kModeRender ? launch_tc<__half, kModeRender>(P, in, n_fixed, n_dev, out, device, st)
                             : launch_tc<__half, kModeQuery>(P, in, n_fixed, n_dev, out, device, st);
}

}  // namespace nr
