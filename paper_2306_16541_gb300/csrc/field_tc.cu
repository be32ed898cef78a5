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
#include "mma.cuh"
#include "render.cuh"

namespace nr {

// Threads per block for MT m-tiles per weight-fragment read (one block per SM).
template <int MT>
struct TcCfg {
  static constexpr int threads = MT == 1 ? 640 : 384;
  static constexpr int warps = threads / 32;
};
constexpr int kGamRow = kResGammaPad + 8;   // 56: gamma tile row stride (elements)
constexpr int kEncRow = kMlpIn + 8;         // 40: encoding tile row stride (elements)

template <typename T, int MODE, int MT>
__global__ void __launch_bounds__(TcCfg<MT>::threads, 1) field_tc_kernel(FieldParams P, const float4 *__restrict__ in,
                                                                 uint32_t n_fixed, const uint32_t *__restrict__ n_dev,
                                                                 float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  T *sW = reinterpret_cast<T *>(smem);                                   // tensor-core weights
  float *sBias = reinterpret_cast<float *>(smem + ((P.tlay.total * sizeof(T) + 15) & ~size_t(15)));
  const TcBias bl = tc_bias_layout(P.hidden);
  float *sG = sBias + ((bl.total + 3) & ~3);
  // per warp: one [32][kGamRow] tile that holds gamma(x_skel) for the residual MLP and,
  // once that is done, the hash encoding (row stride kEncRow) for the canonical MLP
  T *sGam = reinterpret_cast<T *>(sG + kPoseSmem);                       // [warps][32][kGamRow]
  float *sOut = reinterpret_cast<float *>(sGam + TcCfg<MT>::warps * 32 * kGamRow);  // [warps][32][4]

  const float *sBox = nullptr;
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
    sBox = stage_pose(P, sG, threadIdx.x, blockDim.x);
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T *gam = sGam + warp * 32 * kGamRow;
  T *enc = gam;
  float *o4 = sOut + warp * 32 * 4;
  const uint32_t n = n_dev ? *n_dev : n_fixed;
  const uint32_t n_tiles = (n + 31) / 32;
  for (uint32_t tile = blockIdx.x * TcCfg<MT>::warps + warp; tile < n_tiles; tile += gridDim.x * TcCfg<MT>::warps) {
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
    lbs_warp(P, sG, x0, x1, x2, s0, s1, s2, S, sBox);
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
      for (int m0 = 0; m0 < 32; m0 += 16 * MT) {
        uint32_t ag[MT][3][4], a[MT][4][4];
        float acc[MT][8][4];
        load_a<3, MT>(gam, kGamRow, m0, ag);
        init_bias(sBias + bl.r1, acc);
        mma_block<T, 3, 8, MT>(ag, sW + P.tlay.r1, kTcRow, 0, acc);
        relu_to_a<T, MT>(acc, a);
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {   // layers 2 and 3 share one copy of the code
          init_bias(sBias + (q ? bl.r3 : bl.r2), acc);
          mma_block<T, 4, 8, MT>(a, sW + (q ? P.tlay.r3 : P.tlay.r2), kTcRow, 0, acc);
          relu_to_a<T, MT>(acc, a);
        }
        init_bias(sBias + bl.r4, acc);                               // layer 4 sees [h3, gamma]
        mma_block<T, 4, 8, MT>(a, sW + P.tlay.r4, kTcRowWide, 0, acc);
        mma_block<T, 3, 8, MT>(ag, sW + P.tlay.r4, kTcRowWide, kWidth, acc);
        relu_to_a<T, MT>(acc, a);
        float acc5[MT][1][4];
        init_bias(sBias + bl.r5, acc5);
        mma_block<T, 4, 1, MT>(a, sW + P.tlay.r5, kTcRow, 0, acc5);
        store_out4<MT>(acc5, m0, o4);
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
      // one copy of the level body (a runtime loop keeps the kernel's code small)
#pragma unroll 1
      for (int l = 0; l < P.L; ++l) {
        float fa, fb;
        hash_level(P, l, p0, p1, p2, fa, fb);
        row[l] = inside ? TcOps<T>::pack(fa, fb) : 0u;
      }
      for (int l = P.L; l < kMaxLevels; ++l) row[l] = 0u;
    }
    __syncwarp();
#pragma unroll 1
    for (int m0 = 0; m0 < 32; m0 += 16 * MT) {
      uint32_t ae[MT][2][4], a[MT][4][4];
      float acc[MT][8][4];
      load_a<2, MT>(enc, kEncRow, m0, ae);
      init_bias(sBias + bl.c0, acc);
      mma_block<T, 2, 8, MT>(ae, sW + P.tlay.c0, kTcRow, 0, acc);
      relu_to_a<T, MT>(acc, a);
      for (int l = 0; l < P.hidden - 1; ++l) {
        init_bias(sBias + bl.c0 + kWidth * (l + 1), acc);
        mma_block<T, 4, 8, MT>(a, sW + P.tlay.ch[l], kTcRow, 0, acc);
        relu_to_a<T, MT>(acc, a);
      }
      float acco[MT][1][4];
      init_bias(sBias + bl.cl, acco);
      mma_block<T, 4, 1, MT>(a, sW + P.tlay.cl, kTcRow, 0, acco);
      store_out4<MT>(acco, m0, o4);
    }
    __syncwarp();
    if (valid) {
      const float cr = sigmoidf_(o4[lane * 4 + 0]), cg = sigmoidf_(o4[lane * 4 + 1]);
      const float cb = sigmoidf_(o4[lane * 4 + 2]), sigma = softplusf_(o4[lane * 4 + 3]);
      if (MODE == kModeRender) {
        const float al = inside ? -expm1f(-sigma * delta) * fminf(S, 1.f) : 0.f;
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

template <typename T, int MT>
static size_t tc_smem(const FieldParams &P) {
  const TcBias bl = tc_bias_layout(P.hidden);
  size_t b = ((P.tlay.total * sizeof(T) + 15) & ~size_t(15));
  b += sizeof(float) * (((bl.total + 3) & ~3) + kPoseSmem);
  b += sizeof(T) * (size_t)TcCfg<MT>::warps * 32 * kGamRow;
  b += sizeof(float) * (size_t)TcCfg<MT>::warps * 32 * 4;
  return b;
}

template <typename T, int MODE, int MT>
static nr_status launch_tc(const FieldParams &P, const float4 *in, uint32_t n_fixed, const uint32_t *n_dev, float *out,
                           int device, cudaStream_t st) {
  const size_t smem = tc_smem<T, MT>(P);
  NR_CHECK_CUDA(
      cudaFuncSetAttribute(field_tc_kernel<T, MODE, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  field_tc_kernel<T, MODE, MT><<<num_sms(device), TcCfg<MT>::threads, smem, st>>>(P, in, n_fixed, n_dev, out);
  NR_CHECK_CUDA(cudaGetLastError());
  return NR_OK;
}

template <typename T>
static nr_status launch_tc_t(const FieldParams &P, int mode, const float4 *in, uint32_t n_fixed, const uint32_t *n_dev,
                             float *out, int device, cudaStream_t st, int mt) {
  if (mt == 2)
    return mode == kModeRender ? launch_tc<T, kModeRender, 2>(P, in, n_fixed, n_dev, out, device, st)
                               : launch_tc<T, kModeQuery, 2>(P, in, n_fixed, n_dev, out, device, st);
  return mode == kModeRender ? launch_tc<T, kModeRender, 1>(P, in, n_fixed, n_dev, out, device, st)
                             : launch_tc<T, kModeQuery, 1>(P, in, n_fixed, n_dev, out, device, st);
}

nr_status launch_field_tc(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                          const uint32_t *n_dev, float *out, int device, cudaStream_t st, int mt) {
  if (mlp_dtype == NR_BF16) return launch_tc_t<__nv_bfloat16>(P, mode, in, n_fixed, n_dev, out, device, st, mt);
  return launch_tc_t<__half>(P, mode, in, n_fixed, n_dev, out, device, st, mt);
}

}  // namespace nr
