// field_tf32.cu -- the float32 tier on the tensor cores: the per-sample field (render and
// query modes) with both MLPs as warp-level layers at float32 accuracy (three TF32 products
// per step, tf32.cuh) instead of CUDA-core FMAs.
//
// Work split: each warp owns a tile of 32 samples.  The gathers (inverse-LBS warp, PE, hash
// encoding) run one sample per lane in float32 as in the CUDA-core kernel; every layer is a
// C = W X^T product over the tile (M = outputs, N = the 32 samples, K = inputs) on a padded
// shared-memory copy of the float32 weights; a sample's activations live in its thread's
// column of a global scratch buffer (L1/L2 resident), two 64-row buffers used in turn.
#include "field.cuh"
#include "render.cuh"
#include "tf32.cuh"

namespace nr {

// rows of a thread's scratch column
constexpr int kRowGam = 0;                         // gamma(x_skel)
constexpr int kRowA = kRowGam + kResGammaPad;      // hidden activations, two buffers in turn
constexpr int kRowB = kRowA + kWidth;
constexpr int kRowEnc = kRowB + kWidth;            // hash encoding
constexpr int kRowOut = kRowEnc + kMlpIn;          // the four outputs of either MLP
static_assert(kRowOut + 4 == kTf32Rows, "scratch rows");

template <int MODE>
__global__ void __launch_bounds__(kTf32Threads, 1) field_tf32_kernel(FieldParams P, PadLay PL,
                                                                     const float4 *__restrict__ in, uint32_t n_fixed,
                                                                     const uint32_t *__restrict__ n_dev,
                                                                     float *__restrict__ out) {
  extern __shared__ float4 smem4[];
  float *sW = reinterpret_cast<float *>(smem4);    // the weights in the padded layout PL
  float *sG = sW + ((PL.total + 3) & ~3);          // pose (and support boxes)
  float *sB1 = sG + kPoseSmem;                     // residual layer-1 bias with the pose folded in
  for (int q = 0; q < PL.n_seg; ++q) {
    const PadSeg &sg = PL.seg[q];
    for (int i = threadIdx.x; i < sg.rows * sg.cols; i += blockDim.x) {
      const int rr = i / sg.cols, cc = i - rr * sg.cols;
      sW[sg.dst + rr * sg.dstride + cc] = __ldg(P.blob + sg.src + i);
    }
  }
  const float *sBox = stage_pose(P, sG, threadIdx.x, blockDim.x);
  for (int i = threadIdx.x; i < kWidth; i += blockDim.x) sB1[i] = P.bias1[i];
  __syncthreads();

  const int stride = blockDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float *colbase = P.tf32_scratch + (size_t)blockIdx.x * kTf32Rows * stride;
  float *col = colbase + threadIdx.x;               // this thread's column
  float *wcol = colbase + warp * 32;                // the warp's column 0
  const int warps = blockDim.x >> 5;
  const uint32_t n = n_dev ? *n_dev : n_fixed;
  const uint32_t n_tiles = (n + 31) / 32;
  for (uint32_t tile = blockIdx.x * warps + warp; tile < n_tiles; tile += gridDim.x * warps) {
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
      pos_enc(P, s0, s1, s2, col + kRowGam * stride, stride);
      __syncwarp();
      warp_fwd<kWidth, kResGammaPad, 0>(sW + PL.r1, kPadRow, wcol, stride, kRowGam, 0, sB1, nullptr, 0, true, kRowA);
      warp_fwd<kWidth, kWidth, 0>(sW + PL.r2, kPadRow, wcol, stride, kRowA, 0, sW + PL.r2b, nullptr, 0, true, kRowB);
      warp_fwd<kWidth, kWidth, 0>(sW + PL.r3, kPadRow, wcol, stride, kRowB, 0, sW + PL.r3b, nullptr, 0, true, kRowA);
      warp_fwd<kWidth, kWidth, kResGammaPad>(sW + PL.r4, kPadRow, wcol, stride, kRowA, kRowGam, sW + PL.r4b, nullptr,
                                             0, true, kRowB);
      warp_fwd<4, kWidth, 0>(sW + PL.r5, 4, wcol, stride, kRowB, 0, sW + PL.r5b, nullptr, 0, false, kRowOut);
      f0 += col[(kRowOut + 0) * stride];
      f1 += col[(kRowOut + 1) * stride];
      f2 += col[(kRowOut + 2) * stride];
    }
    const bool inside = hash_encode(P, f0, f1, f2, col + kRowEnc * stride, stride);
    __syncwarp();
    warp_fwd<kWidth, kMlpIn, 0>(sW + PL.c0, kPadRow, wcol, stride, kRowEnc, 0, sW + PL.c0b, nullptr, 0, true, kRowA);
    int cur = kRowA, nxt = kRowB;
    for (int l = 1; l < P.hidden; ++l) {
      warp_fwd<kWidth, kWidth, 0>(sW + PL.ch[l - 1], kPadRow, wcol, stride, cur, 0, sW + PL.chb[l - 1], nullptr, 0,
                                  true, nxt);
      const int t = cur;
      cur = nxt;
      nxt = t;
    }
    warp_fwd<4, kWidth, 0>(sW + PL.cl, 4, wcol, stride, cur, 0, sW + PL.clb, nullptr, 0, false, kRowOut);
    if (valid) {
      const float o0 = col[kRowOut * stride], o1 = col[(kRowOut + 1) * stride], o2 = col[(kRowOut + 2) * stride],
                  o3 = col[(kRowOut + 3) * stride];
      const float cr = sigmoidf_(o0), cg = sigmoidf_(o1), cb = sigmoidf_(o2), sigma = softplusf_(o3);
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
    __syncwarp();   // the next tile reuses the warp's rows
  }
}

nr_status launch_field_tf32(const FieldParams &P, int mode, const float4 *in, uint32_t n_fixed, const uint32_t *n_dev,
                            float *out, int device, cudaStream_t st) {
  if (!P.tf32_scratch) {
    set_error("the float32 tensor-core tier has no scratch buffer");
    return NR_ESTATE;
  }
  const PadLay PL = pad_layout(P.lay, P.hidden);
  const size_t smem = sizeof(float) * (((PL.total + 3) & ~3) + kPoseSmem + kWidth);
  const int blocks = num_sms(device);
  if (mode == kModeRender) {
    NR_CHECK_CUDA(
        cudaFuncSetAttribute(field_tf32_kernel<kModeRender>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    field_tf32_kernel<kModeRender><<<blocks, kTf32Threads, smem, st>>>(P, PL, in, n_fixed, n_dev, out);
  } else {
    NR_CHECK_CUDA(
        cudaFuncSetAttribute(field_tf32_kernel<kModeQuery>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    field_tf32_kernel<kModeQuery><<<blocks, kTf32Threads, smem, st>>>(P, PL, in, n_fixed, n_dev, out);
  }
  NR_CHECK_CUDA(cudaGetLastError());
  return NR_OK;
}

}  // namespace nr
