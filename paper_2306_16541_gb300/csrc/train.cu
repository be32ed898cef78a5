// train.cu -- one training step (Sec. 5.2): stratified samples of a batch of
// pixel rays, the float32 field forward, compositing with the squared-error
// loss (or a caller's dL/dC), the hand-written backward (compositing adjoint,
// canonical MLP, hash scatter-add, residual MLP through the positional
// encoding, inverse-LBS scatter-add into the weight volume, and the pose
// refiner's dL/dG) and Adam.
//
// Work split:
//   * the gathers and their adjoints (LBS warp, PE, hash encoding) run one
//     sample per thread; each thread keeps its sample's activations and deltas
//     in its own column of a scratch buffer (rows x threads per block);
//   * both MLPs run per warp of 32 samples on the tensor cores -- forward
//     layers W X^T, layer backprop W^T D^T, weight gradients D^T H -- as
//     m16n8k8 TF32 MMAs with three products per step (hi/lo splits) for
//     float32 accuracy, over a bank-padded shared-memory copy of the weights;
//   * weight gradients of a warp go into its block's private accumulator
//     (fire-and-forget atomics shared by the block's warps); one kernel sums
//     the block accumulators at the end;
//   * hash-table and weight-volume gradients are scattered with float2 /
//     float atomics straight into the gradient buffers, warp-aggregated: the
//     lanes of a run that adds into one cell sum first (run_sum);
//   * thread slots visit the batch's rays in a scattered order (ray_of), so
//     that the rays in flight together do not come from one image patch;
//   * the forward records which slots carry a gradient (live mask); the
//     backward skips the rest.
#include <math.h>
#include <string.h>

#include "field.cuh"
#include "render.cuh"
#include "tf32.cuh"

namespace nr {

constexpr int kBwdThreads = 384;   // ~160 registers a thread (512 threads at 128 measured slower)
constexpr int kFwdThreads = 512;   // the forward fits 128, so twice the warps hide its gathers

// Rows of a thread's scratch column (sized for the subject's hidden depth H).
struct Rows {
  int gam;     // gamma(x_skel)            48
  int rh;      // residual h1..h4          4 x 64
  int enc;     // hash encoding            32
  int ch;      // canonical h1..hH         H x 64
  int db;      // two 64-row delta buffers, used in turn by both MLPs' backward
  int dcl;     // canonical output delta   4
  int dr5;     // residual output delta    4
  int denc;    // dL/d encoding            32
  int dgam;    // dL/d gamma               48
  int dp;      // dL/d p_i per bone (pose refiner)  3 x 24
  int xs;      // the sample position               3
  int total;
};

static Rows make_rows(int H) {
  Rows r{};
  int o = 0;
  r.gam = o; o += kResGammaPad;
  r.rh = o; o += 4 * kWidth;
  r.enc = o; o += kMlpIn;
  r.ch = o; o += H * kWidth;
  r.db = o; o += 2 * kWidth;
  r.dcl = o; o += 4;
  r.dr5 = o; o += 4;
  r.denc = o; o += kMlpIn;
  r.dgam = o; o += kResGammaPad;
  r.dp = o; o += 3 * kBones;
  r.xs = o; o += 3;
  r.total = o;
  return r;
}

struct TrainDev {
  const uint32_t *frame_id, *px, *py;
  const float *target;
  uint32_t n_rays, S;
  uint32_t ray_mul;       // coprime with n_rays: the order in which thread slots visit rays
  float loss_weight;      // lambda_mse
  uint64_t seed;
  float bg[3];
  const Frame *cams;
  const float *fG, *fbias1, *fomega;
  float4 *samp, *out;
  float *T;
  uint32_t *raycnt;
  uint32_t *live;         // per warp of 32 thread slots: bit l set if slot l's sample has a gradient
  float *loss;
  float2 *g_table;
  float *g_wvol;
  float *scratch, *wacc;
  int acc_floats;         // floats per block accumulator
  int n_frames;
  Rows rw;
  float *dG;              // [F][24][12] dL/dG of every frame (pose refiner), or NULL
  int dG_smem;            // 1: the block sums dG in shared memory first
  PadLay pl;              // shared-memory layout of the backward kernel's weights
  float *pred;            // [n][3] composited colours out, or NULL
  const float *grad_rgb;  // [n][3] dL/dC from the caller, or NULL (MSE against target)
  int forward_only;       // stop after compositing
};

// The ray whose samples thread slot q (of the fwd/bwd kernels) evaluates: slot q takes
// sample q mod S of ray (q / S) ray_mul mod n_rays.  With ray_mul near 0.618 n_rays the
// rays in flight at one time lie spread over the batch; taken in batch order they would be
// neighbours from one image patch whose scatter-adds all hit the same table entries and
// voxels at once.  Every ray is visited once since ray_mul is coprime with n_rays.
__device__ __forceinline__ uint32_t ray_of(const TrainDev &T, uint32_t q) {
  return (uint32_t)(((uint64_t)(q / T.S) * T.ray_mul) % T.n_rays);
}

// A multiplier coprime with n near the golden-ratio fraction of n (1 for n <= 2).
static uint32_t ray_multiplier(uint32_t n) {
  if (n <= 2) return 1;
  auto gcd = [](uint32_t a, uint32_t b) {
    while (b) {
      const uint32_t t = a % b;
      a = b;
      b = t;
    }
    return a;
  };
  uint32_t m = (uint32_t)(0.6180339887498949 * (double)n);
  if (m < 1) m = 1;
  while (gcd(m, n) != 1) ++m;
  return m;
}

// ----------------------------------------------------------------- rays
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  // SplitMix64 (Steele, Lea and Flood 2014): output k of the generator seeded with `seed`
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// One thread per (ray, bin): stratified sample t_i = lo + (i + u_i) D inside the
// clipped ray, delta_i = t_{i+1} - t_i, delta_{S-1} = hi - t_{S-1}.
__global__ void __launch_bounds__(256) train_samples_kernel(TrainDev T, float bx, float by, float bz, float Bx,
                                                            float By, float Bz) {
  const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q >= (uint64_t)T.n_rays * T.S) return;
  const uint32_t r = (uint32_t)(q / T.S), i = (uint32_t)(q % T.S);
  const Frame &F = T.cams[T.frame_id[r]];
  CamParams c;
  for (int k = 0; k < 9; ++k) c.R[k] = F.R[k];
  for (int k = 0; k < 3; ++k) c.t[k] = F.t[k];
  c.fx = F.fx; c.fy = F.fy; c.cx = F.cx; c.cy = F.cy; c.t_near = F.t_near; c.t_far = F.t_far;
  const float bmin[3] = {bx, by, bz}, bmax[3] = {Bx, By, Bz};
  float o[3], d[3], lo, hi;
  camera_origin(c, o);
  const bool hit = ray_setup(c, o, bmin, bmax, T.px[r], T.py[r], d, lo, hi);
  if (i == 0) T.raycnt[r] = hit ? T.S : 0u;
  if (!hit) {
    T.samp[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float D = (hi - lo) / (float)T.S;
  auto u_of = [&](uint32_t ii) {
    const uint64_t z = splitmix64(T.seed, (uint64_t)r * T.S + ii + 1);
    return (float)(z >> 40) * (1.0f / 16777216.0f);
  };
  const float t = lo + ((float)i + u_of(i)) * D;
  const float tn = (i + 1 < T.S) ? lo + ((float)(i + 1) + u_of(i + 1)) * D : hi;
  T.samp[q] = make_float4(o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2], tn - t);
}

// ------------------------------------------------- compositing and its adjoint
// Per ray: C = sum_i T_i alpha_i c_i + T_S bg, T_{i+1} = T_i (1 - alpha_i) (Eq. 3),
// loss term sum_k (C_k - C_gt,k)^2 / (3 N), g = dL/dC.  The reverse scan keeps
// B_i = sum_{j>i} alpha_j prod_{i<k<j}(1 - alpha_k) (c_j . g) + prod_{k>i}(1 - alpha_k) (bg . g)
// (B_{S-1} = bg . g, B_{i-1} = alpha_i (c_i . g) + (1 - alpha_i) B_i) so that
//   dL/dc_i = T_i alpha_i g,  dL/dalpha_i = T_i (c_i . g - B_i)
// without dividing by (1 - alpha_i).
__global__ void __launch_bounds__(256) train_composite_kernel(TrainDev T) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  float lsum = 0.f;
  if (r < T.n_rays) {
    const size_t base = (size_t)r * T.S;
    const uint32_t cnt = T.raycnt[r];
    float Tr = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    for (uint32_t i = 0; i < cnt; ++i) {
      const float4 v = T.out[base + i];
      T.T[base + i] = Tr;
      const float w = Tr * v.w;
      c0 = fmaf(w, v.x, c0);
      c1 = fmaf(w, v.y, c1);
      c2 = fmaf(w, v.z, c2);
      Tr *= 1.f - v.w;
    }
    const float C0 = fmaf(Tr, T.bg[0], c0), C1 = fmaf(Tr, T.bg[1], c1), C2 = fmaf(Tr, T.bg[2], c2);
    if (T.pred) {
      T.pred[3 * r] = C0;
      T.pred[3 * r + 1] = C1;
      T.pred[3 * r + 2] = C2;
    }
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (T.grad_rgb) {   // the caller's dL/dC
      g0 = T.grad_rgb[3 * r];
      g1 = T.grad_rgb[3 * r + 1];
      g2 = T.grad_rgb[3 * r + 2];
    } else if (T.target) {
      const float e0 = C0 - T.target[3 * r], e1 = C1 - T.target[3 * r + 1], e2 = C2 - T.target[3 * r + 2];
      lsum = T.loss_weight * (e0 * e0 + e1 * e1 + e2 * e2);
      const float scale = 2.f * T.loss_weight / (3.f * (float)T.n_rays);
      g0 = scale * e0;
      g1 = scale * e1;
      g2 = scale * e2;
    }
    float B = T.bg[0] * g0 + T.bg[1] * g1 + T.bg[2] * g2;
    for (int i = T.forward_only ? -1 : (int)cnt - 1; i >= 0; --i) {
      const float4 v = T.out[base + i];
      const float Ti = T.T[base + i];
      const float cg = v.x * g0 + v.y * g1 + v.z * g2;
      const float ta = Ti * v.w;
      T.out[base + i] = make_float4(ta * g0, ta * g1, ta * g2, Ti * (cg - B));
      B = fmaf(v.w, cg, (1.f - v.w) * B);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(T.loss, lsum / (3.f * (float)T.n_rays));
}

// ------------------------------------------------------- warp-aggregated scatter-add
// The samples of a warp lie in order along one ray (or a few, when S is not a multiple of
// 32), so lanes that add into the same cell (hash level cell, weight-volume cell) are runs of
// consecutive lanes.  run_sum sums the
// values of each run into its first lane (a segmented suffix sum over shuffles, stopping
// once no run is longer than the distance reached) and returns whether this lane heads a
// valid run: only head lanes issue the atomics, with the run's totals.  A run is a maximal
// stretch of valid lanes with equal keys (key_lo, key_hi); invalid lanes are runs of their
// own and add nothing.  Every lane of the warp must call it.
template <int NV>
__device__ __forceinline__ bool run_sum(uint32_t key_lo, uint32_t key_hi, bool valid, float (&v)[NV]) {
  const int lane = threadIdx.x & 31;
  const uint32_t plo = __shfl_up_sync(0xffffffffu, key_lo, 1), phi = __shfl_up_sync(0xffffffffu, key_hi, 1);
  const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
  const bool pvalid = lane > 0 && ((vmask >> (lane - 1)) & 1u);
  const bool head = !valid || !pvalid || plo != key_lo || phi != key_hi;
  const uint32_t heads = __ballot_sync(0xffffffffu, head);
  const int run = __popc(heads & (0xffffffffu >> (31 - lane)));   // heads at lanes 0..lane
#pragma unroll 1
  for (int d = 1; d < 32; d <<= 1) {
    const int rd = __shfl_down_sync(0xffffffffu, run, d);
    const bool take = lane + d < 32 && rd == run;
    if (!__any_sync(0xffffffffu, take)) break;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const float o = __shfl_down_sync(0xffffffffu, v[k], d);
      if (take) v[k] += o;
    }
  }
  return head && valid;
}

// ---------------------------------------------------------------- backward
// Warp-level weight gradient of one layer with 64 outputs over the warp's 32 samples,
// dW[j][k] = sum_s d[s][j] h[s][k], as the product D^T H on the tensor cores
// (m16n8k8 TF32 MMAs, three per step for float32 accuracy): M = the 64 outputs in four
// 16-row tiles, K = the 32 samples in four steps of 8, N = the inputs in tiles of 8.  Each
// finished 16 x 8 tile is added into the block's accumulator acc[wt + k * 64 + j] with
// fire-and-forget atomics (shared by the block's warps); acc[b + j] += sum_s d[s][j].
// `wcol` points at the warp's column 0 (row r of sample s is wcol[r * stride + s]).
__device__ __noinline__ void wgrad64(const float *wcol, int stride, int r_in, int n_in, int r_d, float *acc,
                                        int wt, int b, bool with_bias) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  if (with_bias) {
    const float4 *p0 = reinterpret_cast<const float4 *>(wcol + (r_d + lane) * stride);
    const float4 *p1 = reinterpret_cast<const float4 *>(wcol + (r_d + lane + 32) * stride);
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 a = p0[q], c = p1[q];
      s0 += (a.x + a.y) + (a.z + a.w);
      s1 += (c.x + c.y) + (c.z + c.w);
    }
    atomicAdd(acc + b + lane, s0);
    atomicAdd(acc + b + lane + 32, s1);
  }
  // A = D^T fragments of two row tiles at a time (one per step of 8 samples), so that the
  // hi/lo fragments take 64 registers; H is read once per pair of row tiles
#pragma unroll 1
  for (int mh = 0; mh < 4; mh += 2) {
    uint32_t ah[2][4][4], al[2][4][4];
#pragma unroll
    for (int mm = 0; mm < 2; ++mm) {
      const float *d0 = wcol + (r_d + 16 * (mh + mm) + g) * stride;
      const float *d8 = d0 + 8 * stride;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const int s = 8 * ks + t;
        tf32_split(d0[s], ah[mm][ks][0], al[mm][ks][0]);
        tf32_split(d8[s], ah[mm][ks][1], al[mm][ks][1]);
        tf32_split(d0[s + 4], ah[mm][ks][2], al[mm][ks][2]);
        tf32_split(d8[s + 4], ah[mm][ks][3], al[mm][ks][3]);
      }
    }
#pragma unroll 1
    for (int n0 = 0; n0 < n_in; n0 += 8) {
      uint32_t bh[4][2], bl[4][2];   // B = H fragments of this column tile
      const float *hk = wcol + (r_in + n0 + g) * stride;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        tf32_split(hk[8 * ks + t], bh[ks][0], bl[ks][0]);
        tf32_split(hk[8 * ks + t + 4], bh[ks][1], bl[ks][1]);
      }
#pragma unroll
      for (int mm = 0; mm < 2; ++mm) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          mma_tf32(c, al[mm][ks], bh[ks]);
          mma_tf32(c, ah[mm][ks], bl[ks]);
          mma_tf32(c, ah[mm][ks], bh[ks]);
        }
        // c = C[16m + g][n0 + 2t], C[16m + g][n0 + 2t + 1], C[16m + g + 8][n0 + 2t], C[16m + g + 8][n0 + 2t + 1]
        float *o = acc + wt + (n0 + 2 * t) * kWidth + 16 * (mh + mm) + g;
        atomicAdd(o, c[0]);
        atomicAdd(o + kWidth, c[1]);
        atomicAdd(o + 8, c[2]);
        atomicAdd(o + kWidth + 8, c[3]);
      }
    }
  }
}

// Same for a layer with 4 (padded) outputs and 64 inputs: lane owns input rows k = lane, lane + 32.
__device__ __forceinline__ void wgrad4(const float *wcol, int stride, int r_in, int r_d, int n_out, float *acc, int wt,
                                       int b) {
  const int lane = threadIdx.x & 31;
  float h0[32], h1[32];
  const float4 *p0 = reinterpret_cast<const float4 *>(wcol + (r_in + lane) * stride);
  const float4 *p1 = reinterpret_cast<const float4 *>(wcol + (r_in + lane + 32) * stride);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 a = p0[q], c = p1[q];
    h0[4 * q] = a.x; h0[4 * q + 1] = a.y; h0[4 * q + 2] = a.z; h0[4 * q + 3] = a.w;
    h1[4 * q] = c.x; h1[4 * q + 1] = c.y; h1[4 * q + 2] = c.z; h1[4 * q + 3] = c.w;
  }
  for (int j = 0; j < n_out; ++j) {
    const float4 *pd = reinterpret_cast<const float4 *>(wcol + (r_d + j) * stride);
    float a0 = 0.f, a1 = 0.f, sb = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 d = pd[q];
      a0 = fmaf(h0[4 * q], d.x, fmaf(h0[4 * q + 1], d.y, fmaf(h0[4 * q + 2], d.z, fmaf(h0[4 * q + 3], d.w, a0))));
      a1 = fmaf(h1[4 * q], d.x, fmaf(h1[4 * q + 1], d.y, fmaf(h1[4 * q + 2], d.z, fmaf(h1[4 * q + 3], d.w, a1))));
      sb += d.x + d.y + d.z + d.w;
    }
    atomicAdd(acc + wt + lane * 4 + j, a0);
    atomicAdd(acc + wt + (lane + 32) * 4 + j, a1);
    if (lane == 0) atomicAdd(acc + b + j, sb);
  }
}

// The backward of one layer for the warp's 32 samples on the tensor cores:
//   out[s][i] = (sum_o W^T[i][o] delta[s][o]) * (h[s][i] > 0)     (no mask when r_h < 0)
// as C = W^T D^T with M = IN (16-row tiles of inputs), N = the 32 samples (4 tiles of 8),
// K = OUT (steps of 8; a 4-output layer pads its step with zeros); m16n8k8 TF32 MMAs, three
// per step for float32 accuracy.  W^T comes from the padded shared copy (row i at Wt + i * rs),
// delta from scratch rows r_d.., the mask from rows r_h..; the result goes to rows r_out..
// (added to them when `accumulate`).  Every lane of the warp must take part.
template <int OUT, int IN>
__device__ __noinline__ void warp_back(const float *__restrict__ Wt, int rs, float *wcol, int stride, int r_d,
                                          int r_h, int r_out, bool accumulate) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  constexpr int KS = (OUT + 7) / 8, MT = IN / 16;
  float acc[MT][4][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
#pragma unroll 1
  for (int ks = 0; ks < KS; ++ks) {
    const int o0 = 8 * ks + t, o1 = o0 + 4;
    uint32_t bh[4][2], bl[4][2];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const float u0 = o0 < OUT ? wcol[(r_d + o0) * stride + 8 * n + g] : 0.f;
      const float u1 = o1 < OUT ? wcol[(r_d + o1) * stride + 8 * n + g] : 0.f;
      tf32_split(u0, bh[n][0], bl[n][0]);
      tf32_split(u1, bh[n][1], bl[n][1]);
    }
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const float *w0 = Wt + (16 * m + g) * rs, *w8 = w0 + 8 * rs;
      uint32_t ah[4], al[4];
      tf32_split(o0 < OUT ? w0[o0] : 0.f, ah[0], al[0]);
      tf32_split(o0 < OUT ? w8[o0] : 0.f, ah[1], al[1]);
      tf32_split(o1 < OUT ? w0[o1] : 0.f, ah[2], al[2]);
      tf32_split(o1 < OUT ? w8[o1] : 0.f, ah[3], al[3]);
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
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 16 * m + g + (q >= 2 ? 8 : 0), smp = 8 * n + 2 * t + (q & 1);
        float v = acc[m][n][q];
        if (r_h >= 0 && !(wcol[(r_h + i) * stride + smp] > 0.f)) v = 0.f;
        float *dst = wcol + (r_out + i) * stride + smp;
        *dst = accumulate ? *dst + v : v;
      }
  __syncwarp();   // the next layer reads these rows through other lanes
}

// ------------------------------------------------------------ forward field
// The float32 field with the pose of each sample's frame, laid out like the backward
// kernel: per-sample gathers (LBS warp, PE, hash encoding) one sample per thread, both MLPs
// as warp-level tensor-core layers over the samples' scratch columns (float32 accuracy).
// Writes (r, g, b, alpha) per sample slot (zero for a ray that misses the box).
__global__ void __launch_bounds__(kFwdThreads, 1) train_fwd_kernel(FieldParams P, TrainDev T) {
  extern __shared__ float4 smem4[];
  float *sW = reinterpret_cast<float *>(smem4);        // the weights in the padded layout T.pl
  for (int q = 0; q < T.pl.n_seg; ++q) {
    const PadSeg &sg = T.pl.seg[q];
    for (int i = threadIdx.x; i < sg.rows * sg.cols; i += blockDim.x) {
      const int rr = i / sg.cols, cc = i - rr * sg.cols;
      sW[sg.dst + rr * sg.dstride + cc] = __ldg(P.blob + sg.src + i);
    }
  }
  __syncthreads();
  const PadLay &PL = T.pl;
  const int stride = blockDim.x;
  const int warp = threadIdx.x >> 5;
  const Rows &RW = T.rw;
  const int R_GAM = RW.gam, R_RH = RW.rh, R_ENC = RW.enc, R_CH = RW.ch, D_CL = RW.dcl, D_R5 = RW.dr5;
  float *colbase = T.scratch + (size_t)blockIdx.x * RW.total * stride;
  float *col = colbase + threadIdx.x;
  float *wcol = colbase + warp * 32;
  const int H = P.hidden;
  const uint32_t n = T.n_rays * T.S;
  const uint32_t step = gridDim.x * blockDim.x;
  const uint32_t n_iter = (n + step - 1) / step;
  for (uint32_t it = 0; it < n_iter; ++it) {
    const uint32_t q = it * step + blockIdx.x * blockDim.x + threadIdx.x;   // thread slot
    const uint32_t r = q < n ? ray_of(T, q) : 0;
    const uint32_t j = r * T.S + q % T.S;                                       // sample slot
    const bool active = q < n && T.raycnt[r] != 0;
    if (!__any_sync(0xffffffffu, active)) {   // 32 slots of rays that miss the box
      if (q < n) T.out[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      if ((threadIdx.x & 31) == 0 && q < n) T.live[q >> 5] = 0u;
      continue;
    }
    const uint32_t f = active ? T.frame_id[r] : 0;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    float S = 0.f, f0 = 0.f, f1 = 0.f, f2 = 0.f;
    if (active) {
      s = T.samp[j];
      float s0, s1, s2;
      lbs_warp(P, T.fG + (size_t)f * kBones * 12, s.x, s.y, s.z, s0, s1, s2, S);
      f0 = s0;
      f1 = s1;
      f2 = s2;
      pos_enc(P, s0, s1, s2, col + R_GAM * stride, stride);
    } else {
      for (int q = 0; q < kResGammaPad; ++q) col[(R_GAM + q) * stride] = 0.f;
    }
    __syncwarp();
    if (P.res_enabled) {
      warp_fwd<kWidth, kResGammaPad, 0>(sW + PL.r1, kPadRow, wcol, stride, R_GAM, 0, nullptr, T.fbias1, (int)f,
                                        true, R_RH + 0 * kWidth);
      warp_fwd<kWidth, kWidth, 0>(sW + PL.r2, kPadRow, wcol, stride, R_RH + 0 * kWidth, 0, sW + PL.r2b, nullptr, 0,
                                  true, R_RH + 1 * kWidth);
      warp_fwd<kWidth, kWidth, 0>(sW + PL.r3, kPadRow, wcol, stride, R_RH + 1 * kWidth, 0, sW + PL.r3b, nullptr, 0,
                                  true, R_RH + 2 * kWidth);
      warp_fwd<kWidth, kWidth, kResGammaPad>(sW + PL.r4, kPadRow, wcol, stride, R_RH + 2 * kWidth, R_GAM, sW + PL.r4b,
                                             nullptr, 0, true, R_RH + 3 * kWidth);
      warp_fwd<4, kWidth, 0>(sW + PL.r5, 4, wcol, stride, R_RH + 3 * kWidth, 0, sW + PL.r5b, nullptr, 0, false, D_R5);
    }
    bool inside = false;
    if (active) {
      if (P.res_enabled) {
        f0 += col[(D_R5 + 0) * stride];
        f1 += col[(D_R5 + 1) * stride];
        f2 += col[(D_R5 + 2) * stride];
      }
      inside = hash_encode(P, f0, f1, f2, col + R_ENC * stride, stride);
    } else {
      for (int q = 0; q < kMlpIn; ++q) col[(R_ENC + q) * stride] = 0.f;
    }
    __syncwarp();
    warp_fwd<kWidth, kMlpIn, 0>(sW + PL.c0, kPadRow, wcol, stride, R_ENC, 0, sW + PL.c0b, nullptr, 0, true, R_CH);
    for (int l = 1; l < H; ++l)
      warp_fwd<kWidth, kWidth, 0>(sW + PL.ch[l - 1], kPadRow, wcol, stride, R_CH + (l - 1) * kWidth, 0,
                                  sW + PL.chb[l - 1], nullptr, 0, true, R_CH + l * kWidth);
    warp_fwd<4, kWidth, 0>(sW + PL.cl, 4, wcol, stride, R_CH + (H - 1) * kWidth, 0, sW + PL.clb, nullptr, 0, false,
                           D_CL);
    {
      // the slots whose samples carry a gradient (in the box, warped into the canonical box);
      // the backward skips the others, which add exactly zero
      const uint32_t lw = __ballot_sync(0xffffffffu, active && inside);
      if ((threadIdx.x & 31) == 0 && q < n) T.live[q >> 5] = lw;
    }
    if (q < n) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (active) {
        const float o0 = col[D_CL * stride], o1 = col[(D_CL + 1) * stride], o2 = col[(D_CL + 2) * stride],
                    o3 = col[(D_CL + 3) * stride];
        const float a = inside ? -expm1f(-softplusf_(o3) * s.w) * fminf(S, 1.f) : 0.f;
        v = make_float4(sigmoidf_(o0), sigmoidf_(o1), sigmoidf_(o2), a);
      }
      T.out[j] = v;
    }
  }
}

// The compositing adjoint of train_composite_kernel for the RB rays whose slots a block holds
// (ray slots rs0 .. rs0 + RB - 1; local ray lr's samples at o[lr S ..]), by the block's first
// warp: o[] holds each slot's (r, g, b, alpha) on entry and its (dL/dc, dL/dalpha) on exit,
// Ts[] the transmittance in front of each sample.  Same arithmetic in the same order.
__device__ __forceinline__ void composite_rays(const TrainDev &T, float4 *o, float *Ts, uint32_t rs0, uint32_t RB) {
  const int lane = threadIdx.x & 31;
  float lsum = 0.f;
  for (uint32_t lr = lane; lr < RB; lr += 32) {
    const uint32_t rs = rs0 + lr;
    if (rs >= T.n_rays) break;
    const uint32_t r = (uint32_t)(((uint64_t)rs * T.ray_mul) % T.n_rays);
    float4 *v4 = o + (size_t)lr * T.S;
    float *t4 = Ts + (size_t)lr * T.S;
    const uint32_t cnt = T.raycnt[r];
    float Tr = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    for (uint32_t i = 0; i < cnt; ++i) {
      const float4 v = v4[i];
      t4[i] = Tr;
      const float w = Tr * v.w;
      c0 = fmaf(w, v.x, c0);
      c1 = fmaf(w, v.y, c1);
      c2 = fmaf(w, v.z, c2);
      Tr *= 1.f - v.w;
    }
    const float C0 = fmaf(Tr, T.bg[0], c0), C1 = fmaf(Tr, T.bg[1], c1), C2 = fmaf(Tr, T.bg[2], c2);
    if (T.pred) {
      T.pred[3 * r] = C0;
      T.pred[3 * r + 1] = C1;
      T.pred[3 * r + 2] = C2;
    }
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (T.grad_rgb) {
      g0 = T.grad_rgb[3 * r];
      g1 = T.grad_rgb[3 * r + 1];
      g2 = T.grad_rgb[3 * r + 2];
    } else if (T.target) {
      const float e0 = C0 - T.target[3 * r], e1 = C1 - T.target[3 * r + 1], e2 = C2 - T.target[3 * r + 2];
      lsum += T.loss_weight * (e0 * e0 + e1 * e1 + e2 * e2);
      const float scale = 2.f * T.loss_weight / (3.f * (float)T.n_rays);
      g0 = scale * e0;
      g1 = scale * e1;
      g2 = scale * e2;
    }
    float B = T.bg[0] * g0 + T.bg[1] * g1 + T.bg[2] * g2;
    for (int i = (int)cnt - 1; i >= 0; --i) {
      const float4 v = v4[i];
      const float Ti = t4[i];
      const float cg = v.x * g0 + v.y * g1 + v.z * g2;
      const float ta = Ti * v.w;
      v4[i] = make_float4(ta * g0, ta * g1, ta * g2, Ti * (cg - B));
      B = fmaf(v.w, cg, (1.f - v.w) * B);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
  if (lane == 0 && lsum != 0.f) atomicAdd(T.loss, lsum / (3.f * (float)T.n_rays));
}

// One thread per sample: forward recompute (activations into the thread's scratch
// column), backward, scatter-adds, then the warp's weight-gradient reduction.
// FUSED: the forward and the compositing adjoint run here too, so that neither train_fwd_kernel
// nor train_composite_kernel is needed: the block takes groups of whole rays (RB = blockDim / S
// of them), evaluates every sample once, composites its rays in shared memory and goes straight
// on to the backward with the activations still in its columns.
template <bool FUSED>
__global__ void __launch_bounds__(kBwdThreads, 1) train_bwd_kernel(FieldParams P, TrainDev T) {
  extern __shared__ float4 smem4[];
  float *sW = reinterpret_cast<float *>(smem4);        // the weights in the padded layout T.pl
  float *sdG = sW + T.pl.total;                        // [F][24][12] when T.dG_smem
  // FUSED: each slot's (r, g, b, alpha), then its adjoint [SB], and transmittances [SB]
  float4 *sOut = reinterpret_cast<float4 *>(sdG + (T.dG && T.dG_smem ? T.n_frames * kBones * 12 : 0));
  float *sT = reinterpret_cast<float *>(sOut + blockDim.x);
  for (int q = 0; q < T.pl.n_seg; ++q) {
    const PadSeg &sg = T.pl.seg[q];
    for (int i = threadIdx.x; i < sg.rows * sg.cols; i += blockDim.x) {
      const int rr = i / sg.cols, cc = i - rr * sg.cols;
      sW[sg.dst + rr * sg.dstride + cc] = __ldg(P.blob + sg.src + i);
    }
  }
  if (T.dG && T.dG_smem)
    for (int i = threadIdx.x; i < T.n_frames * kBones * 12; i += blockDim.x) sdG[i] = 0.f;
  __syncthreads();
  const BlobLayout &Ly = P.lay;                        // the gradient accumulators' layout
  const PadLay &PL = T.pl;
  const int stride = blockDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Rows &RW = T.rw;
  const int R_GAM = RW.gam, R_RH = RW.rh, R_ENC = RW.enc, R_CH = RW.ch, D_B = RW.db, D_CL = RW.dcl, D_R5 = RW.dr5,
            R_DENC = RW.denc, R_DGAM = RW.dgam, R_DP = RW.dp, R_XS = RW.xs, kRows = RW.total;
  float *colbase = T.scratch + (size_t)blockIdx.x * kRows * stride;
  float *col = colbase + threadIdx.x;                  // this thread's column
  float *wcol = colbase + warp * 32;                   // the warp's column 0
  float *acc = T.wacc + (size_t)blockIdx.x * T.acc_floats;
  float *accF = acc + Ly.total;                        // per-frame first-layer bias gradients [F][64]
  const int H = P.hidden;
  const uint32_t n = T.n_rays * T.S;
  const uint32_t step = gridDim.x * blockDim.x;
  const uint32_t RB = FUSED ? blockDim.x / T.S : 0u, SB = RB * T.S;   // FUSED: rays and slots a group
  const uint32_t n_units = FUSED ? (T.n_rays + RB - 1) / RB : (n + step - 1) / step;
  for (uint32_t it = FUSED ? blockIdx.x : 0u; it < n_units; it += FUSED ? gridDim.x : 1u) {
    const uint32_t q = FUSED ? it * SB + threadIdx.x : it * step + blockIdx.x * blockDim.x + threadIdx.x;  // slot
    const bool qv = q < n && (!FUSED || threadIdx.x < SB);
    const uint32_t q0 = q - lane;                                               // the warp's first slot
    const uint32_t r = qv ? ray_of(T, q) : 0;
    const uint32_t j = r * T.S + q % T.S;                                       // sample slot
    bool active;
    if constexpr (FUSED) {
      active = qv && T.raycnt[r] != 0;   // every slot of a ray that meets the box is evaluated
    } else {
      // the forward's mask: a slot outside it (no box hit, or warped out of the canonical box)
      // adds exactly zero to every gradient, and a warp without live slots has nothing to do
      const uint32_t lw = q0 < n ? T.live[q0 >> 5] : 0u;
      if (lw == 0u) continue;
      active = (lw >> lane) & 1u;
    }
    const uint32_t f = active ? T.frame_id[r] : 0;
    float4 g4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!FUSED && active) g4 = __ldcs(T.out + j);
    const bool run = !FUSED || __any_sync(0xffffffffu, active);   // warp-uniform
    // per-sample state carried across the warp-level phases below
    const float *G = T.fG + (size_t)f * kBones * 12;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    float xs0 = 0.f, xs1 = 0.f, xs2 = 0.f, S = 0.f, xf0 = 0.f, xf1 = 0.f, xf2 = 0.f, dS_alpha = 0.f;
    bool inside = false;
    if (run) {
    // ---------------- forward recompute: per-sample gathers, warp-level MLP layers
    if (active) {
      s = __ldcs(T.samp + j);
      lbs_warp(P, G, s.x, s.y, s.z, xs0, xs1, xs2, S);
      xf0 = xs0;
      xf1 = xs1;
      xf2 = xs2;
      pos_enc(P, xs0, xs1, xs2, col + R_GAM * stride, stride);
    } else {
      for (int q = 0; q < kResGammaPad; ++q) col[(R_GAM + q) * stride] = 0.f;
    }
    __syncwarp();
    if (P.res_enabled) {
      warp_fwd<kWidth, kResGammaPad, 0>(sW + PL.r1, kPadRow, wcol, stride, R_GAM, 0, nullptr, T.fbias1, (int)f,
                                        true, R_RH + 0 * kWidth);
      warp_fwd<kWidth, kWidth, 0>(sW + PL.r2, kPadRow, wcol, stride, R_RH + 0 * kWidth, 0, sW + PL.r2b, nullptr, 0,
                                  true, R_RH + 1 * kWidth);
      warp_fwd<kWidth, kWidth, 0>(sW + PL.r3, kPadRow, wcol, stride, R_RH + 1 * kWidth, 0, sW + PL.r3b, nullptr, 0,
                                  true, R_RH + 2 * kWidth);
      warp_fwd<kWidth, kWidth, kResGammaPad>(sW + PL.r4, kPadRow, wcol, stride, R_RH + 2 * kWidth, R_GAM, sW + PL.r4b,
                                             nullptr, 0, true, R_RH + 3 * kWidth);
      // x_res into the (not yet used) rows of the residual output's delta
      warp_fwd<4, kWidth, 0>(sW + PL.r5, 4, wcol, stride, R_RH + 3 * kWidth, 0, sW + PL.r5b, nullptr, 0, false, D_R5);
    }
    if (active) {
      if (P.res_enabled) {
        xf0 += col[(D_R5 + 0) * stride];
        xf1 += col[(D_R5 + 1) * stride];
        xf2 += col[(D_R5 + 2) * stride];
      } else {
        for (int q = 0; q < 4 * kWidth; ++q) col[(R_RH + q) * stride] = 0.f;
      }
      inside = hash_encode(P, xf0, xf1, xf2, col + R_ENC * stride, stride);
    } else {
      for (int q = 0; q < kMlpIn; ++q) col[(R_ENC + q) * stride] = 0.f;
    }
    __syncwarp();
    warp_fwd<kWidth, kMlpIn, 0>(sW + PL.c0, kPadRow, wcol, stride, R_ENC, 0, sW + PL.c0b, nullptr, 0, true, R_CH);
    for (int l = 1; l < H; ++l)
      warp_fwd<kWidth, kWidth, 0>(sW + PL.ch[l - 1], kPadRow, wcol, stride, R_CH + (l - 1) * kWidth, 0,
                                  sW + PL.chb[l - 1], nullptr, 0, true, R_CH + l * kWidth);
    // the canonical output o into the rows of its delta, read back by each sample's thread
    warp_fwd<4, kWidth, 0>(sW + PL.cl, 4, wcol, stride, R_CH + (H - 1) * kWidth, 0, sW + PL.clb, nullptr, 0, false,
                           D_CL);
    }
    if constexpr (FUSED) {
      // each slot's (r, g, b, alpha) as train_fwd_kernel forms it, the rays composited in shared
      // memory by the first warp, and each slot's adjoint back
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (active) {
        const float o0 = col[D_CL * stride], o1 = col[(D_CL + 1) * stride], o2 = col[(D_CL + 2) * stride],
                    o3 = col[(D_CL + 3) * stride];
        const float a = inside ? -expm1f(-softplusf_(o3) * s.w) * fminf(S, 1.f) : 0.f;
        v = make_float4(sigmoidf_(o0), sigmoidf_(o1), sigmoidf_(o2), a);
      }
      if (threadIdx.x < SB) sOut[threadIdx.x] = v;
      __syncthreads();
      if (warp == 0) composite_rays(T, sOut, sT, it * RB, RB);
      __syncthreads();
      if (active) g4 = sOut[threadIdx.x];
      if (__ballot_sync(0xffffffffu, active && inside) == 0u) continue;   // no live slot in the warp
    }
    active = active && inside;
    if (active) {
      // ---------------- alpha, rgb, sigma
      float *dcl = col + (D_CL) * stride;
      const float o[4] = {dcl[0], dcl[stride], dcl[2 * stride], dcl[3 * stride]};
      const float sig = softplusf_(o[3]);
      const float e = expf(-sig * s.w);
      const float lk = fminf(S, 1.f);
      const float dsig = g4.w * s.w * e * lk;
      dS_alpha = S < 1.f ? g4.w * -expm1f(-sig * s.w) : 0.f;
      const float gc[3] = {g4.x, g4.y, g4.z};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float c = sigmoidf_(o[k]);
        dcl[k * stride] = gc[k] * c * (1.f - c);
      }
      dcl[3 * stride] = dsig * sigmoidf_(o[3]);
    }
    if (!active)
      for (int k = 0; k < 4; ++k) col[(D_CL + k) * stride] = 0.f;
    __syncwarp();
    // ---------------- canonical MLP backward: the warp's 32 samples on the tensor cores, each
    // layer's weight gradient summed as soon as its delta exists (two delta buffers in turn)
    {
      int cur = D_B, nxt = D_B + kWidth;
      warp_back<4, kWidth>(sW + PL.cl, 4, wcol, stride, D_CL, R_CH + (H - 1) * kWidth, cur, false);
      wgrad4(wcol, stride, R_CH + (H - 1) * kWidth, D_CL, 4, acc, Ly.cl, Ly.clb);
      for (int l = H - 1; l >= 1; --l) {
        warp_back<kWidth, kWidth>(sW + PL.ch[l - 1], kPadRow, wcol, stride, cur, R_CH + (l - 1) * kWidth, nxt, false);
        wgrad64(wcol, stride, R_CH + (l - 1) * kWidth, kWidth, cur, acc, Ly.ch[l - 1], Ly.chb[l - 1], true);
        const int tmp = cur;
        cur = nxt;
        nxt = tmp;
      }
      warp_back<kWidth, kMlpIn>(sW + PL.c0, kPadRow, wcol, stride, cur, -1, R_DENC, false);
      wgrad64(wcol, stride, R_ENC, kMlpIn, cur, acc, Ly.c0, Ly.c0b, true);
    }
    __syncwarp();
    float dx0 = 0.f, dx1 = 0.f, dx2 = 0.f;
    {
      // ---------------- hash backward: warp-aggregated scatter-add and dL/dx_final
      const float p0 = active ? (xf0 - P.bmin[0]) * P.inv_box[0] : 0.f;
      const float p1 = active ? (xf1 - P.bmin[1]) * P.inv_box[1] : 0.f;
      const float p2 = active ? (xf2 - P.bmin[2]) * P.inv_box[2] : 0.f;
      for (int l = 0; l < P.L; ++l) {
        const float da = active ? col[(R_DENC + 2 * l) * stride] : 0.f;
        const float db = active ? col[(R_DENC + 2 * l + 1) * stride] : 0.f;
        const uint32_t N = P.level_res[l];
        const float fn = (float)N;
        const float q0 = p0 * fn, q1 = p1 * fn, q2 = p2 * fn;
        const float a0 = fminf(floorf(q0), fn - 1.f), a1 = fminf(floorf(q1), fn - 1.f),
                    a2 = fminf(floorf(q2), fn - 1.f);
        const float fr[3] = {q0 - a0, q1 - a1, q2 - a2};
        HashCell c;
        hash_cell(P, l, p0, p1, p2, c);
        float v[16];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          v[2 * k] = c.w[k] * da;
          v[2 * k + 1] = c.w[k] * db;
        }
        const uint32_t ka = (uint32_t)a0 | ((uint32_t)a1 << 16), kb = (uint32_t)a2;
        if (run_sum<16>(ka, kb, active, v)) {
#pragma unroll
          for (int k = 0; k < 8; ++k)
            atomicAdd(T.g_table + (size_t)l * (P.T_mask + 1) + c.idx[k], make_float2(v[2 * k], v[2 * k + 1]));
        }
        if (active) {
          float gp0 = 0.f, gp1 = 0.f, gp2 = 0.f;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float2 tv = __ldg(P.table32 + (size_t)l * (P.T_mask + 1) + c.idx[k]);
            const float sv = tv.x * da + tv.y * db;
            const float wx = (k & 1) ? fr[0] : 1.f - fr[0], wy = ((k >> 1) & 1) ? fr[1] : 1.f - fr[1],
                        wz = (k >> 2) ? fr[2] : 1.f - fr[2];
            const float sx = (k & 1) ? 1.f : -1.f, sy = ((k >> 1) & 1) ? 1.f : -1.f, sz = (k >> 2) ? 1.f : -1.f;
            gp0 = fmaf(sv, sx * wy * wz, gp0);
            gp1 = fmaf(sv, wx * sy * wz, gp1);
            gp2 = fmaf(sv, wx * wy * sz, gp2);
          }
          dx0 = fmaf(gp0, fn, dx0);
          dx1 = fmaf(gp1, fn, dx1);
          dx2 = fmaf(gp2, fn, dx2);
        }
      }
      dx0 *= P.inv_box[0];
      dx1 *= P.inv_box[1];
      dx2 *= P.inv_box[2];
    }
    float ds0 = dx0, ds1 = dx1, ds2 = dx2;
    if (P.res_enabled) {
      // ---------------- residual MLP backward (x_final = x_skel + x_res), tensor cores
      float *dr5 = col + D_R5 * stride;
      dr5[0] = dx0;
      dr5[stride] = dx1;
      dr5[2 * stride] = dx2;
      dr5[3 * stride] = 0.f;
      __syncwarp();
      const int b0 = D_B, b1 = D_B + kWidth;   // delta4 -> b0, delta3 -> b1, delta2 -> b0, delta1 -> b1
      warp_back<4, kWidth>(sW + PL.r5, 4, wcol, stride, D_R5, R_RH + 3 * kWidth, b0, false);
      wgrad4(wcol, stride, R_RH + 3 * kWidth, D_R5, 3, acc, Ly.r5, Ly.r5b);
      warp_back<kWidth, kWidth>(sW + PL.r4, kPadRow, wcol, stride, b0, R_RH + 2 * kWidth, b1, false);
      warp_back<kWidth, kResGammaPad>(sW + PL.r4 + kWidth * kPadRow, kPadRow, wcol, stride, b0, -1, R_DGAM, false);
      wgrad64(wcol, stride, R_RH + 2 * kWidth, kWidth, b0, acc, Ly.r4, Ly.r4b, true);
      wgrad64(wcol, stride, R_GAM, kResGammaPad, b0, acc, Ly.r4 + kWidth * kWidth, 0, false);
      warp_back<kWidth, kWidth>(sW + PL.r3, kPadRow, wcol, stride, b1, R_RH + 1 * kWidth, b0, false);
      wgrad64(wcol, stride, R_RH + 1 * kWidth, kWidth, b1, acc, Ly.r3, Ly.r3b, true);
      warp_back<kWidth, kWidth>(sW + PL.r2, kPadRow, wcol, stride, b0, R_RH + 0 * kWidth, b1, false);
      wgrad64(wcol, stride, R_RH + 0 * kWidth, kWidth, b0, acc, Ly.r2, Ly.r2b, true);
      // dL/dgamma += W1_gamma^T delta1 (the pose columns of W1 are reduced per frame below)
      warp_back<kWidth, kResGammaPad>(sW + PL.r1, kPadRow, wcol, stride, b1, -1, R_DGAM, true);
      wgrad64(wcol, stride, R_GAM, kResGammaPad, b1, acc, Ly.r1, Ly.r1b, true);
      {  // per-frame sums of delta1 (for W_Omega): lane owns rows lane, lane + 32
        const float *d0 = wcol + (b1 + lane) * stride, *d1 = wcol + (b1 + lane + 32) * stride;
        int cur = -1;
        float s0 = 0.f, s1 = 0.f;
        for (int sI = 0; sI < 32; ++sI) {
          const uint32_t jj = q0 + sI;
          if (jj >= n || (FUSED && (uint32_t)(warp * 32 + sI) >= SB)) break;
          const int fr = (int)T.frame_id[ray_of(T, jj)];
          if (fr != cur) {
            if (cur >= 0) {
              atomicAdd(accF + cur * kWidth + lane, s0);
              atomicAdd(accF + cur * kWidth + lane + 32, s1);
            }
            cur = fr;
            s0 = s1 = 0.f;
          }
          s0 += d0[sI];
          s1 += d1[sI];
        }
        if (cur >= 0) {
          atomicAdd(accF + cur * kWidth + lane, s0);
          atomicAdd(accF + cur * kWidth + lane + 32, s1);
        }
      }
      __syncwarp();
      if (active) {
          // through gamma: d gamma / d x_skel
          const float *dg = col + R_DGAM * stride;
          const float xh[3] = {(xs0 - P.box_c[0]) * P.box_ih[0], (xs1 - P.box_c[1]) * P.box_ih[1],
                               (xs2 - P.box_c[2]) * P.box_ih[2]};
          float dh[3] = {dg[0], dg[stride], dg[2 * stride]};
          for (int k = 0; k < P.res_freqs; ++k) {
            const float sc = (float)(1 << k);
            const float wk = P.hann[k] * sc * 3.14159265358979f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              float sn, cs;
              sincospif(sc * xh[a], &sn, &cs);
              dh[a] += wk * (dg[(3 + 6 * k + a) * stride] * cs - dg[(6 + 6 * k + a) * stride] * sn);
            }
          }
          ds0 += dh[0] * P.box_ih[0];
          ds1 += dh[1] * P.box_ih[1];
          ds2 += dh[2] * P.box_ih[2];
      }
    }
    {
      // ---------------- inverse-LBS backward: warp-aggregated scatter into the weight volume
      // and, for the pose refiner, dL/dp_i of each candidate p_i = G_i x:
      //   x_skel = sum_i w_i p_i / D,  w_i = W_i(p_i)
      //   dL/dp_i = (w_i / D) dL/dx_skel + dL/dw_i grad W_i(p_i)
      const float D = fmaxf(S, kEpsW);
      // one division per sample: a per-bone quotient with a vanishing numerator (far from the
      // body S, and with it the gradient reaching x_skel, goes to zero) takes the division's
      // slow path 24 times a sample
      const float inv_D = 1.f / D;
      const float m = S > kEpsW ? 1.f : 0.f;
      const int R = P.wres, R3 = R * R * R;
      const size_t QC = quad_channel(R);
      if (T.dG && active) {
        col[(R_XS + 0) * stride] = s.x;
        col[(R_XS + 1) * stride] = s.y;
        col[(R_XS + 2) * stride] = s.z;
      }
      for (int i = 0; i < kBones; ++i) {
        const float *g = G + 12 * i;
        const float p0 = fmaf(g[0], s.x, fmaf(g[1], s.y, fmaf(g[2], s.z, g[3])));
        const float p1 = fmaf(g[4], s.x, fmaf(g[5], s.y, fmaf(g[6], s.z, g[7])));
        const float p2 = fmaf(g[8], s.x, fmaf(g[9], s.y, fmaf(g[10], s.z, g[11])));
        const float dw = (ds0 * (p0 - m * xs0) + ds1 * (p1 - m * xs1) + ds2 * (p2 - m * xs2)) * inv_D + dS_alpha;
        const float ux = (p0 - P.bmin[0]) * P.vol_scale[0];
        const float uy = (p1 - P.bmin[1]) * P.vol_scale[1];
        const float uz = (p2 - P.bmin[2]) * P.vol_scale[2];
        if (T.dG && active) {
          float gx, gy, gz;
          const float w = trilinear_quad_grad(P.wquad + (size_t)i * QC, R, ux, uy, uz, gx, gy, gz);
          const float a = w * inv_D;
          col[(R_DP + 3 * i + 0) * stride] = fmaf(a, ds0, dw * gx * P.vol_scale[0]);
          col[(R_DP + 3 * i + 1) * stride] = fmaf(a, ds1, dw * gy * P.vol_scale[1]);
          col[(R_DP + 3 * i + 2) * stride] = fmaf(a, ds2, dw * gz * P.vol_scale[2]);
        }
        const float fx0 = floorf(ux), fy0 = floorf(uy), fz0 = floorf(uz);
        const bool in_range = fx0 >= -1.f && fy0 >= -1.f && fz0 >= -1.f && fx0 < (float)R && fy0 < (float)R &&
                              fz0 < (float)R;
        const bool valid = active && dw != 0.f && in_range;
        const int ix = valid ? (int)fx0 : 0, iy = valid ? (int)fy0 : 0, iz = valid ? (int)fz0 : 0;
        const float fx = ux - fx0, fy = uy - fy0, fz = uz - fz0;
        float v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
          v[c] = dw * (((c & 1) ? fx : 1.f - fx) * (((c >> 1) & 1) ? fy : 1.f - fy) * ((c >> 2) ? fz : 1.f - fz));
        const uint32_t key = (uint32_t)(ix + 1) | ((uint32_t)(iy + 1) << 10) | ((uint32_t)(iz + 1) << 20);
        if (run_sum<8>(key, 0u, valid, v)) {
          float *chg = T.g_wvol + (size_t)i * R3;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int ax = ix + (c & 1), ay = iy + ((c >> 1) & 1), az = iz + (c >> 2);
            if (ax < 0 || ay < 0 || az < 0 || ax >= R || ay >= R || az >= R) continue;
            atomicAdd(chg + (az * R + ay) * R + ax, v[c]);
          }
        }
      }
    }
    if (T.dG && !active)   // the refiner's reduction reads these rows of every lane
      for (int q = 0; q < 3 * kBones + 3; ++q) col[(R_DP + q) * stride] = 0.f;
    __syncwarp();
    if (T.dG) {
      // dL/dG_i of each frame: dR_i += dp_i x^T, dt_i += dp_i over the warp's 32 samples;
      // lane owns 9 of the 24 x 12 entries and sums them per run of equal frames
      const int fl = qv ? (int)T.frame_id[r] : -1;
      const int f0 = __shfl_sync(0xffffffffu, fl, 0);
      if (__all_sync(0xffffffffu, fl == f0) && f0 >= 0) {
        // one frame in the warp: C[3i + r][c] = sum_s dp_i[s][r] (x_s, y_s, z_s, 1)[c] as one
        // tensor-core product (M = 72 rows of dp in 16-row tiles, N = 4 columns padded to 8,
        // K = the 32 samples; m16n8k8 TF32, three products per step)
        const int g = lane >> 2, t = lane & 3;
        float *dst = (T.dG_smem ? sdG : T.dG) + (size_t)f0 * kBones * 12;
        uint32_t bh[4][2], bl[4][2];   // B[s][c] = (x, y, z, 1)[c] of sample s, zero for c >= 4
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const int s0 = 8 * ks + t;
          const float v0 = g < 3 ? wcol[(R_XS + g) * stride + s0] : (g == 3 ? 1.f : 0.f);
          const float v1 = g < 3 ? wcol[(R_XS + g) * stride + s0 + 4] : (g == 3 ? 1.f : 0.f);
          tf32_split(v0, bh[ks][0], bl[ks][0]);
          tf32_split(v1, bh[ks][1], bl[ks][1]);
        }
#pragma unroll 1
        for (int mt = 0; mt < 5; ++mt) {
          const int o0 = 16 * mt + g, o8 = o0 + 8;
          float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const int s0 = 8 * ks + t;
            uint32_t ah[4], al[4];
            tf32_split(o0 < 3 * kBones ? wcol[(R_DP + o0) * stride + s0] : 0.f, ah[0], al[0]);
            tf32_split(o8 < 3 * kBones ? wcol[(R_DP + o8) * stride + s0] : 0.f, ah[1], al[1]);
            tf32_split(o0 < 3 * kBones ? wcol[(R_DP + o0) * stride + s0 + 4] : 0.f, ah[2], al[2]);
            tf32_split(o8 < 3 * kBones ? wcol[(R_DP + o8) * stride + s0 + 4] : 0.f, ah[3], al[3]);
            mma_tf32(c, al, bh[ks]);
            mma_tf32(c, ah, bl[ks]);
            mma_tf32(c, ah, bh[ks]);
          }
          // c = C[o0][2t], C[o0][2t + 1], C[o8][2t], C[o8][2t + 1]
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int o = q >= 2 ? o8 : o0, cc = 2 * t + (q & 1);
            if (o < 3 * kBones && cc < 4 && c[q] != 0.f) atomicAdd(dst + (o / 3) * 12 + (o % 3) * 4 + cc, c[q]);
          }
        }
      } else {
      for (int o = lane; o < kBones * 12; o += 32) {
        const int i = o / 12, rr = (o % 12) >> 2, c = o & 3;
        const float *dpr = wcol + (R_DP + 3 * i + rr) * stride;
        const float *xr = wcol + (R_XS + (c < 3 ? c : 0)) * stride;
        int cur = -1;
        float v = 0.f;
        for (int sI = 0; sI < 32; ++sI) {
          const int fr = __shfl_sync(0xffffffffu, fl, sI);
          if (fr < 0) break;
          if (fr != cur) {
            if (cur >= 0 && v != 0.f) atomicAdd((T.dG_smem ? sdG : T.dG) + cur * kBones * 12 + o, v);
            cur = fr;
            v = 0.f;
          }
          v = fmaf(dpr[sI], c < 3 ? xr[sI] : 1.f, v);
        }
        if (cur >= 0 && v != 0.f) atomicAdd((T.dG_smem ? sdG : T.dG) + cur * kBones * 12 + o, v);
      }
      }
    }
    __syncwarp();
  }
  if (T.dG && T.dG_smem) {
    __syncthreads();
    for (int i = threadIdx.x; i < T.n_frames * kBones * 12; i += blockDim.x)
      if (sdG[i] != 0.f) atomicAdd(T.dG + i, sdG[i]);
  }
}

// Sum of the per-block accumulators: red[e] = sum_w wacc[w][e].
__global__ void reduce_acc_kernel(const float *__restrict__ wacc, int n_warps, int A, float *__restrict__ red) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= A) return;
  float s = 0.f;
  for (int w = 0; w < n_warps; ++w) s += wacc[(size_t)w * A + e];
  red[e] = s;
}

// Gradients in the packed master layout (W[out][in], b) from the transposed
// blob-shaped sums; the joint-angle columns of the residual first layer get
// dL/dW_Omega[j][m] = sum_f (sum of delta1 over frame f)[j] * Omega_f[m].
struct ScatterArgs {
  MasterOffsets m;
  BlobLayout b;
  int g, pose_dim, n_frames, hidden, mlp_in;
};

__global__ void scatter_res_kernel(const float *__restrict__ red, const float *__restrict__ fomega, ScatterArgs a,
                                   float *__restrict__ g_res) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.m.n_res) return;
  const float *accF = red + a.b.total;
  // find the layer
  const int rin[5] = {a.g + a.pose_dim, kWidth, kWidth, kWidth + a.g, kWidth};
  const int rout[5] = {kWidth, kWidth, kWidth, kWidth, 3};
  const int wt[5] = {a.b.r1, a.b.r2, a.b.r3, a.b.r4, a.b.r5};
  const int bb[5] = {a.b.r1b, a.b.r2b, a.b.r3b, a.b.r4b, a.b.r5b};
  const int ostride[5] = {kWidth, kWidth, kWidth, kWidth, 4};
  for (int l = 0; l < 5; ++l) {
    if (e >= a.m.r[l] && e < a.m.rb[l]) {
      const int q = e - a.m.r[l], j = q / rin[l], k = q % rin[l];
      float v;
      if (l == 0 && k >= a.g) {
        const int mm = k - a.g;
        v = 0.f;
        for (int f = 0; f < a.n_frames; ++f) v = fmaf(accF[f * kWidth + j], fomega[f * a.pose_dim + mm], v);
      } else if (l == 3 && k >= kWidth) {
        v = red[wt[l] + (kWidth + (k - kWidth)) * ostride[l] + j];
      } else {
        v = red[wt[l] + k * ostride[l] + j];
      }
      g_res[e] = v;
      return;
    }
    if (e >= a.m.rb[l] && e < a.m.rb[l] + rout[l]) {
      g_res[e] = red[bb[l] + (e - a.m.rb[l])];
      return;
    }
  }
}

__global__ void scatter_mlp_kernel(const float *__restrict__ red, ScatterArgs a, float *__restrict__ g_mlp) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.m.n_mlp) return;
  const int H = a.hidden;
  for (int l = 0; l <= H; ++l) {
    const int in = l == 0 ? a.mlp_in : kWidth;
    const int out = l == H ? 4 : kWidth;
    const int wt = l == 0 ? a.b.c0 : (l == H ? a.b.cl : a.b.ch[l - 1]);
    const int bb = l == 0 ? a.b.c0b : (l == H ? a.b.clb : a.b.chb[l - 1]);
    const int ostride = l == H ? 4 : kWidth;
    if (e >= a.m.c[l] && e < a.m.cb[l]) {
      const int q = e - a.m.c[l], j = q / in, k = q % in;
      g_mlp[e] = red[wt + k * ostride + j];
      return;
    }
    if (e >= a.m.cb[l] && e < a.m.cb[l] + out) {
      g_mlp[e] = red[bb + (e - a.m.cb[l])];
      return;
    }
  }
}

// Adam with bias correction (Kingma and Ba 2015; Sec. 5.2 uses beta = (0.9, 0.99)):
// m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, p -= lr (m c1) / (sqrt(v c2) + eps),
// c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t).  Every entry is updated.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

template <typename P_>
static nr_status grow(P_ *&ptr, size_t &cap, size_t need) {
  if (need <= cap) return NR_OK;
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  cap = 0;
  NR_CHECK_CUDA(cudaMalloc((void **)&ptr, need * sizeof(P_)));
  cap = need;
  return NR_OK;
}

}  // namespace nr

using namespace nr;

extern "C" nr_status nr_train_step(nr_subject *s, const nr_train_batch *b, float *loss_out, void *stream) {
  NR_REQUIRE(subject_ok(s), "nr_train_step: invalid handle");
  NR_REQUIRE(b, "nr_train_step: NULL batch");
  NR_REQUIRE(b->n_rays >= 1 && b->frame_id && b->px && b->py, "nr_train_step: empty or NULL batch");
  const bool fwd_only = (b->flags & NR_FORWARD_ONLY) != 0;
  NR_REQUIRE(b->target_rgb || b->grad_rgb || fwd_only, "nr_train_step: neither target_rgb nor grad_rgb");
  NR_REQUIRE(b->n_samples >= 1 && b->n_samples <= 1024, "nr_train_step: n_samples must be 1..1024");
  NR_REQUIRE((uint64_t)b->n_rays * b->n_samples <= (1ull << 31), "nr_train_step: batch too large");
  NR_REQUIRE(b->lr >= 0.f && b->beta1 >= 0.f && b->beta1 < 1.f && b->beta2 >= 0.f && b->beta2 < 1.f && b->eps > 0.f,
             "nr_train_step: bad Adam hyper-parameters");
  for (int k = 0; k < 4; ++k) NR_REQUIRE(b->lr_scale[k] >= 0.f, "nr_train_step: negative lr_scale");
  NR_REQUIRE(b->loss_weight >= 0.f && b->lr_scale_refiner >= 0.f && b->lr_scale_cnn >= 0.f,
             "nr_train_step: negative loss_weight or lr scale");
  if (s->n_frames == 0) {
    set_error("nr_train_step: call nr_set_frames first");
    return NR_ESTATE;
  }
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  cudaStream_t st = (cudaStream_t)stream;
  nr_status r;
  if ((r = prepare_params(s, st)) != NR_OK) return r;
  const bool refine = s->ref_layers != 0;
  int launched = 0;
  if (refine) {   // every frame's G and updated angles from its refined pose (Sec. 4.1)
    if ((r = launch_refine_fk(s, s->f_omega, 3 * kBones, s->f_root, 3, (int)s->n_frames, s->f_G, s->f_omega_o,
                              3 * kBones, st)) != NR_OK)
      return r;
    s->fG_refined = true;
  } else if (s->fG_refined) {   // the refiner was switched off: back to the estimated poses
    NR_CHECK_CUDA(cudaMemcpyAsync(s->f_G, s->h_fG.data(), s->h_fG.size() * 4, cudaMemcpyHostToDevice, st));
    NR_CHECK_CUDA(cudaStreamSynchronize(st));
    s->fG_refined = false;
  }
  if ((r = fold_frame_biases(s, st)) != NR_OK) return r;
  nr_render_opts o{};
  o.mlp_dtype = NR_F32;
  o.feat_dtype = NR_F32;
  o.hann_alpha = b->hann_alpha;
  FieldParams P = field_params(s, &o);
  P.bone_box = nullptr;   // training differentiates every bone channel
  const size_t n = (size_t)b->n_rays * b->n_samples;
  const int blocks = num_sms(s->device);
  const int A = s->lay.total + (int)s->n_frames * kWidth;
  if (n > s->tw_samples) {              // the three per-sample buffers grow together
    size_t c0 = 0, c1 = 0, c2 = 0;
    if (s->t_samp) cudaFree(s->t_samp);
    if (s->t_out) cudaFree(s->t_out);
    if (s->t_T) cudaFree(s->t_T);
    s->t_samp = nullptr;
    s->t_out = nullptr;
    s->t_T = nullptr;
    s->tw_samples = 0;
    if ((r = grow(s->t_samp, c0, n)) != NR_OK) return r;
    if ((r = grow(s->t_out, c1, n)) != NR_OK) return r;
    if ((r = grow(s->t_T, c2, n)) != NR_OK) return r;
    s->tw_samples = n;
  }
  if ((r = grow(s->t_raycnt, s->tw_rays, (size_t)b->n_rays)) != NR_OK) return r;
  if ((r = grow(s->t_live, s->tw_live, ((size_t)b->n_rays * b->n_samples + 31) / 32)) != NR_OK) return r;
  const Rows rows = make_rows((int)s->hidden);
  if ((r = grow(s->t_scratch, s->tw_scratch, (size_t)blocks * rows.total * std::max(kFwdThreads, kBwdThreads))) !=
      NR_OK)
    return r;
  const size_t n_acc = (size_t)blocks;                 // one accumulator per block
  if ((r = grow(s->t_wacc, s->tw_acc, n_acc * A)) != NR_OK) return r;
  if ((r = grow(s->t_red, s->tw_red, (size_t)A)) != NR_OK) return r;
  if (!s->loss_acc) NR_CHECK_CUDA(cudaMalloc(&s->loss_acc, sizeof(float)));
  if (!s->adam_m) {
    s->n_params_total = s->n_wvol + s->n_table + s->n_mlp + s->n_res;
    NR_CHECK_CUDA(cudaMalloc(&s->adam_m, s->n_params_total * 4));
    NR_CHECK_CUDA(cudaMalloc(&s->adam_v, s->n_params_total * 4));
    NR_CHECK_CUDA(cudaMemsetAsync(s->adam_m, 0, s->n_params_total * 4, st));
    NR_CHECK_CUDA(cudaMemsetAsync(s->adam_v, 0, s->n_params_total * 4, st));
    s->adam_t = 0;
  }
  NR_CHECK_CUDA(cudaMemsetAsync(s->g_wvol, 0, s->n_wvol * 4, st));
  NR_CHECK_CUDA(cudaMemsetAsync(s->g_table, 0, s->n_table * 4, st));
  NR_CHECK_CUDA(cudaMemsetAsync(s->t_wacc, 0, n_acc * A * 4, st));
  NR_CHECK_CUDA(cudaMemsetAsync(s->loss_acc, 0, sizeof(float), st));
  const size_t n_dG = (size_t)s->n_frames * kBones * 12;
  const bool dG_smem = refine && s->n_frames <= 16;
  if (refine) {
    if ((r = grow(s->f_dG, s->f_dG_cap, n_dG)) != NR_OK) return r;
    NR_CHECK_CUDA(cudaMemsetAsync(s->f_dG, 0, n_dG * 4, st));
    NR_CHECK_CUDA(cudaMemsetAsync(s->g_ref, 0, s->n_ref * 4, st));
  }

  TrainDev T{};
  T.frame_id = b->frame_id;
  T.px = b->px;
  T.py = b->py;
  T.target = b->target_rgb;
  T.n_rays = b->n_rays;
  T.S = b->n_samples;
  T.ray_mul = ray_multiplier(b->n_rays);
  T.loss_weight = b->loss_weight > 0.f ? b->loss_weight : 1.f;
  T.seed = b->step_seed;
  for (int k = 0; k < 3; ++k) T.bg[k] = b->bg[k];
  T.cams = s->f_cam;
  T.fG = s->f_G;
  T.fbias1 = s->f_bias1;
  T.fomega = s->f_omega;
  T.samp = s->t_samp;
  T.out = s->t_out;
  T.T = s->t_T;
  T.raycnt = s->t_raycnt;
  T.live = s->t_live;
  T.loss = s->loss_acc;
  T.g_table = reinterpret_cast<float2 *>(s->g_table);
  T.g_wvol = s->g_wvol;
  T.scratch = s->t_scratch;
  T.wacc = s->t_wacc;
  T.acc_floats = A;
  T.n_frames = (int)s->n_frames;
  T.rw = rows;
  T.dG = refine ? s->f_dG : nullptr;
  T.dG_smem = dG_smem ? 1 : 0;
  T.pl = pad_layout(s->lay, (int)s->hidden);
  T.pred = b->pred_rgb;
  T.grad_rgb = fwd_only ? nullptr : b->grad_rgb;
  T.forward_only = fwd_only ? 1 : 0;

  train_samples_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(T, s->bmin[0], s->bmin[1], s->bmin[2], s->bmax[0],
                                                                     s->bmax[1], s->bmax[2]);
  NR_CHECK_CUDA(cudaGetLastError());
  const size_t smem_f = sizeof(float) * T.pl.total;
  // a step whose rays fit a backward block whole runs forward, compositing and backward in one
  // kernel (train_bwd_kernel<true>); else the forward and the compositing adjoint run first
  const bool fused = !fwd_only && b->n_samples <= (uint32_t)kBwdThreads;
  if (!fused) {
    NR_CHECK_CUDA(cudaFuncSetAttribute(train_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f));
    train_fwd_kernel<<<blocks, kFwdThreads, smem_f, st>>>(P, T);
    NR_CHECK_CUDA(cudaGetLastError());
    train_composite_kernel<<<(b->n_rays + 255) / 256, 256, 0, st>>>(T);
    NR_CHECK_CUDA(cudaGetLastError());
    launched += 2;
  }
  if (fwd_only) {
    count_launches(launched + 2);
    if (loss_out) {
      NR_CHECK_CUDA(cudaMemcpyAsync(loss_out, s->loss_acc, sizeof(float), cudaMemcpyDeviceToHost, st));
      NR_CHECK_CUDA(cudaStreamSynchronize(st));
    }
    return NR_OK;
  }
  const size_t smem_b = sizeof(float) * (T.pl.total + (dG_smem ? n_dG : 0)) + (fused ? kBwdThreads * 20 : 0);
  if (fused) {
    NR_CHECK_CUDA(
        cudaFuncSetAttribute(train_bwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    train_bwd_kernel<true><<<blocks, kBwdThreads, smem_b, st>>>(P, T);
  } else {
    NR_CHECK_CUDA(
        cudaFuncSetAttribute(train_bwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    train_bwd_kernel<false><<<blocks, kBwdThreads, smem_b, st>>>(P, T);
  }
  NR_CHECK_CUDA(cudaGetLastError());
  reduce_acc_kernel<<<(A + 255) / 256, 256, 0, st>>>(s->t_wacc, (int)n_acc, A, s->t_red);
  ScatterArgs sa{};
  sa.m = master_offsets(s);
  sa.b = s->lay;
  sa.g = res_gamma_dims(s);
  sa.pose_dim = 3 * (int)s->K;
  sa.n_frames = (int)s->n_frames;
  sa.hidden = (int)s->hidden;
  sa.mlp_in = (int)s->mlp_in;
  if (s->res_enabled) {
    scatter_res_kernel<<<(sa.m.n_res + 255) / 256, 256, 0, st>>>(s->t_red, refine ? s->f_omega_o : s->f_omega, sa,
                                                                 s->g_res);
  } else {
    NR_CHECK_CUDA(cudaMemsetAsync(s->g_res, 0, s->n_res * 4, st));
  }
  scatter_mlp_kernel<<<(sa.m.n_mlp + 255) / 256, 256, 0, st>>>(s->t_red, sa, s->g_mlp);
  NR_CHECK_CUDA(cudaGetLastError());
  launched += 5;   // samples, backward, reduction, two scatters
  if (refine && (r = launch_refine_bwd(s, s->f_omega, 3 * kBones, s->f_root, 3, (int)s->n_frames, s->f_dG,
                                       s->t_red + s->lay.total, s->g_ref, st)) != NR_OK)
    return r;
  if (s->cnn_on && (r = cnn_backward(s, st)) != NR_OK) return r;   // dL/dW^c -> CNN_skel
  if (!(b->flags & NR_GRAD_ONLY)) {
    const uint32_t mask = b->train_mask ? b->train_mask : NR_TRAIN_ALL;
    s->adam_t += 1;
    const double c1 = 1.0 / (1.0 - pow((double)b->beta1, (double)s->adam_t));
    const double c2 = 1.0 / (1.0 - pow((double)b->beta2, (double)s->adam_t));
    struct G_ {
      uint32_t bit;
      float *p, *g;
      size_t n, off;
      float scale;
    } groups[4] = {{NR_TRAIN_WVOL, s->wvol, s->g_wvol, s->n_wvol, 0, b->lr_scale[0]},
                   {NR_TRAIN_HASH, s->table, s->g_table, s->n_table, s->n_wvol, b->lr_scale[1]},
                   {NR_TRAIN_MLP, s->mlp, s->g_mlp, s->n_mlp, s->n_wvol + s->n_table, b->lr_scale[2]},
                   {NR_TRAIN_RES, s->res, s->g_res, s->n_res, s->n_wvol + s->n_table + s->n_mlp, b->lr_scale[3]}};
    for (const auto &g : groups) {
      if (!(mask & g.bit) || (g.bit == NR_TRAIN_RES && !s->res_enabled)) continue;
      if (g.bit == NR_TRAIN_WVOL && s->cnn_on) continue;   // the volume is generated, not stored
      const float lr = b->lr * (g.scale > 0.f ? g.scale : 1.f);
      const int nb = (int)std::min<size_t>((g.n + 255) / 256, (size_t)blocks * 8);
      adam_kernel<<<nb, 256, 0, st>>>(g.p, g.g, s->adam_m + g.off, s->adam_v + g.off, g.n, lr, b->beta1, b->beta2,
                                      b->eps, (float)c1, (float)c2);
      ++launched;
    }
    if (s->cnn_on && (mask & NR_TRAIN_CNN)) {
      s->cnn_t += 1;
      const double q1 = 1.0 / (1.0 - pow((double)b->beta1, (double)s->cnn_t));
      const double q2 = 1.0 / (1.0 - pow((double)b->beta2, (double)s->cnn_t));
      const float lr = b->lr * (b->lr_scale_cnn > 0.f ? b->lr_scale_cnn : 1.f);
      const int nb = (int)std::min<size_t>((s->n_cnn + 255) / 256, (size_t)blocks * 8);
      adam_kernel<<<nb, 256, 0, st>>>(s->cnn, s->g_cnn, s->cnn_m, s->cnn_v, s->n_cnn, lr, b->beta1, b->beta2, b->eps,
                                      (float)q1, (float)q2);
      ++launched;
      s->cnn_dirty = true;
    }
    if (refine && (mask & NR_TRAIN_REFINER)) {
      s->ref_t += 1;
      const double r1 = 1.0 / (1.0 - pow((double)b->beta1, (double)s->ref_t));
      const double r2 = 1.0 / (1.0 - pow((double)b->beta2, (double)s->ref_t));
      const float lr = b->lr * (b->lr_scale_refiner > 0.f ? b->lr_scale_refiner : 1.f);
      const int nb = (int)std::min<size_t>((s->n_ref + 255) / 256, (size_t)blocks * 8);
      adam_kernel<<<nb, 256, 0, st>>>(s->ref, s->g_ref, s->ref_m, s->ref_v, s->n_ref, lr, b->beta1, b->beta2, b->eps,
                                      (float)r1, (float)r2);
      ++launched;
      s->pose_dirty = s->pose_set;   // the current pose's refinement moved
    }
    NR_CHECK_CUDA(cudaGetLastError());
    s->params_dirty = true;
    s->bias_dirty = true;
  }
  count_launches(launched);
  if (loss_out) {
    NR_CHECK_CUDA(cudaMemcpyAsync(loss_out, s->loss_acc, sizeof(float), cudaMemcpyDeviceToHost, st));
    NR_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  return NR_OK;
}
