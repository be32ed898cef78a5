// cnn.cu -- CNN_skel (Sec. 4.2): the canonical weight volume W^c generated from
// a constant latent z by a fully-connected layer and five 3D transposed
// convolutions (kernel 4, stride 2, padding 1: 1^3 -> 32^3), LeakyReLU(0.2)
// between layers and a softmax over the 25 channels (after adding log(prior)
// when one is given); and its backward from dL/dW^c to the network's weights.
//
// Parameters (float32, packed in this order): W_fc [C0][256], b_fc [C0], then
// for each transposed convolution k = 1..5: W_k [C_{k-1}][C_k][4][4][4],
// b_k [C_k] with C_5 = 25.  Everything runs on CUDA cores in float32: a forward
// is ~1 GFLOP at the default widths, small beside a training step.
//
// Transposed convolution, per axis: output u = 2 i - 1 + k (k = 0..3), so output
// u gathers input i = t (tap k = u + 1 - 2t) and i = t - 1 (tap k + 2), t = (u + 1) / 2.
#include <math.h>
#include <string.h>

#include "render.cuh"

namespace nr {

constexpr int kCnnZ = 256;
constexpr int kCnnOut = kBones + 1;   // 25 channels
constexpr int kCnnRes = 32;
constexpr float kSlope = 0.2f;

__device__ __forceinline__ float leaky(float v) { return v > 0.f ? v : kSlope * v; }
__device__ __forceinline__ float leaky_grad(float post) { return post > 0.f ? 1.f : kSlope; }

// the two (input index, tap) pairs feeding output coordinate u of an axis with r inputs
__device__ __forceinline__ void taps(int u, int r, int *i, int *k) {
  const int t = (u + 1) >> 1;
  i[0] = t;
  k[0] = u + 1 - 2 * t;
  i[1] = t - 1;
  k[1] = k[0] + 2;
  if (i[0] >= r) i[0] = -1;
  if (i[1] < 0) i[1] = -1;
}

__global__ void cnn_fc_fwd(const float *__restrict__ W, const float *__restrict__ b, const float *__restrict__ z,
                           int C0, float *__restrict__ h) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= C0) return;
  float a = b[o];
  for (int k = 0; k < kCnnZ; ++k) a = fmaf(W[(size_t)o * kCnnZ + k], z[k], a);
  h[o] = leaky(a);
}

// out[o][u] = b[o] + sum_i sum_taps in[i][tap] W[i][o][k(tap)]: `split` consecutive lanes per
// output (a power of two up to 32), lane j taking inputs i = j, j + split, ... and the group
// summing over shuffles, so that the first layers' few outputs still fill the GPU
__global__ void __launch_bounds__(256) cnn_convt_fwd(const float *__restrict__ in, const float *__restrict__ W,
                                                     const float *__restrict__ b, int Cin, int Cout, int r,
                                                     int act, int split, float *__restrict__ out) {
  const int R = 2 * r;
  const size_t n = (size_t)Cout * R * R * R;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t idx = t / split;
  const int j = (int)(t % split);
  const bool valid = idx < n;
  float acc = 0.f;
  if (valid) {
    const int x = (int)(idx % R), y = (int)((idx / R) % R), zz = (int)((idx / ((size_t)R * R)) % R);
    const int o = (int)(idx / ((size_t)R * R * R));
    int iz[2], kz[2], iy[2], ky[2], ix[2], kx[2];
    taps(zz, r, iz, kz);
    taps(y, r, iy, ky);
    taps(x, r, ix, kx);
    const size_t r3 = (size_t)r * r * r;
    for (int i = j; i < Cin; i += split) {
      const float *wi = W + ((size_t)i * Cout + o) * 64;
      const float *xi = in + (size_t)i * r3;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        if (iz[a] < 0) continue;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (iy[c] < 0) continue;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            if (ix[e] < 0) continue;
            acc = fmaf(xi[((size_t)iz[a] * r + iy[c]) * r + ix[e]], wi[(kz[a] * 4 + ky[c]) * 4 + kx[e]], acc);
          }
        }
      }
    }
  }
  for (int off = split >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (valid && j == 0) {
    acc += b[idx / ((size_t)R * R * R)];
    out[idx] = act ? leaky(acc) : acc;
  }
}

// W^c[c][v] = softmax_c(logit[c][v] + log_prior[c][v])
__global__ void cnn_softmax_fwd(const float *__restrict__ logit, const float *__restrict__ log_prior, int V,
                                float *__restrict__ w) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  float m = -INFINITY, a[kCnnOut];
#pragma unroll
  for (int c = 0; c < kCnnOut; ++c) {
    a[c] = logit[(size_t)c * V + v] + (log_prior ? log_prior[(size_t)c * V + v] : 0.f);
    m = fmaxf(m, a[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kCnnOut; ++c) {
    a[c] = expf(a[c] - m);
    s += a[c];
  }
  const float inv = 1.f / s;
#pragma unroll
  for (int c = 0; c < kCnnOut; ++c) w[(size_t)c * V + v] = a[c] * inv;
}

// dlogit[c][v] = w[c][v] (g[c][v] - sum_c' w[c'][v] g[c'][v])
__global__ void cnn_softmax_bwd(const float *__restrict__ w, const float *__restrict__ g, int V,
                                float *__restrict__ dlogit) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  float dot = 0.f;
#pragma unroll
  for (int c = 0; c < kCnnOut; ++c) dot = fmaf(w[(size_t)c * V + v], g[(size_t)c * V + v], dot);
#pragma unroll
  for (int c = 0; c < kCnnOut; ++c) {
    const size_t e = (size_t)c * V + v;
    dlogit[e] = w[e] * (g[e] - dot);
  }
}

// din[i][q] = leaky'(in[i][q]) sum_o sum_k W[i][o][k] dout[o][2 q - 1 + k]: `split` lanes per
// input (outputs o = j, j + split, ...), summed over shuffles
__global__ void __launch_bounds__(256) cnn_convt_bwd_data(const float *__restrict__ in, const float *__restrict__ W,
                                                          const float *__restrict__ dout, int Cin, int Cout, int r,
                                                          int split, float *__restrict__ din) {
  const size_t r3 = (size_t)r * r * r;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t idx = t / split;
  const int j = (int)(t % split);
  const bool valid = idx < (size_t)Cin * r3;
  float acc = 0.f;
  if (valid) {
    const int q = (int)(idx % r3), i = (int)(idx / r3);
    const int x = q % r, y = (q / r) % r, zz = q / (r * r);
    const int R = 2 * r;
    const size_t R3 = (size_t)R * R * R;
    for (int o = j; o < Cout; o += split) {
      const float *wi = W + ((size_t)i * Cout + o) * 64;
      const float *go = dout + (size_t)o * R3;
      for (int kz = 0; kz < 4; ++kz) {
        const int uz = 2 * zz - 1 + kz;
        if (uz < 0 || uz >= R) continue;
        for (int ky = 0; ky < 4; ++ky) {
          const int uy = 2 * y - 1 + ky;
          if (uy < 0 || uy >= R) continue;
#pragma unroll
          for (int kx = 0; kx < 4; ++kx) {
            const int ux = 2 * x - 1 + kx;
            if (ux < 0 || ux >= R) continue;
            acc = fmaf(wi[(kz * 4 + ky) * 4 + kx], go[((size_t)uz * R + uy) * R + ux], acc);
          }
        }
      }
    }
  }
  for (int off = split >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (valid && j == 0) din[idx] = acc * leaky_grad(in[idx]);
}

// dW[i][o][k] = sum_q in[i][q] dout[o][2 q - 1 + k], one thread per weight (k fastest)
__global__ void __launch_bounds__(256) cnn_convt_bwd_weight(const float *__restrict__ in, const float *__restrict__ dout,
                                                            int Cin, int Cout, int r, float *__restrict__ dW) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)Cin * Cout * 64) return;
  const int k = (int)(idx % 64);
  const size_t io = idx / 64;
  const int o = (int)(io % Cout), i = (int)(io / Cout);
  const int kx = k & 3, ky = (k >> 2) & 3, kz = k >> 4;
  const int R = 2 * r;
  const size_t R3 = (size_t)R * R * R;
  const float *xi = in + (size_t)i * r * r * r;
  const float *go = dout + (size_t)o * R3;
  float acc = 0.f;
  for (int zz = 0; zz < r; ++zz) {
    const int uz = 2 * zz - 1 + kz;
    if (uz < 0 || uz >= R) continue;
    for (int y = 0; y < r; ++y) {
      const int uy = 2 * y - 1 + ky;
      if (uy < 0 || uy >= R) continue;
      for (int x = 0; x < r; ++x) {
        const int ux = 2 * x - 1 + kx;
        if (ux < 0 || ux >= R) continue;
        acc = fmaf(xi[((size_t)zz * r + y) * r + x], go[((size_t)uz * R + uy) * R + ux], acc);
      }
    }
  }
  dW[idx] = acc;
}

// db[o] = sum_u dout[o][u]: one block per channel
__global__ void cnn_bias_grad(const float *__restrict__ dout, int n_per, float *__restrict__ db) {
  __shared__ float red[256];
  const int o = blockIdx.x;
  float a = 0.f;
  for (int u = threadIdx.x; u < n_per; u += blockDim.x) a += dout[(size_t)o * n_per + u];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int sft = blockDim.x / 2; sft > 0; sft >>= 1) {
    if ((int)threadIdx.x < sft) red[threadIdx.x] += red[threadIdx.x + sft];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[o] = red[0];
}

// fully-connected layer: dW_fc[o][k] = dh[o] z[k], db_fc = dh (dh already through leaky')
__global__ void cnn_fc_bwd(const float *__restrict__ dh, const float *__restrict__ z, int C0, float *__restrict__ dW,
                           float *__restrict__ db) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)C0 * kCnnZ) return;
  const int o = (int)(idx / kCnnZ), k = (int)(idx % kCnnZ);
  dW[idx] = dh[o] * z[k];
  if (k == 0) db[o] = dh[o];
}

struct CnnLayout {
  size_t w[6], b[6];      // offsets of W and b of the fc layer (0) and convolutions 1..5
  int cin[6], cout[6], r[6];   // input channels, output channels, input resolution
  size_t act[6];          // offsets of each layer's output in the activation buffer
  size_t n_params, n_act, max_grad;
};

static CnnLayout cnn_layout(const uint32_t *ch) {
  CnnLayout L{};
  size_t o = 0;
  L.cin[0] = kCnnZ;
  L.cout[0] = (int)ch[0];
  L.r[0] = 1;
  L.w[0] = o;
  o += (size_t)ch[0] * kCnnZ;
  L.b[0] = o;
  o += ch[0];
  int r = 1;
  for (int k = 1; k <= 5; ++k) {
    L.cin[k] = (int)ch[k - 1];
    L.cout[k] = k < 5 ? (int)ch[k] : kCnnOut;
    L.r[k] = r;
    L.w[k] = o;
    o += (size_t)L.cin[k] * L.cout[k] * 64;
    L.b[k] = o;
    o += L.cout[k];
    r *= 2;
  }
  L.n_params = o;
  size_t a = 0, mg = 0;
  for (int k = 0; k <= 5; ++k) {
    const size_t rr = (size_t)(k == 0 ? 1 : 2 * L.r[k]);
    const size_t n = (size_t)L.cout[k] * rr * rr * rr;
    L.act[k] = a;
    a += n;
    mg = std::max(mg, n);
  }
  L.n_act = a;
  L.max_grad = mg;
  return L;
}

static unsigned blocks_for(size_t n) { return (unsigned)((n + 255) / 256); }

// Lanes per output of a layer with n outputs, each a sum over `terms` inputs (or outputs): enough
// that the launch reaches ~2^18 threads, at most 32 and no more than the terms.
static int cnn_split(size_t n, int terms) {
  int sp = 1;
  while (sp < 32 && sp < terms && n * (size_t)sp < (size_t(1) << 18)) sp *= 2;
  return sp;
}

// W^c = CNN_skel(z) into s->wvol; keeps the activations for the backward.
nr_status cnn_forward(nr_subject *s, cudaStream_t st) {
  const CnnLayout L = cnn_layout(s->cnn_ch);
  float *A = s->cnn_act;
  cnn_fc_fwd<<<blocks_for(L.cout[0]), 256, 0, st>>>(s->cnn + L.w[0], s->cnn + L.b[0], s->cnn_z, L.cout[0],
                                                     A + L.act[0]);
  for (int k = 1; k <= 5; ++k) {
    const size_t R = 2 * (size_t)L.r[k];
    const size_t nout = (size_t)L.cout[k] * R * R * R;
    const int sp = cnn_split(nout, L.cin[k]);
    cnn_convt_fwd<<<blocks_for(nout * sp), 256, 0, st>>>(A + L.act[k - 1], s->cnn + L.w[k], s->cnn + L.b[k],
                                                         L.cin[k], L.cout[k], L.r[k], k < 5 ? 1 : 0, sp,
                                                         A + L.act[k]);
  }
  const int V = kCnnRes * kCnnRes * kCnnRes;
  cnn_softmax_fwd<<<blocks_for(V), 256, 0, st>>>(A + L.act[5], s->cnn_prior, V, s->wvol);
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(7);
  return NR_OK;
}

// dL/dtheta_cnn into s->g_cnn from dL/dW^c in s->g_wvol (the forward's activations and
// s->wvol must be those of the current parameters).
nr_status cnn_backward(nr_subject *s, cudaStream_t st) {
  const CnnLayout L = cnn_layout(s->cnn_ch);
  const float *A = s->cnn_act;
  float *d0 = s->cnn_grad, *d1 = s->cnn_grad + L.max_grad;
  const int V = kCnnRes * kCnnRes * kCnnRes;
  cnn_softmax_bwd<<<blocks_for(V), 256, 0, st>>>(s->wvol, s->g_wvol, V, d0);
  int launched = 1;
  for (int k = 5; k >= 1; --k) {
    const size_t R = 2 * (size_t)L.r[k];
    const size_t nout = R * R * R;
    cnn_convt_bwd_weight<<<blocks_for((size_t)L.cin[k] * L.cout[k] * 64), 256, 0, st>>>(
        A + L.act[k - 1], d0, L.cin[k], L.cout[k], L.r[k], s->g_cnn + L.w[k]);
    cnn_bias_grad<<<L.cout[k], 256, 0, st>>>(d0, (int)nout, s->g_cnn + L.b[k]);
    const size_t nin = (size_t)L.cin[k] * L.r[k] * L.r[k] * L.r[k];
    const int sp = cnn_split(nin, L.cout[k]);
    cnn_convt_bwd_data<<<blocks_for(nin * sp), 256, 0, st>>>(A + L.act[k - 1], s->cnn + L.w[k], d0, L.cin[k],
                                                             L.cout[k], L.r[k], sp, d1);
    std::swap(d0, d1);
    launched += 3;
  }
  cnn_fc_bwd<<<blocks_for((size_t)L.cout[0] * kCnnZ), 256, 0, st>>>(d0, s->cnn_z, L.cout[0], s->g_cnn + L.w[0],
                                                                     s->g_cnn + L.b[0]);
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(launched + 1);
  return NR_OK;
}

size_t cnn_param_count(const uint32_t *ch) { return cnn_layout(ch).n_params; }

}  // namespace nr

using namespace nr;

extern "C" nr_status nr_set_weight_cnn(nr_subject *s, const uint32_t *channels, const float *params, const float *z,
                                       const float *log_prior, void *stream) {
  NR_REQUIRE(subject_ok(s), "nr_set_weight_cnn: invalid handle");
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (!params) {   // back to the directly stored volume (it keeps the last generated values)
    s->cnn_on = false;
    return NR_OK;
  }
  NR_REQUIRE(channels && z, "nr_set_weight_cnn: NULL channels or z");
  NR_REQUIRE(s->wres == (uint32_t)kCnnRes, "nr_set_weight_cnn: the subject's weight volume must be 32^3");
  for (int k = 0; k < 5; ++k)
    NR_REQUIRE(channels[k] >= 1 && channels[k] <= 4096, "nr_set_weight_cnn: channels[%d] must be 1..4096", k);
  const CnnLayout L = cnn_layout(channels);
  for (size_t i = 0; i < L.n_params; ++i)
    NR_REQUIRE(isfinite(params[i]), "nr_set_weight_cnn: non-finite weight %zu", i);
  float *bufs[] = {s->cnn, s->g_cnn, s->cnn_m, s->cnn_v, s->cnn_z, s->cnn_prior, s->cnn_act, s->cnn_grad};
  for (float *b : bufs)
    if (b) cudaFree(b);
  s->cnn = s->g_cnn = s->cnn_m = s->cnn_v = s->cnn_z = s->cnn_prior = s->cnn_act = s->cnn_grad = nullptr;
  s->cnn_on = false;
  s->n_cnn = 0;
  const size_t V = (size_t)kCnnRes * kCnnRes * kCnnRes;
  NR_CHECK_CUDA(cudaMalloc(&s->cnn, L.n_params * 4));
  NR_CHECK_CUDA(cudaMalloc(&s->g_cnn, L.n_params * 4));
  NR_CHECK_CUDA(cudaMalloc(&s->cnn_m, L.n_params * 4));
  NR_CHECK_CUDA(cudaMalloc(&s->cnn_v, L.n_params * 4));
  NR_CHECK_CUDA(cudaMalloc(&s->cnn_z, kCnnZ * 4));
  NR_CHECK_CUDA(cudaMalloc(&s->cnn_act, L.n_act * 4));
  NR_CHECK_CUDA(cudaMalloc(&s->cnn_grad, 2 * L.max_grad * 4));
  if (log_prior) NR_CHECK_CUDA(cudaMalloc(&s->cnn_prior, kCnnOut * V * 4));
  NR_CHECK_CUDA(cudaMemcpyAsync(s->cnn, params, L.n_params * 4, cudaMemcpyHostToDevice, st));
  NR_CHECK_CUDA(cudaMemcpyAsync(s->cnn_z, z, kCnnZ * 4, cudaMemcpyHostToDevice, st));
  if (log_prior) NR_CHECK_CUDA(cudaMemcpyAsync(s->cnn_prior, log_prior, kCnnOut * V * 4, cudaMemcpyHostToDevice, st));
  NR_CHECK_CUDA(cudaMemsetAsync(s->g_cnn, 0, L.n_params * 4, st));
  NR_CHECK_CUDA(cudaMemsetAsync(s->cnn_m, 0, L.n_params * 4, st));
  NR_CHECK_CUDA(cudaMemsetAsync(s->cnn_v, 0, L.n_params * 4, st));
  NR_CHECK_CUDA(cudaStreamSynchronize(st));   // the host arrays may be freed on return
  memcpy(s->cnn_ch, channels, sizeof(s->cnn_ch));
  s->n_cnn = L.n_params;
  s->cnn_t = 0;
  s->cnn_on = true;
  s->cnn_dirty = true;
  return NR_OK;
}
