// refine.cu -- the pose refiner (Sec. 4.1): Delta_Omega = MLP_theta(Omega) on
// the joint angles of the non-root joints, the refined local rotations
// Rot(Delta_omega_j) Rot(omega_j), forward kinematics to the bone transforms
// G_i, and the backward of that chain from dL/dG_i to MLP_theta's weights.
//
// One block per pose.  The MLP runs in float32 with its activations in shared
// memory (one thread per unit); rotations and the kinematic chain run in
// float64 (24 joints, a few hundred operations) like the host's forward
// kinematics, and G is rounded to float32 at the end.  The backward block
// recomputes its pose's forward pass instead of storing it.
#include <math.h>
#include <string.h>

#include "render.cuh"

namespace nr {

constexpr int kRefIn = 3 * (kBones - 1);   // 69: non-root joint angles in, corrections out
constexpr int kRefThreads = 256;
constexpr int kRefMaxLayers = 4;

struct RefParams {
  int width, layers;            // hidden width (<= 256), hidden layers (1..4)
  const float *w;               // packed W[out][in] then b[out] per layer
  int parents[kBones];
  double J[kBones * 3];         // rest joints
};

// d = a b for row-major 3 x 3 matrices
__device__ __forceinline__ void mat3_mul(const double *a, const double *b, double *d) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) d[3 * r + c] = a[3 * r] * b[c] + a[3 * r + 1] * b[3 + c] + a[3 * r + 2] * b[6 + c];
}

// Rot(v) = I + A K + B K^2, K = [v]_x, A = sin(th)/th, B = (1 - cos th)/th^2, with
// C = A'(th)/th = (th cos th - sin th)/th^3 and E = B'(th)/th = (th sin th - 2(1 - cos th))/th^4
// for the derivative; Taylor forms below th = 1e-3.
struct RodCoef {
  double A, B, C, E;
};

__device__ __forceinline__ RodCoef rod_coef(const double *v) {
  const double t2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  RodCoef k;
  if (t2 < 1e-6) {
    k.A = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
    k.B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
    k.C = -1.0 / 3.0 + t2 / 30.0;
    k.E = -1.0 / 12.0 + t2 / 180.0;
  } else {
    const double t = sqrt(t2), sn = sin(t), cs = cos(t);
    k.A = sn / t;
    k.B = (1.0 - cs) / t2;
    k.C = (t * cs - sn) / (t2 * t);
    k.E = (t * sn - 2.0 * (1.0 - cs)) / (t2 * t2);
  }
  return k;
}

__device__ __forceinline__ void skew(const double *v, double *K) {
  K[0] = 0.0;   K[1] = -v[2]; K[2] = v[1];
  K[3] = v[2];  K[4] = 0.0;   K[5] = -v[0];
  K[6] = -v[1]; K[7] = v[0];  K[8] = 0.0;
}

__device__ void rodrigues_d(const double *v, double *R) {
  const RodCoef k = rod_coef(v);
  double K[9], K2[9];
  skew(v, K);
  mat3_mul(K, K, K2);
#pragma unroll
  for (int e = 0; e < 9; ++e) R[e] = (e % 4 == 0 ? 1.0 : 0.0) + k.A * K[e] + k.B * K2[e];
}

// dv_a = <dR, dRot/dv_a>, dRot/dv_a = A E_a + B (E_a K + K E_a) + v_a (C K + E K^2), E_a = [e_a]_x
__device__ void rodrigues_grad(const double *v, const double *dR, double *dv) {
  const RodCoef k = rod_coef(v);
  double K[9], K2[9];
  skew(v, K);
  mat3_mul(K, K, K2);
  double dK = 0.0, dK2 = 0.0;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    dK += dR[e] * K[e];
    dK2 += dR[e] * K2[e];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double ea[3] = {0.0, 0.0, 0.0}, Ea[9], EK[9], KE[9];
    ea[a] = 1.0;
    skew(ea, Ea);
    mat3_mul(Ea, K, EK);
    mat3_mul(K, Ea, KE);
    double dE = 0.0, dS = 0.0;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      dE += dR[e] * Ea[e];
      dS += dR[e] * (EK[e] + KE[e]);
    }
    dv[a] = k.A * dE + k.B * dS + v[a] * (k.C * dK + k.E * dK2);
  }
}

// Log of a rotation (angle in [0, pi)): a = (R_32 - R_23, R_13 - R_31, R_21 - R_12) / 2 =
// sin(th) n, cos(th) = (tr R - 1) / 2, v = th / sin(th) a (1 + th^2 / 6 below sin = 1e-8).
__device__ void rot_log(const double *R, double *v) {
  const double a0 = 0.5 * (R[7] - R[5]), a1 = 0.5 * (R[2] - R[6]), a2 = 0.5 * (R[3] - R[1]);
  const double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
  const double s = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
  const double th = atan2(s, c);
  const double k = s < 1e-8 ? 1.0 + th * th / 6.0 : th / s;
  v[0] = k * a0;
  v[1] = k * a1;
  v[2] = k * a2;
}

// y = M^T x for M = I + p K + q K^2, K = [v]_x:  y_r = x_r + sum_c (p K_cr + q (K^2)_cr) x_c.
__device__ __forceinline__ void so3_poly_t(const double *v, double p, double q, const double *x, double *y) {
  double K[9], K2[9];
  skew(v, K);
  mat3_mul(K, K, K2);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    double a = x[r];
#pragma unroll
    for (int c = 0; c < 3; ++c) a += (p * K[3 * c + r] + q * K2[3 * c + r]) * x[c];
    y[r] = a;
  }
}

// Derivative of phi = Log(Rot(d) R0) in d: dphi = J_l^{-1}(phi) J_l(d) dd, with the left
// Jacobian J_l(v) = I + (1 - cos th)/th^2 K + (th - sin th)/th^3 K^2 and its inverse
// J_l^{-1}(phi) = I - K/2 + (1/th^2 - (1 + cos th) / (2 th sin th)) K^2.  Returns dd += J_l(d)^T
// J_l^{-1}(phi)^T g.
__device__ void log_compose_grad(const double *d, const double *phi, const double *g, double *dd) {
  double t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2], q;
  if (t2 < 1e-6) {
    q = 1.0 / 12.0 + t2 / 720.0;
  } else {
    const double t = sqrt(t2);
    q = 1.0 / t2 - (1.0 + cos(t)) / (2.0 * t * sin(t));
  }
  double y[3], z[3];
  so3_poly_t(phi, -0.5, q, g, y);
  t2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double p1, q1;
  if (t2 < 1e-6) {
    p1 = 0.5 - t2 / 24.0;
    q1 = 1.0 / 6.0 - t2 / 120.0;
  } else {
    const double t = sqrt(t2);
    p1 = (1.0 - cos(t)) / t2;
    q1 = (t - sin(t)) / (t2 * t);
  }
  so3_poly_t(d, p1, q1, y, z);
  for (int a = 0; a < 3; ++a) dd[a] += z[a];
}

// Shared state of one pose's forward pass.
struct RefShared {
  float in[kRefIn + 3];
  float h[kRefMaxLayers][kRefThreads];    // post-ReLU activations
  float delta[kRefIn + 3];
  double Ro[kBones][9];                   // Rot(omega_j)
  double Rd[kBones][9];                   // Rot(Delta_omega_j), j >= 1
  double Rl[kBones][9];                   // refined local rotation
  double AR[kBones][9], At[kBones][3];    // world rotation and position of each joint
};

// MLP_theta forward, refined rotations and the kinematic chain of pose `om`
// (72 angles) with root translation `rt`.  Every thread of the block calls it.
__device__ void refine_forward(const RefParams &P, const float *om, const float *rt, RefShared &sh) {
  const int t = threadIdx.x;
  if (t < kRefIn) sh.in[t] = om[3 + t];
  __syncthreads();
  const float *w = P.w;
  int in = kRefIn;
  const float *src = sh.in;
  for (int l = 0; l < P.layers; ++l) {
    const float *W = w, *b = w + (size_t)P.width * in;
    if (t < P.width) {
      float a = b[t];
      for (int k = 0; k < in; ++k) a = fmaf(W[(size_t)t * in + k], src[k], a);
      sh.h[l][t] = fmaxf(a, 0.f);
    }
    __syncthreads();
    w = b + P.width;
    in = P.width;
    src = sh.h[l];
  }
  if (t < kRefIn) {
    const float *W = w, *b = w + (size_t)kRefIn * in;
    float a = b[t];
    for (int k = 0; k < in; ++k) a = fmaf(W[(size_t)t * in + k], src[k], a);
    sh.delta[t] = a;
  }
  __syncthreads();
  if (t < kBones) {
    const double v[3] = {om[3 * t], om[3 * t + 1], om[3 * t + 2]};
    rodrigues_d(v, sh.Ro[t]);
    if (t == 0) {
      for (int e = 0; e < 9; ++e) sh.Rl[0][e] = sh.Ro[0][e];
    } else {
      const double d[3] = {sh.delta[3 * (t - 1)], sh.delta[3 * (t - 1) + 1], sh.delta[3 * (t - 1) + 2]};
      rodrigues_d(d, sh.Rd[t]);
      mat3_mul(sh.Rd[t], sh.Ro[t], sh.Rl[t]);
    }
  }
  __syncthreads();
  if (t == 0) {
    for (int i = 0; i < kBones; ++i) {
      const int p = P.parents[i];
      if (p < 0) {
        for (int e = 0; e < 9; ++e) sh.AR[i][e] = sh.Rl[i][e];
        for (int r = 0; r < 3; ++r) sh.At[i][r] = P.J[3 * i + r] + (double)rt[r];
      } else {
        mat3_mul(sh.AR[p], sh.Rl[i], sh.AR[i]);
        for (int r = 0; r < 3; ++r) {
          double a = sh.At[p][r];
          for (int m = 0; m < 3; ++m) a += sh.AR[p][3 * r + m] * (P.J[3 * i + m] - P.J[3 * p + m]);
          sh.At[i][r] = a;
        }
      }
    }
  }
  __syncthreads();
}

// G_i = (R_i | t_i), R_i = AR_i^T, t_i = J_i - AR_i^T At_i, rows [R | t] in float32, and the
// updated joint angles Omega^o (root: omega_0; j >= 1: Log of the refined local rotation).
__global__ void __launch_bounds__(kRefThreads) refine_fk_kernel(RefParams P, const float *__restrict__ omega,
                                                                int omega_stride, const float *__restrict__ root,
                                                                int root_stride, float *__restrict__ G,
                                                                float *__restrict__ omega_o, int omega_o_stride) {
  __shared__ RefShared sh;
  const int f = blockIdx.x, t = threadIdx.x;
  const float *om = omega + (size_t)f * omega_stride;
  refine_forward(P, om, root + (size_t)f * root_stride, sh);
  if (omega_o && t < kBones) {
    float *oo = omega_o + (size_t)f * omega_o_stride + 3 * t;
    if (t == 0) {
      oo[0] = om[0];
      oo[1] = om[1];
      oo[2] = om[2];
    } else {
      double v[3];
      rot_log(sh.Rl[t], v);
      oo[0] = (float)v[0];
      oo[1] = (float)v[1];
      oo[2] = (float)v[2];
    }
  }
  if (t < kBones) {
    float *g = G + ((size_t)f * kBones + t) * 12;
    for (int r = 0; r < 3; ++r) {
      double tr = P.J[3 * t + r];
      for (int c = 0; c < 3; ++c) {
        const double Rrc = sh.AR[t][3 * c + r];
        g[4 * r + c] = (float)Rrc;
        tr -= Rrc * sh.At[t][c];
      }
      g[4 * r + 3] = (float)tr;
    }
  }
}

// From dL/dG [F][24][12] of each pose to dL/d theta (added into g with atomics).
// dbias: [F][64] dL/d(first residual bias of each frame), W1: residual layer 1, rows of
// w1_stride floats whose columns w1_col.. hold W_Omega (bias1 = b1 + W_Omega Omega^o); NULL
// when the residual MLP is off.
__global__ void __launch_bounds__(kRefThreads) refine_bwd_kernel(RefParams P, const float *__restrict__ omega,
                                                                 int omega_stride, const float *__restrict__ root,
                                                                 int root_stride, const float *__restrict__ dG,
                                                                 const float *__restrict__ dbias,
                                                                 const float *__restrict__ W1, int w1_stride,
                                                                 int w1_col, float *__restrict__ g) {
  __shared__ RefShared sh;
  __shared__ double dAR[kBones][9], dAt[kBones][3], dRl[kBones][9];
  __shared__ float dcur[kRefThreads], dnext[kRefThreads], dout[kRefIn + 3], dom[3 * kBones];
  const int f = blockIdx.x, t = threadIdx.x;
  const float *gG = dG + (size_t)f * kBones * 12;
  const float *gb = dbias ? dbias + (size_t)f * kWidth : nullptr;
  // frames the batch did not touch have dG = 0 and dbias = 0: nothing to do
  bool any = false;
  for (int e = t; e < kBones * 12; e += blockDim.x) any |= gG[e] != 0.f;
  if (gb)
    for (int e = t; e < kWidth; e += blockDim.x) any |= gb[e] != 0.f;
  if (!__syncthreads_or(any)) return;
  refine_forward(P, omega + (size_t)f * omega_stride, root + (size_t)f * root_stride, sh);
  // dL/dOmega^o = W_Omega^T dL/dbias1
  if (t < 3 * kBones) {
    float a = 0.f;
    if (gb)
      for (int q = 0; q < kWidth; ++q) a = fmaf(W1[(size_t)q * w1_stride + w1_col + t], gb[q], a);
    dom[t] = a;
  }
  // G_i -> (AR_i, At_i):  R_i[r][c] = AR_i[c][r],  t_i[r] = J_i[r] - sum_c AR_i[c][r] At_i[c]
  if (t < kBones) {
    const float *d = gG + 12 * t;
    for (int c = 0; c < 3; ++c) {
      double a = 0.0;
      for (int r = 0; r < 3; ++r) {
        dAR[t][3 * c + r] = (double)d[4 * r + c] - (double)d[4 * r + 3] * sh.At[t][c];
        a -= sh.AR[t][3 * c + r] * (double)d[4 * r + 3];
      }
      dAt[t][c] = a;
    }
  }
  __syncthreads();
  // the chain in reverse: children (larger index) before their parent
  if (t == 0) {
    for (int i = kBones - 1; i >= 0; --i) {
      const int p = P.parents[i];
      if (p < 0) {
        for (int e = 0; e < 9; ++e) dRl[i][e] = dAR[i][e];
        continue;
      }
      // AR_i = AR_p Rl_i:  dAR_p += dAR_i Rl_i^T,  dRl_i = AR_p^T dAR_i
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          double a = 0.0, b = 0.0;
          for (int m = 0; m < 3; ++m) {
            a += dAR[i][3 * r + m] * sh.Rl[i][3 * c + m];
            b += sh.AR[p][3 * m + r] * dAR[i][3 * m + c];
          }
          dAR[p][3 * r + c] += a;
          dRl[i][3 * r + c] = b;
        }
      // At_i = AR_p (J_i - J_p) + At_p:  dAR_p += dAt_i (J_i - J_p)^T,  dAt_p += dAt_i
      for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) dAR[p][3 * r + c] += dAt[i][r] * (P.J[3 * i + c] - P.J[3 * p + c]);
        dAt[p][r] += dAt[i][r];
      }
    }
  }
  __syncthreads();
  // Rl_j = Rd_j Ro_j:  dRd_j = dRl_j Ro_j^T, then through Rot(Delta_omega_j)
  if (t >= 1 && t < kBones) {
    double dRd[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double a = 0.0;
        for (int m = 0; m < 3; ++m) a += dRl[t][3 * r + m] * sh.Ro[t][3 * c + m];
        dRd[3 * r + c] = a;
      }
    const double v[3] = {sh.delta[3 * (t - 1)], sh.delta[3 * (t - 1) + 1], sh.delta[3 * (t - 1) + 2]};
    double dv[3];
    rodrigues_grad(v, dRd, dv);
    // omega^o_j = Log(Rot(Delta_j) Rot(omega_j)) feeds the residual MLP
    const double go[3] = {dom[3 * t], dom[3 * t + 1], dom[3 * t + 2]};
    if (go[0] != 0.0 || go[1] != 0.0 || go[2] != 0.0) {
      double phi[3];
      rot_log(sh.Rl[t], phi);
      log_compose_grad(v, phi, go, dv);
    }
    for (int a = 0; a < 3; ++a) dout[3 * (t - 1) + a] = (float)dv[a];
  }
  __syncthreads();
  // MLP_theta backward; layer l has W_l [out][in] at offset off_l, b_l after it
  size_t off[kRefMaxLayers + 1];
  {
    size_t o = 0;
    int in = kRefIn;
    for (int l = 0; l < P.layers; ++l) {
      off[l] = o;
      o += (size_t)P.width * in + P.width;
      in = P.width;
    }
    off[P.layers] = o;
  }
  const int W = P.width;
  // output layer: in = width (h of the last hidden layer), out = 69
  {
    const float *h = sh.h[P.layers - 1];
    float *gW = g + off[P.layers], *gb = gW + (size_t)kRefIn * W;
    for (int e = t; e < kRefIn * W; e += blockDim.x) atomicAdd(gW + e, dout[e / W] * h[e % W]);
    if (t < kRefIn) atomicAdd(gb + t, dout[t]);
    if (t < W) {
      const float *Wo = P.w + off[P.layers];
      float a = 0.f;
      for (int j = 0; j < kRefIn; ++j) a = fmaf(Wo[(size_t)j * W + t], dout[j], a);
      dcur[t] = h[t] > 0.f ? a : 0.f;
    }
  }
  __syncthreads();
  for (int l = P.layers - 1; l >= 0; --l) {
    const int in = l == 0 ? kRefIn : W;
    const float *src = l == 0 ? sh.in : sh.h[l - 1];
    float *gW = g + off[l], *gb = gW + (size_t)W * in;
    for (int e = t; e < W * in; e += blockDim.x) atomicAdd(gW + e, dcur[e / in] * src[e % in]);
    if (t < W) atomicAdd(gb + t, dcur[t]);
    if (l > 0) {
      if (t < W) {
        const float *Wl = P.w + off[l];
        float a = 0.f;
        for (int j = 0; j < W; ++j) a = fmaf(Wl[(size_t)j * in + t], dcur[j], a);
        dnext[t] = sh.h[l - 1][t] > 0.f ? a : 0.f;
      }
      __syncthreads();
      if (t < W) dcur[t] = dnext[t];
      __syncthreads();
    }
  }
}

static RefParams ref_params(const nr_subject *s) {
  RefParams P{};
  P.width = (int)s->ref_width;
  P.layers = (int)s->ref_layers;
  P.w = s->ref;
  for (int i = 0; i < kBones; ++i) {
    P.parents[i] = s->parents[i];
    for (int k = 0; k < 3; ++k) P.J[3 * i + k] = s->rest[3 * i + k];
  }
  return P;
}

nr_status launch_refine_fk(const nr_subject *s, const float *omega, int omega_stride, const float *root,
                           int root_stride, int n, float *G, float *omega_o, int omega_o_stride, cudaStream_t st) {
  refine_fk_kernel<<<n, kRefThreads, 0, st>>>(ref_params(s), omega, omega_stride, root, root_stride, G, omega_o,
                                              omega_o_stride);
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(1);
  return NR_OK;
}

nr_status launch_refine_bwd(const nr_subject *s, const float *omega, int omega_stride, const float *root,
                            int root_stride, int n, const float *dG, const float *dbias, float *g, cudaStream_t st) {
  const int gd = res_gamma_dims(s);
  refine_bwd_kernel<<<n, kRefThreads, 0, st>>>(ref_params(s), omega, omega_stride, root, root_stride, dG,
                                               s->res_enabled ? dbias : nullptr, s->res, gd + 3 * (int)s->K, gd,
                                               g);
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(1);
  return NR_OK;
}

size_t refiner_param_count(uint32_t width, uint32_t layers) {
  size_t n = (size_t)width * kRefIn + width;
  n += (size_t)(layers - 1) * ((size_t)width * width + width);
  n += (size_t)kRefIn * width + kRefIn;
  return n;
}

}  // namespace nr

using namespace nr;

extern "C" nr_status nr_set_pose_refiner(nr_subject *s, uint32_t width, uint32_t hidden_layers, const float *params,
                                         void *stream) {
  NR_REQUIRE(subject_ok(s), "nr_set_pose_refiner: invalid handle");
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (!params) {   // switch the refiner off
    s->ref_width = s->ref_layers = 0;
    s->pose_dirty = s->pose_set;
    return NR_OK;
  }
  NR_REQUIRE(width >= 1 && width <= (uint32_t)kRefThreads, "nr_set_pose_refiner: width must be 1..256");
  NR_REQUIRE(hidden_layers >= 1 && hidden_layers <= (uint32_t)kRefMaxLayers,
             "nr_set_pose_refiner: hidden_layers must be 1..4");
  const size_t n = refiner_param_count(width, hidden_layers);
  for (size_t i = 0; i < n; ++i) NR_REQUIRE(isfinite(params[i]), "nr_set_pose_refiner: non-finite weight %zu", i);
  if (n != s->n_ref) {
    float *bufs[4] = {s->ref, s->g_ref, s->ref_m, s->ref_v};
    for (float *b : bufs)
      if (b) cudaFree(b);
    s->ref = s->g_ref = s->ref_m = s->ref_v = nullptr;
    s->n_ref = 0;
    NR_CHECK_CUDA(cudaMalloc(&s->ref, n * 4));
    NR_CHECK_CUDA(cudaMalloc(&s->g_ref, n * 4));
    NR_CHECK_CUDA(cudaMalloc(&s->ref_m, n * 4));
    NR_CHECK_CUDA(cudaMalloc(&s->ref_v, n * 4));
    s->n_ref = n;
  }
  NR_CHECK_CUDA(cudaMemcpyAsync(s->ref, params, n * 4, cudaMemcpyHostToDevice, st));
  NR_CHECK_CUDA(cudaMemsetAsync(s->g_ref, 0, n * 4, st));
  NR_CHECK_CUDA(cudaMemsetAsync(s->ref_m, 0, n * 4, st));
  NR_CHECK_CUDA(cudaMemsetAsync(s->ref_v, 0, n * 4, st));
  NR_CHECK_CUDA(cudaStreamSynchronize(st));   // params may be freed on return
  s->ref_width = width;
  s->ref_layers = hidden_layers;
  s->ref_t = 0;
  s->pose_dirty = s->pose_set;
  return NR_OK;
}
