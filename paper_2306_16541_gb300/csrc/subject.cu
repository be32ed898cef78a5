// subject.cu -- subject lifetime, pose (forward kinematics, posed occupancy
// bitfield), derived weight layouts and parameter access for libnr.so.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>

#include "field.cuh"
#include "render.cuh"
#include "t5.cuh"

namespace nr {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

nr_status set_error_cuda(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? NR_ENOMEM : NR_ECUDA;
}

bool subject_ok(const nr_subject *s) { return s && s->magic == 0x4e525342u; }

static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ------------------------------------------------------- forward kinematics
// Sec. 4.2: G_i(x) = R_i x + t_i maps observation to canonical space for bone
// i.  With A_i the posed world transform of joint i (A_root = [Rot(w_0) |
// J_0 + root_t], A_i = A_parent o [Rot(w_i) | J_i - J_parent]) and the rest
// pose as canonical pose, G_i = (A_i o [I | -J_i])^{-1}:
//   R_i = A_i.R^T,  t_i = J_i - A_i.R^T A_i.t.
// Rot is the axis-angle rotation (Rodrigues' formula).  float64 on the host.
static void rodrigues(const double a[3], double R[9]) {
  const double th = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  double K[9] = {0, -a[2], a[1], a[2], 0, -a[0], -a[1], a[0], 0};
  double s, c1;
  if (th < 1e-12) {
    s = 1.0;
    c1 = 0.0;
  } else {
    for (double &k : K) k /= th;
    s = sin(th);
    c1 = 1.0 - cos(th);
  }
  double KK[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0;
      for (int m = 0; m < 3; ++m) acc += K[r * 3 + m] * K[m * 3 + c];
      KK[r * 3 + c] = acc;
    }
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + s * K[i] + c1 * KK[i];
}

void forward_kinematics(const nr_subject *s, const float *aa, const float *root_t, float *G) {
  const int K = (int)s->K;
  std::vector<double> AR(K * 9), At(K * 3);
  for (int i = 0; i < K; ++i) {
    double a[3] = {aa[3 * i], aa[3 * i + 1], aa[3 * i + 2]}, Rl[9];
    rodrigues(a, Rl);
    const double *J = &s->rest[3 * i];
    const int p = s->parents[i];
    if (p < 0) {
      for (int k = 0; k < 9; ++k) AR[9 * i + k] = Rl[k];
      for (int k = 0; k < 3; ++k) At[3 * i + k] = J[k] + (root_t ? (double)root_t[k] : 0.0);
    } else {
      const double *Jp = &s->rest[3 * p];
      for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
          double acc = 0;
          for (int m = 0; m < 3; ++m) acc += AR[9 * p + 3 * r + m] * Rl[3 * m + c];
          AR[9 * i + 3 * r + c] = acc;
        }
        double acc = At[3 * p + r];
        for (int m = 0; m < 3; ++m) acc += AR[9 * p + 3 * r + m] * (J[m] - Jp[m]);
        At[3 * i + r] = acc;
      }
    }
  }
  for (int i = 0; i < K; ++i) {
    const double *J = &s->rest[3 * i];
    for (int r = 0; r < 3; ++r) {
      double tr = J[r];
      for (int c = 0; c < 3; ++c) {
        const double Rrc = AR[9 * i + 3 * c + r];  // (A.R^T)[r][c]
        G[12 * i + 4 * r + c] = (float)Rrc;
        tr -= Rrc * At[3 * i + c];
      }
      G[12 * i + 4 * r + 3] = (float)tr;
    }
  }
}

// ------------------------------------------------------------ posed bitfield
// Empty-space skipping (Sec. 2.3) over the performer's box: cell c is set iff
// for some bone i the canonical image q = G_i(centre_c) lies inside canonical
// ellipsoid i dilated by half a cell diagonal.  Every operation is an
// explicitly rounded float32 operation (no contraction into FMA) so that the
// decision is reproducible: see the evaluation order written beside each line.
__global__ void __launch_bounds__(256) posed_bitfield_kernel(const float *__restrict__ G, const float *__restrict__ E,
                                                             float bx, float by, float bz, float Bx, float By,
                                                             float Bz, int grid, uint32_t *__restrict__ bits) {
  __shared__ float sG[kBones * 12], sE[kBones * 15], sC[kBones * 4];
  for (int i = threadIdx.x; i < kBones * 12; i += blockDim.x) sG[i] = G[i];
  for (int i = threadIdx.x; i < kBones * 15; i += blockDim.x) sE[i] = E[i];
  const uint32_t n = (uint32_t)grid * grid * grid;
  const float fg = (float)grid;
  const float h0 = __fdiv_rn(__fsub_rn(Bx, bx), fg);     // (bmax - bmin) / G
  const float h1 = __fdiv_rn(__fsub_rn(By, by), fg);
  const float h2 = __fdiv_rn(__fsub_rn(Bz, bz), fg);
  // 0.5 sqrt(((h0 h0) + (h1 h1)) + (h2 h2))
  const float dil = __fmul_rn(0.5f, __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(h0, h0), __fmul_rn(h1, h1)),
                                                         __fmul_rn(h2, h2))));
  __syncthreads();
  // A filter that never changes the decision: G_i is rigid, so a centre passing the
  // test lies within the largest dilated radius rho_i of ellipsoid i's centre mapped to
  // the observation space, c_i = R_i^T (centre_i - t_i); with a 1 mm margin far above
  // float32 rounding, a centre farther than that skips the exact test.
  if (threadIdx.x < kBones) {
    const int i = threadIdx.x;
    const float *g = sG + 12 * i;
    const float *e = sE + 15 * i;
    const float d0 = e[0] - g[3], d1 = e[1] - g[7], d2 = e[2] - g[11];
    sC[4 * i + 0] = g[0] * d0 + g[4] * d1 + g[8] * d2;
    sC[4 * i + 1] = g[1] * d0 + g[5] * d1 + g[9] * d2;
    sC[4 * i + 2] = g[2] * d0 + g[6] * d1 + g[10] * d2;
    const float rho = fmaxf(fmaxf(e[12], e[13]), e[14]) + dil + 1e-3f;
    // only for a rotation (transforms given as matrices need not be rigid): |R^T R - I| small
    float dev = 0.f;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const float rr = g[a] * g[b] + g[4 + a] * g[4 + b] + g[8 + a] * g[8 + b];
        dev = fmaxf(dev, fabsf(rr - (a == b ? 1.f : 0.f)));
      }
    sC[4 * i + 3] = dev < 1e-4f ? rho * rho : INFINITY;
  }
  __syncthreads();
  // blocks stride over the grid in steps of 256 cells, so the set-up above runs once per block
  for (uint32_t c0 = blockIdx.x * blockDim.x; c0 < n; c0 += gridDim.x * blockDim.x) {
    const uint32_t c = c0 + threadIdx.x;
    bool occ = false;
    if (c < n) {
      const int cx = (int)(c % grid), cy = (int)((c / grid) % grid), cz = (int)(c / (grid * grid));
      // y_k = bmin_k + ((j_k + 0.5) h_k)
      const float y0 = __fadd_rn(bx, __fmul_rn(__fadd_rn((float)cx, 0.5f), h0));
      const float y1 = __fadd_rn(by, __fmul_rn(__fadd_rn((float)cy, 0.5f), h1));
      const float y2 = __fadd_rn(bz, __fmul_rn(__fadd_rn((float)cz, 0.5f), h2));
      for (int i = 0; i < kBones && !occ; ++i) {
        const float *sc = sC + 4 * i;
        const float a0 = y0 - sc[0], a1 = y1 - sc[1], a2 = y2 - sc[2];
        if (a0 * a0 + a1 * a1 + a2 * a2 > sc[3]) continue;
        const float *g = sG + 12 * i;
        const float *e = sE + 15 * i;
        float v[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          // q_r = (((R_r0 y0) + (R_r1 y1)) + (R_r2 y2)) + t_r ; v_r = q_r - centre_r
          const float q = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(g[4 * r], y0), __fmul_rn(g[4 * r + 1], y1)),
                                              __fmul_rn(g[4 * r + 2], y2)),
                                    g[4 * r + 3]);
          v[r] = __fsub_rn(q, e[r]);
        }
        float s2[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          // l_m = ((Q_m0 v0) + (Q_m1 v1)) + (Q_m2 v2) ; s_m = l_m / (r_m + dil)
          const float l = __fadd_rn(__fadd_rn(__fmul_rn(e[3 + 3 * m], v[0]), __fmul_rn(e[3 + 3 * m + 1], v[1])),
                                    __fmul_rn(e[3 + 3 * m + 2], v[2]));
          s2[m] = __fdiv_rn(l, __fadd_rn(e[12 + m], dil));
        }
        // ((s0 s0) + (s1 s1)) + (s2 s2) <= 1
        const float q2 = __fadd_rn(__fadd_rn(__fmul_rn(s2[0], s2[0]), __fmul_rn(s2[1], s2[1])), __fmul_rn(s2[2], s2[2]));
        occ = q2 <= 1.f;
      }
    }
    const unsigned word = __ballot_sync(0xffffffffu, occ);
    if ((threadIdx.x & 31) == 0 && c < n) bits[c >> 5] = word;
  }
}

// Blocks of the posed-bitfield launch: eight 256-thread blocks per SM, striding over the cells.
static unsigned bitfield_blocks(long n, int device) {
  return (unsigned)std::min<long>((n + 255) / 256, 8L * num_sms(device));
}

// ------------------------------------------------------ bone support boxes
// For each bone channel, the index bounds of the vertices whose weight exceeds
// kBoneEps; rendering skips a candidate whose trilinear cell lies outside them.
__global__ void bone_box_init_kernel(int *ibox, int R) {
  const int i = threadIdx.x;
  if (i < kBones * 6) ibox[i] = (i % 6) < 3 ? R : -1;
}

__global__ void bone_box_kernel(const float *__restrict__ wvol, int R, int *__restrict__ ibox) {
  const size_t R3 = (size_t)R * R * R;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kBones * R3) return;
  if (!(wvol[idx] > kBoneEps)) return;
  const int c = (int)(idx / R3);
  const int v = (int)(idx % R3);
  const int x = v % R, y = (v / R) % R, z = v / (R * R);
  int *b = ibox + 6 * c;
  atomicMin(b + 0, x);
  atomicMin(b + 1, y);
  atomicMin(b + 2, z);
  atomicMax(b + 3, x);
  atomicMax(b + 4, y);
  atomicMax(b + 5, z);
}

// u in [lo - 1, hi + 1) may touch a vertex in [lo, hi]; an empty channel skips everywhere
__global__ void bone_box_finish_kernel(const int *__restrict__ ibox, float *__restrict__ box) {
  const int c = threadIdx.x;
  if (c >= kBones) return;
  const int *b = ibox + 6 * c;
  const bool empty = b[0] > b[3];
  for (int k = 0; k < 3; ++k) {
    box[6 * c + k] = empty ? INFINITY : (float)(b[k] - 1);
    box[6 * c + 3 + k] = empty ? -INFINITY : (float)(b[3 + k] + 1);
  }
}

// --------------------------------------------------------- derived layouts
// Transposes rows [0, out) x columns [col0, col0 + n_in) of a packed float32
// W[out][src_stride] into dst[(row0 + k) * out_pad + j]; rows n_in..in_pad-1
// and columns out..out_pad-1 are zero.
__global__ void transpose_layer_kernel(const float *__restrict__ W, int src_stride, int col0, int n_in, int in_pad,
                                       int out, int out_pad, float *__restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= in_pad * out_pad) return;
  const int k = i / out_pad, j = i % out_pad;
  dst[i] = (k < n_in && j < out) ? W[(size_t)j * src_stride + col0 + k] : 0.f;
}

// Row-major [out_pad][in_pad] half-precision copy (rows padded to row_stride):
// dst[j * row_stride + dcol0 + k] = W[j][col0 + k].
template <typename T>
__global__ void pack_tc_kernel(const float *__restrict__ W, int src_stride, int col0, int n_in, int in_pad, int out,
                               int out_pad, int row_stride, int dcol0, T *__restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= in_pad * out_pad) return;
  const int j = i / in_pad, k = i % in_pad;
  const float v = (k < n_in && j < out) ? W[(size_t)j * src_stride + col0 + k] : 0.f;
  dst[(size_t)j * row_stride + dcol0 + k] = T(v);
}

// Corner-block copy of the bone channels (see trilinear_quad in field.cuh).
__global__ void build_quad_kernel(const float *__restrict__ vol, int R, float4 *__restrict__ quad) {
  const size_t QC = quad_channel(R);
  const size_t n = QC * kBones;
  const int R1 = R + 1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / QC);
    size_t r = e % QC;
    const int x = (int)(r % R1) - 1;
    r /= R1;
    const int y = (int)(r % R1) - 1;
    const int z = (int)(r / R1) - 1;
    const float *ch = vol + (size_t)c * R * R * R;
    auto at = [&](int zz, int yy, int xx) -> float {
      return (zz < 0 || yy < 0 || xx < 0 || zz >= R || yy >= R || xx >= R) ? 0.f : ch[((size_t)zz * R + yy) * R + xx];
    };
    quad[e] = make_float4(at(z, y, x), at(z, y, x + 1), at(z, y + 1, x), at(z, y + 1, x + 1));
  }
}

__global__ void copy_kernel(const float *__restrict__ src, int n, float *__restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (i < n) ? src[i] : 0.f;
}

__global__ void zero_kernel(float *__restrict__ dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = 0.f;
}

__global__ void table_to_f16_kernel(const float2 *__restrict__ src, size_t n, __half2 *__restrict__ dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __floats2half2_rn(src[i].x, src[i].y);
}

// Corner blocks of the dense levels of the f16 table: entry (x, y, z) of level l holds the
// vertices (x, y, z), (x + 1, y, z), (x, y + 1, z), (x + 1, y + 1, z) (row-major vertex index
// x + y (N + 1) + z (N + 1)^2), so that a sample reads its eight corners as two 16-byte loads.
struct DenseQuadArgs {
  int n_levels;
  uint32_t level[kMaxLevels], N[kMaxLevels];
  size_t off[kMaxLevels + 1];
  size_t T;
};

__global__ void dense_quad_kernel(const __half2 *__restrict__ t16, DenseQuadArgs a, uint4 *__restrict__ dq) {
  const size_t n = a.off[a.n_levels];
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < a.n_levels && e >= a.off[k + 1]) ++k;
    const size_t N = a.N[k], M = N + 1, q = e - a.off[k];
    const size_t x = q % N, y = (q / N) % N, z = q / (N * N);
    const __half2 *t = t16 + (size_t)a.level[k] * a.T;
    const size_t v = x + y * M + z * M * M;
    uint4 r;
    r.x = *reinterpret_cast<const uint32_t *>(t + v);
    r.y = *reinterpret_cast<const uint32_t *>(t + v + 1);
    r.z = *reinterpret_cast<const uint32_t *>(t + v + M);
    r.w = *reinterpret_cast<const uint32_t *>(t + v + M + 1);
    dq[e] = r;
  }
}

// bias1[f][j] = b1[j] + sum_m W1[j][g + m] * omega[f][m]: the joint angles of
// Omega^o enter the residual MLP's first layer (Fig. S3) as a per-pose bias.
__global__ void fold_pose_bias_kernel(const float *__restrict__ res, int g, int pose_dim,
                                      const float *__restrict__ omega, float *__restrict__ bias1) {
  const int j = threadIdx.x;
  const int f = blockIdx.x;
  const int stride = g + pose_dim;
  if (j >= kWidth) return;
  const float *W1 = res;
  const float *b1 = res + kWidth * stride;
  float acc = b1[j];
  for (int m = 0; m < pose_dim; ++m) acc = fmaf(W1[j * stride + g + m], omega[f * pose_dim + m], acc);
  bias1[f * kWidth + j] = acc;
}

int res_gamma_dims(const nr_subject *s) { return 3 + 6 * (int)s->res_freqs; }

MasterOffsets master_offsets(const nr_subject *s) {
  MasterOffsets m{};
  const int g = res_gamma_dims(s), P = 3 * (int)s->K;
  const int rin[5] = {g + P, kWidth, kWidth, kWidth + g, kWidth};
  const int rout[5] = {kWidth, kWidth, kWidth, kWidth, 3};
  int o = 0;
  for (int l = 0; l < 5; ++l) {
    m.r[l] = o;
    o += rin[l] * rout[l];
    m.rb[l] = o;
    o += rout[l];
  }
  m.n_res = o;
  o = 0;
  const int H = (int)s->hidden;
  for (int l = 0; l <= H; ++l) {
    const int in = l == 0 ? (int)s->mlp_in : kWidth;
    const int out = l == H ? 4 : kWidth;
    m.c[l] = o;
    o += in * out;
    m.cb[l] = o;
    o += out;
  }
  m.n_mlp = o;
  return m;
}

static BlobLayout blob_layout(const nr_subject *s) {
  BlobLayout b{};
  int o = 0;
  auto take = [&](int n) {
    const int r = o;
    o += (n + 3) & ~3;
    return r;
  };
  b.r1 = take(kResGammaPad * kWidth);
  b.r1b = take(kWidth);
  b.r2 = take(kWidth * kWidth);
  b.r2b = take(kWidth);
  b.r3 = take(kWidth * kWidth);
  b.r3b = take(kWidth);
  b.r4 = take((kWidth + kResGammaPad) * kWidth);
  b.r4b = take(kWidth);
  b.r5 = take(kWidth * 4);
  b.r5b = take(4);
  b.c0 = take(kMlpIn * kWidth);
  b.c0b = take(kWidth);
  for (int l = 0; l < (int)s->hidden - 1; ++l) {
    b.ch[l] = take(kWidth * kWidth);
    b.chb[l] = take(kWidth);
  }
  b.cl = take(kWidth * 4);
  b.clb = take(4);
  b.total = o;
  return b;
}

static TcLayout tc_layout(const nr_subject *s) {
  TcLayout t{};
  int o = 0;
  t.r1 = o;
  o += kWidth * kTcRow;          // [64][48] in a 72-wide row
  t.r2 = o;
  o += kWidth * kTcRow;
  t.r3 = o;
  o += kWidth * kTcRow;
  t.r4 = o;
  o += kWidth * kTcRowWide;      // [64][64 + 48]
  t.r5 = o;
  o += 8 * kTcRow;               // [3 -> 8][64]
  t.c0 = o;
  o += kWidth * kTcRow;          // [64][32]
  for (int l = 0; l < (int)s->hidden - 1; ++l) {
    t.ch[l] = o;
    o += kWidth * kTcRow;
  }
  t.cl = o;
  o += 8 * kTcRow;               // [4 -> 8][64]
  t.total = o;
  return t;
}

static inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

template <typename T>
static int pack_tc_all(const nr_subject *s, const MasterOffsets &m, cudaStream_t st, T *dst) {
  const TcLayout &t = s->tlay;
  const int g = res_gamma_dims(s), P = 3 * (int)s->K;
  cudaMemsetAsync(dst, 0, sizeof(T) * t.total, st);
  int launched = 0;
  auto pack = [&](const float *W, int stride, int col0, int n_in, int in_pad, int out, int out_pad, int rs, int dcol0,
                  int off) {
    ++launched;
    pack_tc_kernel<T><<<nblk((long)in_pad * out_pad, 256), 256, 0, st>>>(W, stride, col0, n_in, in_pad, out, out_pad, rs,
                                                                         dcol0, dst + off);
  };
  pack(s->res + m.r[0], g + P, 0, g, kResGammaPad, kWidth, kWidth, kTcRow, 0, t.r1);
  pack(s->res + m.r[1], kWidth, 0, kWidth, kWidth, kWidth, kWidth, kTcRow, 0, t.r2);
  pack(s->res + m.r[2], kWidth, 0, kWidth, kWidth, kWidth, kWidth, kTcRow, 0, t.r3);
  pack(s->res + m.r[3], kWidth + g, 0, kWidth, kWidth, kWidth, kWidth, kTcRowWide, 0, t.r4);
  pack(s->res + m.r[3], kWidth + g, kWidth, g, kResGammaPad, kWidth, kWidth, kTcRowWide, kWidth, t.r4);
  pack(s->res + m.r[4], kWidth, 0, kWidth, kWidth, 3, 8, kTcRow, 0, t.r5);
  pack(s->mlp + m.c[0], (int)s->mlp_in, 0, (int)s->mlp_in, kMlpIn, kWidth, kWidth, kTcRow, 0, t.c0);
  for (int l = 1; l < (int)s->hidden; ++l)
    pack(s->mlp + m.c[l], kWidth, 0, kWidth, kWidth, kWidth, kWidth, kTcRow, 0, t.ch[l - 1]);
  pack(s->mlp + m.c[s->hidden], kWidth, 0, kWidth, kWidth, 4, 8, kTcRow, 0, t.cl);
  return launched;
}

nr_status prepare_params(nr_subject *s, cudaStream_t st) {
  if (s->cnn_on && s->cnn_dirty) {   // the weight volume is generated (Sec. 4.2)
    nr_status r = cnn_forward(s, st);
    if (r != NR_OK) return r;
    s->cnn_dirty = false;
    s->params_dirty = true;
  }
  if (!s->params_dirty) return NR_OK;
  const MasterOffsets m = master_offsets(s);
  const BlobLayout &b = s->lay;
  const int g = res_gamma_dims(s), P = 3 * (int)s->K;
  float *B = s->blob;
  int launched = 0;
  auto tr = [&](const float *W, int stride, int col0, int n_in, int in_pad, int out, int out_pad, int off) {
    ++launched;
    transpose_layer_kernel<<<nblk((long)in_pad * out_pad, 256), 256, 0, st>>>(W, stride, col0, n_in, in_pad, out,
                                                                             out_pad, B + off);
  };
  auto cp = [&](const float *src, int n, int n_pad, int off) {
    launched += 2;
    zero_kernel<<<nblk(n_pad, 256), 256, 0, st>>>(B + off, n_pad);
    copy_kernel<<<nblk(n, 256), 256, 0, st>>>(src, n, B + off);
  };
  // residual MLP
  tr(s->res + m.r[0], g + P, 0, g, kResGammaPad, kWidth, kWidth, b.r1);
  cp(s->res + m.rb[0], kWidth, kWidth, b.r1b);
  tr(s->res + m.r[1], kWidth, 0, kWidth, kWidth, kWidth, kWidth, b.r2);
  cp(s->res + m.rb[1], kWidth, kWidth, b.r2b);
  tr(s->res + m.r[2], kWidth, 0, kWidth, kWidth, kWidth, kWidth, b.r3);
  cp(s->res + m.rb[2], kWidth, kWidth, b.r3b);
  tr(s->res + m.r[3], kWidth + g, 0, kWidth, kWidth, kWidth, kWidth, b.r4);
  tr(s->res + m.r[3], kWidth + g, kWidth, g, kResGammaPad, kWidth, kWidth, b.r4 + kWidth * kWidth);
  cp(s->res + m.rb[3], kWidth, kWidth, b.r4b);
  tr(s->res + m.r[4], kWidth, 0, kWidth, kWidth, 3, 4, b.r5);
  cp(s->res + m.rb[4], 3, 4, b.r5b);
  // canonical MLP
  tr(s->mlp + m.c[0], (int)s->mlp_in, 0, (int)s->mlp_in, kMlpIn, kWidth, kWidth, b.c0);
  cp(s->mlp + m.cb[0], kWidth, kWidth, b.c0b);
  for (int l = 1; l < (int)s->hidden; ++l) {
    tr(s->mlp + m.c[l], kWidth, 0, kWidth, kWidth, kWidth, kWidth, b.ch[l - 1]);
    cp(s->mlp + m.cb[l], kWidth, kWidth, b.chb[l - 1]);
  }
  tr(s->mlp + m.c[s->hidden], kWidth, 0, kWidth, kWidth, 4, 4, b.cl);
  cp(s->mlp + m.cb[s->hidden], 4, 4, b.clb);
  // tensor-core copies
  launched += pack_tc_all<__nv_bfloat16>(s, m, st, s->tc_bf16);
  launched += pack_tc_all<__half>(s, m, st, s->tc_f16);
  // half-precision hash table, corner-block weight volume
  table_to_f16_kernel<<<1024, 256, 0, st>>>(reinterpret_cast<const float2 *>(s->table), s->n_table / 2, s->table16);
  if (s->dense_quad) {
    DenseQuadArgs a{};
    for (uint32_t l = 0; l < s->L; ++l) {
      const double n1 = (double)s->level_res[l] + 1.0;
      if (n1 * n1 * n1 > (double)s->T) continue;
      a.level[a.n_levels] = l;
      a.N[a.n_levels] = s->level_res[l];
      a.off[a.n_levels] = s->dq_off[l];
      ++a.n_levels;
    }
    a.off[a.n_levels] = s->n_dq;
    a.T = s->T;
    dense_quad_kernel<<<1024, 256, 0, st>>>(s->table16, a, s->dense_quad);
    ++launched;
  }
  build_quad_kernel<<<2048, 256, 0, st>>>(s->wvol, (int)s->wres, s->wquad);
  bone_box_init_kernel<<<1, kBones * 6, 0, st>>>(s->bone_ibox, (int)s->wres);
  bone_box_kernel<<<nblk((long)kBones * s->wres * s->wres * s->wres, 256), 256, 0, st>>>(s->wvol, (int)s->wres,
                                                                                        s->bone_ibox);
  bone_box_finish_kernel<<<1, 32, 0, st>>>(s->bone_ibox, s->bone_box);
  launched += 4;
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(launched + 1);
  s->params_dirty = false;
  s->bias_dirty = true;
  s->occ_dirty = true;
  s->fp8_ready = false;
  s->t5_ready = false;
  (void)P;
  return NR_OK;
}

// Canonical occupancy dilated by r cells (Chebyshev distance, clipped at the
// grid's faces): out(c) = OR of raw(c') over |c' - c|_inf <= r.  g^3 is a
// multiple of the block, so every warp writes whole words.
__global__ void __launch_bounds__(256) dilate_bits_kernel(const uint32_t *__restrict__ raw, int g, int r,
                                                          uint32_t *__restrict__ out) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  const int x = (int)(c % g), y = (int)((c / g) % g), z = (int)(c / ((uint32_t)g * g));
  bool occ = false;
  for (int dz = -r; dz <= r && !occ; ++dz) {
    const int zz = z + dz;
    if (zz < 0 || zz >= g) continue;
    for (int dy = -r; dy <= r && !occ; ++dy) {
      const int yy = y + dy;
      if (yy < 0 || yy >= g) continue;
      for (int dx = -r; dx <= r; ++dx) {
        const int xx = x + dx;
        if (xx < 0 || xx >= g) continue;
        const uint32_t q = ((uint32_t)zz * g + yy) * g + xx;
        if ((__ldg(raw + (q >> 5)) >> (q & 31)) & 1u) {
          occ = true;
          break;
        }
      }
    }
  }
  const unsigned word = __ballot_sync(0xffffffffu, occ);
  if ((threadIdx.x & 31) == 0) out[c >> 5] = word;
}

nr_status launch_posed_bitfield(const nr_subject *s, const float *G_dev, const float *bias_dev, uint32_t *bits,
                                cudaStream_t st) {
  if (s->occ_source == kOccGrid) {
    FieldParams P = field_params(s, nullptr);
    P.G = G_dev;
    P.bias1 = bias_dev;
    P.occ_grid = (int)s->occ_grid;
    P.occ_smin = s->occ_smin;
    P.canon_bits = s->canon_bits;
    return launch_occupancy_field(P, kModePose, bits, s->device, st);
  }
  const int g = (int)s->occ_grid;
  const long n = (long)g * g * g;
  posed_bitfield_kernel<<<bitfield_blocks(n, s->device), 256, 0, st>>>(G_dev, s->ellip, s->bmin[0], s->bmin[1],
                                                                       s->bmin[2], s->bmax[0], s->bmax[1], s->bmax[2],
                                                                       g, bits);
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(1);
  return NR_OK;
}

nr_status launch_fold_bias(const nr_subject *s, const float *omega_dev, float *bias_dev, int n_poses, cudaStream_t st) {
  fold_pose_bias_kernel<<<n_poses, kWidth, 0, st>>>(s->res, res_gamma_dims(s), 3 * (int)s->K, omega_dev, bias_dev);
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(1);
  return NR_OK;
}

nr_status ensure_occupancy(nr_subject *s, cudaStream_t st) {
  if (s->occ_source != kOccGrid || !s->occ_dirty || !s->pose_set) return NR_OK;
  nr_status r = launch_posed_bitfield(s, s->d_G, s->d_bias1, s->bits, st);
  if (r == NR_OK) s->occ_dirty = false;
  return r;
}

nr_status ensure_bias(nr_subject *s, cudaStream_t st) {
  if (!s->bias_dirty) return NR_OK;
  fold_pose_bias_kernel<<<1, kWidth, 0, st>>>(s->res, res_gamma_dims(s), 3 * (int)s->K, pose_omega(s), s->d_bias1);
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(1);
  s->bias_dirty = false;
  return NR_OK;
}

nr_status fold_frame_biases(nr_subject *s, cudaStream_t st) {
  if (s->n_frames == 0) return NR_OK;
  fold_pose_bias_kernel<<<s->n_frames, kWidth, 0, st>>>(s->res, res_gamma_dims(s), 3 * (int)s->K,
                                                         s->ref_layers ? s->f_omega_o : s->f_omega, s->f_bias1);
  NR_CHECK_CUDA(cudaGetLastError());
  return NR_OK;
}

FieldParams field_params(const nr_subject *s, const nr_render_opts *o) {
  FieldParams P{};
  for (int k = 0; k < 3; ++k) {
    P.bmin[k] = s->bmin[k];
    P.bmax[k] = s->bmax[k];
    P.vol_scale[k] = (float)((double)(s->wres - 1) / ((double)s->bmax[k] - (double)s->bmin[k]));
    P.inv_box[k] = (float)(1.0 / ((double)s->bmax[k] - (double)s->bmin[k]));
    P.box_c[k] = (float)(0.5 * ((double)s->bmax[k] + (double)s->bmin[k]));
    P.box_ih[k] = (float)(2.0 / ((double)s->bmax[k] - (double)s->bmin[k]));
  }
  P.wres = (int)s->wres;
  P.wvol = s->wvol;
  P.wquad = s->wquad;
  P.L = (int)s->L;
  P.T_mask = s->T - 1;
  for (uint32_t l = 0; l < s->L; ++l) {
    P.level_res[l] = s->level_res[l];
    const double n1 = (double)s->level_res[l] + 1.0;
    if (n1 * n1 * n1 <= (double)s->T) P.dense_mask |= 1u << l;
  }
  P.table32 = reinterpret_cast<const float2 *>(s->table);
  P.table16 = s->table16;
  P.dense_quad = s->dense_quad;
  P.tf32_scratch = s->r_scratch;
  for (uint32_t l = 0; l < s->L; ++l) P.dq_off[l] = s->dq_off[l];
  P.use_f16_table = (o && o->feat_dtype == NR_F16) ? 1 : 0;
  P.hidden = (int)s->hidden;
  P.res_enabled = (int)s->res_enabled;
  P.res_freqs = (int)s->res_freqs;
  const double alpha = (o && o->hann_alpha >= 0.f) ? (double)o->hann_alpha : (double)s->res_freqs;
  for (int k = 0; k < 8; ++k) {
    double a = alpha - k;
    a = a < 0 ? 0 : (a > 1 ? 1 : a);
    P.hann[k] = (float)((1.0 - cos(M_PI * a)) / 2.0);
  }
  P.blob = s->blob;
  P.lay = s->lay;
  P.tc_blob = (o && o->mlp_dtype == NR_F16) ? (const void *)s->tc_f16 : (const void *)s->tc_bf16;
  P.tlay = s->tlay;
  P.G = s->d_G;
  P.bias1 = s->d_bias1;
  P.bone_box = (o && !(o->flags & NR_RENDER_ALL_BONES)) ? s->bone_box : nullptr;
  P.fp8_blob = s->fp8_blob;
  P.fp8_scales = s->fp8_scales;
  P.t5_bf16 = s->t5_bf16;
  P.t5_f16 = s->t5_f16;
  P.t5_fp8 = s->t5_fp8;
  P.t5_err = s->t5_err;
  return P;
}

}  // namespace nr

using namespace nr;

// ====================================================================== ABI

extern "C" const char *nr_last_error(void) { return nr::g_err; }

extern "C" uint64_t nr_launch_count(void) { return nr::g_launches.load(std::memory_order_relaxed); }

extern "C" nr_status nr_field_error_word(nr_subject *s, uint32_t **dev_word) {
  NR_REQUIRE(subject_ok(s) && dev_word, "nr_field_error_word: bad argument");
  *dev_word = s->t5_err;
  return NR_OK;
}

static void free_subject(nr_subject *s) {
  void *bufs[] = {s->wquad,  s->wvol,   s->g_wvol,  s->table,    s->g_table,  s->mlp,       s->g_mlp,     s->res,
                  s->g_res,  s->adam_m,  s->adam_v,   s->table16,  s->dense_quad, s->r_scratch, s->blob,      s->tc_bf16,   s->tc_f16,
                  s->d_G,    s->d_omega, s->d_bias1,  s->ellip,    s->bits,      s->f_G,       s->f_omega,
                  s->f_bias1, s->f_cam,  s->samp,     s->samp_out, s->ray_range, s->counter,   s->out_stage,
                  s->t_samp, s->t_out,   s->t_T,      s->t_raycnt, s->t_live,   s->t_scratch, s->t_wacc,    s->t_red,
                  s->loss_acc, s->f_dbias1, s->fp8_blob, s->fp8_scales, s->fp8_jobs, s->fp8_G,
                  s->t5_bf16,  s->t5_f16,  s->t5_fp8,  s->t5_err,  s->ray_state, s->ray_next, s->canon_bits, s->occ_raw,
                  s->ref, s->g_ref, s->ref_m, s->ref_v, s->f_root, s->f_dG, s->f_omega_o,
                  s->cnn, s->g_cnn, s->cnn_m, s->cnn_v, s->cnn_z, s->cnn_prior, s->cnn_act, s->cnn_grad,
                  s->bone_box, s->bone_ibox};
  for (void *p : bufs)
    if (p) cudaFree(p);
  for (cudaEvent_t &e : s->prof_ev)
    if (e) cudaEventDestroy(e);
  if (s->pose_ev) cudaEventDestroy(s->pose_ev);
  s->magic = 0;
  delete s;
}

extern "C" nr_status nr_create_subject(const nr_subject_desc *d, void *stream, nr_subject **out) {
  NR_REQUIRE(d && out, "nr_create_subject: NULL argument");
  *out = nullptr;
  NR_REQUIRE(d->abi_version == NR_ABI_VERSION, "abi_version %u != %u", d->abi_version, NR_ABI_VERSION);
  NR_REQUIRE(d->n_bones == 24, "n_bones must be 24 (got %u)", d->n_bones);
  NR_REQUIRE(d->parents && d->rest_joints && d->wvol && d->level_res && d->hash_table && d->mlp_params,
             "a required array pointer is NULL");
  NR_REQUIRE(d->hash_feats == 2, "hash_feats must be 2");
  NR_REQUIRE(d->hash_levels >= 1 && d->hash_levels <= 16, "hash_levels must be 1..16");
  NR_REQUIRE(d->log2_T >= 10 && d->log2_T <= 24, "log2_T must be 10..24");
  NR_REQUIRE(d->mlp_in == 32, "mlp_in must be 32");
  NR_REQUIRE(d->mlp_width == 64, "mlp_width must be 64");
  NR_REQUIRE(d->mlp_hidden_layers >= 1 && d->mlp_hidden_layers <= 4, "mlp_hidden_layers must be 1..4");
  NR_REQUIRE(!d->res_enabled || (d->res_params && d->res_pe_freqs <= 6), "residual MLP needs res_params, <=6 bands");
  NR_REQUIRE(d->wvol_res >= 2 && d->wvol_res <= 256, "wvol_res must be 2..256");
  NR_REQUIRE(d->occ_grid == 0 || d->occ_grid == 32 || d->occ_grid == 64 || d->occ_grid == 128 || d->occ_grid == 256,
             "occ_grid must be 32, 64, 128 or 256 (0 = 128)");
  for (int k = 0; k < 3; ++k) NR_REQUIRE(d->box_max[k] > d->box_min[k], "empty box");
  for (uint32_t i = 0; i < d->n_bones; ++i)
    NR_REQUIRE(d->parents[i] < (int32_t)i && d->parents[i] >= -1, "parents[%u] must be -1 or < %u", i, i);
  for (uint32_t l = 0; l < d->hash_levels; ++l)
    NR_REQUIRE(d->level_res[l] >= 1 && d->level_res[l] <= 65536, "level_res must be 1..65536");

  NR_CHECK_CUDA(cudaSetDevice(d->device));
  cudaStream_t st = (cudaStream_t)stream;
  nr_subject *s = new (std::nothrow) nr_subject();
  if (!s) {
    set_error("host allocation failed");
    return NR_ENOMEM;
  }
  s->device = d->device;
  s->K = d->n_bones;
  for (int k = 0; k < 3; ++k) {
    s->bmin[k] = d->box_min[k];
    s->bmax[k] = d->box_max[k];
  }
  s->wres = d->wvol_res;
  s->L = d->hash_levels;
  s->F = d->hash_feats;
  s->log2T = d->log2_T;
  s->T = 1u << d->log2_T;
  for (uint32_t l = 0; l < s->L; ++l) s->level_res[l] = d->level_res[l];
  s->mlp_in = d->mlp_in;
  s->width = d->mlp_width;
  s->hidden = d->mlp_hidden_layers;
  s->res_enabled = d->res_enabled;
  s->res_freqs = d->res_pe_freqs;
  s->occ_grid = d->occ_grid ? d->occ_grid : 128;
  s->has_ellipsoids = d->ellipsoids != nullptr;
  s->occ_source = s->has_ellipsoids ? kOccEllipsoids : kOccNone;
  s->parents.assign(d->parents, d->parents + s->K);
  s->rest.assign(d->rest_joints, d->rest_joints + 3 * s->K);

  const MasterOffsets m = master_offsets(s);
  s->n_wvol = (size_t)(s->K + 1) * s->wres * s->wres * s->wres;
  s->n_table = (size_t)s->L * s->T * 2;
  s->n_mlp = (size_t)m.n_mlp;
  s->n_res = (size_t)m.n_res;
  s->lay = blob_layout(s);
  s->tlay = tc_layout(s);

  auto fail = [&](cudaError_t e, const char *what) {
    nr_status r = set_error_cuda(e, what);
    free_subject(s);
    return r;
  };
#define ALLOC(ptr, bytes)                                            \
  do {                                                               \
    cudaError_t e_ = cudaMalloc((void **)&(ptr), (bytes));           \
    if (e_ != cudaSuccess) return fail(e_, "cudaMalloc " #ptr);      \
  } while (0)
  ALLOC(s->wvol, s->n_wvol * 4);
  ALLOC(s->g_wvol, s->n_wvol * 4);
  ALLOC(s->table, s->n_table * 4);
  ALLOC(s->g_table, s->n_table * 4);
  ALLOC(s->mlp, s->n_mlp * 4);
  ALLOC(s->g_mlp, s->n_mlp * 4);
  ALLOC(s->res, s->n_res * 4);
  ALLOC(s->g_res, s->n_res * 4);
  ALLOC(s->table16, s->n_table * 2);
  for (uint32_t l = 0; l < s->L; ++l) {   // corner blocks of the dense levels: N x N x (N + 1) each
    const double n1 = (double)s->level_res[l] + 1.0;
    if (n1 * n1 * n1 > (double)s->T) continue;
    const size_t N = s->level_res[l];
    s->dq_off[l] = (uint32_t)s->n_dq;
    s->n_dq += N * N * (N + 1);
  }
  if (s->n_dq) ALLOC(s->dense_quad, s->n_dq * sizeof(uint4));
  ALLOC(s->blob, (size_t)s->lay.total * 4);
  ALLOC(s->wquad, quad_channel((int)s->wres) * kBones * sizeof(float4));
  ALLOC(s->bone_box, kBones * 6 * sizeof(float));
  ALLOC(s->bone_ibox, kBones * 6 * sizeof(int));
  ALLOC(s->tc_bf16, (size_t)s->tlay.total * 2);
  ALLOC(s->tc_f16, (size_t)s->tlay.total * 2);
  ALLOC(s->t5_bf16, (size_t)t5_layout((int)s->hidden).total);   // tcgen05 weight blobs, packed on first use
  ALLOC(s->t5_f16, (size_t)t5_layout((int)s->hidden).total);
  ALLOC(s->t5_fp8, (size_t)t5_layout((int)s->hidden).total);
  ALLOC(s->t5_err, sizeof(uint32_t));
  ALLOC(s->d_G, kBones * 12 * 4);
  ALLOC(s->d_omega, (2 * kBones * 3 + 3) * 4);
  ALLOC(s->d_bias1, kWidth * 4);
  ALLOC(s->counter, 16 * 4);
  if (s->has_ellipsoids) {
    ALLOC(s->ellip, kBones * 15 * 4);
    ALLOC(s->bits, (size_t)s->occ_grid * s->occ_grid * s->occ_grid / 8);
  }
#undef ALLOC
  cudaError_t e;
#define H2D(dst, src, bytes)                                                   \
  e = cudaMemcpyAsync((dst), (src), (bytes), cudaMemcpyHostToDevice, st);      \
  if (e != cudaSuccess) return fail(e, "cudaMemcpyAsync " #dst);
  e = cudaMemsetAsync(s->t5_err, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return fail(e, "cudaMemsetAsync t5_err");
  H2D(s->wvol, d->wvol, s->n_wvol * 4);
  H2D(s->table, d->hash_table, s->n_table * 4);
  H2D(s->mlp, d->mlp_params, s->n_mlp * 4);
  if (s->res_enabled) {
    H2D(s->res, d->res_params, s->n_res * 4);
  } else {
    e = cudaMemsetAsync(s->res, 0, s->n_res * 4, st);
    if (e != cudaSuccess) return fail(e, "cudaMemsetAsync res");
  }
  if (s->has_ellipsoids) {
    H2D(s->ellip, d->ellipsoids, kBones * 15 * 4);
  }
#undef H2D
  e = cudaMemsetAsync(s->d_omega, 0, (2 * kBones * 3 + 3) * 4, st);
  if (e != cudaSuccess) return fail(e, "cudaMemsetAsync omega");
  // the call's host arrays may be freed on return: finish the copies first
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e, "cudaStreamSynchronize");
  *out = s;
  return NR_OK;
}

extern "C" nr_status nr_destroy(nr_subject *s) {
  if (!s) return NR_OK;
  NR_REQUIRE(subject_ok(s), "nr_destroy: invalid handle");
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  free_subject(s);
  return NR_OK;
}

// The pose of one nr_set_pose call, passed by value as a kernel argument (1,452 bytes): the
// launch copies it when it is queued, so the call neither stages a host copy nor waits for the
// device.
struct PoseUpload {
  float G[kBones * 12];
  float omega[kBones * 3 + 3];   // joint angles, then the root translation
};

__global__ void __launch_bounds__(128) store_pose_kernel(const PoseUpload u, float *__restrict__ G,
                                                         float *__restrict__ omega) {
  for (int i = threadIdx.x; i < kBones * 12; i += blockDim.x) G[i] = u.G[i];
  for (int i = threadIdx.x; i < kBones * 3 + 3; i += blockDim.x) omega[i] = u.omega[i];
}

extern "C" nr_status nr_set_pose(nr_subject *s, const float *aa, const float *root_t, uint32_t flags, void *stream) {
  NR_REQUIRE(subject_ok(s), "nr_set_pose: invalid handle");
  NR_REQUIRE(aa, "nr_set_pose: NULL pose");
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (flags & NR_POSE_MATRICES) {
    memcpy(s->h_G, aa, sizeof(float) * 12 * s->K);
    memset(s->h_omega, 0, sizeof(s->h_omega));
    memset(s->h_root, 0, sizeof(s->h_root));
  } else {
    for (uint32_t i = 0; i < 3 * s->K; ++i)
      NR_REQUIRE(isfinite(aa[i]), "nr_set_pose: non-finite joint angle at %u", i);
    forward_kinematics(s, aa, root_t, s->h_G);
    memcpy(s->h_omega, aa, sizeof(float) * 3 * s->K);
    for (int k = 0; k < 3; ++k) s->h_root[k] = root_t ? root_t[k] : 0.f;
  }
  s->pose_matrices = (flags & NR_POSE_MATRICES) != 0;
  nr_status r = after_pose(s, st);   // the previous pose's work, if on another stream, comes first
  if (r != NR_OK) return r;
  PoseUpload u;
  memcpy(u.G, s->h_G, sizeof(u.G));
  memcpy(u.omega, s->h_omega, sizeof(float) * 3 * kBones);
  memcpy(u.omega + 3 * kBones, s->h_root, sizeof(float) * 3);
  store_pose_kernel<<<1, 128, 0, st>>>(u, s->d_G, s->d_omega);
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(1);
  s->d_G_host = true;
  s->pose_set = true;
  s->pose_dirty = true;
  s->bias_dirty = true;
  s->pose_ev_live = false;
  if ((r = ensure_pose(s, st)) != NR_OK) return r;
  if (!s->pose_ev) NR_CHECK_CUDA(cudaEventCreateWithFlags(&s->pose_ev, cudaEventDisableTiming));
  NR_CHECK_CUDA(cudaEventRecord(s->pose_ev, st));
  s->pose_stream = st;
  s->pose_ev_live = true;
  return NR_OK;
}

// A consumer of the pose on another stream than the last nr_set_pose waits for that call's
// device work.  Under a stream capture the wait is left out (a capture may not wait on an event
// recorded outside it): the caller orders the capture after the pose.
nr_status nr::after_pose(nr_subject *s, cudaStream_t st) {
  if (!s->pose_ev_live || st == s->pose_stream) return NR_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  NR_CHECK_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs == cudaStreamCaptureStatusNone) NR_CHECK_CUDA(cudaStreamWaitEvent(st, s->pose_ev, 0));
  return NR_OK;
}

// Derives the device transforms of the current pose: the refined pose when
// MLP_theta is on (and the pose came as joint angles), else the host forward
// kinematics; then the posed occupancy of the subject's source.
nr_status nr::ensure_pose(nr_subject *s, cudaStream_t st) {
  nr_status r = after_pose(s, st);
  if (r != NR_OK) return r;
  if (!s->pose_dirty || !s->pose_set) return NR_OK;
  if (s->ref_layers && !s->pose_matrices) {
    if ((r = launch_refine_fk(s, s->d_omega, 3 * kBones, s->d_omega + 3 * kBones, 3, 1, s->d_G,
                              s->d_omega + 3 * kBones + 3, 3 * kBones, st)) != NR_OK)
      return r;
    s->d_G_host = false;
  } else if (!s->d_G_host) {   // the refiner was removed since: back to the host's transforms
    NR_CHECK_CUDA(cudaMemcpyAsync(s->d_G, s->h_G, sizeof(float) * 12 * s->K, cudaMemcpyHostToDevice, st));
    NR_CHECK_CUDA(cudaStreamSynchronize(st));   // h_G is rewritten by the next nr_set_pose
    s->d_G_host = true;
  }
  if (s->occ_source == kOccEllipsoids) {
    const int g = (int)s->occ_grid;
    const long n = (long)g * g * g;
    posed_bitfield_kernel<<<bitfield_blocks(n, s->device), 256, 0, st>>>(s->d_G, s->ellip, s->bmin[0], s->bmin[1],
                                                                         s->bmin[2], s->bmax[0], s->bmax[1],
                                                                         s->bmax[2], g, s->bits);
    NR_CHECK_CUDA(cudaGetLastError());
    count_launches(1);
  }
  s->occ_dirty = true;   // a canonical-grid source is posed lazily, after the bias fold
  s->bias_dirty = true;  // the refined angles condition MLP_res
  s->pose_dirty = false;
  return NR_OK;
}

const float *nr::pose_omega(const nr_subject *s) {
  return (s->ref_layers && !s->pose_matrices) ? s->d_omega + 3 * kBones + 3 : s->d_omega;
}

extern "C" nr_status nr_pose_transforms(nr_subject *s, float *G_out) {
  NR_REQUIRE(subject_ok(s) && G_out, "nr_pose_transforms: bad argument");
  if (!s->pose_set) {
    set_error("nr_pose_transforms: no pose set");
    return NR_ESTATE;
  }
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  nr_status r = ensure_pose(s, nullptr);
  if (r != NR_OK) return r;
  NR_CHECK_CUDA(cudaMemcpy(G_out, s->d_G, sizeof(float) * 12 * s->K, cudaMemcpyDeviceToHost));
  return NR_OK;
}

extern "C" nr_status nr_occupancy(nr_subject *s, uint32_t *bits_out) {
  NR_REQUIRE(subject_ok(s) && bits_out, "nr_occupancy: bad argument");
  if (!s->pose_set || s->occ_source == kOccNone) {
    set_error("nr_occupancy: no pose set or no occupancy source");
    return NR_ESTATE;
  }
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  nr_status r;
  if ((r = prepare_params(s, nullptr)) != NR_OK) return r;
  if ((r = ensure_pose(s, nullptr)) != NR_OK) return r;
  if ((r = ensure_bias(s, nullptr)) != NR_OK) return r;
  if ((r = ensure_occupancy(s, nullptr)) != NR_OK) return r;
  const size_t words = (size_t)s->occ_grid * s->occ_grid * s->occ_grid / 32;
  NR_CHECK_CUDA(cudaMemcpy(bits_out, s->bits, words * 4, cudaMemcpyDeviceToHost));
  return NR_OK;
}

// Allocates the canonical and posed grids of a kOccGrid source on first use.
static nr_status grid_buffers(nr_subject *s) {
  const size_t bytes = (size_t)s->occ_grid * s->occ_grid * s->occ_grid / 8;
  if (!s->bits) NR_CHECK_CUDA(cudaMalloc(&s->bits, bytes));
  if (!s->canon_bits) NR_CHECK_CUDA(cudaMalloc(&s->canon_bits, bytes));
  if (!s->occ_raw) NR_CHECK_CUDA(cudaMalloc(&s->occ_raw, bytes));
  return NR_OK;
}

extern "C" nr_status nr_refresh_occupancy(nr_subject *s, float sigma_threshold, uint32_t dilate, float s_min,
                                          void *stream) {
  NR_REQUIRE(subject_ok(s), "nr_refresh_occupancy: invalid handle");
  NR_REQUIRE(isfinite(sigma_threshold) && sigma_threshold >= 0.f, "nr_refresh_occupancy: bad sigma_threshold");
  NR_REQUIRE(dilate <= 3, "nr_refresh_occupancy: dilate must be 0..3");
  NR_REQUIRE(isfinite(s_min) && s_min >= 0.f, "nr_refresh_occupancy: bad s_min");
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  cudaStream_t st = (cudaStream_t)stream;
  nr_status r;
  if ((r = grid_buffers(s)) != NR_OK) return r;
  if ((r = prepare_params(s, st)) != NR_OK) return r;
  FieldParams P = field_params(s, nullptr);
  P.occ_grid = (int)s->occ_grid;
  P.occ_tau = sigma_threshold;
  if ((r = launch_occupancy_field(P, kModeDensity, s->occ_raw, s->device, st)) != NR_OK) return r;
  const uint32_t cells = s->occ_grid * s->occ_grid * s->occ_grid;
  dilate_bits_kernel<<<cells / 256, 256, 0, st>>>(s->occ_raw, (int)s->occ_grid, (int)dilate, s->canon_bits);
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(1);
  s->occ_source = kOccGrid;
  s->occ_smin = s_min;
  s->occ_dirty = true;
  return NR_OK;
}

extern "C" nr_status nr_set_canonical_occupancy(nr_subject *s, const uint32_t *bits, float s_min, void *stream) {
  NR_REQUIRE(subject_ok(s) && bits, "nr_set_canonical_occupancy: bad argument");
  NR_REQUIRE(isfinite(s_min) && s_min >= 0.f, "nr_set_canonical_occupancy: bad s_min");
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  cudaStream_t st = (cudaStream_t)stream;
  nr_status r;
  if ((r = grid_buffers(s)) != NR_OK) return r;
  const size_t bytes = (size_t)s->occ_grid * s->occ_grid * s->occ_grid / 8;
  NR_CHECK_CUDA(cudaMemcpyAsync(s->canon_bits, bits, bytes, cudaMemcpyHostToDevice, st));
  NR_CHECK_CUDA(cudaStreamSynchronize(st));   // the caller may free bits on return
  s->occ_source = kOccGrid;
  s->occ_smin = s_min;
  s->occ_dirty = true;
  return NR_OK;
}

extern "C" nr_status nr_canonical_occupancy(nr_subject *s, uint32_t *bits_out) {
  NR_REQUIRE(subject_ok(s) && bits_out, "nr_canonical_occupancy: bad argument");
  if (s->occ_source != kOccGrid) {
    set_error("nr_canonical_occupancy: the occupancy source is not a canonical grid");
    return NR_ESTATE;
  }
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  const size_t words = (size_t)s->occ_grid * s->occ_grid * s->occ_grid / 32;
  NR_CHECK_CUDA(cudaMemcpy(bits_out, s->canon_bits, words * 4, cudaMemcpyDeviceToHost));
  return NR_OK;
}

extern "C" nr_status nr_param(nr_subject *s, uint32_t which, float **dev, float **grad, size_t *count) {
  NR_REQUIRE(subject_ok(s), "nr_param: invalid handle");
  float *p = nullptr, *g = nullptr;
  size_t n = 0;
  switch (which) {
    case NR_PARAM_WVOL: p = s->wvol; g = s->g_wvol; n = s->n_wvol; break;
    case NR_PARAM_HASH: p = s->table; g = s->g_table; n = s->n_table; break;
    case NR_PARAM_MLP: p = s->mlp; g = s->g_mlp; n = s->n_mlp; break;
    case NR_PARAM_RES: p = s->res; g = s->g_res; n = s->n_res; break;
    case NR_PARAM_REFINER: p = s->ref; g = s->g_ref; n = s->n_ref; break;
    case NR_PARAM_CNN: p = s->cnn; g = s->g_cnn; n = s->n_cnn; break;
    default: set_error("nr_param: unknown group %u", which); return NR_EINVAL;
  }
  if (dev) *dev = p;
  if (grad) *grad = g;
  if (count) *count = n;
  return NR_OK;
}

extern "C" nr_status nr_params_changed(nr_subject *s) {
  NR_REQUIRE(subject_ok(s), "nr_params_changed: invalid handle");
  s->params_dirty = true;
  s->bias_dirty = true;
  if (s->ref_layers) s->pose_dirty = s->pose_set;
  if (s->cnn_on) s->cnn_dirty = true;
  return NR_OK;
}

extern "C" nr_status nr_set_frames(nr_subject *s, uint32_t n_frames, const float *aa, const float *root_t,
                                   const nr_camera *cams, void *stream) {
  NR_REQUIRE(subject_ok(s), "nr_set_frames: invalid handle");
  NR_REQUIRE(n_frames >= 1 && n_frames <= 65536 && aa && cams, "nr_set_frames: bad arguments");
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<float> G((size_t)n_frames * 12 * s->K), om((size_t)n_frames * 3 * s->K);
  std::vector<Frame> fr(n_frames);
  for (uint32_t f = 0; f < n_frames; ++f) {
    const float *a = aa + (size_t)f * 3 * s->K;
    for (uint32_t i = 0; i < 3 * s->K; ++i) NR_REQUIRE(isfinite(a[i]), "nr_set_frames: non-finite angle");
    forward_kinematics(s, a, root_t ? root_t + 3 * f : nullptr, &G[(size_t)f * 12 * s->K]);
    memcpy(&om[(size_t)f * 3 * s->K], a, sizeof(float) * 3 * s->K);
    const nr_camera &c = cams[f];
    NR_REQUIRE(c.width >= 1 && c.height >= 1 && c.fx != 0.f && c.fy != 0.f, "nr_set_frames: bad camera %u", f);
    memcpy(fr[f].R, c.R, sizeof(fr[f].R));
    memcpy(fr[f].t, c.t, sizeof(fr[f].t));
    fr[f].fx = c.fx;
    fr[f].fy = c.fy;
    fr[f].cx = c.cx;
    fr[f].cy = c.cy;
    fr[f].t_near = c.t_near;
    fr[f].t_far = c.t_far;
    fr[f].width = c.width;
    fr[f].height = c.height;
  }
  if (n_frames > s->frames_cap) {
    if (s->f_G) cudaFree(s->f_G);
    if (s->f_omega) cudaFree(s->f_omega);
    if (s->f_bias1) cudaFree(s->f_bias1);
    if (s->f_dbias1) cudaFree(s->f_dbias1);
    if (s->f_cam) cudaFree(s->f_cam);
    if (s->f_root) cudaFree(s->f_root);
    if (s->f_omega_o) cudaFree(s->f_omega_o);
    s->f_G = s->f_omega = s->f_bias1 = s->f_dbias1 = s->f_root = s->f_omega_o = nullptr;
    s->f_cam = nullptr;
    s->n_frames = s->frames_cap = 0;
    NR_CHECK_CUDA(cudaMalloc(&s->f_root, (size_t)n_frames * 3 * 4));
    NR_CHECK_CUDA(cudaMalloc(&s->f_omega_o, (size_t)n_frames * 3 * kBones * 4));
    NR_CHECK_CUDA(cudaMalloc(&s->f_G, G.size() * 4));
    NR_CHECK_CUDA(cudaMalloc(&s->f_omega, om.size() * 4));
    NR_CHECK_CUDA(cudaMalloc(&s->f_bias1, (size_t)n_frames * kWidth * 4));
    NR_CHECK_CUDA(cudaMalloc(&s->f_dbias1, (size_t)n_frames * kWidth * 4));
    NR_CHECK_CUDA(cudaMalloc(&s->f_cam, (size_t)n_frames * sizeof(Frame)));
    s->frames_cap = n_frames;
  }
  NR_CHECK_CUDA(cudaMemcpyAsync(s->f_G, G.data(), G.size() * 4, cudaMemcpyHostToDevice, st));
  NR_CHECK_CUDA(cudaMemcpyAsync(s->f_omega, om.data(), om.size() * 4, cudaMemcpyHostToDevice, st));
  NR_CHECK_CUDA(cudaMemcpyAsync(s->f_cam, fr.data(), fr.size() * sizeof(Frame), cudaMemcpyHostToDevice, st));
  std::vector<float> rt((size_t)n_frames * 3, 0.f);
  if (root_t) memcpy(rt.data(), root_t, rt.size() * 4);
  NR_CHECK_CUDA(cudaMemcpyAsync(s->f_root, rt.data(), rt.size() * 4, cudaMemcpyHostToDevice, st));
  NR_CHECK_CUDA(cudaStreamSynchronize(st));
  s->h_fG = G;
  s->fG_refined = false;
  s->n_frames = n_frames;
  return NR_OK;
}
