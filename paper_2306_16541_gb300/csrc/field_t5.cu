// field_t5.cu -- the per-sample field with both MLPs on the 5th-generation
// tensor cores: tcgen05.mma with accumulators in tensor memory (TMEM).
//
// A block of 512 threads runs four independent groups of 4 warps; a group
// owns a tile of 128 samples, one per thread, and 64 TMEM columns.  For every
// layer:
//   1. each thread writes its sample's input row (bf16/f16) into the group's
//      A tile in shared memory, in the 128-byte-swizzled K-major layout the
//      tensor core reads (16-byte chunk j of row r stored at chunk j ^ (r % 8));
//   2. fence.proxy.async + a group barrier make the rows visible to the tensor
//      core; one elected thread issues the layer's M = 128 MMAs (K = 16 each)
//      against the layer's weights, also swizzled K-major in shared memory, and
//      commits them to the group's mbarrier;
//   3. every thread waits on the mbarrier (bounded), reads its own row of the
//      accumulator from TMEM (tcgen05.ld 32x32b: warp w of the group reads
//      lanes 32w..32w+31), adds the float32 bias, applies ReLU and writes the
//      next layer's input row.
// Outputs (x_res, the canonical MLP's raw outputs) come back as a 16-column
// accumulator that each thread reads for its own row.  The gathers (inverse
// LBS, PE, hash encoding) run in float32 as in field_tc.cu.
//
// Every mbarrier wait gives up after a bounded number of polls; a group that
// times out records an error word, stops waiting, still reaches the block
// barrier and the TMEM release, and returns.
#include "field.cuh"
#include "mma.cuh"
#include "render.cuh"
#include "t5.cuh"

namespace nr {

constexpr int kT5Groups = 4;
constexpr int kT5Threads = 128 * kT5Groups;
constexpr int kT5TmemCols = 64 * kT5Groups;
constexpr uint32_t kT5MaxPolls = 1u << 24;

__device__ __forceinline__ void t5_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// Bounded wait for the completion of phase `parity`; false once the poll budget is spent.
__device__ __forceinline__ bool t5_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < kT5MaxPolls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void group_sync(int group) {
  asm volatile("bar.sync %0, 128;" ::"r"(group + 1));
}

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,"
      "%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
        "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
        "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
        "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
        "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// Writes 8-column chunk j (values v[0..7]) of row r of a swizzled tile.
template <typename T>
__device__ __forceinline__ void put_chunk(uint8_t *tile, int r, int j, const float *v) {
  const uint4 q = make_uint4(pack2<T>(v[0], v[1]), pack2<T>(v[2], v[3]), pack2<T>(v[4], v[5]), pack2<T>(v[6], v[7]));
  *reinterpret_cast<uint4 *>(tile + r * 128 + ((j ^ (r & 7)) << 4)) = q;
}

// Epilogue: row r of the next input = relu(acc + bias), 64 columns.
template <typename T>
__device__ __forceinline__ void relu_row(const float (&acc)[64], const float *bias, uint8_t *tile, int r) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = fmaxf(acc[8 * j + q] + bias[8 * j + q], 0.f);
    put_chunk<T>(tile, r, j, v);
  }
}

struct T5State {           // per-thread view of its group's synchronisation state
  uint32_t mbar, tmem, phase;
  bool ok;
};

// Makes the group's freshly written rows visible to the tensor core, issues
// `nk` K-steps of A x B^T (and `nk2` more of A2 x B2^T into the same
// accumulator), commits, and waits for completion.
__device__ __forceinline__ void t5_layer(T5State &s, int group, bool leader, uint32_t a, uint32_t b, int nk,
                                         uint32_t a2, uint32_t b2, int nk2, uint32_t idesc, uint32_t *err) {
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  group_sync(group);
  if (leader && s.ok) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint64_t da = t5_desc(a), db = t5_desc(b);
    for (int k = 0; k < nk; ++k) t5_mma(s.tmem, da + 2 * k, db + 2 * k, idesc, k > 0);
    if (nk2) {
      const uint64_t da2 = t5_desc(a2), db2 = t5_desc(b2);
      for (int k = 0; k < nk2; ++k) t5_mma(s.tmem, da2 + 2 * k, db2 + 2 * k, idesc, 1);
    }
    t5_commit(s.mbar);
  }
  if (s.ok) {
    if (!t5_wait(s.mbar, s.phase)) {
      s.ok = false;
      atomicExch(err, 1u);
    }
  }
  s.phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;");
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kT5Threads, 1) field_t5_kernel(FieldParams P, const uint8_t *__restrict__ wblob,
                                                                 const float4 *__restrict__ in, uint32_t n_fixed,
                                                                 const uint32_t *__restrict__ n_dev,
                                                                 float *__restrict__ out, uint32_t *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned base for the swizzled tiles
  uint8_t *smem = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const T5Layout L = t5_layout(P.hidden);
  const TcBias bl = tc_bias_layout(P.hidden);
  uint8_t *sW = smem;                                                 // weights
  uint8_t *sTiles = sW + ((L.total + 1023) & ~1023);                  // [group][gamma 16 KB | h 16 KB]
  float *sBias = reinterpret_cast<float *>(sTiles + kT5Groups * 32768);
  float *sG = sBias + ((bl.total + 3) & ~3);
  uint64_t *sMbar = reinterpret_cast<uint64_t *>(sG + kPoseSmem);
  uint32_t *sTmem = reinterpret_cast<uint32_t *>(sMbar + kT5Groups);

  const int tid = threadIdx.x, warp = tid >> 5, group = warp >> 2, r = tid & 127;
  const float *sBox = nullptr;
  {
    const int4 *src = reinterpret_cast<const int4 *>(wblob);
    int4 *dst = reinterpret_cast<int4 *>(sW);
    for (int i = tid; i < L.total / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    auto copyb = [&](int dsto, const float *s, int n, int npad) {
      for (int i = tid; i < npad; i += blockDim.x) sBias[dsto + i] = i < n ? s[i] : 0.f;
    };
    copyb(bl.r1, P.bias1, kWidth, kWidth);
    copyb(bl.r2, P.blob + P.lay.r2b, kWidth, kWidth);
    copyb(bl.r3, P.blob + P.lay.r3b, kWidth, kWidth);
    copyb(bl.r4, P.blob + P.lay.r4b, kWidth, kWidth);
    copyb(bl.r5, P.blob + P.lay.r5b, 3, 4);
    copyb(bl.c0, P.blob + P.lay.c0b, kWidth, kWidth);
    for (int l = 0; l < P.hidden - 1; ++l) copyb(bl.c0 + kWidth * (l + 1), P.blob + P.lay.chb[l], kWidth, kWidth);
    copyb(bl.cl, P.blob + P.lay.clb, 4, 4);
    sBox = stage_pose(P, sG, tid, blockDim.x);
    if (tid < kT5Groups) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(sMbar + tid)));
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sTmem)),
                   "r"(kT5TmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");

  T5State st;
  st.mbar = smem_u32(sMbar + group);
  st.tmem = *sTmem + (uint32_t)(group * 64);          // this group's 64 columns
  st.phase = 0;
  st.ok = true;
  const uint32_t lane_addr = st.tmem + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's 32 lanes
  const bool leader = r == 0;
  uint8_t *gam = sTiles + group * 32768;
  uint8_t *hh = gam + 16384;
  const uint32_t a_gam = smem_u32(gam), a_h = smem_u32(hh);
  const uint32_t id64 = t5_idesc(64, TcFmt<T>::value), id16 = t5_idesc(16, TcFmt<T>::value);

  const uint32_t n = n_dev ? *n_dev : n_fixed;
  const uint32_t n_tiles = (n + 127) / 128;
  for (uint32_t tile = blockIdx.x * kT5Groups + group; tile < n_tiles; tile += gridDim.x * kT5Groups) {
    const uint32_t j = tile * 128 + r;
    const bool valid = j < n;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, delta = 0.f;
    if (valid) {
      if (MODE == kModeRender) {
        const float4 s = in[j];
        x0 = s.x; x1 = s.y; x2 = s.z; delta = s.w;
      } else {
        const float *q = reinterpret_cast<const float *>(in) + 3 * (size_t)j;
        x0 = q[0]; x1 = q[1]; x2 = q[2];
      }
    }
    float s0, s1, s2, S;
    lbs_warp(P, sG, x0, x1, x2, s0, s1, s2, S, sBox);
    float f0 = s0, f1 = s1, f2 = s2;
    float acc[64];
    if (P.res_enabled) {
      {  // gamma(x_skel): 48 columns (39 used) of this thread's row
        float g[48];
        const float h0 = (s0 - P.box_c[0]) * P.box_ih[0];
        const float h1 = (s1 - P.box_c[1]) * P.box_ih[1];
        const float h2 = (s2 - P.box_c[2]) * P.box_ih[2];
        g[0] = h0; g[1] = h1; g[2] = h2;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float sc = (float)(1 << k);
          float sa, ca, sb, cb, sd, cd;
          sincospif(sc * h0, &sa, &ca);
          sincospif(sc * h1, &sb, &cb);
          sincospif(sc * h2, &sd, &cd);
          const float w = (k < P.res_freqs) ? P.hann[k] : 0.f;
          g[3 + 6 * k + 0] = w * sa; g[3 + 6 * k + 1] = w * sb; g[3 + 6 * k + 2] = w * sd;
          g[3 + 6 * k + 3] = w * ca; g[3 + 6 * k + 4] = w * cb; g[3 + 6 * k + 5] = w * cd;
        }
#pragma unroll
        for (int k = 39; k < 48; ++k) g[k] = 0.f;
#pragma unroll
        for (int c = 0; c < 6; ++c) put_chunk<T>(gam, r, c, g + 8 * c);
      }
      t5_layer(st, group, leader, a_gam, smem_u32(sW + L.r1), 3, 0, 0, 0, id64, err);
      tmem_ld64(lane_addr, acc);
      relu_row<T>(acc, sBias + bl.r1, hh, r);
      t5_layer(st, group, leader, a_h, smem_u32(sW + L.r2), 4, 0, 0, 0, id64, err);
      tmem_ld64(lane_addr, acc);
      relu_row<T>(acc, sBias + bl.r2, hh, r);
      t5_layer(st, group, leader, a_h, smem_u32(sW + L.r3), 4, 0, 0, 0, id64, err);
      tmem_ld64(lane_addr, acc);
      relu_row<T>(acc, sBias + bl.r3, hh, r);
      t5_layer(st, group, leader, a_h, smem_u32(sW + L.r4h), 4, a_gam, smem_u32(sW + L.r4g), 3, id64, err);
      tmem_ld64(lane_addr, acc);
      relu_row<T>(acc, sBias + bl.r4, hh, r);
      t5_layer(st, group, leader, a_h, smem_u32(sW + L.r5), 4, 0, 0, 0, id16, err);
      float o3[4];
      tmem_ld4(lane_addr, o3);
      f0 += o3[0] + sBias[bl.r5 + 0];
      f1 += o3[1] + sBias[bl.r5 + 1];
      f2 += o3[2] + sBias[bl.r5 + 2];
    }
    // canonical field: hash encoding (float32) -> 32 columns of this thread's row
    bool inside;
    {
      float p0 = (f0 - P.bmin[0]) * P.inv_box[0];
      float p1 = (f1 - P.bmin[1]) * P.inv_box[1];
      float p2 = (f2 - P.bmin[2]) * P.inv_box[2];
      inside = p0 >= 0.f && p0 <= 1.f && p1 >= 0.f && p1 <= 1.f && p2 >= 0.f && p2 <= 1.f;
      p0 = fminf(fmaxf(p0, 0.f), 1.f);
      p1 = fminf(fmaxf(p1, 0.f), 1.f);
      p2 = fminf(fmaxf(p2, 0.f), 1.f);
      float e[32];
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
        e[2 * l] = inside ? fa : 0.f;
        e[2 * l + 1] = inside ? fb : 0.f;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) put_chunk<T>(hh, r, c, e + 8 * c);
    }
    t5_layer(st, group, leader, a_h, smem_u32(sW + L.c0), 2, 0, 0, 0, id64, err);
    tmem_ld64(lane_addr, acc);
    relu_row<T>(acc, sBias + bl.c0, hh, r);
    for (int l = 0; l < P.hidden - 1; ++l) {
      t5_layer(st, group, leader, a_h, smem_u32(sW + L.c0 + 8192 * (l + 1)), 4, 0, 0, 0, id64, err);
      tmem_ld64(lane_addr, acc);
      relu_row<T>(acc, sBias + bl.c0 + kWidth * (l + 1), hh, r);
    }
    t5_layer(st, group, leader, a_h, smem_u32(sW + L.cl), 4, 0, 0, 0, id16, err);
    float o[4];
    tmem_ld4(lane_addr, o);
    if (valid) {
      const float cr = sigmoidf_(o[0] + sBias[bl.cl]), cg = sigmoidf_(o[1] + sBias[bl.cl + 1]);
      const float cb = sigmoidf_(o[2] + sBias[bl.cl + 2]), sigma = softplusf_(o[3] + sBias[bl.cl + 3]);
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
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*sTmem), "r"(kT5TmemCols));
  }
}

// Swizzled K-major copy of a layer: rows [0, out) x columns [col0, col0 + n_in) of W into a
// [rows][64] tile at byte offset `dst` (rows out..rows-1 and columns n_in..63 are zero).
template <typename T>
__global__ void pack_t5_kernel(const float *__restrict__ W, int stride, int col0, int n_in, int out, int rows,
                               int dst, uint8_t *__restrict__ blob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * 64) return;
  const int rr = i / 64, k = i % 64;
  const float v = (rr < out && k < n_in) ? W[(size_t)rr * stride + col0 + k] : 0.f;
  *reinterpret_cast<T *>(blob + dst + sw128(rr, k)) = T(v);
}

template <typename T>
static int pack_t5_all(const nr_subject *s, const MasterOffsets &m, cudaStream_t st, uint8_t *blob) {
  const T5Layout L = t5_layout((int)s->hidden);
  const int g = res_gamma_dims(s), P3 = 3 * (int)s->K, H = (int)s->hidden;
  int launched = 0;
  auto pack = [&](const float *W, int stride, int col0, int n_in, int out, int rows, int dst) {
    pack_t5_kernel<T><<<(rows * 64 + 255) / 256, 256, 0, st>>>(W, stride, col0, n_in, out, rows, dst, blob);
    ++launched;
  };
  pack(s->res + m.r[0], g + P3, 0, g, kWidth, 64, L.r1);
  pack(s->res + m.r[1], kWidth, 0, kWidth, kWidth, 64, L.r2);
  pack(s->res + m.r[2], kWidth, 0, kWidth, kWidth, 64, L.r3);
  pack(s->res + m.r[3], kWidth + g, 0, kWidth, kWidth, 64, L.r4h);
  pack(s->res + m.r[3], kWidth + g, kWidth, g, kWidth, 64, L.r4g);
  pack(s->res + m.r[4], kWidth, 0, kWidth, 3, 16, L.r5);
  pack(s->mlp + m.c[0], (int)s->mlp_in, 0, (int)s->mlp_in, kWidth, 64, L.c0);
  for (int l = 1; l < H; ++l) pack(s->mlp + m.c[l], kWidth, 0, kWidth, kWidth, 64, L.ch[l - 1]);
  pack(s->mlp + m.c[H], kWidth, 0, kWidth, 4, 16, L.cl);
  return launched;
}

nr_status prepare_t5(nr_subject *s, cudaStream_t st) {
  if (s->t5_ready) return NR_OK;
  const T5Layout L = t5_layout((int)s->hidden);
  if (!s->t5_bf16 || !s->t5_f16) {   // allocated with the subject
    set_error("tcgen05 weight blobs missing");
    return NR_ESTATE;
  }
  NR_CHECK_CUDA(cudaMemsetAsync(s->t5_bf16, 0, (size_t)L.total, st));
  NR_CHECK_CUDA(cudaMemsetAsync(s->t5_f16, 0, (size_t)L.total, st));
  const MasterOffsets m = master_offsets(s);
  int launched = pack_t5_all<__nv_bfloat16>(s, m, st, s->t5_bf16);
  launched += pack_t5_all<__half>(s, m, st, s->t5_f16);
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(launched);
  s->t5_ready = true;
  return NR_OK;
}

static size_t t5_smem(int hidden) {
  const T5Layout L = t5_layout(hidden);
  const TcBias bl = tc_bias_layout(hidden);
  size_t b = 1024 + (size_t)((L.total + 1023) & ~1023) + (size_t)kT5Groups * 32768;
  b += sizeof(float) * (((bl.total + 3) & ~3) + kPoseSmem);
  b += sizeof(uint64_t) * kT5Groups + 16;
  return b;
}

template <typename T, int MODE>
static nr_status launch_t5_mode(const FieldParams &P, const uint8_t *blob, const float4 *in, uint32_t n_fixed,
                                const uint32_t *n_dev, float *out, uint32_t *err, int device, cudaStream_t st) {
  const size_t smem = t5_smem(P.hidden);
  NR_CHECK_CUDA(cudaFuncSetAttribute(field_t5_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  field_t5_kernel<T, MODE><<<num_sms(device), kT5Threads, smem, st>>>(P, blob, in, n_fixed, n_dev, out, err);
  NR_CHECK_CUDA(cudaGetLastError());
  return NR_OK;
}

nr_status launch_field_t5(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                          const uint32_t *n_dev, float *out, int device, cudaStream_t st) {
  if (!P.t5_bf16 || !P.t5_f16 || !P.t5_err) {
    set_error("tcgen05 weights not prepared");
    return NR_ESTATE;
  }
  if (mlp_dtype == NR_BF16)
    return mode == kModeRender
               ? launch_t5_mode<__nv_bfloat16, kModeRender>(P, P.t5_bf16, in, n_fixed, n_dev, out, P.t5_err, device, st)
               : launch_t5_mode<__nv_bfloat16, kModeQuery>(P, P.t5_bf16, in, n_fixed, n_dev, out, P.t5_err, device, st);
  return mode == kModeRender
             ? launch_t5_mode<__half, kModeRender>(P, P.t5_f16, in, n_fixed, n_dev, out, P.t5_err, device, st)
             : launch_t5_mode<__half, kModeQuery>(P, P.t5_f16, in, n_fixed, n_dev, out, P.t5_err, device, st);
}

}  // namespace nr
