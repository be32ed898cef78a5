// field_ws.cu -- the per-sample field (Sec. 4.2 - 4.4) with both MLPs on the
// 5th-generation tensor cores and the activations kept in tensor memory (TMEM)
// between layers, as a warp-specialised pipeline.
//
// A block (one per SM) holds kWsGroups worker groups of 4 warps and one
// warpgroup of issuer warps, one per worker group.  Each worker group owns a
// 128-sample tile at a time, one sample per thread (thread r of the group <->
// TMEM lane r), and a slot of kWsSlotCols TMEM columns:
//   [kWsAcc, +64)   float32 accumulator D of the current layer (N <= 64);
//   [kWsAct, +32)   the layer input A as packed bf16/f16 pairs (K <= 64);
//   [kWsOne, +8)    the constant input (1, 1, 0, ..., 0) (K = 16);
//   [kWsGam, +24)   gamma(x_skel) (K = 48, inputs 39 and 40 held at 1), read
//                   by residual layers 1 and 4.
// The bias of a hidden layer enters its product through the constant inputs,
// split as b = hi + lo with both parts in the operand type (about 16
// significant bits): residual layers 1 and 4 read it from weight columns 39
// and 40 against gamma's ones, the others take one more K step of the
// constant block against a bias tile (products and sums in float32).  So per
// layer the group's threads read their accumulator row (tcgen05.ld), convert
// it with ReLU to the next layer's packed input (one cvt.rn.relu per pair),
// write it back into TMEM (tcgen05.st) and arrive, one arrive per warp, on the
// group's "input ready" mbarrier; the group's issuer warp then sends the layer
// as M = 128 MMAs with A read from TMEM and the weights (B) from shared memory
// and commits them to the group's "layer done" mbarrier, which the workers
// wait on.  The two output layers (x_res and the four raw outputs) keep their
// float32 bias.  A thread that issues tcgen05.mma is held while the tensor
// core takes the instructions, and one issuer keeps only about half of a
// tensor core busy with these short (K = 64, N = 64) layers: so every group has
// its own issuer, and the issuers are not the workers, who would otherwise sit
// in the issue.  The issuer warpgroup gives its registers to the workers
// (setmaxnreg: 32 per issuer thread, 112 per worker thread).
// While one group waits for its MMAs the others run their gathers (inverse
// LBS, positional encoding, hash encoding, in float32 as in field_tc.cu), so
// gathers and MMAs of different tiles overlap; no activation passes through
// shared memory and the weights are read by the tensor core alone.
//
// Every mbarrier wait is bounded (kWsTimeoutNs of the global timer).  A warp
// whose wait gives up records an error word and stops waiting and arriving; an
// issuer whose input does not arrive stops issuing.  Before the block releases
// its TMEM each issuer commits once more and waits (bounded) for every MMA it
// issued.
#include "field.cuh"
#include "gather.cuh"
#include "mma.cuh"
#include "render.cuh"
#include "t5.cuh"

namespace nr {

constexpr int kWsGroups = 4;
constexpr int kWsWorkers = 128 * kWsGroups;
constexpr int kWsThreads = kWsWorkers + 128;                 // + the issuer warpgroup
constexpr int kWsRegsWorker = 112, kWsRegsIssuer = 32;      // 4 x 128 x 112 + 128 x 32 = 640 x 96
constexpr uint32_t kWsSlotCols = 128;
constexpr uint32_t kWsTmemCols = kWsSlotCols * kWsGroups;   // 512: the whole of TMEM
constexpr uint32_t kWsAcc = 0, kWsAct = 64, kWsOne = 96, kWsGam = 104;
constexpr int kWsBiasTile = 64 * 128;     // bytes of one bias tile: 64 rows of one swizzled 128-byte row
constexpr int kWsMaxLayers = 5 + kMaxHidden + 1;
constexpr unsigned long long kWsTimeoutNs = 500000000ull;
// The fp8 tier's table in shared memory (floats): m' per layer, then b' [layer][64] from a
// 16-byte aligned offset (read as float4), then 1 / s_a of gamma and of the encoding.
constexpr int kWsF8Bias = (kWsMaxLayers + 3) & ~3;
constexpr int kWsF8Inv = kWsF8Bias + kWsMaxLayers * 64;

// One layer as the issuing thread sends it: nk K-steps of A (TMEM column a_col) x B (weights at
// byte offset b_off of the shared blob), then nk2 K-steps of a second pair into the same
// accumulator (residual layer 4: [h3 | gamma]).
struct WsLayer {
  uint32_t a_col, b_off, nk, a2_col, b2_off, nk2, idesc, pad;
};

__device__ __forceinline__ uint64_t ws_now() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for the completion of phase `parity`; false once kWsTimeoutNs have passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = ws_now();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (ws_now() - t0 > kWsTimeoutNs) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}

// The fp8 tier's operand type: e4m3 operands of tcgen05.mma kind::f8f6f4 (format code 0).
struct E4M3 {};
template <>
struct TcFmt<E4M3> {
  static constexpr int value = 0;
};
template <typename T>
constexpr bool kIsF8 = false;
template <>
constexpr bool kIsF8<E4M3> = true;

// D[128 x N] (+)= A[128 x K] B^T with A in TMEM (columns a .. a + 7: K = 16 bf16/f16 or 32 e4m3
// values) and B in shared memory.
template <bool F8>
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if constexpr (F8)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// Four float32 values as e4m3 bytes 0..3 of a word (rounded, saturated to +-448; with ReLU when
// RELU).
template <bool RELU>
__device__ __forceinline__ uint32_t e4m3x4(float a0, float a1, float a2, float a3) {
  uint32_t d;
  if constexpr (RELU)
    asm("{\n.reg .b16 lo, hi;\ncvt.rn.satfinite.relu.e4m3x2.f32 lo, %2, %1;\n"
        "cvt.rn.satfinite.relu.e4m3x2.f32 hi, %4, %3;\nmov.b32 %0, {lo, hi};\n}\n"
        : "=r"(d) : "f"(a0), "f"(a1), "f"(a2), "f"(a3));
  else
    asm("{\n.reg .b16 lo, hi;\ncvt.rn.satfinite.e4m3x2.f32 lo, %2, %1;\n"
        "cvt.rn.satfinite.e4m3x2.f32 hi, %4, %3;\nmov.b32 %0, {lo, hi};\n}\n"
        : "=r"(d) : "f"(a0), "f"(a1), "f"(a2), "f"(a3));
  return d;
}

// 32 columns of this warp's 32 lanes; the wait carries the registers so that no use of
// them is scheduled before the load has completed.
__device__ __forceinline__ void tm_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
      "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

__device__ __forceinline__ void tm_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3) : : "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
}

__device__ __forceinline__ void tm_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]));
}

__device__ __forceinline__ void tm_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]));
}

__device__ __forceinline__ void tm_st1(uint32_t taddr, uint32_t v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(v));
}

struct WsGroup {
  uint32_t a_bar;       // the group's "input ready" mbarrier (one arrive per worker warp)
  uint32_t d_bar;       // the group's "layer done" mbarrier (the issuer's commit)
};

// One layer of a worker group: this thread's TMEM stores complete, one arrive per warp hands the
// slot to the issuer, `overlap` runs while the tensor core works, and every thread waits (bounded)
// for the result.  ok stays warp-uniform; a warp whose wait gave up stops arriving.
template <typename Overlap>
__device__ __forceinline__ void ws_layer(const WsGroup &G, uint32_t &phase, bool &ok, uint32_t *err,
                                         Overlap &&overlap) {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncwarp();
  if ((threadIdx.x & 31) == 0 && ok) mbar_arrive(G.a_bar);
  overlap();
  if (ok && !mbar_wait_bounded(G.d_bar, phase)) {
    ok = false;
    atomicExch(err, 1u);
  }
  ok = __all_sync(0xffffffffu, ok);
  phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// The issuer of one group: for each of its n layer steps, wait (bounded) for the group's input,
// send the layer's MMAs and commit them; then commit once more and wait until every MMA it issued
// has completed.  One thread.
template <bool F8>
__device__ __forceinline__ void ws_issue(uint32_t slot, uint32_t a_bar, uint32_t d_bar, uint32_t drain,
                                         const WsLayer *__restrict__ lay, int n_layers, uint32_t n_steps,
                                         const uint8_t *sW, uint32_t *err) {
  uint32_t phase = 0;
  for (uint32_t i = 0; i < n_steps; ++i) {
    if (!mbar_wait_bounded(a_bar, phase)) {
      atomicExch(err, 2u);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const WsLayer &Ly = lay[i % (uint32_t)n_layers];
    const uint64_t db = t5_desc(smem_u32(sW + Ly.b_off));
    for (uint32_t k = 0; k < Ly.nk; ++k) mma_ts<F8>(slot + kWsAcc, slot + Ly.a_col + 8 * k, db + 2 * k, Ly.idesc, k);
    if (Ly.nk2) {
      const uint64_t db2 = t5_desc(smem_u32(sW + Ly.b2_off));
      for (uint32_t k = 0; k < Ly.nk2; ++k)
        mma_ts<F8>(slot + kWsAcc, slot + Ly.a2_col + 8 * k, db2 + 2 * k, Ly.idesc, 1u);
    }
    t5_commit(d_bar);
  }
  t5_commit(drain);
  if (!mbar_wait_bounded(drain, 0)) atomicExch(err, 3u);
}

// Two float32 values with ReLU as one packed bf16/f16 pair (lo in the low half).
template <typename T>
__device__ __forceinline__ uint32_t relu_pack(float lo, float hi);
template <>
__device__ __forceinline__ uint32_t relu_pack<__nv_bfloat16>(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
template <>
__device__ __forceinline__ uint32_t relu_pack<__half>(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// Epilogue of a 64-wide hidden layer (bias already in the accumulator): row = relu(acc)
// packed into the input columns.
template <typename T>
__device__ __forceinline__ void ws_relu_layer(uint32_t my) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t v[32];
    tm_ld32(my + kWsAcc + 32 * h, v);
    uint32_t p[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) p[i] = relu_pack<T>(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
    tm_st16(my + kWsAct + 16 * h, p);
  }
}

// Epilogue of a 64-wide hidden layer of the fp8 tier: row = e4m3(relu(m' acc + b')) with
// m' = s_w s_a / s_a,next and b' = b / s_a,next (the next layer's input scale), 4 bytes a column.
__device__ __forceinline__ void ws_relu_layer_f8(uint32_t my, float m, const float *__restrict__ b) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t v[32];
    tm_ld32(my + kWsAcc + 32 * h, v);
    uint32_t p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 bb = reinterpret_cast<const float4 *>(b)[8 * h + i];   // one broadcast load per 4 columns
      p[i] = e4m3x4<true>(fmaf(__uint_as_float(v[4 * i]), m, bb.x), fmaf(__uint_as_float(v[4 * i + 1]), m, bb.y),
                          fmaf(__uint_as_float(v[4 * i + 2]), m, bb.z), fmaf(__uint_as_float(v[4 * i + 3]), m, bb.w));
    }
    tm_st8(my + kWsAct + 8 * h, p);
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kWsThreads, 1) field_ws_kernel(FieldParams P, const uint8_t *__restrict__ wblob,
                                                                 const float4 *__restrict__ in, uint32_t n_fixed,
                                                                 const uint32_t *__restrict__ n_dev,
                                                                 float *__restrict__ out, uint32_t *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const T5Layout L = t5_layout(P.hidden);
  const TcBias bl = tc_bias_layout(P.hidden);
  const int n_bt = P.hidden + 2;                                          // bias tiles: r2, r3, c0, ch[]
  const int bt0 = (L.total + 1023) & ~1023;                               // their offset from sW
  uint8_t *sW = smem;                                                     // swizzled weights (B operands)
  float *sBias = reinterpret_cast<float *>(sW + bt0 + n_bt * kWsBiasTile);
  float *sG = sBias + ((bl.total + 3) & ~3);
  uint64_t *sBar = reinterpret_cast<uint64_t *>(sG + kPoseSmem);         // input ready[G], done[G], drain[G]
  WsLayer *sLay = reinterpret_cast<WsLayer *>(sBar + 3 * kWsGroups);
  uint32_t *sTmem = reinterpret_cast<uint32_t *>(sLay + kWsMaxLayers);
  float *sF8 = reinterpret_cast<float *>(sTmem + 4);   // fp8 tier's table (16-byte aligned)
  constexpr bool F8 = kIsF8<T>;

  {  // a block with no tile leaves before any set-up (the live count is known only here)
    const uint32_t n0 = n_dev ? *n_dev : n_fixed;
    if ((uint64_t)blockIdx.x * kWsGroups * 128 >= n0) return;
  }
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool res = P.res_enabled != 0;
  const int H = P.hidden;
  const float *sBox = nullptr;
  {  // weights, biases, pose; barriers and the layer table; TMEM
    const int4 *src = reinterpret_cast<const int4 *>(wblob);
    int4 *dst = reinterpret_cast<int4 *>(sW);
    for (int i = tid; i < L.total / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    for (int i = tid; i < n_bt * kWsBiasTile / 16; i += blockDim.x) dst[bt0 / 16 + i] = make_int4(0, 0, 0, 0);
    auto copyb = [&](int dsto, const float *s, int nv, int npad) {
      for (int i = tid; i < npad; i += blockDim.x) sBias[dsto + i] = i < nv ? s[i] : 0.f;
    };
    copyb(bl.r1, P.bias1, kWidth, kWidth);
    copyb(bl.r2, P.blob + P.lay.r2b, kWidth, kWidth);
    copyb(bl.r3, P.blob + P.lay.r3b, kWidth, kWidth);
    copyb(bl.r4, P.blob + P.lay.r4b, kWidth, kWidth);
    copyb(bl.r5, P.blob + P.lay.r5b, 3, 4);
    copyb(bl.c0, P.blob + P.lay.c0b, kWidth, kWidth);
    for (int l = 0; l < H - 1; ++l) copyb(bl.c0 + kWidth * (l + 1), P.blob + P.lay.chb[l], kWidth, kWidth);
    copyb(bl.cl, P.blob + P.lay.clb, 4, 4);
    sBox = stage_pose(P, sG, tid, blockDim.x);
    __syncthreads();
    // biases into the B operands: columns 39 and 40 of residual layers 1 (the pose-folded bias)
    // and 4 (its gamma part), columns 0 and 1 of the bias tiles
    if constexpr (F8) {
      // fp8: per layer m' = m / s_a,next and b' = b / s_a,next for the epilogue (no bias in the
      // products: e4m3 would keep 3 bits of it)
      const int nl = (res ? 5 : 0) + H + 1, c0l = res ? 5 : 0;
      const float *sc = P.fp8_scales;
      auto bias_of = [&](int li, int n) -> float {
        if (li < c0l) {
          if (li == 0) return P.bias1[n];
          if (li == 4) return n < 3 ? P.blob[P.lay.r5b + n] : 0.f;
          return P.blob[(li == 1 ? P.lay.r2b : li == 2 ? P.lay.r3b : P.lay.r4b) + n];
        }
        const int c = li - c0l;
        if (c == 0) return P.blob[P.lay.c0b + n];
        if (c == H) return n < 4 ? P.blob[P.lay.clb + n] : 0.f;
        return P.blob[P.lay.chb[c - 1] + n];
      };
      for (int i = tid; i < nl * kWidth; i += blockDim.x) {
        const int li = i / kWidth, n = i % kWidth;
        sF8[kWsF8Bias + i] = bias_of(li, n) * sc[kF8SlotWs + 2 * li + 1];
      }
      if (tid < nl) sF8[tid] = sc[kF8SlotWs + 2 * tid] * sc[kF8SlotWs + 2 * tid + 1];
      if (tid == 0) {   // 1 / s_a of gamma and of the hash encoding (the inputs the workers quantise)
        sF8[kWsF8Inv] = sc[kF8SlotInvGam];
        sF8[kWsF8Inv + 1] = sc[kF8SlotInvEnc];
      }
    } else if (tid < kWidth) {
      const int n = tid;
      // b = hi + lo, both rounded to the operand type, in columns k and k + 1
      auto put = [&](int tile, int k, float v) {
        const T hi = TcOps<T>::cvt(v);
        *reinterpret_cast<T *>(sW + tile + sw128(n, k)) = hi;
        *reinterpret_cast<T *>(sW + tile + sw128(n, k + 1)) = TcOps<T>::cvt(v - (float)hi);
      };
      put(L.r1, 39, P.bias1[n]);
      put(L.r4g, 39, P.blob[P.lay.r4b + n]);
      put(bt0 + 0 * kWsBiasTile, 0, P.blob[P.lay.r2b + n]);
      put(bt0 + 1 * kWsBiasTile, 0, P.blob[P.lay.r3b + n]);
      put(bt0 + 2 * kWsBiasTile, 0, P.blob[P.lay.c0b + n]);
      for (int l = 0; l < P.hidden - 1; ++l) put(bt0 + (3 + l) * kWsBiasTile, 0, P.blob[P.lay.chb[l] + n]);
    }
    if (tid == 0) {
      for (int g = 0; g < 3 * kWsGroups; ++g)   // input ready: four worker warps; the others: one commit
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(sBar + g)), "r"(g < kWsGroups ? 4 : 1));
      const int fmt = TcFmt<T>::value;
      int k = 0;
      auto add = [&](uint32_t a, int b, int nk, uint32_t a2, int b2, int nk2, int nout) {
        sLay[k++] = WsLayer{a, (uint32_t)b, (uint32_t)nk, a2, (uint32_t)b2, (uint32_t)nk2, t5_idesc(nout, fmt), 0u};
      };
      if constexpr (F8) {   // K = 32 e4m3 values a step; gamma padded to 64
        if (res) {
          add(kWsGam, L.r1, 2, 0, 0, 0, 64);
          add(kWsAct, L.r2, 2, 0, 0, 0, 64);
          add(kWsAct, L.r3, 2, 0, 0, 0, 64);
          add(kWsAct, L.r4h, 2, kWsGam, L.r4g, 2, 64);
          add(kWsAct, L.r5, 2, 0, 0, 0, 16);
        }
        add(kWsAct, L.c0, 1, 0, 0, 0, 64);
        for (int l = 0; l < H - 1; ++l) add(kWsAct, L.ch[l], 2, 0, 0, 0, 64);
        add(kWsAct, L.cl, 2, 0, 0, 0, 16);
      } else {
        if (res) {
          add(kWsGam, L.r1, 3, 0, 0, 0, 64);
          add(kWsAct, L.r2, 4, kWsOne, bt0 + 0 * kWsBiasTile, 1, 64);
          add(kWsAct, L.r3, 4, kWsOne, bt0 + 1 * kWsBiasTile, 1, 64);
          add(kWsAct, L.r4h, 4, kWsGam, L.r4g, 3, 64);
          add(kWsAct, L.r5, 4, 0, 0, 0, 16);
        }
        add(kWsAct, L.c0, kMlpIn / 16, kWsOne, bt0 + 2 * kWsBiasTile, 1, 64);
        for (int l = 0; l < H - 1; ++l) add(kWsAct, L.ch[l], 4, kWsOne, bt0 + (3 + l) * kWsBiasTile, 1, 64);
        add(kWsAct, L.cl, 4, 0, 0, 0, 16);
      }
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sTmem)),
                   "r"(kWsTmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  const uint32_t tmem0 = *sTmem;
  const uint32_t n = n_dev ? *n_dev : n_fixed;
  const uint32_t n_tiles = (n + 127) / 128;
  const uint32_t tstride = gridDim.x * kWsGroups;

  if (tid >= kWsWorkers) {
    // ------------------------------------------------------------- issuers
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kWsRegsIssuer));
    const int g = warp - kWsWorkers / 32;
    if ((tid & 31) == 0) {
      const uint32_t t0 = blockIdx.x * kWsGroups + g;
      const uint32_t tiles = t0 < n_tiles ? (n_tiles - t0 + tstride - 1) / tstride : 0u;
      const int n_layers = (res ? 5 : 0) + H + 1;
      ws_issue<F8>(tmem0 + (uint32_t)g * kWsSlotCols, smem_u32(sBar + g), smem_u32(sBar + kWsGroups + g),
               smem_u32(sBar + 2 * kWsGroups + g), sLay, n_layers, tiles * (uint32_t)n_layers, sW, err);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------- workers
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kWsRegsWorker));
    const int g = warp >> 2, q = warp & 3, r = tid & 127;
    WsGroup G;
    G.a_bar = smem_u32(sBar + g);
    G.d_bar = smem_u32(sBar + kWsGroups + g);
    const uint32_t my = tmem0 + (uint32_t)g * kWsSlotCols + ((uint32_t)(q * 32) << 16);   // this warp's lanes
    uint32_t phase = 0;
    bool ok = true;
    if constexpr (!F8) {  // the constant input block (1, 1, 0, ..., 0) of this thread's row; no layer writes it
      const uint32_t c[8] = {pack2<T>(1.f, 1.f), 0u, 0u, 0u, 0u, 0u, 0u, 0u};
      tm_st8(my + kWsOne, c);
    }
    const int n_layers = (res ? 5 : 0) + H + 1;
    bool nx_valid = false;
    // this thread's sample of a tile: position and spacing (zero beyond n)
    auto load_in = [&](uint32_t t, LbsState &st, float &dl) {
      const uint32_t jj = t * 128 + r;
      st.x0 = st.x1 = st.x2 = dl = 0.f;
      nx_valid = jj < n;
      if (jj < n) {
        if (MODE == kModeRender) {
          const float4 v = in[jj];
          st.x0 = v.x; st.x1 = v.y; st.x2 = v.z; dl = v.w;
        } else {
          const float *qv = reinterpret_cast<const float *>(in) + 3 * (size_t)jj;
          st.x0 = qv[0]; st.x1 = qv[1]; st.x2 = qv[2];
        }
      }
    };
    // The inverse-LBS warp of the next tile runs in this tile's MLP waits: its support-box tests
    // in the first wait, one round of four bones in each later one; what is left when the next
    // tile starts is finished then.
    uint32_t tile = blockIdx.x * kWsGroups + g;
    LbsState nx;
    float d_next = 0.f;
    if (tile < n_tiles) {
      load_in(tile, nx, d_next);
      lbs_begin(P, sG, sBox, nx, nx_valid);
    }
    for (; tile < n_tiles; tile += tstride) {
      const uint32_t j = tile * 128 + r;
      const bool valid = j < n;
      const float delta = d_next;
      float s0, s1, s2, S;
      lbs_end(P, sG, nx, s0, s1, s2, S);
      if (P.kept_count) {   // profiled renders: the bone channels this warp's samples read
        uint32_t c = valid ? (uint32_t)__popc(nx.mine) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((tid & 31) == 0) atomicAdd(P.kept_count, c);
      }
      const bool more = tile + tstride < n_tiles;
      if (more) load_in(tile + tstride, nx, d_next);
      int stage = 0;
      auto overlap = [&]() {
        if (!more) return;
        if (stage == 0)
          lbs_begin(P, sG, sBox, nx, nx_valid);
        else
          lbs_round(P, sG, nx);
        ++stage;
      };
      if (res) {  // gamma(x_skel): 48 columns (39 used) as 24 packed TMEM columns
        float gm[48];
        const float h0 = (s0 - P.box_c[0]) * P.box_ih[0];
        const float h1 = (s1 - P.box_c[1]) * P.box_ih[1];
        const float h2 = (s2 - P.box_c[2]) * P.box_ih[2];
        gm[0] = h0; gm[1] = h1; gm[2] = h2;
        // band 0 from sincospif, band k + 1 from band k by the double-angle identities
        // sin 2a = 2 sin a cos a, cos 2a = (cos a - sin a)(cos a + sin a); the absolute error at
        // most doubles per band (below 1e-5 at band 5, against the 2^-9 of the bf16/f16 operand)
        float sa, ca, sb, cb, sd, cd;
        sincospif(h0, &sa, &ca);
        sincospif(h1, &sb, &cb);
        sincospif(h2, &sd, &cd);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float w = (k < P.res_freqs) ? P.hann[k] : 0.f;
          gm[3 + 6 * k + 0] = w * sa; gm[3 + 6 * k + 1] = w * sb; gm[3 + 6 * k + 2] = w * sd;
          gm[3 + 6 * k + 3] = w * ca; gm[3 + 6 * k + 4] = w * cb; gm[3 + 6 * k + 5] = w * cd;
          if (k < 5) {
            const float na = 2.f * sa * ca, nb = 2.f * sb * cb, nd = 2.f * sd * cd;
            ca = (ca - sa) * (ca + sa);
            cb = (cb - sb) * (cb + sb);
            cd = (cd - sd) * (cd + sd);
            sa = na; sb = nb; sd = nd;
          }
        }
#pragma unroll
        for (int k = 41; k < 48; ++k) gm[k] = 0.f;
        if constexpr (F8) {   // 64 e4m3 values (39 used) in 16 columns, scaled by 1 / s_a
          const float inv_gam = sF8[kWsF8Inv];
          gm[39] = gm[40] = 0.f;
          uint32_t pa[16];
#pragma unroll
          for (int k = 0; k < 12; ++k)
            pa[k] = e4m3x4<false>(gm[4 * k] * inv_gam, gm[4 * k + 1] * inv_gam, gm[4 * k + 2] * inv_gam,
                                  gm[4 * k + 3] * inv_gam);
#pragma unroll
          for (int k = 12; k < 16; ++k) pa[k] = 0u;
          tm_st16(my + kWsGam, pa);
        } else {
          gm[39] = 1.f;                                     // against the weights' bias columns
          gm[40] = 1.f;
          uint32_t pa[16], pb[8];
#pragma unroll
          for (int k = 0; k < 16; ++k) pa[k] = pack2<T>(gm[2 * k], gm[2 * k + 1]);
#pragma unroll
          for (int k = 0; k < 8; ++k) pb[k] = pack2<T>(gm[32 + 2 * k], gm[32 + 2 * k + 1]);
          tm_st16(my + kWsGam, pa);
          tm_st8(my + kWsGam + 16, pb);
        }
      }
      // the layers: residual 1 .. 5 (with MLP_res), then canonical 0 .. H; before canonical
      // layer 0 the hash encoding of x_final = x_skel + x_res fills the input columns
      const int c0i = res ? 5 : 0;
      float f0 = s0, f1 = s1, f2 = s2;
      bool inside = false;
      for (int li = 0; li < n_layers; ++li) {
        if (li == c0i) {
          float p0 = (f0 - P.bmin[0]) * P.inv_box[0];
          float p1 = (f1 - P.bmin[1]) * P.inv_box[1];
          float p2 = (f2 - P.bmin[2]) * P.inv_box[2];
          inside = p0 >= 0.f && p0 <= 1.f && p1 >= 0.f && p1 <= 1.f && p2 >= 0.f && p2 <= 1.f;
          p0 = fminf(fmaxf(p0, 0.f), 1.f);
          p1 = fminf(fmaxf(p1, 0.f), 1.f);
          p2 = fminf(fmaxf(p2, 0.f), 1.f);
          if constexpr (F8) {
            // e4m3 pairs scaled by 1 / s_a, two levels to a column
            const float inv_enc = sF8[kWsF8Inv + 1];
            uint32_t pend = 0u;
            auto emit8 = [&](int l, float fa, float fb) {
              const uint32_t q = e4m3x4<false>(fa * inv_enc, fb * inv_enc, 0.f, 0.f) & 0xFFFFu;
              if (l & 1)
                tm_st1(my + kWsAct + (uint32_t)(l >> 1), pend | (q << 16));
              else
                pend = q;
            };
            if (grouped_apply(P)) {
              hash_encode_f16_grouped<T>(P, p0, p1, p2, inside, [&](int l, uint32_t v) {
                const float2 f = h2f2(v);
                emit8(l, f.x, f.y);
              });
            } else {
#pragma unroll 1
              for (int l = 0; l < P.L; ++l) {
                float fa, fb;
                hash_level(P, l, p0, p1, p2, fa, fb);
                emit8(l, inside ? fa : 0.f, inside ? fb : 0.f);
              }
            }
            if (P.L & 1) tm_st1(my + kWsAct + (uint32_t)(P.L >> 1), pend);
            for (int c = (P.L + 1) >> 1; c < kMaxLevels / 2; ++c) tm_st1(my + kWsAct + (uint32_t)c, 0u);
          } else {
            if (grouped_apply(P)) {
              hash_encode_f16_grouped<T>(P, p0, p1, p2, inside,
                                         [&](int l, uint32_t v) { tm_st1(my + kWsAct + (uint32_t)l, v); });
            } else {
#pragma unroll 1
              for (int l = 0; l < P.L; ++l) {
                float fa, fb;
                hash_level(P, l, p0, p1, p2, fa, fb);
                tm_st1(my + kWsAct + (uint32_t)l, inside ? pack2<T>(fa, fb) : 0u);
              }
            }
            for (int l = P.L; l < kMaxLevels; ++l) tm_st1(my + kWsAct + (uint32_t)l, 0u);
          }
        }
        ws_layer(G, phase, ok, err, overlap);
        if (li == n_layers - 1) break;
        if (res && li == 4) {                                 // residual layer 5: x_res
          float o3[4];
          tm_ld4(my + kWsAcc, o3);
          if constexpr (F8) {
            const float *b8 = sF8 + kWsF8Bias + 4 * kWidth;
            f0 += fmaf(o3[0], sF8[4], b8[0]);
            f1 += fmaf(o3[1], sF8[4], b8[1]);
            f2 += fmaf(o3[2], sF8[4], b8[2]);
          } else {
            f0 += o3[0] + sBias[bl.r5 + 0];
            f1 += o3[1] + sBias[bl.r5 + 1];
            f2 += o3[2] + sBias[bl.r5 + 2];
          }
        } else if constexpr (F8) {
          ws_relu_layer_f8(my, sF8[li], sF8 + kWsF8Bias + li * kWidth);
        } else {
          ws_relu_layer<T>(my);
        }
      }
      float o[4];
      tm_ld4(my + kWsAcc, o);
      if constexpr (F8) {
        const int lo = n_layers - 1;
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = fmaf(o[k], sF8[lo], sF8[kWsF8Bias + lo * kWidth + k]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] += sBias[bl.cl + k];
      }
      if (valid) {
        const float cr = sigmoidf_(o[0]), cg = sigmoidf_(o[1]);
        const float cb = sigmoidf_(o[2]), sigma = softplusf_(o[3]);
        if (MODE == kModeRender) {
          const float al = inside ? -expm1f(-sigma * delta) * fminf(S, 1.f) : 0.f;
          reinterpret_cast<float4 *>(out)[j] = make_float4(cr, cg, cb, al);
        } else {
          float *qo = out + (size_t)NR_QUERY_STRIDE * j;
          qo[0] = s0; qo[1] = s1; qo[2] = s2; qo[3] = S;
          qo[4] = f0; qo[5] = f1; qo[6] = f2; qo[7] = inside ? 1.f : 0.f;
          qo[8] = cr; qo[9] = cg; qo[10] = cb; qo[11] = sigma;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem0), "r"(kWsTmemCols));
  }
}

static size_t ws_smem(int hidden) {
  const T5Layout L = t5_layout(hidden);
  const TcBias bl = tc_bias_layout(hidden);
  size_t b = 1024 + (size_t)((L.total + 1023) & ~1023) + (size_t)(hidden + 2) * kWsBiasTile;
  b += sizeof(float) * (((bl.total + 3) & ~3) + kPoseSmem);
  b += sizeof(uint64_t) * (3 * kWsGroups) + sizeof(WsLayer) * kWsMaxLayers + 16;
  b += sizeof(float) * (kWsF8Inv + 4);               // the fp8 tier's m', b' and input scales
  return b;
}

template <typename T, int MODE>
static nr_status launch_ws_mode(const FieldParams &P, const uint8_t *blob, const float4 *in, uint32_t n_fixed,
                                const uint32_t *n_dev, float *out, uint32_t *err, int device, cudaStream_t st) {
  const size_t smem = ws_smem(P.hidden);
  NR_CHECK_CUDA(cudaFuncSetAttribute(field_ws_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  field_ws_kernel<T, MODE><<<num_sms(device), kWsThreads, smem, st>>>(P, blob, in, n_fixed, n_dev, out, err);
  NR_CHECK_CUDA(cudaGetLastError());
  return NR_OK;
}

nr_status launch_field_ws(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                          const uint32_t *n_dev, float *out, int device, cudaStream_t st) {
  if (!P.t5_bf16 || !P.t5_f16 || !P.t5_err || (mlp_dtype == NR_FP8E4M3 && (!P.t5_fp8 || !P.fp8_scales))) {
    set_error("tcgen05 weights not prepared");
    return NR_ESTATE;
  }
  if (P.hidden < 1 || P.hidden > kMaxHidden) {
    set_error("tcgen05 pipeline: %d hidden layers (1..%d supported)", P.hidden, kMaxHidden);
    return NR_EUNSUPPORTED;
  }
  if (mlp_dtype == NR_FP8E4M3)
    return mode == kModeRender
               ? launch_ws_mode<E4M3, kModeRender>(P, P.t5_fp8, in, n_fixed, n_dev, out, P.t5_err, device, st)
               : launch_ws_mode<E4M3, kModeQuery>(P, P.t5_fp8, in, n_fixed, n_dev, out, P.t5_err, device, st);
  if (mlp_dtype == NR_BF16)
    return mode == kModeRender
               ? launch_ws_mode<__nv_bfloat16, kModeRender>(P, P.t5_bf16, in, n_fixed, n_dev, out, P.t5_err, device, st)
               : launch_ws_mode<__nv_bfloat16, kModeQuery>(P, P.t5_bf16, in, n_fixed, n_dev, out, P.t5_err, device, st);
  return mode == kModeRender
             ? launch_ws_mode<__half, kModeRender>(P, P.t5_f16, in, n_fixed, n_dev, out, P.t5_err, device, st)
             : launch_ws_mode<__half, kModeQuery>(P, P.t5_f16, in, n_fixed, n_dev, out, P.t5_err, device, st);
}

}  // namespace nr
