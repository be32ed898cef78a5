// common.cuh -- subject state, launch parameters and error plumbing shared by
// the translation units of libnr.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/nr.h"

namespace nr {

constexpr int kBones = 24;
constexpr int kPoseSmem = kBones * 12 + kBones * 6;   // bone transforms then support boxes (floats)
constexpr float kBoneEps = 1e-7f;   // bone-channel values at or below this are skipped when rendering
constexpr int kWidth = 64;          // hidden width of both MLPs
constexpr int kMlpIn = 32;          // canonical MLP input (hash features, zero-padded)
constexpr int kMaxLevels = 16;
constexpr int kResGammaPad = 48;    // 3 + 6 * 6 = 39 PE dims, padded to a multiple of 16
constexpr int kMaxHidden = 4;
// Slots of the fp8 tier's scale array read by the tcgen05 pipeline (written by field_fp8.cu):
// 1 / s_a of gamma and of the hash encoding, residual layer 4's common multiplier, then per layer
// of the pipeline's table the multiplier s_w s_a and the next input's 1 / s_a.
constexpr int kF8SlotInvGam = 28, kF8SlotInvEnc = 29, kF8SlotC4 = 30, kF8SlotWs = 32;
constexpr float kEpsW = 1e-4f;      // floor of the LBS denominator

void set_error(const char *fmt, ...);

#define NR_CHECK_CUDA(call)                                                      \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      ::nr::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                      __FILE__, __LINE__);                                       \
      return e_ == cudaErrorMemoryAllocation ? NR_ENOMEM : NR_ECUDA;             \
    }                                                                            \
  } while (0)

#define NR_REQUIRE(cond, ...)                                                    \
  do {                                                                           \
    if (!(cond)) {                                                               \
      ::nr::set_error(__VA_ARGS__);                                              \
      return NR_EINVAL;                                                          \
    }                                                                            \
  } while (0)

// Offsets (in floats) of each layer inside the float32 kernel weight blob.
// Every matrix is stored transposed, [in][out], so that one thread's
// activation times one row is a run of broadcast float4 reads.
struct BlobLayout {
  // residual MLP
  int r1, r1b, r2, r2b, r3, r3b, r4, r4b, r5, r5b;
  // canonical MLP: first, hidden (H - 1 of them), last
  int c0, c0b, ch[kMaxHidden], chb[kMaxHidden], cl, clb;
  int total;
};

// Offsets (in bf16/f16 elements) of the tensor-core weight blob: every
// matrix is [out][in] row-major with rows padded to kTcRow elements so that
// ldmatrix row reads are free of bank conflicts.
constexpr int kTcRow = 72;          // 64 + 8
constexpr int kTcRowWide = 120;     // 112 + 8 (residual layer 4: [h3 | gamma])
struct TcLayout {
  int r1, r2, r3, r4, r5, c0, ch[kMaxHidden], cl;
  int total;                         // elements
};

// Everything one field evaluation needs; passed to kernels by value.
struct FieldParams {
  float bmin[3], bmax[3];
  float vol_scale[3];                // (R - 1) / (bmax - bmin)
  float inv_box[3];                  // 1 / (bmax - bmin)
  float box_c[3], box_ih[3];         // box centre and 2 / (bmax - bmin)
  int wres;
  const float *wvol;                 // [25][R^3]
  const float4 *wquad;               // [24][(R+2)(R+1)(R+1)] corner blocks (see build_quad_kernel)
  int L;
  uint32_t T_mask;
  uint32_t dense_mask;               // bit l set if level l is dense
  uint32_t level_res[kMaxLevels];
  const float2 *table32;             // [L][T] float2
  const __half2 *table16;            // [L][T] half2
  // dense levels of the f16 table as corner blocks: entry (x, y, z) of level l, at
  // dq_off[l] + (z N + y) N + x for x, y < N and z <= N, holds the half2 values of the
  // vertices (x, y), (x + 1, y), (x, y + 1), (x + 1, y + 1) on plane z (dense_quad_kernel)
  const uint4 *dense_quad;
  uint32_t dq_off[kMaxLevels];
  int use_f16_table;
  int hidden;                        // canonical hidden layers
  int res_enabled, res_freqs;
  float hann[8];
  const float *blob;                 // float32 weight blob (BlobLayout)
  BlobLayout lay;
  const void *tc_blob;               // bf16/f16 weight blob (TcLayout)
  TcLayout tlay;
  const float *G;                    // [24][12] of the current pose
  const float *bias1;                // [64] residual layer-1 bias with the pose folded in
  const uint8_t *fp8_blob;           // e4m3 weight blob (field_fp8.cu)
  const float *fp8_scales;           // its weight and activation scales
  const uint8_t *t5_bf16, *t5_f16;   // swizzled K-major weight blobs of the tcgen05 path (field_t5.cu)
  const uint8_t *t5_fp8;             // the same layout in e4m3 with the fp8 tier's scales (field_fp8.cu)
  uint32_t *t5_err;                  // set by the tcgen05 path when a bounded wait gives up
  const float *bone_box;             // [24][6] per-bone support box in volume-index units, or NULL
  // occupancy from the field's density (kModeDensity / kModePose of the FP32 kernel)
  int occ_grid;                      // cells per axis
  float occ_tau;                     // density threshold
  float occ_smin;                    // least bone-weight sum S of a posed cell
  const uint32_t *canon_bits;        // canonical bitfield read by kModePose
  float *tf32_scratch;               // activation columns of the float32 tensor-core tier (or NULL)
  uint32_t *kept_count;              // profiled renders: bone channels read, summed over samples (or NULL)
};

struct Frame {                       // a training frame's camera (decoded)
  float R[9], t[3];
  float fx, fy, cx, cy, t_near, t_far;
  uint32_t width, height;
};

}  // namespace nr

// ----------------------------------------------------------------- subject
struct nr_subject {
  uint32_t magic = 0x4e525342u;
  int device = 0;
  // configuration
  uint32_t K = 24;
  float bmin[3], bmax[3];
  uint32_t wres = 0;
  uint32_t L = 0, F = 2, log2T = 0, T = 0;
  uint32_t level_res[nr::kMaxLevels] = {0};
  uint32_t mlp_in = 32, width = 64, hidden = 2;
  uint32_t res_enabled = 0, res_freqs = 0;
  uint32_t occ_grid = 128;
  bool has_ellipsoids = false;
  uint32_t occ_source = 0;           // kOccNone, kOccEllipsoids or kOccGrid
  std::vector<int> parents;
  std::vector<double> rest;          // [K][3]
  // float32 master parameters and their gradients
  float *wvol = nullptr, *g_wvol = nullptr;
  float *table = nullptr, *g_table = nullptr;
  float *mlp = nullptr, *g_mlp = nullptr;
  float *res = nullptr, *g_res = nullptr;
  size_t n_wvol = 0, n_table = 0, n_mlp = 0, n_res = 0;
  // Adam moments (allocated at the first training step)
  float *adam_m = nullptr, *adam_v = nullptr;
  size_t n_params_total = 0;
  uint32_t adam_t = 0;
  // derived, rebuilt when parameters change
  __half2 *table16 = nullptr;
  uint4 *dense_quad = nullptr;       // corner blocks of the dense levels of table16 (or NULL)
  float *r_scratch = nullptr;        // activation columns of the float32 tensor-core tier
  size_t rw_scratch = 0;             // its capacity (floats)
  size_t n_dq = 0;                   // its entries
  uint32_t dq_off[nr::kMaxLevels] = {};  // per dense level: first entry
  float *blob = nullptr;
  float4 *wquad = nullptr;           // corner-block copy of the bone channels of wvol
  float *bone_box = nullptr;         // [24][6] support boxes of the bone channels (render skip)
  int *bone_ibox = nullptr;          // [24][6] their voxel bounds
  nr::BlobLayout lay{};
  __nv_bfloat16 *tc_bf16 = nullptr;
  __half *tc_f16 = nullptr;
  nr::TcLayout tlay{};
  bool params_dirty = true;
  uint8_t *fp8_blob = nullptr;       // e4m3 weights, their scales, calibration buffers
  float *fp8_scales = nullptr;
  void *fp8_jobs = nullptr;
  float *fp8_G = nullptr;
  bool fp8_ready = false;
  uint8_t *t5_bf16 = nullptr, *t5_f16 = nullptr, *t5_fp8 = nullptr;
  uint32_t *t5_err = nullptr;
  bool t5_ready = false;
  // current pose
  bool pose_set = false;
  bool pose_matrices = false;        // the pose was given as G (NR_POSE_MATRICES)
  bool pose_dirty = false;           // d_G (and the posed bitfield) must be re-derived
  bool d_G_host = false;             // d_G holds h_G (not a refined pose)
  cudaEvent_t pose_ev = nullptr;     // recorded after the last nr_set_pose's device work
  cudaStream_t pose_stream = nullptr;  // the stream of that work
  bool pose_ev_live = false;
  float h_G[24 * 12];                // host forward kinematics of the estimated pose
  float h_omega[24 * 3];
  float h_root[3] = {0.f, 0.f, 0.f};
  float *d_G = nullptr;              // [24][12]
  float *d_omega = nullptr;          // [72] joint angles, [3] root translation, [72] refined angles
  float *d_bias1 = nullptr;          // [64]
  bool bias_dirty = true;
  float *ellip = nullptr;            // [24][15]
  uint32_t *bits = nullptr;          // occ_grid^3 / 32, posed
  uint32_t *canon_bits = nullptr;    // occ_grid^3 / 32, canonical (kOccGrid)
  uint32_t *occ_raw = nullptr;       // occ_grid^3 / 32, undilated density test
  float occ_smin = 0.f;              // least bone-weight sum of a posed cell (kOccGrid)
  bool occ_dirty = false;            // posed grid stale (kOccGrid)
  // pose refiner MLP_theta (Sec. 4.1); ref_layers == 0: off
  uint32_t ref_width = 0, ref_layers = 0;
  float *ref = nullptr, *g_ref = nullptr, *ref_m = nullptr, *ref_v = nullptr;
  size_t n_ref = 0;
  uint32_t ref_t = 0;                // Adam steps of the refiner
  // CNN_skel weight-volume generator (Sec. 4.2); cnn_on: wvol = CNN(z)
  bool cnn_on = false, cnn_dirty = false;
  uint32_t cnn_ch[5] = {0, 0, 0, 0, 0};
  float *cnn = nullptr, *g_cnn = nullptr, *cnn_m = nullptr, *cnn_v = nullptr;
  float *cnn_z = nullptr, *cnn_prior = nullptr, *cnn_act = nullptr, *cnn_grad = nullptr;
  size_t n_cnn = 0;
  uint32_t cnn_t = 0;                // Adam steps of the generator
  // training frames
  uint32_t n_frames = 0, frames_cap = 0;
  std::vector<float> h_fG;           // host forward kinematics of the estimated frame poses
  bool fG_refined = false;           // f_G holds refined poses
  float *f_root = nullptr;           // [F][3]
  float *f_omega_o = nullptr;        // [F][72] refined joint angles (refiner)
  float *f_dG = nullptr;             // [F][24][12] dL/dG (refiner)
  size_t f_dG_cap = 0;
  float *f_G = nullptr;              // [F][24][12]
  float *f_omega = nullptr;          // [F][72]
  float *f_bias1 = nullptr;          // [F][64]
  nr::Frame *f_cam = nullptr;        // [F]
  // render workspace (grow-only)
  size_t ws_samples = 0, ws_rays = 0;
  float4 *samp = nullptr;            // [max samples] x, y, z, delta
  float4 *samp_out = nullptr;        // [max samples] r, g, b, alpha
  uint2 *ray_range = nullptr;        // [max rays] offset, count
  uint32_t *counter = nullptr;       // [4] device counters
  float *out_stage = nullptr;        // [max rays][4] staging for host outputs
  size_t stage_cap = 0;
  float4 *ray_state = nullptr;       // [max rays] running (C, T) of round-based early termination
  uint32_t *ray_next = nullptr;      // [max rays] next slot of each ray, top bit = retired
  // stage profiling (NR_RENDER_PROFILE): an event per launch boundary, tagged by the stage it ends
  static constexpr int kProfEvents = 512;
  cudaEvent_t prof_ev[kProfEvents] = {};
  int prof_stage[kProfEvents] = {};
  int prof_used = 0;                 // events recorded by the last profiled render
  bool prof_overflow = false;
  // training workspace (grow-only)
  size_t tw_samples = 0;             // capacity of t_samp / t_out / t_T
  size_t tw_rays = 0;                // capacity of t_raycnt
  size_t tw_live = 0;                // capacity of t_live
  size_t tw_acc = 0;                 // capacity of t_wacc (floats)
  size_t tw_red = 0, tw_scratch = 0;  // capacities of t_red, t_scratch (floats)
  float4 *t_samp = nullptr;          // [n_rays * S] x, y, z, delta
  float4 *t_out = nullptr;           // [n_rays * S] (r, g, b, alpha), then (dL/dc, dL/dalpha)
  float *t_T = nullptr;              // [n_rays * S] transmittance before each sample
  uint32_t *t_raycnt = nullptr;      // [n_rays] S if the ray meets the box, else 0
  uint32_t *t_live = nullptr;        // [n_rays * S / 32] per 32 thread slots: which carry gradient
  float *t_scratch = nullptr;        // per-thread activation columns of the backward kernel
  float *t_wacc = nullptr;           // per-warp private MLP-gradient accumulators
  float *t_red = nullptr;            // their sum (float32 blob layout + per-frame bias rows)
  float *loss_acc = nullptr;         // [1]
  float *f_dbias1 = nullptr;         // [F][64] (unused, kept for layout)
};

namespace nr {
// Offsets (floats) of each layer's W[out][in] and b[out] in the packed master parameters.
struct MasterOffsets {
  int r[5], rb[5];                   // residual MLP layers 1..5
  int c[kMaxHidden + 2], cb[kMaxHidden + 2];   // canonical MLP layers 0..H
  int n_res, n_mlp;
};
MasterOffsets master_offsets(const nr_subject *s);
int res_gamma_dims(const nr_subject *s);
void count_launches(uint64_t n);                              // kernels launched by the library
void forward_kinematics(const nr_subject *s, const float *aa, const float *root_t, float *G);   // host, fp64 -> fp32
constexpr uint32_t kOccNone = 0, kOccEllipsoids = 1, kOccGrid = 2;   // nr_subject::occ_source
nr_status launch_posed_bitfield(const nr_subject *s, const float *G_dev, const float *bias_dev, uint32_t *bits,
                                cudaStream_t st);
nr_status ensure_occupancy(nr_subject *s, cudaStream_t st);    // posed grid of the current pose (kOccGrid)
nr_status ensure_pose(nr_subject *s, cudaStream_t st);         // d_G (refined if MLP_theta is on), bitfields
nr_status after_pose(nr_subject *s, cudaStream_t st);          // orders st after the last nr_set_pose
nr_status launch_refine_fk(const nr_subject *s, const float *omega, int omega_stride, const float *root,
                           int root_stride, int n, float *G, float *omega_o, int omega_o_stride, cudaStream_t st);
nr_status launch_refine_bwd(const nr_subject *s, const float *omega, int omega_stride, const float *root,
                            int root_stride, int n, const float *dG, const float *dbias, float *g, cudaStream_t st);
const float *pose_omega(const nr_subject *s);   // angles conditioning MLP_res for the current pose (device)
size_t refiner_param_count(uint32_t width, uint32_t layers);
nr_status cnn_forward(nr_subject *s, cudaStream_t st);         // wvol = CNN_skel(z)
nr_status cnn_backward(nr_subject *s, cudaStream_t st);        // g_cnn from g_wvol
nr_status launch_occupancy_field(const FieldParams &P, int mode, uint32_t *bits, int device, cudaStream_t st);
nr_status launch_fold_bias(const nr_subject *s, const float *omega_dev, float *bias_dev, int n_poses, cudaStream_t st);
bool subject_ok(const nr_subject *s);
nr_status prepare_params(nr_subject *s, cudaStream_t st);      // derived blobs
nr_status ensure_bias(nr_subject *s, cudaStream_t st);         // pose-folded bias
nr_status prepare_fp8(nr_subject *s, cudaStream_t st);         // e4m3 weights + calibrated scales
nr_status prepare_t5(nr_subject *s, cudaStream_t st);          // swizzled weights of the tcgen05 path
FieldParams field_params(const nr_subject *s, const nr_render_opts *o);
nr_status set_error_cuda(cudaError_t e, const char *what);
}  // namespace nr
