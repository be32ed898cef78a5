/*
 * nr.h -- C ABI of the GB300 dynamic-human NeRF renderer (libnr.so).
 *
 * The library renders one performer, held as a canonical radiance field plus
 * a skeleton-driven motion field, from a pose and a camera, and trains that
 * field against images.  The operations follow the paper's statement of the
 * problem:
 *   - a subject is a canonical field and its motion field (Sec. 4, Fig. 2:
 *     M = M_skel + M_res; Sec. 4.2 weight volume W^c; Sec. 4.3 residual
 *     MLP; Sec. 4.4 MLP_nerf);
 *   - it is driven by a body pose theta = (J, Omega) (Sec. 4.1);
 *   - it is rendered from a pinhole camera K with extrinsics (Fig. 2,
 *     Sec. 5.1) by volume rendering (Sec. 2.1, Eq. 2-3) with empty-space
 *     skipping and early ray termination (Sec. 2.3);
 *   - it is trained on a squared photometric error with Adam (Sec. 5.2).
 *
 * Conventions for every call:
 *   - every call returns an nr_status; nothing aborts the process;
 *     nr_last_error() gives a thread-local message for the last failure;
 *   - host pointers passed in are read during the call only (the library
 *     copies what it keeps); device pointers passed in are read in stream
 *     order on `stream` (a cudaStream_t, NULL = the legacy default stream);
 *   - output buffers are owned by the caller;
 *   - the subject owns all of its device state until nr_destroy();
 *   - a subject may be used by one host thread at a time;
 *   - all arrays are dense, C order, little-endian; floats are IEEE binary32.
 */
#ifndef NR_H
#define NR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NR_ABI_VERSION 1u

typedef enum {
  NR_OK = 0,
  NR_EINVAL = 1,        /* an argument is NULL, out of range or inconsistent */
  NR_ENOMEM = 2,        /* a device or host allocation failed */
  NR_ECUDA = 3,         /* a CUDA runtime call failed (message in nr_last_error) */
  NR_ESTATE = 4,        /* wrong order of calls (e.g. render before nr_set_pose) */
  NR_ETIMEOUT = 5,      /* a bounded wait gave up */
  NR_EBUSY = 6,         /* the resource is in use */
  NR_EUNSUPPORTED = 7   /* a valid request this build does not implement */
} nr_status;

typedef enum { NR_F32 = 0, NR_F16 = 1, NR_BF16 = 2, NR_FP8E4M3 = 3 } nr_dtype;

typedef struct nr_subject nr_subject;   /* opaque, library-owned */

/* Everything that defines one performer.  All pointers are host pointers,
 * read during nr_create_subject only.
 *
 * Skeleton (Sec. 4.1, SMPL topology): n_bones joints, parents[i] < i or -1
 * for the root, rest_joints[n_bones][3] in metres; the canonical pose is the
 * rest pose.
 * Box: the performer's axis-aligned bounding box (Sec. 4.4).
 * Weight volume W^c (Sec. 4.2, Fig. S2): wvol[n_bones + 1][r][r][r] float32,
 *   indexed [channel][z][y][x], r = wvol_res; vertex (i, j, k) sits at
 *   box_min + (i, j, k) * (box_max - box_min) / (r - 1); the last channel is
 *   the background and is not a bone.
 * Hash grid (canonical encoding): hash_levels levels of 2^log2_T entries with
 *   hash_feats features each; level_res[l] is the grid resolution N_l (1..65536);
 *   hash_table[L][T][F] float32 initial values.
 * Canonical MLP (MLP_nerf, Sec. 4.4): mlp_in -> mlp_width (ReLU) x
 *   mlp_hidden_layers -> 4; mlp_params packs, per layer, W[out][in] row-major
 *   then b[out], float32.  Output: rgb = sigmoid(o[0:3]), sigma = softplus(o[3]).
 * Residual MLP (MLP_res, Sec. 4.3, Fig. S3): if res_enabled, 5 layers of
 *   width 64 on gamma(x_skel) (3 + 6 * res_pe_freqs dims) and the joint angles
 *   Omega (3 * n_bones), skip of gamma into layer 4, output x_res[3]; packed as
 *   the canonical MLP: W1[64][g + 3K], b1, W2[64][64], b2, W3[64][64], b3,
 *   W4[64][64 + g], b4, W5[3][64], b5.
 * Occupancy: ellipsoids[n_bones][15] (centre[3], rotation rows[9] mapping
 *   canonical to the ellipsoid's local frame, radii[3]) in canonical space, or
 *   NULL; occ_grid cells per axis of the occupancy grids (32, 64, 128 or 256;
 *   0 = 128), used by the ellipsoids or by a canonical density grid
 *   (nr_refresh_occupancy).
 */
typedef struct {
  uint32_t abi_version;          /* NR_ABI_VERSION */
  uint32_t n_bones;              /* 24 */
  const int32_t *parents;
  const float *rest_joints;
  float box_min[3], box_max[3];
  uint32_t wvol_res;
  const float *wvol;
  uint32_t hash_levels, hash_feats, log2_T;
  const uint32_t *level_res;
  const float *hash_table;
  uint32_t mlp_in, mlp_width, mlp_hidden_layers;
  const float *mlp_params;
  uint32_t res_enabled, res_pe_freqs;
  const float *res_params;
  const float *ellipsoids;
  uint32_t occ_grid;
  int32_t device;                /* CUDA device ordinal */
} nr_subject_desc;

/* Limits of this build: n_bones == 24, hash_feats == 2, hash_levels <= 16,
 * 10 <= log2_T <= 24, mlp_in == 32 with hash_levels * 2 <= 32,
 * mlp_width == 64, 1 <= mlp_hidden_layers <= 4, res_pe_freqs <= 6,
 * 2 <= wvol_res <= 256, occ_grid in {32, 64, 128, 256}.
 * Errors: NR_EINVAL for a NULL or out-of-range field, NR_ENOMEM when device
 * memory runs out (nothing is leaked), NR_ECUDA for other CUDA failures. */
nr_status nr_create_subject(const nr_subject_desc *desc, void *stream, nr_subject **out);

/* Releases every device buffer of the subject.  NULL is a no-op.  The
 * handle must not be used afterwards. */
nr_status nr_destroy(nr_subject *s);

#define NR_POSE_MATRICES 1u   /* axis_angle holds G[n_bones][12] (rows [R | t]) instead */

/* Sets the observed pose theta^o used by nr_render and nr_query.
 * axis_angle[n_bones][3]: per-joint rotation (axis times angle, radians) in
 * the parent's frame; root_t[3]: root translation (may be NULL = 0).
 * The library computes, by forward kinematics in float64 on the host, the
 * per-bone observation-to-canonical transforms G_i(x) = R_i x + t_i
 * (Sec. 4.2), rounds them to float32, folds the joint angles into the
 * residual MLP's first-layer bias, and, if the subject has ellipsoids,
 * rebuilds the posed occupancy bitfield on the device: a cell is set iff for
 * some bone i the canonical image G_i(c) of its centre lies in ellipsoid i
 * dilated by half a cell diagonal.  With NR_POSE_MATRICES, axis_angle is
 * G[n_bones][12] float32 and used as given; the joint angles are then taken
 * as zero for the residual MLP.  With a pose refiner installed
 * (nr_set_pose_refiner) and joint angles given, G is that of the refined pose,
 * computed on the device, and is re-derived after every training step that
 * updates the refiner.  Host pointers, read during the call.  The call does
 * not wait for the device: the transforms travel as a kernel argument and the
 * device work is queued on `stream`.  A later call that uses the pose on
 * another stream waits for that work (an event), except inside a stream
 * capture, which the caller must order after the pose.  The reverse order is
 * the caller's: a render still running on another stream reads the pose
 * buffers this call rewrites, so order the call after it. */
nr_status nr_set_pose(nr_subject *s, const float *axis_angle, const float *root_t,
                      uint32_t flags, void *stream);

/* Pose refiner (Sec. 4.1): Delta_Omega = MLP_theta(Omega) corrects the
 * estimated joint angles before forward kinematics.  MLP_theta sees the
 * 3 (n_bones - 1) = 69 angles of the non-root joints and returns one
 * axis-angle correction per non-root joint; hidden_layers (1..4) ReLU layers
 * of `width` (1..256) units, then a linear layer to 69.  params (host) packs,
 * per layer, W[out][in] row-major then b[out] (69 -> width, width -> width,
 * ..., width -> 69).  The refined local rotation of joint j >= 1 is
 * Rot(Delta_omega_j) Rot(omega_j); the root keeps its estimate; the residual
 * MLP is conditioned on the updated angles Omega^o, omega^o_j = Log of the
 * refined local rotation (angles below pi).  Training (nr_train_step) then
 * back-propagates dL/dG_i of every frame, reduced over the batch's samples,
 * through the kinematic chain, and dL/dOmega^o through the rotation log,
 * into MLP_theta (Adam group NR_TRAIN_REFINER, parameters NR_PARAM_REFINER).  params == NULL switches
 * the refiner off.  The Adam moments restart at each call. */
nr_status nr_set_pose_refiner(nr_subject *s, uint32_t width, uint32_t hidden_layers, const float *params,
                              void *stream);

/* Weight-volume generator CNN_skel (Sec. 4.2): W^c = CNN_skel(z) replaces the
 * stored weight volume.  A fully-connected layer maps the constant latent
 * z[256] to channels[0] values (a channels[0] x 1^3 tensor); five transposed
 * convolutions (kernel 4, stride 2, padding 1) take it to 32^3 with channels
 * channels[1..4] and then 25; LeakyReLU(0.2) follows the fully-connected layer
 * and every transposed convolution but the last; the 25 channels pass through
 * a softmax over channels after adding log_prior [25][32][32][32] (may be
 * NULL).  params (host) packs W_fc [channels[0]][256], b_fc, then per
 * convolution W [C_in][C_out][4][4][4], b [C_out].  Requires wvol_res == 32.
 * The volume is regenerated whenever the generator's parameters change;
 * training (nr_train_step) back-propagates dL/dW^c through it (Adam group
 * NR_TRAIN_CNN, parameters NR_PARAM_CNN) and no longer updates the volume
 * directly.  params == NULL switches the generator off (the volume keeps its
 * last generated values).  Host pointers, copied; the Adam moments restart. */
nr_status nr_set_weight_cnn(nr_subject *s, const uint32_t *channels, const float *params, const float *z,
                            const float *log_prior, void *stream);

/* Pinhole camera, OpenCV convention (x right, y down, z forward).
 * Pixel (u, v) looks along R^T ((u + 0.5 - cx) / fx, (v + 0.5 - cy) / fy, 1)
 * from o = -R^T t.  Each ray is clipped to [t_near, t_far] and to the
 * subject's box; n_samples equal bins split the clipped segment and a
 * rendered sample sits at each bin's midpoint. */
typedef struct {
  uint32_t width, height;
  float fx, fy, cx, cy;
  float R[9];          /* world -> camera rotation, row-major */
  float t[3];          /* world -> camera translation */
  float t_near, t_far;
  uint32_t n_samples;  /* 1 .. 1024 */
  float bg[3];         /* background colour composited behind the performer */
} nr_camera;

typedef struct {
  nr_dtype mlp_dtype;      /* NR_F32 (CUDA cores), NR_BF16, NR_F16, NR_FP8E4M3 (tensor cores;
                              e4m3 uses per-matrix weight scales and static per-subject
                              activation scales calibrated once on a seeded probe) */
  nr_dtype feat_dtype;     /* hash-table storage read by the encoder: NR_F32 or NR_F16 */
  uint32_t use_occupancy;  /* skip samples whose posed occupancy cell is empty */
  float t_min;             /* early ray termination once transmittance < t_min; 0 = off */
  float hann_alpha;        /* residual PE window position; < 0 = all bands */
  uint32_t flags;          /* NR_RENDER_PROFILE | NR_RENDER_TCGEN05 | NR_RENDER_MMA2 |
                              NR_RENDER_ALL_BONES | NR_RENDER_F32_TC, or 0 */
} nr_render_opts;

/* Renders the current pose from `cam` into out_rgba[height][width][4]
 * (rgb = sum_i T_i alpha_i c_i + T_final bg, a = 1 - T_final), where
 * alpha_i = (1 - exp(-sigma_i delta_i)) * min(S_i, 1) and S_i is the sum of
 * the bone weights at the sample (the likelihood augmentation of Sec. 4.4).
 * out_rgba may be a device or a host pointer; a host buffer is filled before
 * the call returns, a device buffer in stream order.  Errors: NR_ESTATE
 * before nr_set_pose; NR_EINVAL for bad sizes or options; NR_ENOMEM if the
 * work queues cannot grow. */
nr_status nr_render(nr_subject *s, const nr_camera *cam, const nr_render_opts *opts,
                    float *out_rgba, void *stream);

/* nr_render without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot let the library call
 * cudaMalloc at render time -- a real-time serving thread that must not
 * stall on the implicit device synchronisation of an allocation, or a
 * process that has already handed all free device memory to its own pool,
 * where a late allocation would fail.
 * It renders the same image as nr_render (same kernels, same compositing
 * order), but its work queues live in one fixed, file-scope device array of
 * 8.5 MiB per device (every GPU that loads the library holds it until the
 * process exits) instead of buffers the subject allocates.
 * Limits: width * height <= 65,536 rays and width * height * n_samples
 * <= 262,144 sample slots; larger frames return NR_EINVAL with a message
 * saying which limit was exceeded.  out_rgba must be device memory
 * (NR_EINVAL otherwise); the subject and its pose must already exist.
 * Flags: NR_RENDER_MMA_SYNC, NR_RENDER_MMA2, NR_RENDER_TCGEN05 and
 * NR_RENDER_ALL_BONES are honoured; NR_RENDER_F32_TC and NR_RENDER_PROFILE
 * need buffers or events created on first use and return NR_EUNSUPPORTED;
 * NR_FP8E4M3 returns NR_EINVAL.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and must come before any stream capture; the
 * address is kept for the process, so the device must not be reset
 * (cudaDeviceReset) afterwards.
 * All calls on a device share the one array and leave the last call's data
 * in it: calls whose GPU work overlaps (other streams or host threads) race
 * and corrupt each other's results, so serialise them. */
nr_status nr_render_static(nr_subject *s, const nr_camera *cam, const nr_render_opts *opts,
                           float *out_rgba, void *stream);

#define NR_QUERY_STRIDE 12
/* Evaluates the field at n observation-space points x_obs[n][3] (device) for
 * the current pose and writes out[n][12] (device):
 *   x_skel[3], S, x_final[3], inside (1 or 0), rgb[3], sigma.
 * Same dtype options as nr_render (use_occupancy and t_min are ignored). */
nr_status nr_query(nr_subject *s, uint32_t n, const float *x_obs, const nr_render_opts *opts,
                   float *out, void *stream);

/* Stores the training frames: per frame a pose (axis_angle[F][n_bones][3],
 * root_t[F][3]) and a camera cams[F]; host pointers.  Replaces earlier frames. */
nr_status nr_set_frames(nr_subject *s, uint32_t n_frames, const float *axis_angle,
                        const float *root_t, const nr_camera *cams, void *stream);

#define NR_GRAD_ONLY 1u        /* compute gradients into the grad buffers, skip Adam */
#define NR_FORWARD_ONLY 2u     /* composite the batch (into pred_rgb) and stop: no gradient, no Adam */

#define NR_TRAIN_WVOL 1u
#define NR_TRAIN_HASH 2u
#define NR_TRAIN_MLP 4u
#define NR_TRAIN_RES 8u
#define NR_TRAIN_REFINER 16u
#define NR_TRAIN_CNN 32u
#define NR_TRAIN_ALL 63u

/* One training batch of pixel rays.  frame_id, px, py: device uint32[n];
 * target_rgb: device float32[n][3].  Samples are stratified: bin i of the
 * clipped ray gets t_i = lo + (i + u_i) * (hi - lo) / S with u_i from the
 * SplitMix64 generator seeded with step_seed (output k = ray * S + i + 1,
 * u = top 24 bits * 2^-24); delta_i = t_{i+1} - t_i, delta_{S-1} = hi - t_{S-1}. */
typedef struct {
  uint32_t n_rays;
  const uint32_t *frame_id, *px, *py;
  const float *target_rgb;
  uint32_t n_samples;
  float bg[3];
  uint64_t step_seed;
  float lr, beta1, beta2, eps;   /* Adam (Sec. 5.2: beta = (0.9, 0.99)) */
  float hann_alpha;              /* residual PE window; < 0 = all bands */
  uint32_t flags;                /* NR_GRAD_ONLY, NR_FORWARD_ONLY */
  uint32_t train_mask;           /* NR_TRAIN_* groups that are updated; 0 = all */
  float lr_scale[4];             /* per-group multiplier of lr: weight volume, hash table,
                                    canonical MLP, residual MLP; 0 means 1.  Sec. 5.2 trains
                                    the NeRF network with a 10x larger rate than the others. */
  float loss_weight;             /* lambda_mse: L = lambda_mse * MSE (Sec. 5.2 uses 0.2 beside
                                    LPIPS); 0 means 1 */
  float lr_scale_refiner;        /* lr multiplier of the pose refiner; 0 means 1 */
  float lr_scale_cnn;            /* lr multiplier of the weight-volume generator; 0 means 1 */
  float *pred_rgb;               /* optional device float32[n][3]: receives each ray's colour
                                    C^ + T_final bg */
  const float *grad_rgb;         /* optional device float32[n][3]: dL/dC^ of each ray from the
                                    caller's own loss; replaces the MSE and its gradient
                                    (target_rgb is then not read and *loss_out is 0) */
} nr_train_batch;

/* Forward, loss L = loss_weight * mean over rays and channels of (C^ - C_gt)^2, the
 * hand-written backward into the gradient buffers (overwritten, not
 * accumulated), then one Adam step (bias-corrected, every entry updated)
 * on the selected groups.  loss_out (host, may be NULL) receives L after
 * the step completes.  Errors: NR_ESTATE before nr_set_frames. */
nr_status nr_train_step(nr_subject *s, const nr_train_batch *batch, float *loss_out, void *stream);

#define NR_PARAM_WVOL 0u    /* [n_bones + 1][r][r][r] */
#define NR_PARAM_HASH 1u    /* [L][T][F] (float32 master copy) */
#define NR_PARAM_MLP 2u     /* canonical MLP, packed as in the descriptor */
#define NR_PARAM_RES 3u     /* residual MLP, packed as in the descriptor */
#define NR_PARAM_REFINER 4u /* pose refiner MLP_theta, packed as in nr_set_pose_refiner */
#define NR_PARAM_CNN 5u     /* weight-volume generator CNN_skel, packed as in nr_set_weight_cnn */
/* Device pointers of a parameter group (float32) and of its gradient buffer,
 * and its element count.  Writing the parameters through *dev_ptr is allowed
 * between calls; call nr_params_changed() afterwards. */
nr_status nr_param(nr_subject *s, uint32_t which, float **dev_ptr, float **grad_ptr, size_t *count);
nr_status nr_params_changed(nr_subject *s);

/* ---------------------------------------------------------------- serving
 * A persistent render server for the multi-user conferencing scenario the
 * paper envisions (Sec. 3, Sec. 6: many people rendered for many viewers).
 * Registered subjects stay resident on the device.  Requests (subject,
 * camera, pose, options, output) are admitted in arrival order into slots,
 * each with its own stream, pose buffers, posed occupancy bitfield and work
 * queues; a slot is created only while the device-memory budget (max_bytes)
 * and the slot limit allow, and is reused afterwards.  A request is enqueued
 * on its slot's stream as soon as it is admitted, so requests arriving while
 * others are on the GPU start at once and their kernels overlap (continuous
 * batching).  Each result is the same as rendering the request alone with
 * nr_set_pose + nr_render.  Latency is measured from nr_server_submit to the
 * completion of the request's last GPU operation.  Every wait is bounded. */
typedef struct nr_server nr_server;   /* opaque */

typedef struct {
  uint32_t subject;          /* index from nr_server_add_subject */
  nr_camera cam;
  float axis_angle[72];      /* pose: [24][3] joint rotations (axis * angle) */
  float root_t[3];
  nr_render_opts opts;       /* NR_RENDER_PROFILE is ignored */
  float *out_rgba;           /* caller-owned [H][W][4]: device memory or pinned host memory,
                                valid until the request completes */
} nr_request;

typedef struct {
  uint64_t submitted, completed, failed, rejected;
  uint32_t active;           /* requests on the GPU now */
  uint32_t queued;           /* requests waiting for a slot */
  uint32_t slots, peak_active;
  uint64_t bytes_in_use;     /* device memory held by slots */
  double rays_done;
} nr_server_stats;

/* Creates a server on `device` with a device-memory budget for its slots and a
 * slot limit (1..256); starts its worker thread.  A slot renders a request in
 * chunks of rays: the server takes the largest chunk from 2^17 rays (a slot of
 * ~138 MB) to 2^20 rays (~1.10 GB, a 1024 x 1024 frame in one pass) for which
 * max_slots slots fit max_bytes; fewer, larger passes cost less per frame.
 * Queued requests are dispatched earliest deadline first (nr_server_set_policy
 * changes the order).  Few slots serve the latency tail best (2 measured best
 * at 240 req/s of the conferencing mix): every field launch occupies all SMs,
 * so requests running side by side stretch one another.  NR_EINVAL if
 * max_bytes cannot hold one slot of the smallest chunk. */
nr_status nr_server_create(int device, uint64_t max_bytes, uint32_t max_slots, nr_server **out);
/* Dispatch policy of a server: the order in which queued requests are admitted
 * into free slots, and whether small requests run on high-priority streams. */
#define NR_SERVE_SMALLEST_FIRST 0u  /* fewest pixel x sample slots first; a request queued
                                       age_ms or longer goes first (arrival order) */
#define NR_SERVE_FIFO 1u            /* arrival order */
#define NR_SERVE_EDF 2u             /* earliest deadline first, deadline = arrival + deadline_ms
                                       + deadline_ms_per_mpixel x width x height / 1e6 */
typedef struct {
  uint32_t order;                 /* NR_SERVE_* (default NR_SERVE_EDF) */
  float age_ms;                   /* smallest first: the aging bound (default 40) */
  float deadline_ms;              /* EDF: the deadline's constant part (default 20) */
  float deadline_ms_per_mpixel;   /* EDF: its part per megapixel (default 5) */
  uint32_t priority_streams;      /* 1: requests of at most 512 x 512 pixels on high-priority
                                     streams, the rest on low-priority ones; 0: all alike (default) */
} nr_server_policy;
/* Sets the dispatch policy (applies to requests dispatched afterwards).  NR_EINVAL for an
 * unknown order or a negative time. */
nr_status nr_server_set_policy(nr_server *srv, const nr_server_policy *policy);

/* Registers a subject (not owned; it must outlive the server and must not be
 * trained or given new parameters while the server runs).  All subjects must
 * share one occupancy grid size. */
nr_status nr_server_add_subject(nr_server *srv, nr_subject *s, uint32_t *index);
/* Queues a request (copied); *id identifies it.  NR_EINVAL for bad fields or a
 * pageable host output; NR_ESTATE once the server is stopping. */
nr_status nr_server_submit(nr_server *srv, const nr_request *req, uint64_t *id);
/* state: 0 queued, 1 running, 2 done, -1 failed; a finished request is
 * forgotten after it has been reported once. */
nr_status nr_server_poll(nr_server *srv, uint64_t id, int32_t *state, double *latency_ms);
/* Waits at most timeout_ms for request `id`: NR_OK when done (latency in
 * *latency_ms, may be NULL), NR_ETIMEOUT if still pending, NR_ECUDA if the
 * request failed. */
nr_status nr_server_wait(nr_server *srv, uint64_t id, uint32_t timeout_ms, double *latency_ms);
nr_status nr_server_get_stats(nr_server *srv, nr_server_stats *out);
/* Refuses new requests and waits at most timeout_ms for the queued and running
 * ones to finish: NR_OK when drained (the worker has exited), NR_ETIMEOUT
 * otherwise (call again to keep waiting). */
nr_status nr_server_stop(nr_server *srv, uint32_t timeout_ms);
/* Stops (draining, waiting up to 10 minutes), then frees every slot.  NULL is a no-op. */
nr_status nr_server_destroy(nr_server *srv);

/* Copies the current pose's float32 transforms G[n_bones][12] (host). */
nr_status nr_pose_transforms(nr_subject *s, float *G_out);
/* Copies the current posed occupancy bitfield (occ_grid^3 / 32 uint32, host);
 * cell (x, y, z) is bit (z * g + y) * g + x.  NR_ESTATE without a pose or an
 * occupancy source. */
nr_status nr_occupancy(nr_subject *s, uint32_t *bits_out);

/* Occupancy from the field's own density: empty-space skipping (Sec. 2.3) for
 * subjects with no ellipsoids, or after training has moved the performer's
 * surface.  Both calls make a canonical grid the subject's occupancy source
 * (ellipsoids, if any, are no longer used); the grid has occ_grid^3 cells over
 * the box, in the layout of nr_occupancy.
 *
 * nr_refresh_occupancy evaluates, in float32 on CUDA cores with the float32
 * hash table, the canonical density sigma = softplus(o_3) of MLP_nerf at the
 * centre bmin + (j + 0.5) h of every canonical cell (h = (bmax - bmin) /
 * occ_grid), marks the cells with sigma > sigma_threshold and dilates the set
 * by `dilate` cells (0..3, Chebyshev distance, clipped at the grid's faces).
 * Call it again whenever the parameters have moved far enough (a periodic
 * refresh during training).  nr_set_canonical_occupancy installs a given
 * canonical bitfield (host, occ_grid^3 / 32 words) instead.
 *
 * Posing: observed cell c is set iff at its centre y the bone-weight sum
 * S(y) >= s_min and the canonical cell clamp(floor((x_final - bmin) / h), 0,
 * occ_grid - 1) is set, x_final(y) being the canonical point of Eq. lbs and
 * MLP_res with every PE band on (float32).  The posed grid is rebuilt lazily by the
 * next render, query of nr_occupancy or served request after nr_set_pose, a
 * training step, nr_params_changed or either call here.
 * Errors: NR_EINVAL for a bad threshold, dilate or s_min; NR_ENOMEM. */
nr_status nr_refresh_occupancy(nr_subject *s, float sigma_threshold, uint32_t dilate, float s_min, void *stream);
nr_status nr_set_canonical_occupancy(nr_subject *s, const uint32_t *bits, float s_min, void *stream);
/* Copies the canonical bitfield of a canonical-grid source (host); NR_ESTATE otherwise. */
nr_status nr_canonical_occupancy(nr_subject *s, uint32_t *bits_out);

#define NR_RENDER_PROFILE 1u  /* nr_render_opts.flags: time each stage with CUDA events */
#define NR_RENDER_TCGEN05 2u  /* nr_render_opts.flags: bf16/f16 MLPs on tcgen05.mma with one group of
                                 four warps per 128-sample tile issuing its own MMAs and the
                                 activations passed through shared memory (an earlier design, kept for
                                 comparison) instead of the default pipeline below */
#define NR_RENDER_MMA2 4u     /* nr_render_opts.flags: warp-level mma.sync over two 16-row tiles per
                                 weight-fragment read (12 warps/SM) instead of the default pipeline */
#define NR_RENDER_ALL_BONES 8u /* nr_render_opts.flags: evaluate all 24 bone channels at every sample.
                                 By default a candidate G_i x is skipped when its trilinear cell lies
                                 outside the index box of channel i's vertices above 1e-7 (weights
                                 that small change S by at most 2.4e-6); training never skips. */
#define NR_RENDER_MMA_SYNC 32u /* nr_render_opts.flags: bf16/f16 MLPs as warp-level mma.sync m16n8k16 over
                                 one 16-row tile per weight-fragment read (20 warps/SM, activations in
                                 registers), fp8 MLPs as mma.sync m16n8k32 with the activations
                                 requantised through shared memory, instead of the default pipeline.
                                 The default for NR_BF16 / NR_F16 / NR_FP8E4M3 is the warp-specialised
                                 tcgen05 pipeline: per SM four 128-sample tiles in flight, both MLPs as
                                 M = 128 MMAs (kind::f16, or kind::f8f6f4 with the same per-matrix and
                                 per-input scales) with the activations in tensor memory, one issuing
                                 warp per tile.  Its waits are bounded; a wait that gives up makes the
                                 call return NR_ETIMEOUT (the same holds for NR_RENDER_TCGEN05). */
#define NR_RENDER_F32_TC 16u  /* nr_render_opts.flags with mlp_dtype NR_F32 (nr_render, nr_query):
                                 both MLPs as warp-level tensor-core layers at float32 accuracy
                                 (each product as three TF32 products of hi/lo parts) instead of
                                 CUDA-core FMAs.  The first such call allocates a scratch buffer of
                                 one 212-float column per thread of one 512-thread block per SM
                                 (66 MB on 152 SMs); nr_render_static refuses the flag
                                 (NR_EUNSUPPORTED).  Ignored for the other dtypes and by the
                                 server, whose slots render concurrently. */

/* Stage times in milliseconds of the subject's last nr_render call made with
 * NR_RENDER_PROFILE: ms_out[0] ray marching, [1] the per-sample field,
 * [2] compositing (each summed over ray chunks), [3] the number of field
 * launches (ray chunks), [4] the number of live samples the field evaluated,
 * [5] the mean number of weight-volume bone channels the field read per live
 * sample (channels whose support holds the candidate; the default bf16/f16
 * pipeline counts them, other paths report 0).
 * ms_out holds 6 floats.  A CUDA event on the render's stream marks every
 * boundary between its launches (a stage's time runs from the mark before its
 * launch to the mark after it); this call waits for them.  NR_ESTATE if no profiled render has run. */
nr_status nr_stage_times(nr_subject *s, float *ms_out);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all subjects, all threads). */
uint64_t nr_launch_count(void);

/* Device address of the subject's field error word (one uint32, allocated with
 * the subject): the tcgen05 kernels (the bf16/f16 default, NR_RENDER_TCGEN05) set
 * it when one of their bounded waits gives up; the render or query that launched
 * them reads it back, returns NR_ETIMEOUT when it is non-zero and clears it.
 * Instrumentation for tests and monitoring; writing it makes the next such call
 * report a timeout. */
nr_status nr_field_error_word(nr_subject *s, uint32_t **dev_word);

/* Measured ceiling of the field kernel's gathers (instrumentation; the paper has
 * no counterpart): the rate, in bytes requested by the threads per second, at
 * which `device` serves independent random loads of load_bytes (4 or 16,
 * aligned) from a table of table_bytes (a power of two, 1 MiB .. 1 GiB) that
 * stays resident in L2 -- the access pattern of the hash-table corners (4 B)
 * and of the corner blocks (16 B).  Best of three timed launches (CUDA events)
 * after a warm-up launch; allocates and frees the table. */
nr_status nr_l2_gather_rate(int device, uint64_t table_bytes, uint32_t load_bytes, double *bytes_per_s);

/* Thread-local description of the last error ("" if none). */
const char *nr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NR_H */
