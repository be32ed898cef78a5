// serve.cu -- the multi-user render server: a persistent loop that batches
// render requests of different subjects and resolutions as they arrive
// (continuous batching), for the conferencing scenario of Sec. 3 and Sec. 6.
//
// Structure:
//   * subjects are registered once; their tables, weights, weight volume and
//     derived layouts stay resident on the device;
//   * a request (subject, camera, pose, options, output buffer) is queued by
//     nr_server_submit from any host thread;
//   * one worker thread admits queued requests into slots in the order of the
//     server's policy (nr_server_set_policy): earliest deadline first (deadline
//     = arrival + deadline_ms + deadline_ms_per_mpixel x megapixels, 20 ms +
//     5 ms per megapixel by default), smallest first (fewest pixel x sample
//     slots; a request queued longer than age_ms goes first), or first come
//     first served.  Few slots serve the tail best: each field launch holds
//     every SM, so requests running side by side stretch each other.  A
//     slot owns two CUDA streams (with priority streams on: high priority for
//     requests of at most kSmallPixels pixels, low priority for the rest), the request's pose buffers (bone transforms,
//     folded residual bias, posed occupancy bitfield) and its sample queues,
//     sized for the largest chunk of rays (2^17 .. 2^20) that max_slots slots
//     fit in the budget.
//     Slots are created on demand while the device-memory budget allows and are
//     reused afterwards: admission is by memory and by slot count;
//   * the worker enqueues the whole request on the slot's stream (pose upload,
//     bias fold, bitfield, ray-chunked march / field / composite, copy-out) and
//     returns to the queue at once, so requests that arrive while others are on
//     the GPU start immediately and their kernels overlap on the device;
//   * a host callback on the slot's stream marks the request done, stamps its
//     latency (submit to completion, steady clock) and frees the slot.
// Every wait is bounded (NR_ETIMEOUT); a request that fails is marked failed
// and the others continue.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string.h>
#include <thread>
#include <unordered_map>
#include <vector>

#include "render.cuh"

namespace nr {

using Clock = std::chrono::steady_clock;

// A slot renders a request in chunks of at most its rays per chunk, with a sample queue of 32
// entries per ray (one round of early termination at 128 samples per ray).  The server takes the
// largest chunk in [kSlotRaysMin, kSlotRaysMax] for which max_slots slots fit its budget: a
// 1024 x 1024 frame in one pass at 2^20 rays (~1.07 GB per slot), eight passes at 2^17 (~137 MB).
constexpr size_t kSlotRaysMin = size_t(1) << 17, kSlotRaysMax = size_t(1) << 20;
constexpr size_t kSlotSamplesPerRay = 32;
constexpr double kAgeMs = 40.0;                      // a request queued this long is dispatched first
constexpr uint64_t kSmallPixels = 512 * 512;         // requests up to this size run on high-priority streams

struct Slot {
  int index = 0;
  cudaStream_t stream = nullptr;     // high priority: small requests
  cudaStream_t stream_lo = nullptr;  // low priority: large requests
  cudaStream_t cur = nullptr;        // the stream of the request in flight
  float *d_G = nullptr, *d_omega = nullptr, *d_bias1 = nullptr;
  uint32_t *bits = nullptr;
  FrameWork w{};
  float *h_pose = nullptr;          // pinned: G [24*12], omega [72], root translation [3]
  uint32_t *d_err = nullptr;        // the field kernels' error word of the request in flight
  uint32_t *h_err = nullptr;        // pinned copy, read by the completion callback
  size_t bytes = 0;
  bool busy = false;
  uint64_t req = 0;
};

struct Request {
  nr_request r;
  Clock::time_point t_submit;
  int32_t state = 0;                // 0 queued, 1 running, 2 done, -1 failed
  double latency_ms = 0.0;
  std::string err;
};

struct DoneCtx;

}  // namespace nr

struct nr_server {
  uint32_t magic = 0x4e525356u;
  int device = 0;
  uint64_t max_bytes = 0;
  uint32_t max_slots = 0;
  size_t slot_rays = 0;               // rays per chunk of every slot of this server
  std::vector<nr_subject *> subjects;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, nr::Request> reqs;
  std::vector<nr::Slot *> slots;
  std::vector<nr::DoneCtx *> ctxs;
  uint64_t next_id = 1;
  uint64_t bytes_in_use = 0;
  bool stopping = false, worker_exit = false;
  std::thread worker;
  nr_server_stats st{};
  nr_server_policy pol{NR_SERVE_EDF, (float)nr::kAgeMs, 20.f, 5.f, 0u};
};

namespace nr {

struct DoneCtx {
  nr_server *srv;
  Slot *slot;
};

static bool server_ok(const nr_server *s) { return s && s->magic == 0x4e525356u; }

static size_t slot_bytes(int grid, size_t rays) {
  return rays * kSlotSamplesPerRay * 2 * sizeof(float4) + rays * (sizeof(uint2) + sizeof(float4) + sizeof(uint32_t)) +
         256 + (size_t)grid * grid * grid / 8 + (kBones * 12 + kBones * 3 + kWidth) * sizeof(float);
}

static void free_slot(Slot *sl) {
  if (!sl) return;
  if (sl->stream) cudaStreamSynchronize(sl->stream);
  if (sl->stream_lo) cudaStreamSynchronize(sl->stream_lo);
  void *bufs[] = {sl->d_G,       sl->d_omega,   sl->d_bias1,      sl->bits,   sl->w.samp,
                  sl->w.samp_out, sl->w.ray_range, sl->w.counter, sl->w.state, sl->w.next, sl->d_err};
  for (void *p : bufs)
    if (p) cudaFree(p);
  if (sl->h_pose) cudaFreeHost(sl->h_pose);
  if (sl->h_err) cudaFreeHost(sl->h_err);
  if (sl->stream) cudaStreamDestroy(sl->stream);
  if (sl->stream_lo) cudaStreamDestroy(sl->stream_lo);
  delete sl;
}

static nr_status make_slot(nr_server *srv, int grid, Slot **out) {
  Slot *sl = new Slot();
  auto fail = [&](cudaError_t e, const char *what) {
    nr_status r = set_error_cuda(e, what);
    free_slot(sl);
    return r;
  };
  cudaError_t e;
#define SLOT_ALLOC(p, n)                                   \
  if ((e = cudaMalloc((void **)&(p), (n))) != cudaSuccess) \
    return fail(e, "slot allocation " #p);
  int least = 0, greatest = 0;
  if ((e = cudaDeviceGetStreamPriorityRange(&least, &greatest)) != cudaSuccess) return fail(e, "stream priorities");
  if ((e = cudaStreamCreateWithPriority(&sl->stream, cudaStreamNonBlocking, greatest)) != cudaSuccess)
    return fail(e, "stream");
  if ((e = cudaStreamCreateWithPriority(&sl->stream_lo, cudaStreamNonBlocking, least)) != cudaSuccess)
    return fail(e, "stream");
  SLOT_ALLOC(sl->d_G, kBones * 12 * sizeof(float));
  SLOT_ALLOC(sl->d_omega, (2 * kBones * 3 + 3) * sizeof(float));
  SLOT_ALLOC(sl->d_bias1, kWidth * sizeof(float));
  SLOT_ALLOC(sl->bits, (size_t)grid * grid * grid / 8);
  const size_t rays = srv->slot_rays, samples = rays * kSlotSamplesPerRay;
  SLOT_ALLOC(sl->w.samp, samples * sizeof(float4));
  SLOT_ALLOC(sl->w.samp_out, samples * sizeof(float4));
  SLOT_ALLOC(sl->w.ray_range, rays * sizeof(uint2));
  SLOT_ALLOC(sl->w.counter, 256);
  SLOT_ALLOC(sl->w.state, rays * sizeof(float4));
  SLOT_ALLOC(sl->w.next, rays * sizeof(uint32_t));
  SLOT_ALLOC(sl->d_err, sizeof(uint32_t));
#undef SLOT_ALLOC
  if ((e = cudaMallocHost((void **)&sl->h_pose, (kBones * 12 + kBones * 3 + 3) * sizeof(float))) != cudaSuccess)
    return fail(e, "pinned pose buffer");
  if ((e = cudaMallocHost((void **)&sl->h_err, sizeof(uint32_t))) != cudaSuccess) return fail(e, "pinned error word");
  *sl->h_err = 0;
  sl->w.cap_samples = samples;
  sl->w.cap_rays = rays;
  sl->bytes = slot_bytes(grid, rays);
  sl->index = (int)srv->slots.size();
  *out = sl;
  return NR_OK;
}

// Host callback at the end of a request's work on its slot stream (no CUDA calls here).
static void CUDART_CB on_request_done(void *p) {
  DoneCtx *c = static_cast<DoneCtx *>(p);
  nr_server *srv = c->srv;
  std::lock_guard<std::mutex> lock(srv->mu);
  Slot *sl = c->slot;
  auto it = srv->reqs.find(sl->req);
  if (it != srv->reqs.end()) {
    Request &q = it->second;
    q.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - q.t_submit).count();
    if (*sl->h_err) {   // a bounded wait of a tcgen05 field kernel gave up: the image is invalid
      q.state = -1;
      q.err = "field kernel: a bounded wait on the tensor-core pipeline gave up";
      srv->st.failed += 1;
    } else {
      q.state = 2;
      srv->st.completed += 1;
      srv->st.rays_done += (double)q.r.cam.width * q.r.cam.height;
    }
  }
  sl->busy = false;
  srv->st.active -= 1;
  srv->cv_work.notify_all();
  srv->cv_done.notify_all();
}

// Enqueues one request on a slot (worker thread, mu not held).  On failure the
// request is marked failed by the caller.
static nr_status launch_request(nr_server *srv, Slot *sl, Request &q, DoneCtx *ctx) {
  const nr_request &r = q.r;
  nr_subject *s = srv->subjects[r.subject];
  cudaStream_t st = sl->cur;
  memcpy(sl->h_pose + kBones * 12, r.axis_angle, sizeof(float) * kBones * 3);
  memcpy(sl->h_pose + kBones * 15, r.root_t, sizeof(float) * 3);
  NR_CHECK_CUDA(cudaMemcpyAsync(sl->d_omega, sl->h_pose + kBones * 12, sizeof(float) * (kBones * 3 + 3),
                                cudaMemcpyHostToDevice, st));
  nr_status rc;
  const float *omega_res = sl->d_omega;
  if (s->ref_layers) {   // the refined pose and updated angles (Sec. 4.1), on the device
    if ((rc = launch_refine_fk(s, sl->d_omega, 3 * kBones, sl->d_omega + 3 * kBones, 3, 1, sl->d_G,
                               sl->d_omega + 3 * kBones + 3, 3 * kBones, st)) != NR_OK)
      return rc;
    omega_res = sl->d_omega + 3 * kBones + 3;
  } else {
    forward_kinematics(s, r.axis_angle, r.root_t, sl->h_pose);
    NR_CHECK_CUDA(cudaMemcpyAsync(sl->d_G, sl->h_pose, sizeof(float) * kBones * 12, cudaMemcpyHostToDevice, st));
  }
  if ((rc = launch_fold_bias(s, omega_res, sl->d_bias1, 1, st)) != NR_OK) return rc;
  if (r.opts.use_occupancy && (rc = launch_posed_bitfield(s, sl->d_G, sl->d_bias1, sl->bits, st)) != NR_OK) return rc;
  FieldParams P = field_params(s, &r.opts);
  P.G = sl->d_G;
  P.bias1 = sl->d_bias1;
  P.t5_err = sl->d_err;             // this slot's own error word: slots render concurrently
  NR_CHECK_CUDA(cudaMemsetAsync(sl->d_err, 0, sizeof(uint32_t), st));
  // the composite kernel writes the pixels straight into out_rgba (device memory, or
  // pinned host memory reached through the unified address space)
  if ((rc = render_frame(s, P, sl->bits, &r.cam, &r.opts, sl->w, reinterpret_cast<float4 *>(r.out_rgba), st)) !=
      NR_OK)
    return rc;
  NR_CHECK_CUDA(cudaMemcpyAsync(sl->h_err, sl->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  NR_CHECK_CUDA(cudaLaunchHostFunc(st, on_request_done, ctx));
  return NR_OK;
}

static void worker_main(nr_server *srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lock(srv->mu);
  while (true) {
    // admit the oldest queued request into a free slot, or a new slot the budget allows
    Slot *slot = nullptr;
    if (!srv->queue.empty()) {
      for (Slot *sl : srv->slots)
        if (!sl->busy) {
          slot = sl;
          break;
        }
      if (!slot && srv->slots.size() < srv->max_slots) {
        const int grid = srv->subjects.empty() ? 128 : (int)srv->subjects[0]->occ_grid;
        if (srv->bytes_in_use + slot_bytes(grid, srv->slot_rays) <= srv->max_bytes) {
          Slot *ns = nullptr;
          if (make_slot(srv, grid, &ns) == NR_OK) {
            srv->slots.push_back(ns);
            srv->ctxs.push_back(new DoneCtx{srv, ns});
            srv->bytes_in_use += ns->bytes;
            srv->st.slots = (uint32_t)srv->slots.size();
            srv->st.bytes_in_use = srv->bytes_in_use;
            slot = ns;
          }
        }
      }
    }
    if (slot) {
      auto pick = srv->queue.begin();   // the queue is in arrival order: first come first served
      const nr_server_policy &pol = srv->pol;
      if (pol.order == NR_SERVE_SMALLEST_FIRST) {
        // smallest first, unless the oldest request has waited age_ms
        const double oldest_ms =
            std::chrono::duration<double, std::milli>(Clock::now() - srv->reqs[*pick].t_submit).count();
        if (oldest_ms < pol.age_ms) {
          uint64_t best = UINT64_MAX;
          for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it) {
            const nr_camera &c = srv->reqs[*it].r.cam;
            const uint64_t work = (uint64_t)c.width * c.height * c.n_samples;
            if (work < best) {
              best = work;
              pick = it;
            }
          }
        }
      } else if (pol.order == NR_SERVE_EDF) {
        // earliest deadline first: arrival + deadline_ms + deadline_ms_per_mpixel x megapixels
        double best = 1e300;
        const Clock::time_point t0 = srv->reqs[*pick].t_submit;
        for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it) {
          const Request &q = srv->reqs[*it];
          const double mpix = (double)q.r.cam.width * q.r.cam.height * 1e-6;
          const double due = std::chrono::duration<double, std::milli>(q.t_submit - t0).count() + pol.deadline_ms +
                             pol.deadline_ms_per_mpixel * mpix;
          if (due < best) {
            best = due;
            pick = it;
          }
        }
      }
      const uint64_t id = *pick;
      srv->queue.erase(pick);
      Request &q = srv->reqs[id];
      slot->cur = (srv->pol.priority_streams && (uint64_t)q.r.cam.width * q.r.cam.height <= kSmallPixels)
                      ? slot->stream
                      : slot->stream_lo;
      q.state = 1;
      slot->busy = true;
      slot->req = id;
      srv->st.active += 1;
      srv->st.peak_active = std::max(srv->st.peak_active, srv->st.active);
      DoneCtx *ctx = srv->ctxs[slot->index];
      Request copy = q;
      lock.unlock();
      const nr_status rc = launch_request(srv, slot, copy, ctx);
      lock.lock();
      if (rc != NR_OK) {
        // nothing (or only part of the work) reached the stream: wait for it, then fail the request
        lock.unlock();
        cudaStreamSynchronize(slot->cur);
        lock.lock();
        Request &qq = srv->reqs[id];
        qq.state = -1;
        qq.err = nr_last_error();
        srv->st.failed += 1;
        srv->st.active -= 1;
        slot->busy = false;
        srv->cv_done.notify_all();
      }
      continue;
    }
    if (srv->stopping && srv->queue.empty() && srv->st.active == 0) break;
    srv->cv_work.wait_for(lock, std::chrono::milliseconds(5));
  }
  srv->worker_exit = true;
  srv->cv_done.notify_all();
}

}  // namespace nr

using namespace nr;

extern "C" nr_status nr_server_create(int device, uint64_t max_bytes, uint32_t max_slots, nr_server **out) {
  NR_REQUIRE(out, "nr_server_create: NULL out");
  *out = nullptr;
  NR_REQUIRE(max_slots >= 1 && max_slots <= 256, "nr_server_create: max_slots must be 1..256");
  NR_REQUIRE(max_bytes >= slot_bytes(32, kSlotRaysMin), "nr_server_create: max_bytes below one slot (%zu bytes)",
             slot_bytes(32, kSlotRaysMin));
  NR_CHECK_CUDA(cudaSetDevice(device));
  nr_server *srv = new nr_server();
  srv->device = device;
  srv->max_bytes = max_bytes;
  srv->max_slots = max_slots;
  // the largest chunk for which max_slots slots (128^3 occupancy grids) fit the budget
  srv->slot_rays = kSlotRaysMin;
  while (srv->slot_rays < kSlotRaysMax && slot_bytes(128, 2 * srv->slot_rays) * max_slots <= max_bytes)
    srv->slot_rays *= 2;
  srv->worker = std::thread(worker_main, srv);
  *out = srv;
  return NR_OK;
}

extern "C" nr_status nr_server_set_policy(nr_server *srv, const nr_server_policy *policy) {
  NR_REQUIRE(server_ok(srv) && policy, "nr_server_set_policy: bad argument");
  NR_REQUIRE(policy->order == NR_SERVE_SMALLEST_FIRST || policy->order == NR_SERVE_FIFO ||
                 policy->order == NR_SERVE_EDF,
             "nr_server_set_policy: unknown order %u", policy->order);
  NR_REQUIRE(policy->age_ms >= 0.f && policy->deadline_ms >= 0.f && policy->deadline_ms_per_mpixel >= 0.f,
             "nr_server_set_policy: negative time");
  std::lock_guard<std::mutex> lock(srv->mu);
  srv->pol = *policy;
  return NR_OK;
}

extern "C" nr_status nr_server_add_subject(nr_server *srv, nr_subject *s, uint32_t *index) {
  NR_REQUIRE(server_ok(srv) && subject_ok(s) && index, "nr_server_add_subject: bad argument");
  NR_REQUIRE(s->device == srv->device, "nr_server_add_subject: subject lives on device %d, server on %d", s->device,
             srv->device);
  NR_CHECK_CUDA(cudaSetDevice(srv->device));
  nr_status r;
  if ((r = prepare_params(s, nullptr)) != NR_OK) return r;
  if ((r = prepare_fp8(s, nullptr)) != NR_OK) return r;
  if ((r = prepare_t5(s, nullptr)) != NR_OK) return r;
  NR_CHECK_CUDA(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lock(srv->mu);
  NR_REQUIRE(srv->subjects.empty() || srv->subjects[0]->occ_grid == s->occ_grid,
             "nr_server_add_subject: all subjects must share one occupancy grid size");
  srv->subjects.push_back(s);
  *index = (uint32_t)srv->subjects.size() - 1;
  return NR_OK;
}

extern "C" nr_status nr_server_submit(nr_server *srv, const nr_request *req, uint64_t *id) {
  NR_REQUIRE(server_ok(srv) && req && id, "nr_server_submit: bad argument");
  const nr_camera &c = req->cam;
  NR_REQUIRE(req->out_rgba, "nr_server_submit: NULL output");
  NR_REQUIRE(c.width >= 1 && c.height >= 1 && (uint64_t)c.width * c.height <= (1ull << 24),
             "nr_server_submit: image size out of range");
  NR_REQUIRE(c.n_samples >= 1 && c.n_samples <= 1024 && c.fx != 0.f && c.fy != 0.f, "nr_server_submit: bad camera");
  NR_REQUIRE(req->opts.mlp_dtype == NR_F32 || req->opts.mlp_dtype == NR_BF16 || req->opts.mlp_dtype == NR_F16 ||
                 req->opts.mlp_dtype == NR_FP8E4M3,
             "nr_server_submit: unknown mlp_dtype");
  NR_REQUIRE(req->opts.feat_dtype == NR_F32 || req->opts.feat_dtype == NR_F16, "nr_server_submit: bad feat_dtype");
  NR_REQUIRE(req->opts.t_min >= 0.f && req->opts.t_min < 1.f, "nr_server_submit: t_min must be in [0, 1)");
  for (int i = 0; i < kBones * 3; ++i) NR_REQUIRE(isfinite(req->axis_angle[i]), "nr_server_submit: non-finite pose");
  cudaPointerAttributes attr{};
  const cudaError_t e = cudaPointerGetAttributes(&attr, req->out_rgba);
  cudaGetLastError();
  NR_REQUIRE(e == cudaSuccess && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeHost),
             "nr_server_submit: out_rgba must be device memory or pinned host memory");
  std::lock_guard<std::mutex> lock(srv->mu);
  NR_REQUIRE(req->subject < srv->subjects.size(), "nr_server_submit: unknown subject %u", req->subject);
  NR_REQUIRE(!req->opts.use_occupancy || srv->subjects[req->subject]->occ_source != kOccNone,
             "nr_server_submit: occupancy requested for a subject without it");
  if (srv->stopping) {
    set_error("nr_server_submit: the server is stopping");
    srv->st.rejected += 1;
    return NR_ESTATE;
  }
  const uint64_t nid = srv->next_id++;
  Request &q = srv->reqs[nid];
  q.r = *req;
  q.t_submit = Clock::now();
  srv->queue.push_back(nid);
  srv->st.submitted += 1;
  *id = nid;
  srv->cv_work.notify_all();
  return NR_OK;
}

extern "C" nr_status nr_server_poll(nr_server *srv, uint64_t id, int32_t *state, double *latency_ms) {
  NR_REQUIRE(server_ok(srv) && state, "nr_server_poll: bad argument");
  std::lock_guard<std::mutex> lock(srv->mu);
  auto it = srv->reqs.find(id);
  NR_REQUIRE(it != srv->reqs.end(), "nr_server_poll: unknown request %llu", (unsigned long long)id);
  *state = it->second.state;
  if (latency_ms) *latency_ms = it->second.latency_ms;
  if (it->second.state == 2 || it->second.state == -1) {
    if (it->second.state == -1) set_error("request failed: %s", it->second.err.c_str());
    srv->reqs.erase(it);
  }
  return NR_OK;
}

extern "C" nr_status nr_server_wait(nr_server *srv, uint64_t id, uint32_t timeout_ms, double *latency_ms) {
  NR_REQUIRE(server_ok(srv), "nr_server_wait: bad server");
  std::unique_lock<std::mutex> lock(srv->mu);
  auto it = srv->reqs.find(id);
  NR_REQUIRE(it != srv->reqs.end(), "nr_server_wait: unknown request %llu", (unsigned long long)id);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  while (true) {
    it = srv->reqs.find(id);
    if (it->second.state == 2 || it->second.state == -1) break;
    if (srv->cv_done.wait_until(lock, deadline) == std::cv_status::timeout) {
      it = srv->reqs.find(id);
      if (it->second.state == 2 || it->second.state == -1) break;
      set_error("nr_server_wait: request %llu not done after %u ms", (unsigned long long)id, timeout_ms);
      return NR_ETIMEOUT;
    }
  }
  const int32_t state = it->second.state;
  if (latency_ms) *latency_ms = it->second.latency_ms;
  std::string err = it->second.err;
  srv->reqs.erase(it);
  if (state == -1) {
    set_error("request failed: %s", err.c_str());
    return NR_ECUDA;
  }
  return NR_OK;
}

extern "C" nr_status nr_server_get_stats(nr_server *srv, nr_server_stats *out) {
  NR_REQUIRE(server_ok(srv) && out, "nr_server_get_stats: bad argument");
  std::lock_guard<std::mutex> lock(srv->mu);
  *out = srv->st;
  out->queued = (uint32_t)srv->queue.size();
  return NR_OK;
}

extern "C" nr_status nr_server_stop(nr_server *srv, uint32_t timeout_ms) {
  NR_REQUIRE(server_ok(srv), "nr_server_stop: bad server");
  std::unique_lock<std::mutex> lock(srv->mu);
  srv->stopping = true;
  srv->cv_work.notify_all();
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  while (!srv->worker_exit) {
    if (srv->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && !srv->worker_exit) {
      set_error("nr_server_stop: %u requests still queued or running after %u ms",
                (unsigned)(srv->queue.size() + srv->st.active), timeout_ms);
      return NR_ETIMEOUT;
    }
  }
  lock.unlock();
  if (srv->worker.joinable()) srv->worker.join();
  return NR_OK;
}

extern "C" nr_status nr_server_destroy(nr_server *srv) {
  if (!srv) return NR_OK;
  NR_REQUIRE(server_ok(srv), "nr_server_destroy: bad server");
  nr_status r = nr_server_stop(srv, 600000);
  if (r != NR_OK) return r;
  cudaSetDevice(srv->device);
  for (Slot *sl : srv->slots) free_slot(sl);
  for (DoneCtx *c : srv->ctxs) delete c;
  srv->magic = 0;
  delete srv;
  return NR_OK;
}
