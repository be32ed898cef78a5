// render_static.cu -- nr_render_static: the frame render of nr_render with its
// work queues in a fixed, file-scope device array instead of memory the
// library allocates, for callers that must not trigger a device allocation.
//
// Why: nr_render grows the subject's sample queues with cudaMalloc the first
// time a frame of a new size arrives.  Some callers cannot allow that at render
// time: a real-time serving thread where cudaMalloc's implicit device
// synchronisation would stall every other stream, or a process that has handed
// all free device memory to its own pool, so that a late allocation fails.
// This entry point allocates nothing: its scratch is the static array below,
// created when the module loads, and held by every GPU that loads the library
// until exit.  Everything else it touches (parameters, their derived copies,
// the pose buffers and the occupancy bitfield) was allocated with the subject.
//
// Limits: n_rays = width * height <= kStaticRays (65,536) and
// n_rays * n_samples <= kStaticSamples (262,144 sample slots).  Scratch size:
// 2 x 262,144 x 16 B (sample queue and per-sample outputs) + 65,536 x 8 B
// (ray ranges) + 256 B (counters) = 8.5 MiB per device.
//
// Sharing: every call on a device uses the same array and leaves the last
// call's contents in it.  Two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it and corrupt each other's
// results; serialise them.  The live-sample counter is cleared by each call.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress while that device is current (the host-side name of
// a __device__ variable is not a device address) and keeps it for the process.
// That look-up may not run under a stream capture: make the first call on each
// device before any capture.  The kept address belongs to the device's primary
// context: do not reset the device (cudaDeviceReset) after the first call.
//
// Kernel paths: the default path of the MLP dtype (for bf16/f16 the tcgen05
// pipeline, whose weight blobs and error word come with the subject),
// NR_RENDER_MMA_SYNC, NR_RENDER_MMA2 and NR_RENDER_TCGEN05 are honoured; NR_RENDER_F32_TC (a scratch buffer
// allocated on first use) and NR_RENDER_PROFILE (events created on first use)
// are refused with NR_EUNSUPPORTED.
#include <mutex>

#include "render.cuh"

namespace nr {

constexpr size_t kStaticSamples = size_t(1) << 18;
constexpr size_t kStaticRays = size_t(1) << 16;

struct StaticScratch {
  float4 samp[kStaticSamples];       // live samples: x, y, z, delta
  float4 samp_out[kStaticSamples];   // per-sample r, g, b, alpha
  uint2 ray_range[kStaticRays];      // per ray: first sample, count
  uint32_t counter[64];              // live-sample counter (word 0)
};

static __device__ __align__(256) StaticScratch g_static_scratch;

static std::mutex g_static_mu;
static StaticScratch *g_static_ptr[64] = {nullptr};

// Device address of g_static_scratch on `device` (current), looked up once.
static nr_status static_scratch(int device, StaticScratch **out) {
  NR_REQUIRE(device >= 0 && device < 64, "nr_render_static: device ordinal %d out of range", device);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return set_error_cuda(e, "nr_render_static: cudaGetSymbolAddress");
    g_static_ptr[device] = static_cast<StaticScratch *>(p);
  }
  *out = g_static_ptr[device];
  return NR_OK;
}

}  // namespace nr

using namespace nr;

extern "C" nr_status nr_render_static(nr_subject *s, const nr_camera *cam, const nr_render_opts *opts,
                                      float *out_rgba, void *stream) {
  NR_REQUIRE(subject_ok(s), "nr_render_static: invalid handle");
  NR_REQUIRE(cam && opts && out_rgba, "nr_render_static: NULL argument");
  NR_REQUIRE(opts->mlp_dtype == NR_F32 || opts->mlp_dtype == NR_BF16 || opts->mlp_dtype == NR_F16,
             "nr_render_static: mlp_dtype must be NR_F32, NR_BF16 or NR_F16");
  NR_REQUIRE(opts->feat_dtype == NR_F32 || opts->feat_dtype == NR_F16, "nr_render_static: bad feat_dtype");
  if (opts->mlp_dtype == NR_F32 && (opts->flags & NR_RENDER_F32_TC)) {
    set_error("nr_render_static: NR_RENDER_F32_TC needs a scratch buffer the static path does not allocate");
    return NR_EUNSUPPORTED;
  }
  if (opts->flags & NR_RENDER_PROFILE) {
    set_error("nr_render_static: NR_RENDER_PROFILE needs events the static path does not create");
    return NR_EUNSUPPORTED;
  }
  NR_REQUIRE(opts->t_min >= 0.f && opts->t_min < 1.f, "nr_render_static: t_min must be in [0, 1)");
  NR_REQUIRE(!opts->use_occupancy || s->occ_source != kOccNone, "nr_render_static: the subject has no occupancy");
  NR_REQUIRE(cam->width >= 1 && cam->height >= 1 && cam->n_samples >= 1 && cam->n_samples <= 1024,
             "nr_render_static: empty image or n_samples outside 1..1024");
  NR_REQUIRE(cam->fx != 0.f && cam->fy != 0.f, "nr_render_static: zero focal length");
  const uint64_t n_rays = (uint64_t)cam->width * cam->height;
  NR_REQUIRE(n_rays <= kStaticRays, "nr_render_static: %llu rays exceed the static limit of %llu",
             (unsigned long long)n_rays, (unsigned long long)kStaticRays);
  NR_REQUIRE(n_rays * cam->n_samples <= kStaticSamples,
             "nr_render_static: %llu sample slots exceed the static limit of %llu",
             (unsigned long long)(n_rays * cam->n_samples), (unsigned long long)kStaticSamples);
  if (!s->pose_set) {
    set_error("nr_render_static: call nr_set_pose first");
    return NR_ESTATE;
  }
  NR_CHECK_CUDA(cudaSetDevice(s->device));
  cudaPointerAttributes attr{};
  const bool dev_out = cudaPointerGetAttributes(&attr, out_rgba) == cudaSuccess && attr.type == cudaMemoryTypeDevice;
  cudaGetLastError();
  NR_REQUIRE(dev_out, "nr_render_static: out_rgba must be device memory");
  StaticScratch *sc = nullptr;
  nr_status r = static_scratch(s->device, &sc);
  if (r != NR_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if ((r = prepare_params(s, st)) != NR_OK) return r;
  if ((r = ensure_pose(s, st)) != NR_OK) return r;
  if ((r = ensure_bias(s, st)) != NR_OK) return r;
  if (opts->use_occupancy && (r = ensure_occupancy(s, st)) != NR_OK) return r;
  const int path = render_path(opts);
  const bool t5 = path_uses_tcgen05(opts, path);
  if (t5 && (r = prepare_t5(s, st)) != NR_OK) return r;
  const FieldParams P = field_params(s, opts);
  const CamParams C = cam_params(cam);
  MarchParams mp{};
  for (int k = 0; k < 3; ++k) {
    mp.bmin[k] = s->bmin[k];
    mp.bmax[k] = s->bmax[k];
  }
  mp.grid = (int)s->occ_grid;
  mp.bits = opts->use_occupancy ? s->bits : nullptr;
  mp.ray0 = 0;
  mp.ray_end = (uint32_t)n_rays;
  NR_CHECK_CUDA(cudaMemsetAsync(sc->counter, 0, sizeof(uint32_t), st));
  const uint32_t nr_ = (uint32_t)n_rays;
  march_kernel<<<(nr_ + 255) / 256, 256, 0, st>>>(C, mp, sc->samp, sc->ray_range, sc->counter);
  NR_CHECK_CUDA(cudaGetLastError());
  if ((r = launch_field(P, opts->mlp_dtype, kModeRender, sc->samp, 0, sc->counter, (float *)sc->samp_out, s->device,
                        st, path)) != NR_OK)
    return r;
  composite_kernel<<<(nr_ + 255) / 256, 256, 0, st>>>(sc->ray_range, sc->samp_out, nr_, opts->t_min, cam->bg[0],
                                                      cam->bg[1], cam->bg[2], reinterpret_cast<float4 *>(out_rgba));
  NR_CHECK_CUDA(cudaGetLastError());
  count_launches(3);
  return t5 ? check_field_timeouts(s, st) : NR_OK;
}
