// C ABI entry points (declared in include/gs2d.h): plan layout, argument
// checks, launch sequencing and the frame-fitting loop.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gs2d_internal.cuh"

using namespace gs2d;

namespace {

thread_local char g_err[512] = "";

gs2d_status fail(gs2d_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

gs2d_status ok() {
  g_err[0] = 0;
  return GS2D_OK;
}

gs2d_status cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) return fail(GS2D_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return ok();
}

uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// Size limits that keep every 32-bit index of the kernels in range: the
// parameter rows (9 n), the per-pair records (8 floats per entry) and the
// render-queue ranks (28 bits).
constexpr int64_t kMaxGaussians = int64_t(1) << 27;
constexpr int64_t kMaxEntries = (int64_t(1) << 28) - 1;

gs2d_status check_plan(const gs2d_plan* p, const void* ws) {
  if (!p || p->magic != kPlanMagic) return fail(GS2D_ERR_INVALID_ARG, "plan not initialised");
  if (!ws) return fail(GS2D_ERR_INVALID_ARG, "workspace is NULL");
  if ((uintptr_t)ws % 256 != 0) return fail(GS2D_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  return GS2D_OK;
}

bool cfg_valid(const gs2d_config& c) {
  return (c.tile == 8 || c.tile == 16 || c.tile == 32) &&
         (c.stage == 0 || c.stage == 32 || c.stage == 64 || c.stage == 128 || c.stage == 256) &&
         (c.launch == GS2D_LAUNCH_PERSISTENT || c.launch == GS2D_LAUNCH_GRID) &&
         c.sigma_cut > 0.0f && isfinite(c.sigma_cut) && c.alpha_min > 0.0f &&
         isfinite(c.alpha_min) && c.det_eps >= 0.0f && isfinite(c.det_eps) && c.lr > 0.0f &&
         isfinite(c.lr) && c.beta1 >= 0.0f && c.beta1 < 1.0f && c.beta2 >= 0.0f &&
         c.beta2 < 1.0f && c.eps > 0.0f && isfinite(c.eps) && c.lr_mu >= 0.0f &&
         isfinite(c.lr_mu) && c.lr_shape >= 0.0f && isfinite(c.lr_shape) && c.lr_color >= 0.0f &&
         isfinite(c.lr_color) && c.lr_weight >= 0.0f && isfinite(c.lr_weight) &&
         c.lr_decay > 0.0f && c.lr_decay <= 1.0f && isfinite(c.bin_margin) &&
         (c.reduce == GS2D_REDUCE_SLOTS || c.reduce == GS2D_REDUCE_ATOMIC);
}

}  // namespace

namespace gs2d {
gs2d_status set_error(gs2d_status st, const char* msg) {
  snprintf(g_err, sizeof(g_err), "%s", msg);
  return st;
}
}  // namespace gs2d

extern "C" {

void gs2d_config_default(gs2d_config* cfg) {
  if (!cfg) return;
  cfg->tile = kTileDefault;
  cfg->sigma_cut = 4.5f;
  cfg->alpha_min = 1.0f / 255.0f;
  cfg->det_eps = 1e-8f;
  cfg->lr = 1e-2f;
  cfg->beta1 = 0.9f;
  cfg->beta2 = 0.999f;
  cfg->eps = 1e-8f;
  cfg->stage = kStageDefault;
  cfg->launch = GS2D_LAUNCH_GRID;
  cfg->lr_mu = cfg->lr_shape = cfg->lr_color = cfg->lr_weight = 1.0f;
  cfg->lr_decay = 1.0f;
  cfg->bin_margin = 4.0f;
  cfg->reduce = GS2D_REDUCE_SLOTS;
}

size_t gs2d_sizeof_plan(void) { return sizeof(gs2d_plan); }
size_t gs2d_sizeof_config(void) { return sizeof(gs2d_config); }

gs2d_status gs2d_plan_init(gs2d_plan* plan, int32_t width, int32_t height, int32_t n,
                           int64_t max_entries, const gs2d_config* cfg) {
  if (!plan) return fail(GS2D_ERR_INVALID_ARG, "plan is NULL");
  gs2d_clip clip;
  memset(&clip, 0, sizeof(clip));
  clip.width = width;
  clip.height = height;
  clip.n = n;
  return gs2d_plan_init_batch(plan, &clip, 1, max_entries, cfg);
}

gs2d_status gs2d_plan_init_batch(gs2d_plan* plan, gs2d_clip* clips, int32_t num_clips,
                                 int64_t max_entries, const gs2d_config* cfg) {
  if (!plan) return fail(GS2D_ERR_INVALID_ARG, "plan is NULL");
  memset(plan, 0, sizeof(*plan));
  if (!clips || num_clips < 1 || num_clips > 65536)
    return fail(GS2D_ERR_INVALID_ARG, "num_clips = %d out of range (or clips is NULL)", num_clips);
  gs2d_config c;
  gs2d_config_default(&c);
  if (cfg) c = *cfg;
  if (!cfg_valid(c))
    return fail(GS2D_ERR_INVALID_ARG,
                "invalid config (tile 8, 16 or 32; stage 0, 32, 64, 128 or 256; reduce 0 or 1)");
  if (c.stage == 0) c.stage = kStageDefault;
  const int T = c.tile;
  int64_t n_total = 0, tiles = 0, pixels = 0;
  for (int k = 0; k < num_clips; k++) {
    gs2d_clip& cl = clips[k];
    if (cl.width < 1 || cl.height < 1 || cl.width > 65536 || cl.height > 65536)
      return fail(GS2D_ERR_INVALID_ARG, "clip %d: image size %d x %d out of range", k, cl.width,
                  cl.height);
    if (cl.n < 0) return fail(GS2D_ERR_INVALID_ARG, "clip %d: n = %d < 0", k, cl.n);
    cl.tiles_x = (cl.width + T - 1) / T;
    cl.tiles_y = (cl.height + T - 1) / T;
    cl.g_off = (int32_t)n_total;
    cl.tile_off = (int32_t)tiles;
    cl.reserved = 0;
    cl.pix_off = 3 * pixels;
    n_total += cl.n;
    tiles += (int64_t)cl.tiles_x * cl.tiles_y;
    pixels += (int64_t)cl.width * cl.height;
    if (n_total > kMaxGaussians || tiles > (1 << 28))
      return fail(GS2D_ERR_INVALID_ARG, "batch too large (%lld Gaussians, %lld tiles)",
                  (long long)n_total, (long long)tiles);
  }
  if (max_entries == 0)
    max_entries = std::min<int64_t>(
        kMaxEntries, std::max<int64_t>(1 << 20, 16 * n_total * (T == 8 ? 4 : 1)));
  if (max_entries < 1 || max_entries > kMaxEntries)
    return fail(GS2D_ERR_INVALID_ARG, "max_entries = %lld out of range (1 .. %lld)",
                (long long)max_entries, (long long)kMaxEntries);
  // a one-clip plan is a single frame: its kernels take the clip from these
  plan->width = num_clips == 1 ? clips[0].width : 0;
  plan->height = num_clips == 1 ? clips[0].height : 0;
  plan->n = (int32_t)n_total;
  plan->tile = T;
  plan->tiles_x = num_clips == 1 ? clips[0].tiles_x : 0;
  plan->tiles_y = num_clips == 1 ? clips[0].tiles_y : 0;
  plan->num_tiles = (int32_t)tiles;
  int bits = 0;
  while ((int64_t(1) << bits) < tiles) bits++;
  plan->tile_bits = bits;
  plan->num_clips = num_clips;
  plan->stage = c.stage;
  plan->max_entries = max_entries;
  plan->pixels = pixels;
  plan->cfg = c;
  const uint64_t nn = (uint64_t)n_total, me = (uint64_t)max_entries, nt = (uint64_t)tiles;
  uint64_t sz[kNumSections];
  sz[kOffHeader] = sizeof(WsHeader);
  sz[kOffClips] = (uint64_t)num_clips * sizeof(gs2d_clip);
  sz[kOffRec] = 3 * nn * sizeof(float4);
  sz[kOffRect] = nn * sizeof(int4);
  sz[kOffCount] = (nn + 1) * sizeof(int);
  sz[kOffBlockSum] = (nn / 32 + 1) * sizeof(long long);  // blocks of >= 32 Gaussians
  sz[kOffTileCnt] = nt * sizeof(int);
  sz[kOffCursor] = nt * sizeof(int);
  sz[kOffLong] = (nt + 1) * sizeof(int);
  sz[kOffList] = me * sizeof(uint32_t);
  sz[kOffRanges] = nt * sizeof(int2);
  sz[kOffOrder] = nt * sizeof(int);
  sz[kOffRank] = nt * sizeof(uint32_t);
  sz[kOffBucket] = 2 * kBuckets * sizeof(int);
  sz[kOffPartial] = me * kPartials * sizeof(float);
  sz[kOffLossPart] = nt * sizeof(float2);
  sz[kOffClipLoss] = (uint64_t)num_clips * sizeof(float2);
  sz[kOffActive] = nt;
  sz[kOffActOrder] = (nt + 1) * sizeof(int);
  sz[kOffQuant] = 9 * nn * sizeof(float);
  sz[kOffGrad] = 9 * nn * sizeof(float);
  sz[kOffLRect] = nn * sizeof(int4);
  sz[kOffTileCnt2] = nt * sizeof(int);
  sz[kOffAcc] = 8 * nn * sizeof(float);
  uint64_t off = 0;
  for (int sec = 0; sec < kNumSections; sec++) {
    plan->off[sec] = off;
    off = align256(off + sz[sec]);
  }
  plan->ws_bytes = off;
  plan->magic = kPlanMagic;
  return ok();
}

gs2d_status gs2d_ws_set_clips(const gs2d_plan* plan, void* ws, const gs2d_clip* clips,
                              void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!clips) return fail(GS2D_ERR_INVALID_ARG, "clips is NULL");
  // the table must be the one this plan was laid out from
  int64_t tiles = 0, n = 0;
  for (int k = 0; k < plan->num_clips; k++) {
    const gs2d_clip& cl = clips[k];
    if (cl.tile_off != tiles || cl.g_off != n ||
        cl.tiles_x != (cl.width + plan->tile - 1) / plan->tile ||
        cl.tiles_y != (cl.height + plan->tile - 1) / plan->tile)
      return fail(GS2D_ERR_INVALID_ARG, "clip %d does not match the plan", k);
    tiles += (int64_t)cl.tiles_x * cl.tiles_y;
    n += cl.n;
  }
  if (tiles != plan->num_tiles || n != plan->n)
    return fail(GS2D_ERR_INVALID_ARG, "clip table does not match the plan");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(ws_ptr<gs2d_clip>(ws, *plan, kOffClips), clips,
                                  (size_t)plan->num_clips * sizeof(gs2d_clip),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_check(e, "gs2d_ws_set_clips");
}

gs2d_status gs2d_project(const gs2d_plan* plan, void* ws, const float* params, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!params && plan->n > 0) return fail(GS2D_ERR_INVALID_ARG, "params is NULL");
  return cuda_check(launch_project(*plan, ws, params, (cudaStream_t)stream), "gs2d_project");
}

gs2d_status gs2d_bin_sort(const gs2d_plan* plan, void* ws, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  return cuda_check(launch_bin_sort(*plan, ws, (cudaStream_t)stream), "gs2d_bin_sort");
}

gs2d_status gs2d_prepare(const gs2d_plan* plan, void* ws, const float* params, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!params && plan->n > 0) return fail(GS2D_ERR_INVALID_ARG, "params is NULL");
  return cuda_check(launch_prepare(*plan, ws, params, false, (cudaStream_t)stream),
                    "gs2d_prepare");
}

gs2d_status gs2d_render_fwd(const gs2d_plan* plan, void* ws, float* img, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!img) return fail(GS2D_ERR_INVALID_ARG, "img is NULL");
  return cuda_check(launch_render_fwd(*plan, ws, img, (cudaStream_t)stream), "gs2d_render_fwd");
}

gs2d_status gs2d_render_bwd(const gs2d_plan* plan, void* ws, const float* params,
                            const float* dimg, float* grads, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!dimg) return fail(GS2D_ERR_INVALID_ARG, "dimg is NULL");
  if (plan->n > 0 && (!params || !grads))
    return fail(GS2D_ERR_INVALID_ARG, "params or grads is NULL");
  return cuda_check(launch_render_bwd(*plan, ws, params, dimg, grads, (cudaStream_t)stream),
                    "gs2d_render_bwd");
}

gs2d_status gs2d_render_l2(const gs2d_plan* plan, void* ws, const float* params,
                           const float* target, float* grads, float* img, float* loss,
                           void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!target) return fail(GS2D_ERR_INVALID_ARG, "target is NULL");
  if (plan->n > 0 && (!params || !grads))
    return fail(GS2D_ERR_INVALID_ARG, "params or grads is NULL");
  return cuda_check(
      launch_render_l2(*plan, ws, params, target, grads, img, loss, (cudaStream_t)stream),
      "gs2d_render_l2");
}

gs2d_status gs2d_adam_step(float* params, const float* grads, float* m, float* v, int64_t count,
                           int32_t step, const uint8_t* mask, const gs2d_config* cfg,
                           void* stream) {
  gs2d_config c;
  gs2d_config_default(&c);
  if (cfg) c = *cfg;
  if (!cfg_valid(c)) return fail(GS2D_ERR_INVALID_ARG, "invalid config");
  if (count < 0) return fail(GS2D_ERR_INVALID_ARG, "count < 0");
  if (step < 1) return fail(GS2D_ERR_INVALID_ARG, "step must be >= 1");
  if (count > 0 && (!params || !grads || !m || !v))
    return fail(GS2D_ERR_INVALID_ARG, "NULL array");
  if (mask && count % 9 != 0)
    return fail(GS2D_ERR_INVALID_ARG, "mask needs count to be a multiple of 9");
  return cuda_check(launch_adam(params, grads, m, v, count, step, mask, c, (cudaStream_t)stream),
                    "gs2d_adam_step");
}

uint64_t gs2d_roi_init_scratch_bytes(int32_t width, int32_t height, int32_t n) {
  if (width < 1 || height < 1 || n < 0) return 0;
  return roi_init_scratch_bytes(width, height, n);
}

static gs2d_status roi_init_checked(const float* frame, const uint8_t* mask, int32_t width,
                                    int32_t height, int32_t n, float roi_frac, const float* bg_xy,
                                    float* params, int32_t* n_roi, void* scratch,
                                    uint64_t scratch_bytes, void* stream, float* cen_trace,
                                    int32_t* label_trace, const char* what) {
  // (its kernels index pixels with 32-bit integers)
  if (width < 1 || height < 1 || width > 65536 || height > 65536 ||
      (int64_t)width * height > (int64_t(1) << 30) || n < 0 || n > kMaxGaussians)
    return fail(GS2D_ERR_INVALID_ARG, "%s: sizes out of range", what);
  if (!(roi_frac >= 0.0f && roi_frac <= 1.0f))
    return fail(GS2D_ERR_INVALID_ARG, "%s: roi_frac must be in [0, 1]", what);
  if (!frame || !mask || (n > 0 && (!params || !bg_xy)) || !scratch)
    return fail(GS2D_ERR_INVALID_ARG, "%s: NULL pointer", what);
  if ((uintptr_t)scratch % 256) return fail(GS2D_ERR_INVALID_ARG, "scratch not 256-byte aligned");
  char msg[256] = "";
  const gs2d_status st = roi_init(frame, mask, width, height, n, roi_frac, bg_xy, params, n_roi,
                                  scratch, scratch_bytes, (cudaStream_t)stream, msg, sizeof(msg),
                                  cen_trace, label_trace);
  if (st != GS2D_OK) return fail(st, "%s", msg);
  return ok();
}

gs2d_status gs2d_roi_init(const float* frame, const uint8_t* mask, int32_t width, int32_t height,
                          int32_t n, float roi_frac, const float* bg_xy, float* params,
                          int32_t* n_roi, void* scratch, uint64_t scratch_bytes, void* stream) {
  return roi_init_checked(frame, mask, width, height, n, roi_frac, bg_xy, params, n_roi, scratch,
                          scratch_bytes, stream, nullptr, nullptr, "gs2d_roi_init");
}

gs2d_status gs2d_roi_init_trace(const float* frame, const uint8_t* mask, int32_t width,
                                int32_t height, int32_t n, float roi_frac, const float* bg_xy,
                                float* params, int32_t* n_roi, void* scratch,
                                uint64_t scratch_bytes, float* cen_trace, int32_t* label_trace,
                                void* stream) {
  return roi_init_checked(frame, mask, width, height, n, roi_frac, bg_xy, params, n_roi, scratch,
                          scratch_bytes, stream, cen_trace, label_trace, "gs2d_roi_init_trace");
}

static cudaError_t fit_iteration(const gs2d_plan& p, void* ws, const float* target, float* params,
                                 float* m, float* v, cudaStream_t s) {
  cudaError_t e = launch_prepare_fit(p, ws, params, s);
  if (e == cudaSuccess) e = launch_fit_step(p, ws, target, params, m, v, s);
  return e;
}

// Zeroes the Adam moments and the workspace header (step counter, status,
// render queue): the optimiser restarts for every frame.
static cudaError_t reset_fit(const gs2d_plan& p, void* ws, float* m, float* v, cudaStream_t s) {
  const size_t pbytes = (size_t)9 * p.n * sizeof(float);
  cudaError_t e = cudaSuccess;
  if (pbytes) e = cudaMemsetAsync(m, 0, pbytes, s);
  if (e == cudaSuccess && pbytes) e = cudaMemsetAsync(v, 0, pbytes, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(ws_ptr<WsHeader>(ws, p, kOffHeader), 0, sizeof(WsHeader), s);
  return e;
}

// One fit iteration captured as a CUDA graph (non-default streams), or NULL:
// the caller then launches the iterations directly.
static cudaGraphExec_t capture_fit(const gs2d_plan& p, void* ws, const float* target,
                                   float* params, float* m, float* v, int iters, cudaStream_t s) {
  cudaGraphExec_t exec = nullptr;
  if (s == nullptr || iters <= 0 || prime_fit_launches(p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    cudaError_t ce = fit_iteration(p, ws, target, params, m, v, s);
    cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (ce == cudaSuccess && ee == cudaSuccess && graph) {
      if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
  }
  cudaGetLastError();  // a failed capture falls back to plain launches
  return exec;
}

gs2d_status gs2d_fit_step(const gs2d_plan* plan, void* ws, const float* target, float* params,
                          float* adam_m, float* adam_v, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!target) return fail(GS2D_ERR_INVALID_ARG, "target is NULL");
  if (plan->n > 0 && (!params || !adam_m || !adam_v))
    return fail(GS2D_ERR_INVALID_ARG, "params or Adam state is NULL");
  return cuda_check(fit_iteration(*plan, ws, target, params, adam_m, adam_v, (cudaStream_t)stream),
                    "gs2d_fit_step");
}


// An auxiliary stream per host thread and device for the frame's upload, so
// that it overlaps the projection and binning (which need only the params).
// Created on the thread's first call on that device (one non-blocking stream
// and two events) and kept for the life of the process.
struct AuxStream {
  cudaStream_t stream = nullptr;
  cudaEvent_t start = nullptr, frame = nullptr;
};
constexpr int kAuxDevices = 64;

static cudaError_t aux_stream(AuxStream** out) {
  static thread_local AuxStream aux[kAuxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kAuxDevices) return cudaErrorInvalidDevice;
  AuxStream& a = aux[dev];
  if (!a.stream) {
    e = cudaStreamCreateWithFlags(&a.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.frame, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  *out = &a;
  return cudaSuccess;
}

gs2d_status gs2d_fit_step_rgb8(const gs2d_plan* plan, void* ws, const uint8_t* rgb_host,
                               uint8_t* rgb_dev, float* frame_dev, const float* params_host,
                               float* params, float* adam_m, float* adam_v, float* params_out_host,
                               void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  const gs2d_plan& p = *plan;
  if (p.num_clips != 1) return fail(GS2D_ERR_INVALID_ARG, "gs2d_fit_step_rgb8: one-clip plans only");
  if (!rgb_host || !rgb_dev || !frame_dev || (p.n > 0 && (!params || !adam_m || !adam_v)))
    return fail(GS2D_ERR_INVALID_ARG, "gs2d_fit_step_rgb8: NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t rgb_bytes = (size_t)3 * p.width * p.height;
  const size_t pbytes = (size_t)9 * p.n * sizeof(float);
  AuxStream* aux = nullptr;
  cudaError_t e = aux_stream(&aux);
  // the frame on the auxiliary stream, after everything queued on s so far
  // (the previous iteration's render reads frame_dev)
  if (e == cudaSuccess) e = cudaEventRecord(aux->start, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(aux->stream, aux->start, 0);
  // pinned host memory the device can address: the conversion reads it over
  // the host link itself, one pass instead of a copy and then a conversion;
  // other host memory goes through rgb_dev
  const uint8_t* src = rgb_dev;
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, rgb_host) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
      pa.devicePointer) {
    src = static_cast<const uint8_t*>(pa.devicePointer);
  } else {
    cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rgb_dev, rgb_host, rgb_bytes, cudaMemcpyHostToDevice, aux->stream);
  }
  if (e != cudaSuccess) return cuda_check(e, "gs2d_fit_step_rgb8");
  st = gs2d_frame_from_rgb8(src, p.width, p.height, (int64_t)3 * p.width, frame_dev,
                            aux->stream);
  if (st) return st;
  e = cudaEventRecord(aux->frame, aux->stream);
  // the params, projection and binning on s meanwhile
  if (e == cudaSuccess && params_host && pbytes)
    e = cudaMemcpyAsync(params, params_host, pbytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_prepare_fit(p, ws, params, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, aux->frame, 0);
  // pinned output the device can address: the Adam kernel stores the new
  // parameters there as well, in place of a download after it
  float* host_out = nullptr;
  if (params_out_host && pbytes) {
    if (cudaPointerGetAttributes(&pa, params_out_host) == cudaSuccess &&
        pa.type == cudaMemoryTypeHost && pa.devicePointer)
      host_out = static_cast<float*>(pa.devicePointer);
    else
      cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = launch_fit_step(p, ws, frame_dev, params, adam_m, adam_v, s, nullptr, host_out);
  if (e == cudaSuccess && params_out_host && pbytes && !host_out)
    e = cudaMemcpyAsync(params_out_host, params, pbytes, cudaMemcpyDeviceToHost, s);
  return cuda_check(e, "gs2d_fit_step_rgb8");
}

gs2d_status gs2d_fit_reset(const gs2d_plan* plan, void* ws, float* adam_m, float* adam_v,
                           void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (plan->n > 0 && (!adam_m || !adam_v)) return fail(GS2D_ERR_INVALID_ARG, "Adam state is NULL");
  return cuda_check(reset_fit(*plan, ws, adam_m, adam_v, (cudaStream_t)stream), "gs2d_fit_reset");
}

// Sets the optimiser state of the fit loop in the workspace header (a
// checkpoint's values) and marks the tile lists as not yet built.
__global__ void k_set_fit_state(WsHeader* __restrict__ hdr, int32_t step, double pw1, double pw2,
                                double pwd) {
  hdr->step = step;
  hdr->pw1 = pw1;
  hdr->pw2 = pw2;
  hdr->pwd = pwd;
  hdr->lists_valid = 0;
}

gs2d_status gs2d_fit_state_get(const gs2d_plan* plan, const void* ws, gs2d_fit_state* state,
                               void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!state) return fail(GS2D_ERR_INVALID_ARG, "state is NULL");
  WsHeader h;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&h, ws_ptr<WsHeader>(ws, *plan, kOffHeader), sizeof(h),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "gs2d_fit_state_get");
  memset(state, 0, sizeof(*state));
  state->step = h.step;
  state->beta1_pow = h.pw1;
  state->beta2_pow = h.pw2;
  state->decay_pow = h.pwd;
  return ok();
}

gs2d_status gs2d_fit_state_set(const gs2d_plan* plan, void* ws, const gs2d_fit_state* state,
                               void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!state || state->step < 0) return fail(GS2D_ERR_INVALID_ARG, "state is NULL or step < 0");
  k_set_fit_state<<<1, 1, 0, (cudaStream_t)stream>>>(ws_ptr<WsHeader>(ws, *plan, kOffHeader),
                                                     state->step, state->beta1_pow,
                                                     state->beta2_pow, state->decay_pow);
  return cuda_check(cudaGetLastError(), "gs2d_fit_state_set");
}

gs2d_status gs2d_fit_rebins(const gs2d_plan* plan, const void* ws, int64_t* rebins,
                            void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!rebins) return fail(GS2D_ERR_INVALID_ARG, "rebins is NULL");
  int32_t r = 0;
  const WsHeader* hdr = ws_ptr<WsHeader>(ws, *plan, kOffHeader);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&r, &hdr->rebins, sizeof(r), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "gs2d_fit_rebins");
  *rebins = r;
  return ok();
}

// Device-driven fit loop: the body of a conditional WHILE graph node is one
// fit iteration followed by this kernel.  It counts the iteration; every
// check_every iterations (and at the last) it sums the render's per-tile loss
// partials, writes the PSNR of the clamped image to the trace and clears the
// loop condition once the target is met, the cap is reached or a kernel has
// recorded an error.  The host reads the header and the trace once, at the
// end.
struct LoopArgs {
  int num_tiles, iters, check_every;
  float target_psnr;
  const float2* loss_part;
  WsHeader* hdr;
  float* trace;  // device, one float per check
  cudaGraphConditionalHandle handle;
};

__global__ void __launch_bounds__(1024) k_loop_control(LoopArgs a) {
  pdl_begin();
  __shared__ int s_it;
  __shared__ double s_a[32], s_b[32];
  if (threadIdx.x == 0) s_it = ++a.hdr->loop_iter;
  __syncthreads();
  const int it = s_it;
  if (it % a.check_every != 0 && it < a.iters) return;
  double x = 0.0, y = 0.0;
  for (int t = threadIdx.x; t < a.num_tiles; t += blockDim.x) {
    x += a.loss_part[t].x;
    y += a.loss_part[t].y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_a[wid] = x;
    s_b[wid] = y;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double sa = 0.0, sb = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
    sa += s_a[w];
    sb += s_b[w];
  }
  a.hdr->loss[0] = (float)sa;
  a.hdr->loss[1] = (float)sb;
  const double mse = (double)a.hdr->loss[1];
  const float psnr = mse > 0.0 ? (float)(10.0 * log10(1.0 / mse)) : INFINITY;
  a.trace[a.hdr->loop_checks++] = psnr;
  const bool stop = it >= a.iters || a.hdr->status != 0 ||
                    (a.target_psnr > 0.0f && psnr >= a.target_psnr);
  if (stop) cudaGraphSetConditional(a.handle, 0u);
}

// The whole fit loop as one executable graph: a WHILE node whose body is one
// fit iteration and k_loop_control; NULL when the stream cannot be captured,
// the trace does not fit the gradient scratch or the driver declines the
// graph (the caller then drives the loop from the host).
static cudaGraphExec_t capture_fit_loop(const gs2d_plan& p, void* ws, const float* target,
                                        float* params, float* m, float* v, int iters,
                                        int check_every, float target_psnr, cudaStream_t s) {
  const int checks = iters / check_every + 1;
  if (s == nullptr || iters <= 0 || (size_t)checks > (size_t)9 * p.n ||
      prime_fit_launches(p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle handle;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e == cudaSuccess)
    e = cudaGraphConditionalHandleCreate(&handle, graph, 1u, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  }
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t ce = fit_iteration(p, ws, target, params, m, v, s);
      if (ce == cudaSuccess) {
        LoopArgs la;
        la.num_tiles = p.num_tiles;
        la.iters = iters;
        la.check_every = check_every;
        la.target_psnr = target_psnr;
        la.loss_part = ws_ptr<float2>(ws, p, kOffLossPart);
        la.hdr = ws_ptr<WsHeader>(ws, p, kOffHeader);
        la.trace = ws_ptr<float>(ws, p, kOffGrad);
        la.handle = handle;
        ce = launch_pdl(k_loop_control, 1, 1024, 0, s, la);
      }
      cudaGraph_t captured = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(s, &captured);
      e = ce != cudaSuccess ? ce : ee;
    }
  }
  if (e == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  return exec;
}

gs2d_status gs2d_encode_frame(const gs2d_plan* plan, void* ws, const float* target, float* params,
                              float* adam_m, float* adam_v, int32_t iters, float target_psnr,
                              int32_t check_every, float* psnr_trace, int32_t* iters_done,
                              float* final_psnr, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!target) return fail(GS2D_ERR_INVALID_ARG, "target is NULL");
  if (plan->n > 0 && (!params || !adam_m || !adam_v))
    return fail(GS2D_ERR_INVALID_ARG, "params or Adam state is NULL");
  if (iters < 0 || check_every < 1) return fail(GS2D_ERR_INVALID_ARG, "iters / check_every");
  if (plan->num_clips != 1)
    return fail(GS2D_ERR_INVALID_ARG,
                "gs2d_encode_frame takes a one-clip plan (gs2d_encode_batch)");
  const gs2d_plan& p = *plan;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = reset_fit(p, ws, adam_m, adam_v, s);
  if (e != cudaSuccess) return cuda_check(e, "gs2d_encode_frame: reset");
  WsHeader* hdr = ws_ptr<WsHeader>(ws, p, kOffHeader);
  // the device drives the loop (one graph launch, one read at the end) ...
  cudaGraphExec_t loop = capture_fit_loop(p, ws, target, params, adam_m, adam_v, iters,
                                          check_every, target_psnr, s);
  if (loop) {
    e = cudaGraphLaunch(loop, s);
    WsHeader h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaGraphExecDestroy(loop);
    if (e != cudaSuccess) return cuda_check(e, "gs2d_encode_frame");
    const int checks = h.loop_checks;
    float last = 0.0f;
    if (checks > 0) {
      e = cudaMemcpy(&last, ws_ptr<float>(ws, p, kOffGrad) + (checks - 1), sizeof(float),
                     cudaMemcpyDeviceToHost);
      if (e == cudaSuccess && psnr_trace)
        e = cudaMemcpy(psnr_trace, ws_ptr<float>(ws, p, kOffGrad), (size_t)checks * sizeof(float),
                       cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_check(e, "gs2d_encode_frame: trace");
    }
    if (iters_done) *iters_done = h.loop_iter;
    if (final_psnr) *final_psnr = last;
    if (h.status != 0)
      return fail((gs2d_status)h.status, "device status %d after %d iterations", h.status,
                  h.loop_iter);
    return ok();
  }
  // ... or, where that graph is unavailable, the host polls every check_every
  cudaGraphExec_t exec = capture_fit(p, ws, target, params, adam_m, adam_v, iters, s);

  int done = 0, checks = 0;
  float psnr = 0.0f;
  gs2d_status result = GS2D_OK;
  while (done < iters) {
    const int k = std::min(check_every, iters - done);
    for (int it = 0; it < k && e == cudaSuccess; it++)
      e = exec ? cudaGraphLaunch(exec, s) : fit_iteration(p, ws, target, params, adam_m, adam_v, s);
    if (e != cudaSuccess) break;
    done += k;
    e = launch_loss_reduce(p, ws, nullptr, s);
    WsHeader h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    const double mse = h.loss[1];
    psnr = mse > 0.0 ? (float)(10.0 * log10(1.0 / mse)) : INFINITY;
    if (psnr_trace) psnr_trace[checks] = psnr;
    checks++;
    if (h.status != 0) {
      result = fail((gs2d_status)h.status, "device status %d after %d iterations", h.status, done);
      break;
    }
    if (target_psnr > 0.0f && psnr >= target_psnr) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (iters_done) *iters_done = done;
  if (final_psnr) *final_psnr = psnr;
  if (e != cudaSuccess) return cuda_check(e, "gs2d_encode_frame");
  if (result != GS2D_OK) return result;
  return ok();
}

gs2d_status gs2d_select_changed(const gs2d_plan* plan, void* ws, const float* reference,
                                const float* frame, float threshold, uint8_t* selected,
                                int32_t* n_selected, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!reference || !frame || (plan->n > 0 && !selected))
    return fail(GS2D_ERR_INVALID_ARG, "gs2d_select_changed: NULL pointer");
  if (!(threshold >= 0.0f)) return fail(GS2D_ERR_INVALID_ARG, "threshold must be >= 0");
  const gs2d_plan& p = *plan;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = p.n > 0 ? cudaMemsetAsync(selected, 0, (size_t)p.n, s) : cudaSuccess;
  if (e == cudaSuccess) e = launch_select_changed(p, ws, reference, frame, threshold, selected, s);
  if (e == cudaSuccess && n_selected) {
    int* cnt = ws_ptr<int>(ws, p, kOffActOrder) + p.num_tiles;  // free outside P-frame steps
    e = launch_count_flags(p.n, selected, cnt, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(n_selected, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  return cuda_check(e, "gs2d_select_changed");
}

static cudaError_t pframe_iteration(const gs2d_plan& p, void* ws, const float* target,
                                    float* params, float* m, float* v, const uint8_t* select,
                                    cudaStream_t s) {
  cudaError_t e = launch_prepare(p, ws, params, true, s);
  if (e == cudaSuccess) e = launch_pframe_step(p, ws, target, params, m, v, select, s);
  return e;
}

gs2d_status gs2d_pframe_step(const gs2d_plan* plan, void* ws, const float* target, float* params,
                             float* adam_m, float* adam_v, const uint8_t* selected,
                             void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!target || (plan->n > 0 && (!params || !adam_m || !adam_v || !selected)))
    return fail(GS2D_ERR_INVALID_ARG, "gs2d_pframe_step: NULL pointer");
  return cuda_check(pframe_iteration(*plan, ws, target, params, adam_m, adam_v, selected,
                                     (cudaStream_t)stream),
                    "gs2d_pframe_step");
}

gs2d_status gs2d_encode_pframe(const gs2d_plan* plan, void* ws, const float* target,
                               float* params, float* adam_m, float* adam_v,
                               const uint8_t* selected, int32_t iters, float* final_psnr,
                               void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!target || (plan->n > 0 && (!params || !adam_m || !adam_v || !selected)))
    return fail(GS2D_ERR_INVALID_ARG, "gs2d_encode_pframe: NULL pointer");
  if (iters < 0) return fail(GS2D_ERR_INVALID_ARG, "iters < 0");
  const gs2d_plan& p = *plan;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = reset_fit(p, ws, adam_m, adam_v, s);
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess && s != nullptr && iters > 0 && prime_fit_launches(p) == cudaSuccess) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t ce = pframe_iteration(p, ws, target, params, adam_m, adam_v, selected, s);
      cudaError_t ee = cudaStreamEndCapture(s, &graph);
      if (ce == cudaSuccess && ee == cudaSuccess && graph &&
          cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
    }
  }
  cudaGetLastError();  // a failed capture falls back to plain launches
  for (int it = 0; it < iters && e == cudaSuccess; it++)
    e = exec ? cudaGraphLaunch(exec, s)
             : pframe_iteration(p, ws, target, params, adam_m, adam_v, selected, s);
  if (exec) cudaGraphExecDestroy(exec);
  // full-frame PSNR of the result
  if (e == cudaSuccess) e = launch_prepare(p, ws, params, false, s);
  if (e == cudaSuccess)
    e = launch_render_l2(p, ws, params, target, ws_ptr<float>(ws, p, kOffGrad), nullptr,
                         nullptr, s);
  if (e == cudaSuccess) e = launch_loss_reduce(p, ws, nullptr, s);
  WsHeader h;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h, ws_ptr<WsHeader>(ws, p, kOffHeader), sizeof(h),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "gs2d_encode_pframe");
  if (final_psnr) {
    const double mse = h.loss[1];
    *final_psnr = mse > 0.0 ? (float)(10.0 * log10(1.0 / mse)) : INFINITY;
  }
  if (h.status != 0) return fail((gs2d_status)h.status, "device status %d", h.status);
  return ok();
}

gs2d_status gs2d_clip_losses(const gs2d_plan* plan, void* ws, float* out, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!out) return fail(GS2D_ERR_INVALID_ARG, "out is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_clip_losses(*plan, ws, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, ws_ptr<float2>(ws, *plan, kOffClipLoss),
                        (size_t)plan->num_clips * sizeof(float2), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_check(e, "gs2d_clip_losses");
}

gs2d_status gs2d_encode_batch(const gs2d_plan* plan, void* ws, const float* targets,
                              float* params, float* adam_m, float* adam_v, int32_t iters,
                              float* clip_psnr, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  if (!targets) return fail(GS2D_ERR_INVALID_ARG, "targets is NULL");
  if (plan->n > 0 && (!params || !adam_m || !adam_v))
    return fail(GS2D_ERR_INVALID_ARG, "params or Adam state is NULL");
  if (iters < 0) return fail(GS2D_ERR_INVALID_ARG, "iters < 0");
  const gs2d_plan& p = *plan;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = reset_fit(p, ws, adam_m, adam_v, s);
  cudaGraphExec_t exec = e == cudaSuccess ? capture_fit(p, ws, targets, params, adam_m, adam_v,
                                                        iters, s)
                                          : nullptr;
  for (int it = 0; it < iters && e == cudaSuccess; it++)
    e = exec ? cudaGraphLaunch(exec, s)
             : fit_iteration(p, ws, targets, params, adam_m, adam_v, s);
  if (exec) cudaGraphExecDestroy(exec);
  // evaluate the fitted Gaussians (gradients into the scratch section)
  if (e == cudaSuccess) e = launch_prepare(p, ws, params, false, s);
  if (e == cudaSuccess)
    e = launch_render_l2(p, ws, params, targets, ws_ptr<float>(ws, p, kOffGrad), nullptr,
                         nullptr, s);
  if (e == cudaSuccess) e = launch_clip_losses(p, ws, s);
  std::vector<float2> cl((size_t)p.num_clips);
  WsHeader h;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cl.data(), ws_ptr<float2>(ws, p, kOffClipLoss), cl.size() * sizeof(float2),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h, ws_ptr<WsHeader>(ws, p, kOffHeader), sizeof(h),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "gs2d_encode_batch");
  if (clip_psnr)
    for (int k = 0; k < p.num_clips; k++) {
      const double mse = cl[k].y;
      clip_psnr[k] = mse > 0.0 ? (float)(10.0 * log10(1.0 / mse)) : INFINITY;
    }
  if (h.status != 0) return fail((gs2d_status)h.status, "device status %d", h.status);
  return ok();
}

gs2d_status gs2d_read_bins(const gs2d_plan* plan, const void* ws, int64_t* n_entries,
                           uint32_t* keys, uint32_t* values, int64_t max_keys, int32_t* ranges,
                           int32_t* counts, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  const gs2d_plan& p = *plan;
  cudaStream_t s = (cudaStream_t)stream;
  WsHeader h;
  cudaError_t e = cudaMemcpyAsync(&h, ws_ptr<WsHeader>(ws, p, kOffHeader), sizeof(h),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "gs2d_read_bins");
  if (n_entries) *n_entries = h.n_entries;
  const int64_t k = std::min<int64_t>(h.n_entries, std::max<int64_t>(max_keys, 0));
  if (values && k > 0)
    e = cudaMemcpyAsync(values, ws_ptr<uint32_t>(ws, p, kOffList), k * sizeof(uint32_t),
                        cudaMemcpyDeviceToHost, s);
  std::vector<int2> rg((size_t)p.num_tiles);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(rg.data(), ws_ptr<int2>(ws, p, kOffRanges), rg.size() * sizeof(int2),
                        cudaMemcpyDeviceToHost, s);
  std::vector<int> offs;
  if (e == cudaSuccess && counts && p.n > 0) {
    offs.resize((size_t)p.n + 1);
    e = cudaMemcpyAsync(offs.data(), ws_ptr<int>(ws, p, kOffCount), offs.size() * sizeof(int),
                        cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "gs2d_read_bins");
  if (counts)
    for (int i = 0; i < p.n; i++) counts[i] = offs[i + 1] - offs[i];
  if (ranges)
    for (int t = 0; t < p.num_tiles; t++) {
      ranges[2 * t] = rg[t].x;
      ranges[2 * t + 1] = rg[t].y;
    }
  // the key of a list position is the tile whose range holds it
  if (keys)
    for (int t = 0; t < p.num_tiles; t++)
      for (int64_t i = rg[t].x; i < rg[t].y && i < k; i++) keys[i] = (uint32_t)t;
  return ok();
}

gs2d_status gs2d_count_pairs(const gs2d_plan* plan, void* ws, int64_t* pairs, int64_t* hits,
                             void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_count_pairs(*plan, ws, s);
  WsHeader h;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h, ws_ptr<WsHeader>(ws, *plan, kOffHeader), sizeof(h),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "gs2d_count_pairs");
  if (pairs) *pairs = (int64_t)h.pairs;
  if (hits) *hits = (int64_t)h.hits;
  return ok();
}

gs2d_status gs2d_ws_status(const gs2d_plan* plan, void* ws, int32_t reset, void* stream) {
  gs2d_status st = check_plan(plan, ws);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  WsHeader* hdr = ws_ptr<WsHeader>(ws, *plan, kOffHeader);
  int32_t status = 0;
  cudaError_t e = cudaMemcpyAsync(&status, &hdr->status, sizeof(status), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(&hdr->status, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(e, "gs2d_ws_status");
  if (status) return fail((gs2d_status)status, "device status %d", status);
  return ok();
}

gs2d_status gs2d_last_error(char* buf, size_t len) {
  if (!buf || len == 0) return GS2D_ERR_INVALID_ARG;
  strncpy(buf, g_err, len - 1);
  buf[len - 1] = 0;
  return GS2D_OK;
}

}  // extern "C"
