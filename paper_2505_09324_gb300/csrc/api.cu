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

gs2d_status check_plan(const gs2d_plan* p, const void* ws) {
  if (!p || p->magic != kPlanMagic) return fail(GS2D_ERR_INVALID_ARG, "plan not initialised");
  if (!ws) return fail(GS2D_ERR_INVALID_ARG, "workspace is NULL");
  if ((uintptr_t)ws % 256 != 0) return fail(GS2D_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  return GS2D_OK;
}

bool cfg_valid(const gs2d_config& c) {
  return c.tile == kTile && c.sigma_cut > 0.0f && isfinite(c.sigma_cut) && c.alpha_min > 0.0f &&
         isfinite(c.alpha_min) && c.det_eps >= 0.0f && isfinite(c.det_eps) && c.lr > 0.0f &&
         isfinite(c.lr) && c.beta1 >= 0.0f && c.beta1 < 1.0f && c.beta2 >= 0.0f &&
         c.beta2 < 1.0f && c.eps > 0.0f && isfinite(c.eps);
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
  cfg->tile = kTile;
  cfg->sigma_cut = 4.5f;
  cfg->alpha_min = 1.0f / 255.0f;
  cfg->det_eps = 1e-8f;
  cfg->lr = 1e-2f;
  cfg->beta1 = 0.9f;
  cfg->beta2 = 0.999f;
  cfg->eps = 1e-8f;
}

size_t gs2d_sizeof_plan(void) { return sizeof(gs2d_plan); }
size_t gs2d_sizeof_config(void) { return sizeof(gs2d_config); }

gs2d_status gs2d_plan_init(gs2d_plan* plan, int32_t width, int32_t height, int32_t n,
                           int64_t max_entries, const gs2d_config* cfg) {
  if (!plan) return fail(GS2D_ERR_INVALID_ARG, "plan is NULL");
  memset(plan, 0, sizeof(*plan));
  gs2d_config c;
  gs2d_config_default(&c);
  if (cfg) c = *cfg;
  if (!cfg_valid(c)) return fail(GS2D_ERR_INVALID_ARG, "invalid config (tile must be 16)");
  if (width < 1 || height < 1 || width > 65536 || height > 65536)
    return fail(GS2D_ERR_INVALID_ARG, "image size %d x %d out of range", width, height);
  if (n < 0 || n > (1 << 28)) return fail(GS2D_ERR_INVALID_ARG, "n = %d out of range", n);
  if (max_entries == 0) max_entries = std::max<int64_t>(1 << 20, 16 * (int64_t)n);
  if (max_entries < 1 || max_entries > (int64_t(1) << 30))
    return fail(GS2D_ERR_INVALID_ARG, "max_entries = %lld out of range", (long long)max_entries);
  const int tx = (width + kTile - 1) / kTile, ty = (height + kTile - 1) / kTile;
  plan->width = width;
  plan->height = height;
  plan->n = n;
  plan->tile = kTile;
  plan->tiles_x = tx;
  plan->tiles_y = ty;
  plan->num_tiles = tx * ty;
  int bits = 0;
  while ((int64_t(1) << bits) < plan->num_tiles) bits++;
  plan->tile_bits = bits;
  plan->sort_passes = 1;  // one counting pass over the whole tile id
  plan->sort_blocks = 0;
  plan->max_entries = max_entries;
  plan->cfg = c;
  const uint64_t nn = (uint64_t)n, me = (uint64_t)max_entries, nt = (uint64_t)plan->num_tiles;
  uint64_t sz[kNumSections];
  sz[kOffHeader] = sizeof(WsHeader);
  sz[kOffRec] = 3 * nn * sizeof(float4);
  sz[kOffRect] = nn * sizeof(int4);
  sz[kOffCount] = (nn + 1) * sizeof(int);
  sz[kOffBlockSum] = (nn / 256 + 1) * sizeof(long long);
  sz[kOffTileCnt] = nt * sizeof(int);
  sz[kOffCursor] = nt * sizeof(int);
  sz[kOffLong] = (nt + 1) * sizeof(int);
  sz[kOffList] = me * sizeof(uint32_t);
  sz[kOffRanges] = nt * sizeof(int2);
  sz[kOffPartial] = me * kPartials * sizeof(float);
  sz[kOffLossPart] = nt * sizeof(float2);
  sz[kOffGrad] = 9 * nn * sizeof(float);
  uint64_t off = 0;
  for (int s = 0; s < kNumSections; s++) {
    plan->off[s] = off;
    off = align256(off + sz[s]);
  }
  plan->ws_bytes = off;
  plan->magic = kPlanMagic;
  return ok();
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

gs2d_status gs2d_roi_init(const float* frame, const uint8_t* mask, int32_t width, int32_t height,
                          int32_t n, float roi_frac, const float* bg_xy, float* params,
                          int32_t* n_roi, void* scratch, uint64_t scratch_bytes, void* stream) {
  if (width < 1 || height < 1 || width > 65536 || height > 65536 || n < 0 || n > (1 << 28))
    return fail(GS2D_ERR_INVALID_ARG, "gs2d_roi_init: sizes out of range");
  if (!(roi_frac >= 0.0f && roi_frac <= 1.0f))
    return fail(GS2D_ERR_INVALID_ARG, "gs2d_roi_init: roi_frac must be in [0, 1]");
  if (!frame || !mask || (n > 0 && (!params || !bg_xy)) || !scratch)
    return fail(GS2D_ERR_INVALID_ARG, "gs2d_roi_init: NULL pointer");
  if ((uintptr_t)scratch % 256) return fail(GS2D_ERR_INVALID_ARG, "scratch not 256-byte aligned");
  char msg[256] = "";
  const gs2d_status st = roi_init(frame, mask, width, height, n, roi_frac, bg_xy, params, n_roi,
                                  scratch, scratch_bytes, (cudaStream_t)stream, msg, sizeof(msg));
  if (st != GS2D_OK) return fail(st, "%s", msg);
  return ok();
}

static cudaError_t fit_iteration(const gs2d_plan& p, void* ws, const float* target, float* params,
                                 float* m, float* v, cudaStream_t s) {
  cudaError_t e = launch_prepare(p, ws, params, true, s);
  if (e == cudaSuccess) e = launch_fit_step(p, ws, target, params, m, v, s);
  return e;
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
  const gs2d_plan& p = *plan;
  cudaStream_t s = (cudaStream_t)stream;
  WsHeader* hdr = ws_ptr<WsHeader>(ws, p, kOffHeader);
  const size_t pbytes = (size_t)9 * p.n * sizeof(float);
  cudaError_t e = cudaSuccess;
  if (pbytes) e = cudaMemsetAsync(adam_m, 0, pbytes, s);
  if (e == cudaSuccess && pbytes) e = cudaMemsetAsync(adam_v, 0, pbytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s);
  if (e != cudaSuccess) return cuda_check(e, "gs2d_encode_frame: reset");

  cudaGraphExec_t exec = nullptr;
  if (s != nullptr && iters > 0) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t ce = fit_iteration(p, ws, target, params, adam_m, adam_v, s);
      cudaError_t ee = cudaStreamEndCapture(s, &graph);
      if (ce == cudaSuccess && ee == cudaSuccess && graph) {
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();  // a failed capture falls back to plain launches
  }

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
