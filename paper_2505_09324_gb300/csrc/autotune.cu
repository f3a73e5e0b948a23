// Autotuner of the render schedule: for a given batch of clips, times one fit
// iteration (projection, binning, fused render + L2 + backward, per-Gaussian
// reduction) for every (tile edge, stage, launch form) candidate with CUDA
// events on the caller's stream and reports the fastest.  The schedule never
// changes a result (only which pixels and Gaussians a block handles together),
// so the choice is purely a matter of speed: small tiles waste less of each listed
// Gaussian's box on pixels it does not reach, large tiles list each Gaussian
// fewer times and share each staged batch among more pixels.
#include <math.h>
#include <stdio.h>

#include <vector>

#include "gs2d_internal.cuh"

using namespace gs2d;

namespace {

gs2d_status err(gs2d_status st, const char* what) { return set_error(st, what); }

}  // namespace

extern "C" uint64_t gs2d_autotune_ws_bytes(const gs2d_clip* clips, int32_t num_clips,
                                           int64_t max_entries, const gs2d_config* cfg,
                                           const int32_t* tiles, int32_t num_tiles_c) {
  if (!clips || num_clips < 1 || !tiles || num_tiles_c < 1) return 0;
  std::vector<gs2d_clip> tmp(clips, clips + num_clips);
  gs2d_config c;
  gs2d_config_default(&c);
  if (cfg) c = *cfg;
  uint64_t most = 0;
  for (int i = 0; i < num_tiles_c; i++) {
    c.tile = tiles[i];
    gs2d_plan p;
    if (gs2d_plan_init_batch(&p, tmp.data(), num_clips, max_entries, &c) != GS2D_OK) return 0;
    if (p.ws_bytes > most) most = p.ws_bytes;
  }
  return most;
}

extern "C" gs2d_status gs2d_autotune(gs2d_clip* clips, int32_t num_clips, int64_t max_entries,
                                     const gs2d_config* cfg, const float* params,
                                     const float* targets, void* ws, uint64_t ws_bytes,
                                     const int32_t* tiles, int32_t num_tiles_c,
                                     const int32_t* stages, int32_t num_stages,
                                     const int32_t* launches, int32_t num_launches, int32_t reps,
                                     float* ms, int32_t* best_tile, int32_t* best_stage,
                                     int32_t* best_launch, void* stream) {
  if (!clips || num_clips < 1 || !tiles || num_tiles_c < 1 || !stages || num_stages < 1 ||
      !launches || num_launches < 1 || !ms || reps < 1)
    return err(GS2D_ERR_INVALID_ARG, "gs2d_autotune: empty candidate list or bad arguments");
  if (!ws || (uintptr_t)ws % 256 || !targets)
    return err(GS2D_ERR_INVALID_ARG, "gs2d_autotune: NULL or misaligned workspace / targets");
  gs2d_config c;
  gs2d_config_default(&c);
  if (cfg) c = *cfg;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  float best = INFINITY;
  int bt = 0, bs = 0, bl = 0;
  gs2d_status result = GS2D_OK;
  char msg[256];
  for (int i = 0; i < num_tiles_c && e == cudaSuccess && result == GS2D_OK; i++) {
    for (int jl = 0; jl < num_stages * num_launches && e == cudaSuccess; jl++) {
      const int j = jl / num_launches, l = jl % num_launches;
      c.tile = tiles[i];
      c.stage = stages[j];
      c.launch = launches[l];
      gs2d_plan p;
      result = gs2d_plan_init_batch(&p, clips, num_clips, max_entries, &c);
      if (result != GS2D_OK) break;
      if (p.n > 0 && !params) {
        result = err(GS2D_ERR_INVALID_ARG, "gs2d_autotune: params is NULL");
        break;
      }
      if (p.ws_bytes > ws_bytes) {
        snprintf(msg, sizeof(msg), "gs2d_autotune: workspace of %llu bytes, tile %d needs %llu",
                 (unsigned long long)ws_bytes, c.tile, (unsigned long long)p.ws_bytes);
        result = err(GS2D_ERR_INVALID_ARG, msg);
        break;
      }
      e = cudaMemsetAsync(ws, 0, p.ws_bytes, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws_ptr<gs2d_clip>(ws, p, kOffClips), clips,
                            (size_t)num_clips * sizeof(gs2d_clip), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // clips is host memory
      if (e == cudaSuccess) e = prime_fit_launches(p);
      float* grads = ws_ptr<float>(ws, p, kOffGrad);
      for (int it = 0; it < reps + 2 && e == cudaSuccess; it++) {
        if (it == 2) e = cudaEventRecord(ev[0], s);
        if (e == cudaSuccess) e = launch_prepare(p, ws, params, false, s);
        if (e == cudaSuccess)
          e = launch_render_l2(p, ws, params, targets, grads, nullptr, nullptr, s);
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
      float t = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
      int32_t status = 0;
      if (e == cudaSuccess)
        e = cudaMemcpy(&status, ws_ptr<WsHeader>(ws, p, kOffHeader), sizeof(status),
                       cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) break;
      const float per = status == 0 ? t / (float)reps : -1.0f;
      ms[i * num_stages * num_launches + jl] = per;
      if (per >= 0.0f && per < best) {
        best = per;
        bt = c.tile;
        bs = c.stage;
        bl = c.launch;
      }
    }
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (result != GS2D_OK) return result;
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "gs2d_autotune: %s", cudaGetErrorString(e));
    return err(GS2D_ERR_CUDA, msg);
  }
  if (!(best < INFINITY))
    return err(GS2D_ERR_CAPACITY, "gs2d_autotune: every candidate exceeded max_entries");
  if (best_tile) *best_tile = bt;
  if (best_stage) *best_stage = bs;
  if (best_launch) *best_launch = bl;
  return err(GS2D_OK, "");
}
