// Internal definitions shared by the gs2d CUDA translation units (not part of
// the C ABI).  Workspace layout, the per-Gaussian render record, status codes
// and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs2d.h"

namespace gs2d {

constexpr uint64_t kPlanMagic = 0x67733264706c616eull;  // "gs2dplan"
constexpr int kTileDefault = 16;   // tile edge (pixels)
constexpr int kStageDefault = 64;  // Gaussians per shared-memory batch
constexpr int kPartials = 8;       // backward accumulators per (tile, Gaussian)
constexpr int kBuckets = 16;       // list-length classes of the render queue

constexpr float kLn2 = 0.69314718055994530942f;

// Workspace sections (byte offsets stored in gs2d_plan::off).
enum WsSection {
  kOffHeader = 0,   // WsHeader
  kOffClips,        // gs2d_clip[num_clips] (batch plans)
  kOffRec,          // float4[3][n]  render records (SoA of float4 rows)
  kOffRect,         // int4[n]       tile rectangle (first tile, row stride, w, h)
  kOffCount,        // int32[n + 1]  per-Gaussian tile counts, then exclusive offsets
  kOffBlockSum,     // int64[n / 32 + 1]  entry counts per block of Gaussians
  kOffTileCnt,      // int32[num_tiles]  entries per tile (zero between calls)
  kOffCursor,       // int32[num_tiles]  next free slot of each tile's list
  kOffLong,         // int32[num_tiles + 1]  tiles whose list needs the CTA sort
  kOffList,         // uint32[max_entries]  Gaussian indices, tile-major
  kOffRanges,       // int2[num_tiles]
  kOffOrder,        // int32[num_tiles]  render queue: tiles, longest list first
  kOffRank,         // uint32[num_tiles]  (class << 28 | rank in class) of each tile
  kOffBucket,       // int32[2][kBuckets]  queue class sizes (zero between calls)
  kOffPartial,      // float[max_entries][kPartials] backward sums per (tile, Gaussian)
  kOffLossPart,     // float2[num_tiles]  per-tile (sse, clamped sse) / (3 W H of the clip)
  kOffClipLoss,     // float2[num_clips]
  kOffActive,       // uint8[num_tiles] P-frame: tile touched by a selected Gaussian
  kOffActOrder,     // int32[num_tiles + 1] P-frame: active tiles (count last)
  kOffQuant,        // float[9 n] quantisation-aware fitting: the fake-quantised parameters
  kOffGrad,         // float[9 n] gradient scratch
  kOffLRect,        // int4[n]  fit loop: the (widened) rectangle each Gaussian is listed in
  kOffTileCnt2,     // int32[num_tiles]  fit loop: tight-rectangle entries per tile (zero
                    //                   between calls; the fallback of a list rebuild)
  kOffAcc,          // float[n][kPartials]  GS2D_REDUCE_ATOMIC: per-Gaussian backward sums
                    //                      (zero between calls)
  kNumSections
};
static_assert(kNumSections <= 24, "gs2d_plan::off holds 24 sections");

struct WsHeader {
  int32_t status;       // first device-detected error (gs2d_status), 0 if none
  int32_t n_entries;    // entries in the sorted list (0 when over capacity)
  int64_t entries_raw;  // total entries requested by the tile counts
  int32_t step;         // Adam step counter of the fit loop
  float bc1, bc2;       // Adam bias corrections for that step
  int32_t long_count;   // tiles queued for the long-list sort
  float loss[2];        // last reduced {loss, clamped mse}
  unsigned long long pairs, hits;  // gs2d_count_pairs results
  double pw1, pw2;      // beta1^step, beta2^step
  int32_t queue;        // next render-queue ticket (reset by the last block)
  int32_t done;         // render blocks that have left the queue
  double pwd;           // lr_decay^(step - 1)
  float lr_now;         // lr * lr_decay^(step - 1)
  int32_t lists_valid;  // the fit loop's tile lists hold every Gaussian's box
  int32_t rebins;       // times the fit loop rebuilt its lists
  int32_t lists_tight;  // the last rebuild listed tight rectangles (widened ones overflowed)
  int32_t loop_iter;    // device-driven fit loop: iterations run
  int32_t loop_checks;  // device-driven fit loop: PSNR checks made
  int32_t pad[36];
};
static_assert(sizeof(WsHeader) == 256, "header is one 256-byte block");

// The clips a kernel sees: a one-clip plan passes its clip by value, a batch
// the device table (clips ordered by g_off and tile_off).
struct ClipSet {
  int count;
  const gs2d_clip* table;
  gs2d_clip one;
};

// Clip owning Gaussian i: the last clip whose g_off <= i (clips without
// Gaussians share g_off with their successor, which then owns i).
__device__ __forceinline__ gs2d_clip clip_of_gaussian(const ClipSet& cs, int i) {
  if (cs.count == 1) return cs.one;
  int lo = 0, hi = cs.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cs.table[mid].g_off <= i) lo = mid; else hi = mid - 1;
  }
  return cs.table[lo];
}

// Clip owning global tile t (every clip has at least one tile).
__device__ __forceinline__ gs2d_clip clip_of_tile(const ClipSet& cs, int t) {
  if (cs.count == 1) return cs.one;
  int lo = 0, hi = cs.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cs.table[mid].tile_off <= t) lo = mid; else hi = mid - 1;
  }
  return cs.table[lo];
}

// Per-Gaussian render record, three float4 rows.
//   r0 = (mu_x, mu_y, a1, a2)      a1 = s/l1, a2 = s/l3, s = sqrt(log2(e)/2)
//   r1 = (kappa, tau2, c'_r, c'_g) kappa = -(l2/l3) a1, tau2 = tau * log2(e), c' = w c
//   r2 = (c'_b, hx, hy, 0)         half extents of the tau-ellipse (+ slack)
// With dx = px - mu_x, dy = py - mu_y (Eq. 1: Sigma^-1 = L^-T L^-1):
//   u1 = a1 dx, u2 = a2 dy + kappa dx, q = u1^2 + u2^2 = sigma log2(e),
//   contribution c' 2^-q if q <= tau2.
struct Rec {
  float4 r0, r1, r2;
};

template <typename T>
__host__ __device__ inline T* ws_ptr(void* ws, const gs2d_plan& p, int sec) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + p.off[sec]);
}
template <typename T>
__host__ __device__ inline const T* ws_ptr(const void* ws, const gs2d_plan& p, int sec) {
  return reinterpret_cast<const T*>(static_cast<const char*>(ws) + p.off[sec]);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Programmatic dependent launch (sm_90 and later).  A kernel started by
// launch_pdl may become resident while its predecessor on the stream is still
// running; its first statement must be pdl_begin(), which waits until the
// predecessor has completed and its writes are visible, then lets the next
// kernel start launching.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, A... args) {
  cudaLaunchConfig_t c = {};
  c.gridDim = grid;
  c.blockDim = block;
  c.dynamicSmemBytes = smem;
  c.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  c.attrs = at;
#ifdef GS2D_NO_PDL
  c.numAttrs = 0;
#else
  c.numAttrs = 1;
#endif
  return cudaLaunchKernelEx(&c, kernel, static_cast<P>(args)...);
}

__device__ __forceinline__ void set_status(WsHeader* h, int code) {
  atomicCAS(&h->status, 0, code);
}

// Projection of Gaussian i (Sec. 3.1 parameters -> screen-space record, tile
// rectangle and tile count) in the frame of its clip.  The rectangle uses only
// single-rounded operations (no FMA contraction) so it is reproducible on the
// host; the rest of the record is ordinary FP32.  Culled Gaussians
// (non-finite, det <= det_eps, |w| < alpha_min, off-image) get count 0.
// The rectangle is stored as (first tile, tile-row stride, width, height) in
// the plan's tile numbering: tile (x0 + dx, y0 + dy) of the clip is
// first + dy * stride + dx.
// Tile rectangle [tx0, tx1) x [ty0, ty1) of Gaussian i in its clip: the pixel
// span of the bounding box of its cut-off ellipse (sigma <= sigma_cut reaches
// sqrt(2 sigma_cut Sxx) along x and sqrt(2 sigma_cut Syy) along y: 3 sqrt(Sxx),
// 3 sqrt(Syy) at 4.5), widened by `margin` pixels, clipped to the clip.  false
// when the Gaussian is culled (non-finite, degenerate, too faint) or off the
// clip.  Single-rounded FP32 operations (the oracle's rule).
__device__ __forceinline__ bool gaussian_tiles(int i, int n, const gs2d_clip& cl, int tile_shift,
                                               float sigma_cut, float alpha_min, float det_eps,
                                               const float* __restrict__ params, float margin,
                                               int& tx0, int& ty0, int& tx1, int& ty1) {
  const int W = cl.width, H = cl.height;
  const float mx = params[i], my = params[n + i];
  const float l1 = params[2 * n + i], l2 = params[3 * n + i], l3 = params[4 * n + i];
  const float cr = params[5 * n + i], cg = params[6 * n + i], cb = params[7 * n + i];
  const float w = params[8 * n + i];
  const bool finite = isfinite(mx) && isfinite(my) && isfinite(l1) && isfinite(l2) &&
                      isfinite(l3) && isfinite(cr) && isfinite(cg) && isfinite(cb) && isfinite(w);
  const float sxx = __fmul_rn(l1, l1);
  const float syy = __fadd_rn(__fmul_rn(l2, l2), __fmul_rn(l3, l3));
  const float a = __fmul_rn(l1, l3);
  const float det = __fmul_rn(a, a);
  if (!(finite && (det > det_eps) && (fabsf(w) >= alpha_min))) return false;
  const float kc = __fsqrt_rn(__fmul_rn(2.0f, sigma_cut));
  const float rx = __fadd_rn(ceilf(__fmul_rn(kc, __fsqrt_rn(sxx))), margin);
  const float ry = __fadd_rn(ceilf(__fmul_rn(kc, __fsqrt_rn(syy))), margin);
  float fx0 = floorf(__fsub_rn(mx, rx)), fx1 = floorf(__fadd_rn(mx, rx));
  float fy0 = floorf(__fsub_rn(my, ry)), fy1 = floorf(__fadd_rn(my, ry));
  fx0 = fx0 < 0.0f ? 0.0f : fx0;
  fy0 = fy0 < 0.0f ? 0.0f : fy0;
  fx1 = fx1 > (float)(W - 1) ? (float)(W - 1) : fx1;
  fy1 = fy1 > (float)(H - 1) ? (float)(H - 1) : fy1;
  if (!(fx0 <= fx1 && fy0 <= fy1)) return false;
  tx0 = (int)fx0 >> tile_shift;
  ty0 = (int)fy0 >> tile_shift;
  tx1 = ((int)fx1 >> tile_shift) + 1;
  ty1 = ((int)fy1 >> tile_shift) + 1;
  return true;
}

// The render record of Gaussian i (zeros when it is not visible).
__device__ __forceinline__ void write_record(int i, int n, bool visible, float sigma_cut,
                                             float alpha_min, const float* __restrict__ params,
                                             float4* __restrict__ rec) {
  float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
  if (visible) {
    const float mx = params[i], my = params[n + i];
    const float l1 = params[2 * n + i], l2 = params[3 * n + i], l3 = params[4 * n + i];
    const float cr = params[5 * n + i], cg = params[6 * n + i], cb = params[7 * n + i];
    const float w = params[8 * n + i];
    const float sxx = __fmul_rn(l1, l1);
    const float syy = __fadd_rn(__fmul_rn(l2, l2), __fmul_rn(l3, l3));
    const float s = 0.84932180028801904272f;  // sqrt(log2(e) / 2)
    const float log2e = 1.44269504088896340736f;
    float tau2 = fminf(sigma_cut * log2e, log2f(fabsf(w) / alpha_min));
    tau2 = fmaxf(tau2, 0.0f);
    const float tau = tau2 * kLn2;
    // half extents of {sigma <= tau}: sqrt(2 tau Sxx), sqrt(2 tau Syy), padded so
    // the box stays conservative under FP32 rounding
    const float hx = sqrtf(2.0f * tau * sxx) * 1.001f + 0.0039f;
    const float hy = sqrtf(2.0f * tau * syy) * 1.001f + 0.0039f;
    const float a1 = s / l1;
    r0 = make_float4(mx, my, a1, s / l3);
    r1 = make_float4((-l2 / l3) * a1, tau2, w * cr, w * cg);
    r2 = make_float4(w * cb, hx, hy, 0.0f);
  }
  rec[i] = r0;
  rec[n + i] = r1;
  rec[2 * n + i] = r2;
}

__device__ __forceinline__ void project_one(int i, int n, const gs2d_clip& cl, int tile_shift,
                                            float sigma_cut, float alpha_min, float det_eps,
                                            const float* __restrict__ params,
                                            float4* __restrict__ rec, int4* __restrict__ rect,
                                            int* __restrict__ count) {
  int tx0 = 0, ty0 = 0, tx1 = 0, ty1 = 0;
  const bool vis = gaussian_tiles(i, n, cl, tile_shift, sigma_cut, alpha_min, det_eps, params,
                                  0.0f, tx0, ty0, tx1, ty1);
  const int4 rc = vis ? make_int4(cl.tile_off + ty0 * cl.tiles_x + tx0, cl.tiles_x, tx1 - tx0,
                                  ty1 - ty0)
                      : make_int4(0, 0, 0, 0);
  rect[i] = rc;
  count[i] = rc.z * rc.w;
  write_record(i, n, vis, sigma_cut, alpha_min, params, rec);
}

__host__ __device__ inline int tile_shift_of(int tile) {
  return tile == 8 ? 3 : (tile == 32 ? 5 : 4);
}

// Clip set of a plan (the table lives in the workspace of a batch plan).
inline ClipSet clip_set(const gs2d_plan& p, const void* ws) {
  ClipSet cs;
  cs.count = p.num_clips;
  cs.table = ws_ptr<gs2d_clip>(ws, p, kOffClips);
  cs.one = gs2d_clip{p.width, p.height, p.n, p.tiles_x, p.tiles_y, 0, 0, 0, 0};
  return cs;
}

// Arguments of the render kernels (csrc/render_impl.cuh).
enum RenderMode { kModeFwd = 0, kModeBwd = 1, kModeL2 = 2, kModeCount = 3, kModeSelect = 4 };

struct RenderArgs {
  ClipSet clips;
  int n, num_tiles;
  const int2* ranges;
  const uint32_t* list;
  const float4* rec;
  const int4* rect;
  const int* offs;
  const int* order;
  WsHeader* hdr;
  float* img;            // fwd, l2 (optional)
  const float* target;   // l2
  const float* dimg;     // bwd
  float* partial;        // bwd, l2
  float2* loss_part;     // l2
  const int* active;     // device count of tiles in `order` to render, or NULL (all)
  const float* ref;      // select: reference render
  const float* frame;    // select: current frame
  float threshold;       // select: change threshold on max_c |ref - frame|
  uint8_t* selected;     // select: per-Gaussian flag out
  float* acc;            // bwd, l2 with GS2D_REDUCE_ATOMIC: per-Gaussian sums (else NULL:
                         // one record per pair in `partial`)
};

// One instantiation set per tile edge (render_t8.cu, render_t16.cu, render_t32.cu).
cudaError_t launch_render_t8(int stage, int launch, RenderMode mode, const RenderArgs& a,
                              cudaStream_t s);
cudaError_t launch_render_t16(int stage, int launch, RenderMode mode, const RenderArgs& a,
                              cudaStream_t s);
cudaError_t launch_render_t32(int stage, int launch, RenderMode mode, const RenderArgs& a,
                              cudaStream_t s);

cudaError_t prime_render_t8(int stage, int launch);
cudaError_t prime_render_t16(int stage, int launch);
cudaError_t prime_render_t32(int stage, int launch);
// One-time per-device setup of the binning launches (shared-memory opt-in).
cudaError_t prime_binning();
// prime_binning + the render occupancy query of the plan's fit loop.
cudaError_t prime_fit_launches(const gs2d_plan& p);

// Opt-in to `bytes` of dynamic shared memory for `kernel` on the current
// device (once per kernel and device; thread-safe).
cudaError_t opt_in_smem(const void* kernel, int bytes);
// Thread blocks of a persistent launch: resident blocks per SM x SMs of the
// current device, at most `work` blocks.
int persistent_grid(const void* kernel, int threads, int work);

// ---- launchers implemented in the .cu files (return cudaGetLastError) ----
cudaError_t launch_project(const gs2d_plan& p, void* ws, const float* params, cudaStream_t s);
cudaError_t launch_bin_sort(const gs2d_plan& p, void* ws, cudaStream_t s);
cudaError_t launch_render_fwd(const gs2d_plan& p, void* ws, float* img, cudaStream_t s);
cudaError_t launch_render_bwd(const gs2d_plan& p, void* ws, const float* params,
                              const float* dimg, float* grads, cudaStream_t s);
cudaError_t launch_render_l2(const gs2d_plan& p, void* ws, const float* params,
                             const float* target, float* grads, float* img, float* loss,
                             cudaStream_t s);
// Follows launch_prepare_fit (it marks retained lists valid).  params_eval:
// the values the render used, when they differ from params (the chain rule is
// taken there; Adam updates params).  host_out: a device view of pinned host
// memory that receives the parameters after the step, or NULL.
cudaError_t launch_fit_step(const gs2d_plan& p, void* ws, const float* target, float* params,
                            float* m, float* v, cudaStream_t s,
                            const float* params_eval = nullptr, float* host_out = nullptr);
cudaError_t launch_adam(float* params, const float* grads, float* m, float* v, int64_t count,
                        int32_t step, const uint8_t* mask, const gs2d_config& cfg,
                        cudaStream_t s);
cudaError_t launch_loss_reduce(const gs2d_plan& p, void* ws, float* loss, cudaStream_t s);
cudaError_t launch_count_pairs(const gs2d_plan& p, void* ws, cudaStream_t s);
cudaError_t launch_clip_losses(const gs2d_plan& p, void* ws, cudaStream_t s);
cudaError_t launch_select_changed(const gs2d_plan& p, void* ws, const float* ref,
                                  const float* frame, float threshold, uint8_t* selected,
                                  cudaStream_t s);
cudaError_t launch_count_flags(int n, const uint8_t* flags, int* out, cudaStream_t s);
// Quantisation (quant.cu): codes, dequantised values and ranges of params.
cudaError_t launch_quantize(const float* params, int n, const gs2d_quant& q, uint16_t* codes,
                            float* dequant, float* ranges, cudaStream_t s);
cudaError_t launch_pframe_step(const gs2d_plan& p, void* ws, const float* target,
                               float* params, float* m, float* v, const uint8_t* select,
                               cudaStream_t s);
// project + bin_sort; with adam_tick the fit loop's Adam step counter and bias
// corrections advance in the same launch.
cudaError_t launch_prepare(const gs2d_plan& p, void* ws, const float* params, bool adam_tick,
                           cudaStream_t s);
// The fit loop's projection and binning (Adam tick included): tile lists kept
// across iterations and rebuilt only when a Gaussian leaves them
// (cfg.bin_margin >= 0), else launch_prepare.
inline bool fit_lists_retained(const gs2d_config& c) { return c.bin_margin >= 0.0f; }
cudaError_t launch_prepare_fit(const gs2d_plan& p, void* ws, const float* params,
                               cudaStream_t s);

uint64_t roi_init_scratch_bytes(int W, int H, int n);
// cen_trace / label_trace (device, or NULL): per K-means iteration the
// centres the assignment used ([10][5][n]) and the labels it made ([10][H][W]).
constexpr int kRoiIterations = 10;
gs2d_status roi_init(const float* frame, const uint8_t* mask, int W, int H, int n, float roi_frac,
                     const float* bg_xy, float* params, int32_t* n_roi, void* scratch,
                     uint64_t scratch_bytes, cudaStream_t s, char* err, size_t err_len,
                     float* cen_trace = nullptr, int32_t* label_trace = nullptr);

// Records msg as the calling thread's last error (gs2d_last_error); returns st.
gs2d_status set_error(gs2d_status st, const char* msg);

}  // namespace gs2d
