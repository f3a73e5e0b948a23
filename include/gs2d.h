/*
 * gs2d.h -- C ABI of the GB300 (sm_103a) 2D Gaussian-splatting frame encoder.
 *
 * The library implements the hot path of the video encoder of "Neural Video
 * Compression using 2D Gaussian Splatting" (arXiv 2505.09324): fitting N 2D
 * Gaussians to a frame by gradient steps (Sec. 3.2 A), through a
 * differentiable tile-based rasterizer (Sec. 3) that blends by the
 * accumulated-sum rule of Eq. 2 over Gaussians parametrised by mean, Cholesky
 * factor (Eq. 1) and colour (Sec. 3.1).
 *
 * Conventions shared by every call
 * --------------------------------
 * Parameters: one float32 array of 9*n values, structure-of-arrays, row r at
 *   params + r*n, rows (mu_x, mu_y, l1, l2, l3, c_r, c_g, c_b, w).  mu is in
 *   pixels; L = [[l1, 0], [l2, l3]] and Sigma = L L^T (Eq. 1); the colour
 *   coefficient c'_n of Eq. 2 is w_n * c_n.
 * Images: float32 [3][H][W] planar, pixel (x, y) centred at (x + 0.5, y + 0.5).
 * Blending (Eq. 2): C(p) = sum_n w_n c_n exp(-sigma_n(p)) with
 *   sigma_n(p) = 1/2 (p - mu_n)^T Sigma_n^{-1} (p - mu_n), over the Gaussians
 *   with finite parameters, det Sigma > det_eps and sigma_n(p) <= tau_n,
 *   tau_n = min(sigma_cut, ln(|w_n| / alpha_min)); ascending n, FP32.
 * Memory: the caller allocates and owns every buffer.  Pointers marked
 *   "device" must be CUDA device (or managed) memory on the current device;
 *   "host" pointers are ordinary host memory.  The library allocates no device
 *   memory.  `ws` is a device workspace of gs2d_plan.ws_bytes bytes, 256-byte
 *   aligned, laid out by gs2d_plan_init, and zero-filled by the caller before
 *   its first use (its status word must start at GS2D_OK); one workspace serves
 *   one plan and one stream at a time.
 * Streams: every device call is asynchronous and ordered on `stream`
 *   (a cudaStream_t passed as void*; NULL is the legacy default stream).
 * Errors: argument errors are detected on the host and returned at once
 *   (GS2D_ERR_INVALID_ARG).  Launch failures return GS2D_ERR_CUDA.  Errors
 *   found by kernels (entry capacity exceeded) are recorded in a status word in
 *   the workspace; gs2d_ws_status() reads it (synchronising the stream).
 *   gs2d_last_error() returns a message for the calling thread's last error.
 */
#ifndef GS2D_H
#define GS2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS2D_OK = 0,
  GS2D_ERR_INVALID_ARG = 1, /* bad size, pointer, plan or alignment        */
  GS2D_ERR_CUDA = 2,        /* a CUDA call or kernel launch failed          */
  GS2D_ERR_CAPACITY = 3,    /* more (tile, Gaussian) pairs than max_entries */
  GS2D_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up           */
  GS2D_ERR_BOUNDS = 5       /* a device-side bounds check failed            */
} gs2d_status;

/* Rasterizer and optimiser constants.  The paper fixes none of them; these
 * are the project's readings (gs2d_config_default): tile 16, stage 64,
 * launch GS2D_LAUNCH_GRID, learning-rate scales and decay 1,
 * sigma_cut 4.5 (the 3-sigma ellipse), alpha_min 1/255, det_eps 1e-8, Adam
 * lr 1e-2, betas (0.9, 0.999), eps 1e-8.  Tile, stage and launch change only the
 * schedule (which pixels and Gaussians a thread block handles together), never
 * a result: the image, loss and gradients are identical for every choice up to
 * the order of FP32 additions inside a tile (tests hold each against the same
 * oracle). */
typedef struct {
  int32_t tile;      /* tile edge in pixels: 8, 16 or 32 */
  float sigma_cut;   /* sigma cut-off, > 0 */
  float alpha_min;   /* minimum |w| exp(-sigma), > 0 */
  float det_eps;     /* minimum det Sigma, >= 0 */
  float lr, beta1, beta2, eps; /* Adam */
  int32_t stage;     /* Gaussians staged per shared-memory batch: 32, 64, 128
                        or 256 (0 means 64) */
  int32_t launch;    /* render launch form: GS2D_LAUNCH_PERSISTENT (one wave of
                        blocks taking tiles from a queue) or GS2D_LAUNCH_GRID
                        (one block per tile, in queue order) */
  /* Learning-rate schedule of the fit loop (gs2d_fit_step, gs2d_encode_*):
   * parameter row r of step t moves with lr * scale(r) * lr_decay^(t-1),
   * scale = lr_mu (rows mu_x, mu_y), lr_shape (l1, l2, l3), lr_color
   * (c_r, c_g, c_b), lr_weight (w); all 1 by default (plain Adam).
   * gs2d_adam_step ignores them. */
  float lr_mu, lr_shape, lr_color, lr_weight, lr_decay;
  /* Re-binning of the fit loop (gs2d_fit_step, gs2d_fit_step_rgb8,
   * gs2d_fit_step_qat, gs2d_encode_frame, gs2d_encode_batch): each Gaussian is
   * listed in the tiles its pixel box, widened by bin_margin pixels, covers,
   * and the lists are rebuilt only in an iteration where some Gaussian's box
   * has left its listed tiles (checked on the device every iteration).  The
   * results are the same as binning every iteration (tiles a Gaussian does
   * not reach contribute nothing; a rebuild whose widened lists would not
   * fit max_entries lists the tight boxes instead).  Negative: bin every
   * iteration.  Default 4. */
  float bin_margin;
  /* Backward reduction to per-Gaussian sums: GS2D_REDUCE_SLOTS (default: one
   * record per (tile, Gaussian) pair, summed per Gaussian in a fixed order,
   * so every result is reproducible bit for bit) or GS2D_REDUCE_ATOMIC
   * (floating-point atomic additions into per-Gaussian sums: the same sums
   * up to the order of the additions, which varies from run to run). */
  int32_t reduce;
} gs2d_config;

enum { GS2D_LAUNCH_PERSISTENT = 0, GS2D_LAUNCH_GRID = 1 };
enum { GS2D_REDUCE_SLOTS = 0, GS2D_REDUCE_ATOMIC = 1 };

/* One clip of a batch: a W x H frame fitted by n Gaussians.  The caller sets
 * width, height and n; gs2d_plan_init_batch fills the rest.  A batch stores
 * the clips' parameters side by side (clip c owns columns [g_off, g_off + n) of
 * every parameter row of the batch's 9 x n_total array) and their images one
 * after another (clip c's planar [3][H][W] image starts pix_off floats into the
 * batch's image buffer). */
typedef struct {
  int32_t width, height, n;
  int32_t tiles_x, tiles_y;
  int32_t g_off;     /* first Gaussian (column) of the clip */
  int32_t tile_off;  /* first tile of the clip in the batch's tile numbering */
  int32_t reserved;
  int64_t pix_off;   /* first float of the clip's image */
} gs2d_clip;

/* Host-side plan: image size(s), Gaussian count, capacity and the workspace
 * layout.  Filled by gs2d_plan_init (one frame) or gs2d_plan_init_batch;
 * treat as read-only afterwards. */
typedef struct {
  int32_t width, height; /* the frame of a one-clip plan; 0, 0 for several clips */
  int32_t n;             /* Gaussians (all clips) */
  int32_t tile, tiles_x, tiles_y; /* tile edge; tile grid of a one-clip plan */
  int32_t num_tiles;     /* tiles of all clips */
  int32_t tile_bits;     /* bits of a tile id */
  int32_t num_clips;     /* 1 for gs2d_plan_init */
  int32_t stage;         /* Gaussians per shared-memory batch of the render */
  int64_t max_entries;   /* capacity for (tile, Gaussian) pairs */
  int64_t pixels;        /* sum of W H over the clips */
  gs2d_config cfg;
  uint64_t ws_bytes;     /* device workspace size the caller must allocate */
  uint64_t off[24];      /* internal: byte offsets of workspace sections */
  uint64_t magic;        /* internal: set by the plan_init calls */
} gs2d_plan;

/* Fills *cfg with the defaults listed above. */
void gs2d_config_default(gs2d_config* cfg);

/* sizeof(gs2d_plan) and sizeof(gs2d_config) as compiled into the library, so
 * that foreign-language bindings can verify their struct layouts. */
size_t gs2d_sizeof_plan(void);
size_t gs2d_sizeof_config(void);

/* Lays out a workspace for a W x H frame and n Gaussians with room for
 * max_entries (tile, Gaussian) pairs (0 picks max(2^20, 16 n), 64 n for tile 8,
 * at most 2^28 - 1).  cfg may be NULL (defaults).  Host only; no CUDA call.
 * Errors: W, H < 1 or > 65536, n < 0 or more than 2^27 Gaussians in all,
 * max_entries < 0 or > 2^28 - 1, tile not 8, 16 or 32, stage not 0, 32, 64,
 * 128 or 256, unknown launch form, non-positive constants. */
gs2d_status gs2d_plan_init(gs2d_plan* plan, int32_t width, int32_t height, int32_t n,
                           int64_t max_entries, const gs2d_config* cfg);

/* Lays out one workspace for a batch of independent clips (frames of
 * different sizes and Gaussian counts fitted together: every step of the path
 * runs once over all clips, each clip keeping its own loss).  clips: host
 * array of num_clips (1 ... 65536) entries whose width, height and n the caller
 * set; the call fills their other fields.  max_entries 0 picks
 * max(2^20, 16 n_total), 64 n_total for tile 8.  Host only; no CUDA call.  After
 * zero-filling the workspace, the caller uploads the clip table once with
 * gs2d_ws_set_clips.  Every call taking a plan accepts a batch plan, with
 * images in the batch layout of gs2d_clip; gs2d_render_l2's loss is then the
 * sum over clips of each clip's mean squared error (so each clip's gradient is
 * that of its own loss). */
gs2d_status gs2d_plan_init_batch(gs2d_plan* plan, gs2d_clip* clips, int32_t num_clips,
                                 int64_t max_entries, const gs2d_config* cfg);

/* Copies the clip table of a batch plan (host, as filled by
 * gs2d_plan_init_batch) into the workspace.  Synchronises the stream.  A
 * one-clip plan from gs2d_plan_init needs no table. */
gs2d_status gs2d_ws_set_clips(const gs2d_plan* plan, void* ws, const gs2d_clip* clips,
                              void* stream);

/* Projection (Sec. 3: the per-Gaussian step of tile-based rasterization).
 * Reads params (device, 9n floats) and writes, into ws, each Gaussian's
 * screen-space record (conic in Cholesky form, cut-off, weighted colour), its
 * tile rectangle and tile count; culls non-finite, degenerate (det <= det_eps),
 * invisible (|w| < alpha_min) and off-image Gaussians (count 0). */
gs2d_status gs2d_project(const gs2d_plan* plan, void* ws, const float* params, void* stream);

/* Binning and sort (Sec. 3 tile-based rasterization; 2D has no depth, so the
 * order inside a tile is the Gaussian index): per-tile entry counts, exclusive
 * scans (per-Gaussian offsets and per-tile ranges [start, end) into the sorted
 * list), one (tile, n) entry per covered tile placed in its tile's range, and
 * a per-tile sort by Gaussian index -- the (tile, index) key order.  Also
 * orders the tiles by list length (longest first) for the render's work
 * queue.  Needs gs2d_project on the same ws first.  If the entries exceed
 * max_entries, the status word is set to GS2D_ERR_CAPACITY and the sorted list
 * is empty (renders then produce zero). */
gs2d_status gs2d_bin_sort(const gs2d_plan* plan, void* ws, void* stream);

/* gs2d_project followed by gs2d_bin_sort, with the same results, with the
 * projection and the tile counts fused into one launch. */
gs2d_status gs2d_prepare(const gs2d_plan* plan, void* ws, const float* params, void* stream);

/* Forward render, Eq. 2.  img: device [3][H][W] output (every pixel written).
 * Needs gs2d_bin_sort first.  Tiles are rendered in the queue order of
 * gs2d_bin_sort (longest list first), by one thread block per tile
 * (GS2D_LAUNCH_GRID, the default) or by one wave of persistent blocks that
 * take tiles from a queue (GS2D_LAUNCH_PERSISTENT), as gs2d_config.launch
 * says. */
gs2d_status gs2d_render_fwd(const gs2d_plan* plan, void* ws, float* img, void* stream);

/* Forward render that allocates nothing (the paper has no counterpart; this
 * is an integration convenience).  For callers that cannot allocate device
 * memory when they render: a real-time pipeline that must not stall on the
 * allocator, a host application or plugin that forbids libraries to allocate
 * from its memory budget, or code that must not call allocation routines while
 * a CUDA graph is being captured.  Runs projection, binning and the forward
 * render of params (device, 9n floats, layout as above) into img (device
 * [3][H][W], every pixel written) with cfg (NULL: defaults), using as scratch
 * a fixed 16 MiB array that the library reserves on every GPU that loads it,
 * held until the process exits.  Frames and Gaussian counts whose workspace
 * (with room for at least 1024 tile entries) exceeds 16 MiB are rejected with
 * GS2D_ERR_INVALID_ARG and a message; the entry capacity is the largest that
 * fits the array (about 3.5e5 entries at 1920x1080 with 20 000 Gaussians),
 * and an overflow renders zero and reports GS2D_ERR_CAPACITY through status
 * (device int32, may be NULL), written on the stream after the render.
 * Makes no cudaMalloc, cudaFree or other allocating call.  The first call on
 * each device, with that device current, looks up the array's device address
 * (a CUDA runtime query) and caches it: make that first call before any
 * stream capture.  Every call shares the one array and it keeps the previous
 * call's contents (the call clears what must start at zero): calls that may
 * overlap on the GPU (different streams, or host threads without ordering)
 * race and must be serialised by the caller. */
gs2d_status gs2d_render_fwd_noalloc(const float* params, int32_t n, int32_t width, int32_t height,
                                    const gs2d_config* cfg, float* img, int32_t* status,
                                    void* stream);

/* Backward render: given dimg = dL/dC (device [3][H][W]), writes grads
 * (device, 9n floats, same layout as params) = dL/dparams through Eq. 2 and
 * Eq. 1.  Recomputes the blend from the saved per-tile lists (no per-pixel
 * state is stored by the forward pass).  params must be the values given to
 * gs2d_project.  Culled Gaussians get zero gradient. */
gs2d_status gs2d_render_bwd(const gs2d_plan* plan, void* ws, const float* params,
                            const float* dimg, float* grads, void* stream);

/* Fused forward + L2 loss + backward for fitting: L = mean over 3HW of
 * (C - target)^2 (a batch plan: the sum of that over the clips).
 * target: device [3][H][W].  grads: device 9n floats
 * (dL/dparams).  img: device [3][H][W] or NULL (the rendered image is then not
 * stored).  loss: device, 2 floats or NULL: {L, mean squared error of C
 * clamped to [0, 1]} (the latter gives PSNR = -10 log10).  Needs
 * gs2d_bin_sort first. */
gs2d_status gs2d_render_l2(const gs2d_plan* plan, void* ws, const float* params,
                           const float* target, float* grads, float* img, float* loss,
                           void* stream);

/* One Adam step (the "optimization steps" of Sec. 4.1; Adam with bias
 * correction is a project reading) over count floats: m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, p -= lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
 * params, grads, m, v: device, count floats each.  step >= 1.  mask: device
 * uint8 per Gaussian (count / 9 entries, parameter k belongs to Gaussian
 * k % (count / 9)) or NULL; masked-out Gaussians keep params, m and v.
 * cfg NULL means defaults. */
gs2d_status gs2d_adam_step(float* params, const float* grads, float* m, float* v, int64_t count,
                           int32_t step, const uint8_t* mask, const gs2d_config* cfg, void* stream);

/* One iteration of the fitting loop of gs2d_encode_frame / gs2d_encode_batch
 * (Sec. 3.2 A), as those loops run it: projection and binning of params, the
 * fused forward + L2 loss + backward render, and the per-Gaussian reduction
 * fused with the Adam update of params, adam_m, adam_v (device, 9n floats
 * each).  The Adam step counter lives in the workspace header: it starts at
 * zero in a zero-filled workspace and advances by one per call;
 * gs2d_fit_reset restarts the optimiser.  The tile lists are kept from call
 * to call while every Gaussian stays inside them (gs2d_config.bin_margin;
 * gs2d_fit_rebins counts the rebuilds), with the results of binning every
 * call.  target: device, the plan's image layout. */
gs2d_status gs2d_fit_step(const gs2d_plan* plan, void* ws, const float* target, float* params,
                          float* adam_m, float* adam_v, void* stream);

/* Optimiser state of the fit loop kept in the workspace header: the Adam
 * step counter and the running powers beta1^step, beta2^step and
 * lr_decay^(step - 1) (kept as products, so a checkpoint holds them exactly).
 * Together with params, adam_m and adam_v it is a checkpoint of a fit. */
typedef struct {
  int32_t step;
  int32_t reserved;
  double beta1_pow, beta2_pow, decay_pow;
} gs2d_fit_state;

/* Reads the fit loop's optimiser state (host out); synchronises the stream. */
gs2d_status gs2d_fit_state_get(const gs2d_plan* plan, const void* ws, gs2d_fit_state* state,
                               void* stream);

/* Resumes a fit from a checkpoint: sets the optimiser state (host in, step
 * >= 0) in the workspace, stream-ordered, and marks the tile lists unbuilt
 * (the next gs2d_fit_step bins afresh, which gives the results of the
 * retained lists).  With params, adam_m and adam_v restored by the caller,
 * the following gs2d_fit_step calls give bit for bit what the interrupted
 * fit would have.  (Checkpoint/resume is the library's; the paper has no
 * counterpart.) */
gs2d_status gs2d_fit_state_set(const gs2d_plan* plan, void* ws, const gs2d_fit_state* state,
                               void* stream);

/* Restarts the optimiser of gs2d_fit_step: zeroes adam_m and adam_v (device,
 * 9n floats each) and the workspace header (step counter, status word). */
gs2d_status gs2d_fit_reset(const gs2d_plan* plan, void* ws, float* adam_m, float* adam_v,
                           void* stream);

/* P-frames (Sec. 3.2 C, selective Gaussian optimisation): the residual
 * between the current frame and the reference marks the changed pixels
 * (max over channels of |reference - frame| > threshold; reading: the
 * reference is the render of the reference Gaussians, what a decoder holds);
 * the per-tile lists of the current binning (the paper's pixel-to-Gaussian
 * metadata) give the Gaussians that contribute to a changed pixel (the
 * renderer's cut-off predicate).  reference, frame: device, the plan's image
 * layout.  selected: device uint8[n] out (1 = selected).  n_selected: host
 * int32 out or NULL (synchronises the stream when given).  Needs
 * gs2d_prepare of the reference Gaussians on ws. */
gs2d_status gs2d_select_changed(const gs2d_plan* plan, void* ws, const float* reference,
                                const float* frame, float threshold, uint8_t* selected,
                                int32_t* n_selected, void* stream);

/* One P-frame fit iteration: projection and binning of all Gaussians, the
 * fused render + L2 + backward over only the tiles that the selected
 * Gaussians' rectangles cover (every pixel a selected Gaussian reaches, so
 * their gradients are those of the full-frame loss), and the reduction + Adam
 * of only the selected Gaussians (the others keep params, adam_m, adam_v).
 * Adam step counter as for gs2d_fit_step. */
gs2d_status gs2d_pframe_step(const gs2d_plan* plan, void* ws, const float* target, float* params,
                             float* adam_m, float* adam_v, const uint8_t* selected,
                             void* stream);

/* Fits a P-frame: `iters` gs2d_pframe_step iterations replayed as a captured
 * CUDA graph (moments zeroed first), then final_psnr (host, may be NULL) = the
 * full-frame PSNR of the result.  Synchronises the stream. */
gs2d_status gs2d_encode_pframe(const gs2d_plan* plan, void* ws, const float* target,
                               float* params, float* adam_m, float* adam_v,
                               const uint8_t* selected, int32_t iters, float* final_psnr,
                               void* stream);

/* Quantisation of Gaussians (Sec. 3.3 A: distinct quantisers for the mean,
 * the Cholesky factor and the colour; the paper adopts GaussianImage's, which
 * it does not specify).  Per parameter row r (mu_x, mu_y, l1, l2, l3, c_r,
 * c_g, c_b, w): bits[r] = -16 stores the row as IEEE half (round to nearest
 * even, NaN coded 0x7E00); bits[r] in 1 ... 16 is a uniform scalar quantiser
 * over [lo[r], hi[r]]:
 * code = clamp(rint((x - lo) * scale), 0, 2^b - 1), value = lo + code * step,
 * in single-rounded float operations, with scale = (2^b - 1) / (hi - lo) and
 * step = (hi - lo) / (2^b - 1) evaluated in double and rounded to float;
 * bits[r] = 0 keeps float32.  Non-finite inputs are coded 0.
 * refine = 0: lo, scale and step are the caller's (hi documents the range).
 * refine != 0: each uniform row's range is [min, max] of the row's finite
 * values, derived on the device for every call (QAT's quantisation
 * parameters follow the Gaussians); a row with no spread gets scale = step = 0
 * (every code 0, value lo). */
typedef struct {
  int32_t bits[9];
  int32_t refine;
  float lo[9], hi[9];
  float scale[9], step[9];
} gs2d_quant;

/* Post-training quantisation: codes (device uint16 [9][n], or NULL; halves as
 * their bit patterns, unquantised rows as 0), dequantised parameters (device
 * float [9][n], or NULL) and the ranges used (device float [2][9]: lo row, hi
 * row; 0 for rows that are not uniform; or NULL) of params (device float
 * [9][n]).  For n > 0 at least one of codes and dequant must be given. */
gs2d_status gs2d_quantize(const float* params, int32_t n, const gs2d_quant* q, uint16_t* codes,
                          float* dequant, float* ranges, void* stream);

/* Post-training calibration (Sec. 3.3 A: the quantisation parameters are
 * fixed after fitting, from a representative set of fitted frames): for
 * every uniform row (bits[r] in 1 ... 16; host int32 [9]) of params (device
 * float [9][n], the frames' Gaussians side by side), the central `coverage`
 * interval of the row's finite values, coverage in (0, 1]: lo and hi are the
 * (1 - coverage)/2 and (1 + coverage)/2 quantiles with linear interpolation
 * between order statistics (coverage 1: the row's minimum and maximum).  The
 * order statistics are found on the device (a radix select on the values'
 * order-preserving 32-bit keys); the interpolation is formed in double and
 * rounded once.  Rows without spread (or without finite values) get
 * hi = lo + 1; other rows get lo = hi = 0.  lo, hi: host float [9] out.
 * scratch: device, gs2d_quant_calibrate_scratch_bytes() bytes.
 * Synchronises the stream (an offline, training-stage step). */
size_t gs2d_quant_calibrate_scratch_bytes(void);
gs2d_status gs2d_quant_calibrate(const float* params, int32_t n, const int32_t* bits,
                                 double coverage, void* scratch, size_t scratch_bytes, float* lo,
                                 float* hi, void* stream);

/* Quantisation-aware fit iteration (Sec. 3.3 A, QAT): params are
 * fake-quantised with q, the frame is rendered from the quantised values and
 * the gradient taken there, and Adam updates the float params (the
 * straight-through estimator).  Otherwise as gs2d_fit_step. */
gs2d_status gs2d_fit_step_qat(const gs2d_plan* plan, void* ws, const float* target, float* params,
                              float* adam_m, float* adam_v, const gs2d_quant* q, void* stream);

/* Bitstream accounting (Sec. 3.3 B, Eq. 3-4).
 *
 * gs2d_code_entropy: ideal order-0 code length, per parameter row, of the
 * [9][n] codes of gs2d_quantize (device uint16), counting only the columns
 * with select[i] != 0 when select (device uint8 [n]) is given: for each row,
 * T log2 T - sum over symbols of c log2 c, with T the counted columns and c
 * each symbol's count (a vanilla entropy coder with one static model per row
 * approaches it; the model is not counted).  bits (host int32 [9]) are the
 * quantiser's widths: 16-bit symbols for half rows, 2^b for uniform rows
 * (codes masked to that width), 32 bits per value for rows with bits 0.
 * out_bits: device double [9].  scratch: device memory of at least
 * gs2d_code_entropy_scratch_bytes(), cleared by the call.  Deterministic. */
size_t gs2d_code_entropy_scratch_bytes(void);
gs2d_status gs2d_code_entropy(const uint16_t* codes, int32_t n, const int32_t* bits,
                              const uint8_t* select, void* scratch, size_t scratch_bytes,
                              double* out_bits, void* stream);

/* Coded size of one frame (Sec. 3.3 B): the sum over rows of
 * gs2d_code_entropy's code lengths (over the selected columns when select is
 * given), plus, when select (device uint8 [n]) is given (a P-frame), each
 * selected Gaussian's index of ceil(log2 max(n, 2)) bits, plus, when refine
 * != 0, the frame's own ranges (two float32 per uniform row).  out_bits:
 * device double [1].  scratch: device, gs2d_frame_bits_scratch_bytes()
 * bytes.  Other arguments as gs2d_code_entropy. */
size_t gs2d_frame_bits_scratch_bytes(void);
gs2d_status gs2d_frame_bits(const uint16_t* codes, int32_t n, const int32_t* bits,
                            const uint8_t* select, int32_t refine, void* scratch,
                            size_t scratch_bytes, double* out_bits, void* stream);

/* Totals of a coded sequence (host arithmetic, Eq. 3-4).  counts[k] (host
 * int32 [frames]): Gaussians coded in frame k; payload_bits[k] (host double
 * [frames]): its size before bits-back coding.  Frame k is an I-frame when
 * k % gop == 0 (vanilla coding of all Gaussians); every other frame is a
 * P-frame whose bits-back coding saves log2(m!) - log2(m) bits for m =
 * counts[k] (Eq. 3; 0 for m <= 1), summed over the P-frames (Eq. 4). */
typedef struct {
  double i_bits, p_bits, savings, total_bits;
  int32_t i_frames, p_frames;
} gs2d_seq_bits;
gs2d_status gs2d_sequence_bits(const int32_t* counts, const double* payload_bits, int32_t frames,
                               int32_t gop, gs2d_seq_bits* out);

/* Frame input (the video frame a fit targets, Sec. 3.2): 8-bit interleaved
 * RGB (device, row y at rgb + y * row_bytes, pixel x at 3 * x; row_bytes >=
 * 3 * width) to the planar float32 frame [3][H][W] (device) with value c /
 * 255 correctly rounded; height at most 65535.  Stream-ordered; nothing is
 * allocated. */
gs2d_status gs2d_frame_from_rgb8(const uint8_t* rgb, int32_t width, int32_t height,
                                 int64_t row_bytes, float* frame, void* stream);

/* One fit iteration end to end, as an encoder on the host drives it: the
 * 8-bit RGB frame (host, H x W x 3, packed rows) is converted into frame_dev
 * (device [3][H][W] float32, as gs2d_frame_from_rgb8): read over the host
 * link by the conversion itself when rgb_host is pinned memory the device can
 * address (cudaHostAlloc / cudaHostRegister), else first copied to rgb_dev
 * (device, 3 W H bytes); params_host (pinned host, 9n floats, or
 * NULL to keep the device params) is copied to params; then gs2d_fit_step;
 * params after the step also go to params_out_host (host, or NULL): stored
 * there by the Adam kernel itself when it is pinned memory the device can
 * address, else copied after it.  The
 * frame's upload and conversion run on an auxiliary stream and overlap the
 * projection and binning; the render waits for them, and they wait for the
 * work queued on `stream` before the call, so the call is ordered on
 * `stream` like the others.  The auxiliary stream and its two events are
 * the only CUDA objects the library creates: one set per host thread and
 * device, on that thread's first call with the device current, reused by
 * every later call and kept until the process exits.  A cudaDeviceReset
 * destroys them without the library knowing: after one, do not call
 * gs2d_fit_step_rgb8 on that device again in the same process.  One-clip
 * plans only. */
gs2d_status gs2d_fit_step_rgb8(const gs2d_plan* plan, void* ws, const uint8_t* rgb_host,
                               uint8_t* rgb_dev, float* frame_dev, const float* params_host,
                               float* params, float* adam_m, float* adam_v, float* params_out_host,
                               void* stream);

/* Number of times the fit loop has rebuilt its tile lists in this workspace
 * (see gs2d_config.bin_margin) since it was zero-filled or gs2d_fit_reset;
 * synchronises the stream. */
gs2d_status gs2d_fit_rebins(const gs2d_plan* plan, const void* ws, int64_t* rebins,
                            void* stream);

/* Device scratch (bytes, 256-byte aligned start) that gs2d_roi_init needs for
 * a W x H frame and n Gaussians. */
uint64_t gs2d_roi_init_scratch_bytes(int32_t width, int32_t height, int32_t n);

/* Region-of-interest superpixel initialiser (Sec. 3.2 A: the region is cut
 * into superpixels by K-means; each segment's centre, covariance and mean
 * colour give one Gaussian's mean, Cholesky factor and colour).  Readings:
 * about roi_frac * n segments from seeds on a square grid of step
 * S = max(1, sqrt(A / (roi_frac n))) over the mask (A = mask pixels), 10 K-means
 * iterations in (r, g, b, x, y) with distance
 * |dcol|^2 + (0.2 / S)^2 |dxy|^2 among centres within S of the pixel (centres
 * held within S of their seeds), Sigma = 4 (pixel covariance + I/12) (the
 * factor 4 keeps the additive blend of the segments flat), weight =
 * area / (2 pi sqrt(det Sigma)).  Arithmetic: distances decided in FP32
 * (centres kept as float32; where two candidates' distances lie within FP32
 * rounding of each other either may win), segment sums exact in integers
 * (pixel centres as 2x + 1 - 2 floor(seed); colours quantised to 2^-20,
 * clamped to [-32, 32], so a mean colour is within 2^-21 of the plain mean),
 * so the result is reproducible bit for bit.  The other n - n_roi Gaussians
 * are isotropic (variance = 4 x background area per Gaussian / (2 pi),
 * weight 1/4, colour of the frame) at bg_xy (random positions are inputs).
 * frame: device [3][H][W] float32.  mask: device [H][W] uint8 (non-zero = in
 * the region).  bg_xy: device [2][n] float32 (row x, row y); the first
 * n - n_roi columns are used.  params: device, 9n floats out (region
 * Gaussians first, in seed raster order).  n_roi: host int32 out, may be NULL.
 * scratch: device, gs2d_roi_init_scratch_bytes bytes.  All work runs on the
 * device; the call synchronises the stream once at the end to return n_roi.
 * Errors: W or H < 1 or > 65536, W H > 2^30, n < 0 or > 2^27, roi_frac
 * outside [0, 1], NULL pointers, a misaligned or short scratch. */
gs2d_status gs2d_roi_init(const float* frame, const uint8_t* mask, int32_t width, int32_t height,
                          int32_t n, float roi_frac, const float* bg_xy, float* params,
                          int32_t* n_roi, void* scratch, uint64_t scratch_bytes, void* stream);

/* gs2d_roi_init that also writes out the K-means iterations (Sec. 3.2 A), for
 * inspecting or checking the segmentation step by step.  cen_trace: device
 * float32 [10][5][n] or NULL: for iteration k the centres its assignment
 * used, rows r, g, b, x, y of n floats (the first n_roi columns are the
 * centres; iteration 0 holds the seeds with the frame's colour there).
 * label_trace: device int32 [10][H][W] or NULL: for iteration k the centre
 * each pixel joined (-1 outside the mask).  The final Gaussians come from the
 * labels of iteration 9.  Other arguments, results and errors as
 * gs2d_roi_init. */
gs2d_status gs2d_roi_init_trace(const float* frame, const uint8_t* mask, int32_t width,
                                int32_t height, int32_t n, float roi_frac, const float* bg_xy,
                                float* params, int32_t* n_roi, void* scratch,
                                uint64_t scratch_bytes, float* cen_trace, int32_t* label_trace,
                                void* stream);

/* Fits the plan's n Gaussians to a frame (Sec. 3.2 A: optimise N Gaussians
 * to the frame; I-frames start from an initialiser's output, P-frames from the
 * previous frame's Gaussians).  Runs up to `iters` iterations of
 * project -> bin_sort -> render_l2 -> adam_step.  Every check_every
 * iterations (>= 1, and after the last) the PSNR of the clamped render is
 * taken; the loop stops once it reaches target_psnr (<= 0 disables the test)
 * or a kernel records an error.  On a non-default stream the device drives
 * the loop: the whole fit is one CUDA graph whose WHILE node repeats one
 * iteration and a control kernel that counts iterations, takes the PSNR
 * checks and ends the loop, with one host read at the end (the trace is kept
 * in the workspace's gradient scratch, so it needs iters / check_every + 1
 * <= 9n).  Otherwise (the legacy default stream, a longer trace, or a driver
 * that declines the graph) the host replays one captured iteration, or
 * launches it plainly on the legacy stream, and reads the PSNR back at each
 * check.  Both give the same results bit for bit.
 * target: device [3][H][W].  params: device 9n floats, in: start, out: fitted.
 * adam_m, adam_v: device 9n floats each, zeroed by this call (the optimiser
 * state restarts per frame).  psnr_trace: host, NULL or room for
 * iters / check_every + 1 floats (PSNR after each check).  iters_done,
 * final_psnr: host, may be NULL.  Synchronises the stream before returning.
 * Returns GS2D_ERR_CAPACITY if the entry capacity was exceeded (iters_done
 * tells where; re-plan with more max_entries and continue from params). */
gs2d_status gs2d_encode_frame(const gs2d_plan* plan, void* ws, const float* target, float* params,
                              float* adam_m, float* adam_v, int32_t iters, float target_psnr,
                              int32_t check_every, float* psnr_trace, int32_t* iters_done,
                              float* final_psnr, void* stream);

/* Per-clip losses of the last gs2d_render_l2 on this workspace: out (host,
 * 2 num_clips floats) gets, per clip,
 * {mean squared error, mean squared error of the render clamped to [0, 1]}.
 * Synchronises the stream. */
gs2d_status gs2d_clip_losses(const gs2d_plan* plan, void* ws, float* out, void* stream);

/* Fits every clip of a batch plan for `iters` iterations (Sec. 3.2 A applied
 * to many independent frames at once: one launch per step of the path covers
 * all clips), replayed as one captured CUDA graph.  Each clip's Gaussians get
 * exactly the updates a gs2d_encode_frame of that clip alone would give them.
 * targets: device, the batch image layout.  params, adam_m, adam_v: device
 * 9 n_total floats each (moments zeroed by this call).  clip_psnr: host,
 * num_clips floats or NULL: PSNR of each clip's fitted Gaussians (one more
 * evaluation after the last update).  Synchronises the stream. */
gs2d_status gs2d_encode_batch(const gs2d_plan* plan, void* ws, const float* targets,
                              float* params, float* adam_m, float* adam_v, int32_t iters,
                              float* clip_psnr, void* stream);

/* Autotuner of the render schedule: times one fit iteration (projection,
 * binning, fused render + L2 + backward, reduction) of the given batch for
 * every (tile, stage, launch) candidate and reports the fastest.  clips:
 * host, widths, heights and n set (the other fields are overwritten).
 * params: device 9 n_total floats; targets: device, batch image layout.
 * tiles, stages, launches: host candidate lists (tile 8, 16 or 32; stage 32,
 * 64, 128 or 256; launch GS2D_LAUNCH_*).  cfg (or the defaults) gives every
 * other field, the backward reduction included.  ws: device scratch of
 * gs2d_autotune_ws_bytes bytes (contents are overwritten).  reps timed
 * iterations per candidate after two warm-up iterations.  ms: host,
 * num_tiles_c x num_stages x num_launches floats out (row-major: tile, then
 * stage, then launch; -1 if the candidate overflowed max_entries).
 * best_tile, best_stage, best_launch: host out.  params are not modified.
 * Synchronises the stream. */
uint64_t gs2d_autotune_ws_bytes(const gs2d_clip* clips, int32_t num_clips, int64_t max_entries,
                                const gs2d_config* cfg, const int32_t* tiles,
                                int32_t num_tiles_c);
gs2d_status gs2d_autotune(gs2d_clip* clips, int32_t num_clips, int64_t max_entries,
                          const gs2d_config* cfg, const float* params, const float* targets,
                          void* ws, uint64_t ws_bytes, const int32_t* tiles, int32_t num_tiles_c,
                          const int32_t* stages, int32_t num_stages, const int32_t* launches,
                          int32_t num_launches, int32_t reps, float* ms, int32_t* best_tile,
                          int32_t* best_stage, int32_t* best_launch, void* stream);

/* ---------------------------------------------------------------------------
 * Learned initialiser (Sec. 3.2 B: a regressor from the frame to the N
 * Gaussians' parameters, trained with a Chamfer loss on the means).  Its
 * convolutions run as GEMMs on the BF16 tensor cores.
 * ------------------------------------------------------------------------- */

/* C[M][N] = A[M][K] . B[N][K]^T (+ bias[N], then max(., 0) if relu) with BF16
 * A and B (device, row-major, K contiguous, leading dimensions lda, ldb in
 * elements, multiples of 8; 16-byte aligned), FP32 accumulation, output
 * either FP32 (out_f32) or BF16 (out_bf16), exactly one non-NULL, leading
 * dimension ldc.  splits > 1 splits K over thread blocks; partial (device,
 * gs2d_gemm_partial_bytes bytes) then holds FP32 partial sums that a second
 * kernel adds in split order (deterministic).  status: device int32 or NULL;
 * a block whose pipeline stalls for more than a second sets it to
 * GS2D_ERR_TIMEOUT and leaves its output tile unwritten. */
gs2d_status gs2d_gemm_bf16(const void* A, int32_t lda, const void* B, int32_t ldb, int32_t M,
                           int32_t N, int32_t K, const float* bias, int32_t relu, float* out_f32,
                           void* out_bf16, int32_t ldc, int32_t splits, float* partial,
                           int32_t* status, void* stream);
uint64_t gs2d_gemm_partial_bytes(int32_t M, int32_t N, int32_t ldc, int32_t K, int32_t splits);

/* Failure-detection check of the GEMM's bounded waits (not part of the
 * paper's method).  Launches the gs2d_gemm_bf16 kernel on one 128 x 32 x 64
 * tile (A: device bf16 [128][64], B: device bf16 [32][64], 16-byte aligned;
 * out: device float [128][32]) with every operand load withheld and each
 * mbarrier wait limited to wait_ns (1 ms ... 1 s): the MMA warp's wait for
 * the first stage runs out while no copy or MMA is in flight, so the kernel
 * records GS2D_ERR_TIMEOUT in *status (device int32, should hold GS2D_OK),
 * leaves out unwritten, frees its tensor memory and returns; the context
 * stays usable.  Asynchronous on stream. */
gs2d_status gs2d_gemm_wait_check(const void* A, const void* B, float* out, int32_t* status,
                                 uint64_t wait_ns, void* stream);

/* The same check for the persistent convolution kernels.  kernel:
 * GS2D_CHECK_CONV_FRAME (gs2d_conv_frame_bf16's kernel; x: device float
 * frame [1][3][16][256], W: device bf16 [32][80], out: device bf16
 * [8 x 128][32]), GS2D_CHECK_CONV_TAP (the TMA-tap kernel of gs2d_conv_bf16)
 * or GS2D_CHECK_CONV_ROWS (its row-box kernel), both with x: device bf16
 * NHWC [1][16][256][32], W: device bf16 [64][296], out: device bf16
 * [8 x 128][64]; all 16-byte aligned.  Every
 * load is withheld and each wait limited to wait_ns (1 ms ... 1 s): every
 * role's first wait runs out with no copy or MMA in flight, the groups that
 * share a named barrier leave together, the kernel records GS2D_ERR_TIMEOUT
 * in *status, leaves out unwritten, frees its tensor memory and returns.
 * Asynchronous on stream. */
enum { GS2D_CHECK_CONV_FRAME = 0, GS2D_CHECK_CONV_TAP = 1, GS2D_CHECK_CONV_ROWS = 2 };
gs2d_status gs2d_conv_wait_check(int32_t kernel, const void* x, const void* W, void* out,
                                 int32_t* status, uint64_t wait_ns, void* stream);

/* Network input: frames (device, B x [3][H][W] float32) and masks (device,
 * B x [H][W] uint8, or NULL = all zero) -> x (device, [B][H][W][8] BF16 NHWC:
 * r, g, b, mask, 0, 0, 0, 0; 16-byte aligned). */
gs2d_status gs2d_cnn_input(const float* frames, const uint8_t* masks, int32_t B, int32_t H,
                           int32_t W, void* x, void* stream);

/* im2col of x (device, [B][Hi][Wi][C] BF16, C a multiple of 8) for a ks x ks
 * convolution with stride and zero padding pad: col (device, BF16
 * [B Ho Wo][ldk], Ho = (Hi + 2 pad - ks) / stride + 1, likewise Wo) with
 * col[p][(ky ks + kx) C + ci] = x at (oy stride + ky - pad, ox stride + kx -
 * pad), zero outside the image, 1 at column ks^2 C (the bias column of the
 * weights) and 0 up to ldk (a multiple of 8, > ks^2 C).  A convolution is then
 * gs2d_gemm_bf16(col, W) with W [Co][ldk]. */
gs2d_status gs2d_im2col(const void* x, int32_t B, int32_t Hi, int32_t Wi, int32_t C, int32_t ks,
                        int32_t stride, int32_t pad, void* col, int32_t ldk, void* stream);

/* Implicit-GEMM convolution on the tensor cores: out = gs2d_gemm_bf16 of
 * gs2d_im2col(x) and W (the same sums in the same order, bit for bit) without
 * writing the im2col operand: the kernel gathers each 128-row tile of it from
 * x into shared memory.  x: device NHWC BF16 [B][Hi][Wi][C], C a multiple of
 * 8; W: device BF16 [N][ldk], ldk a multiple of 8 and >= ks^2 C + 1 (the
 * bias in column ks^2 C); relu applies max(., 0); exactly one of out_f32 /
 * out_bf16 ([B Ho Wo][ldc], device) is non-NULL.  status as gs2d_gemm_bf16. */
gs2d_status gs2d_conv_bf16(const void* x, int32_t B, int32_t Hi, int32_t Wi, int32_t C,
                           int32_t ks, int32_t stride, int32_t pad, const void* W, int32_t ldk,
                           int32_t N, int32_t relu, float* out_f32, void* out_bf16, int32_t ldc,
                           int32_t* status, void* stream);

/* The first convolution of the learned initialiser straight from the frames:
 * out = gs2d_conv_bf16 of gs2d_cnn_input(frames, masks) (C = 8: R, G, B, mask
 * != 0, four zeros), the same sums in the same order, bit for bit, without the
 * 8-channel image in memory (paper section 3.2 B).  frames: device float
 * [B][3][H][W]; masks: device uint8 [B][H][W] or NULL (channel 3 zero); both
 * 16-byte aligned.  Wt: device BF16 [N][ldk], ldk a multiple of 8, >= 8 ks^2
 * + 1 (the bias in column 8 ks^2) and <= 192.  Requires W a multiple of 16,
 * ks <= 3, 127 stride + ks <= 257 (stride 1 or 2) and N <= 128, else
 * GS2D_ERR_INVALID_ARG.  relu, out_f32 / out_bf16, ldc and status as
 * gs2d_conv_bf16. */
gs2d_status gs2d_conv_frame_bf16(const float* frames, const uint8_t* masks, int32_t B, int32_t H,
                                 int32_t W, int32_t ks, int32_t stride, int32_t pad,
                                 const void* Wt, int32_t ldk, int32_t N, int32_t relu,
                                 float* out_f32, void* out_bf16, int32_t ldc, int32_t* status,
                                 void* stream);

/* Gradient of gs2d_im2col: dx[b][iy][ix][ci] = sum over the taps that read
 * (iy, ix) of dcol (device, float32 [B Ho Wo][ldk]), multiplied by (act > 0)
 * when act (device, [B][Hi][Wi][C] BF16, the ReLU output fed to the im2col) is
 * not NULL (the ReLU backward); dx: device BF16, same shape as act.
 * Deterministic (a gather, no atomics). */
gs2d_status gs2d_col2im(const float* dcol, int32_t ldk, int32_t B, int32_t Hi, int32_t Wi,
                        int32_t C, int32_t ks, int32_t stride, int32_t pad, const void* act,
                        void* dx, void* stream);

/* out[c][r] = in[r][c] for a BF16 R x C matrix (device; leading dimensions
 * ld_in >= C, ld_out >= R). */
gs2d_status gs2d_transpose_bf16(const void* in, int32_t R, int32_t C, int32_t ld_in, void* out,
                                int32_t ld_out, void* stream);

/* dz = dx * (act > 0) over rows x cols: dx float32, act and dz BF16 (device,
 * leading dimensions ldx, lda, ldz). */
gs2d_status gs2d_relu_bwd(const float* dx, int32_t rows, int32_t cols, int32_t ldx,
                          const void* act, int32_t lda, void* dz, int32_t ldz, void* stream);

/* FP32 master weights w (device [co][ldk]) -> BF16 copy wb ([co][ldk]) and
 * BF16 transpose wt ([ldk][co]); either output may be NULL. */
gs2d_status gs2d_cast_weights(const float* w, int32_t co, int32_t ldk, void* wb, void* wt,
                              void* stream);

/* Head of the learned initialiser.  out (device float32 [B gh gw][ldo]): per
 * cell of a gh x gw grid of cell_px-pixel cells, `slots` groups of nine
 * numbers o0 .. o8 (columns 9 s .. 9 s + 8) decoding to one Gaussian:
 * mu = cell origin + anchor(s) + cell_px/2 tanh(o0, o1) with slot anchors on a
 * q x r grid inside the cell (q = ceil(sqrt(slots)), r = ceil(slots / q),
 * anchor(s) = cell_px ((s mod q + 1/2) / q, (s div q + 1/2) / r)),
 * l1 = scale exp(o2), l2 = scale o3, l3 = scale exp(o4) (exponents clamped to
 * [-4, 3]), colour 0.5 + o5..o7, w = 0.25 + o8.  Each frame keeps the n slots
 * with the largest |w| (ties: lower slot index first), in slot order: params
 * (device float32 [9][ldp], frame b in columns b n ... b n + n - 1; ldp >= B n:
 * the batch layout of gs2d_plan_init_batch for equal clips) and sel (device
 * int32 B x n, slot = cell slots + s).  Needs gh gw slots 4 bytes of shared
 * memory (at most 200 KB). */
gs2d_status gs2d_head_decode(const float* out, int32_t ldo, int32_t B, int32_t gh, int32_t gw,
                             int32_t slots, int32_t cell_px, float scale, int32_t n,
                             float* params, int32_t ldp, int32_t* sel, void* stream);
uint64_t gs2d_head_smem_bytes(int32_t gh, int32_t gw, int32_t slots);

/* Backward of gs2d_head_decode: dparams (device float32 [9][ldp], layout of
 * params) -> dout (device BF16 [B gh gw][ldo]; zero for unselected slots and
 * unused columns). */
gs2d_status gs2d_head_decode_bwd(const float* out, int32_t ldo, int32_t B, int32_t gh,
                                 int32_t gw, int32_t slots, int32_t cell_px, float scale,
                                 int32_t n, const int32_t* sel, const float* dparams,
                                 int32_t ldp, void* dout, void* stream);

/* Chamfer distance (Sec. 3.2 B) between the predicted means (rows 0, 1 of
 * params, device float32 [9][ldp], frame b in columns b n ...) and target
 * means (rows 0, 1 of targets, [9][ldq], frame b in columns b m ...), per
 * frame: mean over predictions of the squared distance to the nearest target
 * plus mean over targets of the squared distance to the nearest prediction
 * (brute force).  loss: device float32[B] or NULL.  dparams: device, layout
 * of params, or NULL; rows 0, 1 get += lambda d(Chamfer)/d(mu) (float
 * atomics: the order of additions varies between runs).  scratch: device,
 * gs2d_chamfer_scratch_bytes(n, m, B). */
gs2d_status gs2d_chamfer(const float* params, int32_t n, int32_t ldp, const float* targets,
                         int32_t m, int32_t ldq, int32_t B, float lambda, float* dparams,
                         float* loss, void* scratch, void* stream);
uint64_t gs2d_chamfer_scratch_bytes(int32_t n, int32_t m, int32_t B);

/* Copies the sorted list state to host memory for inspection (tests and
 * tools): n_entries (host, int64), keys (host, may be NULL: tile ids of the
 * sorted list, max_keys entries at most), values (host, may be NULL: Gaussian
 * index of each sorted entry), ranges (host, may be NULL: [num_tiles][2]
 * int32), counts (host, may be NULL: per-Gaussian tile count, n int32).
 * Synchronises the stream. */
gs2d_status gs2d_read_bins(const gs2d_plan* plan, const void* ws, int64_t* n_entries,
                           uint32_t* keys, uint32_t* values, int64_t max_keys, int32_t* ranges,
                           int32_t* counts, void* stream);

/* Work statistics of the current sorted list (diagnostics, autotuning and
 * roofline accounting): pairs = sum over tiles of (pixels of the tile inside
 * the image) x (list length), i.e. the (pixel, Gaussian) pairs a tile
 * rasterizer visits; hits = the pairs that contribute to Eq. 2 (the cut-off
 * predicate holds).  After a fit step the list is the fit loop's retained
 * one (widened rectangles: more pairs, the same hits); after gs2d_prepare
 * or gs2d_bin_sort it is the tight one.  Writes host int64 values (either may be NULL).  Launches
 * one counting kernel and synchronises the stream. */
gs2d_status gs2d_count_pairs(const gs2d_plan* plan, void* ws, int64_t* pairs, int64_t* hits,
                             void* stream);

/* Synchronises the stream and returns the workspace status word
 * (GS2D_OK or the first device-detected error); reset != 0 clears it. */
gs2d_status gs2d_ws_status(const gs2d_plan* plan, void* ws, int32_t reset, void* stream);

/* Throughput probes (not part of the paper's method): the issue-limited peak
 * rates of the two pipes the render kernels are bound by, measured on the
 * current device at its current clock, for roofline accounting.
 * gs2d_probe_peak enqueues one launch of `blocks` blocks on `stream` that
 * executes gs2d_probe_ops(blocks, iters) FP32 fused multiply-adds
 * (GS2D_PROBE_FFMA) or MUFU ex2 evaluations (GS2D_PROBE_EX2) in independent
 * dependency chains; time it with events on the stream.  sink: device, at
 * least `blocks` floats (one result per block, so no work is dead code).
 * gs2d_probe_ops returns 0 for blocks or iters < 1. */
enum { GS2D_PROBE_FFMA = 0, GS2D_PROBE_EX2 = 1 };
int64_t gs2d_probe_ops(int32_t blocks, int32_t iters);
gs2d_status gs2d_probe_peak(int32_t kind, int32_t blocks, int32_t iters, float* sink,
                            void* stream);

/* Message for the calling thread's last error ("" if none).  Copies at most
 * len - 1 characters and a terminating NUL into buf (host). */
gs2d_status gs2d_last_error(char* buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* GS2D_H */
