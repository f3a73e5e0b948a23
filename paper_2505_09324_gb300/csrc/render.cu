// Per-Gaussian reduction of the backward partials, the chain rule to the
// parameters, the fused Adam update of the fit loop, loss reductions, and the
// dispatch of the templated render kernels (render_impl.cuh) by tile edge,
// stage and mode.
#include <map>
#include <mutex>
#include <utility>

#include "gs2d_internal.cuh"

namespace gs2d {

// ---------------------------------------------------------------------------
// Per-Gaussian reduction of the slot partials (fixed order) and the chain rule
// from the eight sums to (mu, l, c, w):
//   e = 2^-q, q = u1^2 + u2^2, u1 = s dx / l1, u2 = s (dy - l2 dx / l1) / l3,
//   dL/dq = -ln2 S, S = (g . c') e; sums G = sum g e, A1 = sum S u1,
//   A2 = sum S u2, A11 = sum S u1^2, A12 = sum S u1 u2, A22 = sum S u2^2.
__device__ __forceinline__ void chain_grads(const float* __restrict__ params, int n, int i,
                                            const float a[kPartials], float gr[9]) {
  const float l1 = params[2 * n + i], l2 = params[3 * n + i], l3 = params[4 * n + i];
  const float cr = params[5 * n + i], cg = params[6 * n + i], cb = params[7 * n + i];
  const float w = params[8 * n + i];
  const float k2 = 1.17741002251547469101f;  // 2 ln2 s = sqrt(2 ln 2)
  const float c2 = 2.0f * kLn2;
  const float il1 = 1.0f / l1, il3 = 1.0f / l3, r = l2 * il3;
  gr[0] = k2 * (a[3] - r * a[4]) * il1;
  gr[1] = k2 * a[4] * il3;
  gr[2] = c2 * (a[5] - r * a[6]) * il1;
  gr[3] = c2 * a[6] * il3;
  gr[4] = c2 * a[7] * il3;
  gr[5] = w * a[0];
  gr[6] = w * a[1];
  gr[7] = w * a[2];
  gr[8] = fmaf(cr, a[0], fmaf(cg, a[1], cb * a[2]));
}

// kRL lanes share one Gaussian: lane `sub` sums slots s0 + sub, s0 + sub + kRL,
// ..., then the group adds its kRL partial sums (a fixed order: deterministic).
constexpr int kRL = 4;

__device__ __forceinline__ bool gather_partials(const float4* __restrict__ partial,
                                                const int* __restrict__ offs, int i, bool valid,
                                                int sub, float a[kPartials]) {
  int s0 = 0, s1 = 0;
  if (valid) {
    s0 = offs[i];
    s1 = offs[i + 1];
  }
#pragma unroll
  for (int k = 0; k < kPartials; k++) a[k] = 0.0f;
  for (int sl = s0 + sub; sl < s1; sl += kRL) {
    const float4 p = partial[2 * sl], q = partial[2 * sl + 1];
    a[0] += p.x;
    a[1] += p.y;
    a[2] += p.z;
    a[3] += p.w;
    a[4] += q.x;
    a[5] += q.y;
    a[6] += q.z;
    a[7] += q.w;
  }
#pragma unroll
  for (int o = 1; o < kRL; o <<= 1)
#pragma unroll
    for (int k = 0; k < kPartials; k++) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
  return s1 > s0;
}

// GS2D_REDUCE_ATOMIC: the render added the Gaussian's sums up itself; every
// lane of the group reads them, then lane 0 clears them for the next pass.
// `any`: the Gaussian had a (tile, Gaussian) pair.  Every lane of the warp
// must take part.
__device__ __forceinline__ bool gather_acc(float* __restrict__ acc, const int* __restrict__ offs,
                                           int i, bool valid, int sub, float a[kPartials]) {
  bool any = false;
#pragma unroll
  for (int k = 0; k < kPartials; k++) a[k] = 0.0f;
  float4* q = reinterpret_cast<float4*>(acc + (size_t)kPartials * i);
  if (valid) {
    const float4 x = q[0], y = q[1];
    a[0] = x.x;
    a[1] = x.y;
    a[2] = x.z;
    a[3] = x.w;
    a[4] = y.x;
    a[5] = y.y;
    a[6] = y.z;
    a[7] = y.w;
    any = offs[i + 1] > offs[i];
  }
  __syncwarp();  // every lane of the group has read the sums
  if (valid && sub == 0) q[0] = q[1] = make_float4(0.f, 0.f, 0.f, 0.f);
  return any;
}

__global__ void __launch_bounds__(256)
k_reduce_chain(int n, const float* __restrict__ params, const int* __restrict__ offs,
               const float4* __restrict__ partial, const WsHeader* __restrict__ hdr,
               float* __restrict__ grads, float* __restrict__ acc) {
  pdl_begin();
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gt / kRL, sub = gt % kRL;
  const bool valid = i < n && hdr->entries_raw == (int64_t)hdr->n_entries;
  float a[kPartials], gr[9];
  const bool any = acc ? gather_acc(acc, offs, i, valid, sub, a)
                       : gather_partials(partial, offs, i, valid, sub, a);
  if (i >= n) return;
  if (any) chain_grads(params, n, i, a, gr);
#pragma unroll
  for (int r = sub; r < 9; r += kRL) grads[(size_t)r * n + i] = any ? gr[r] : 0.0f;
}

// Fit loop: reduction + chain + Adam on the Gaussian's nine parameters (lane
// `sub` of the group updates rows sub, sub + kRL, ...).  host_out (device
// view of pinned host memory, or NULL): every Gaussian's parameters after
// the step are also stored there, so that no separate download is needed.
__global__ void __launch_bounds__(256)
k_reduce_chain_adam(int n, float* __restrict__ params, const int* __restrict__ offs,
                    const float4* __restrict__ partial, const WsHeader* __restrict__ hdr,
                    float* __restrict__ m, float* __restrict__ v, float4 lr_rows, float b1,
                    float b2, float eps, const uint8_t* __restrict__ select,
                    const float* __restrict__ params_eval, WsHeader* hdr_w,
                    float* __restrict__ acc, float* __restrict__ host_out) {
  pdl_begin();
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gt / kRL, sub = gt % kRL;
  const bool ok = hdr->entries_raw == (int64_t)hdr->n_entries;  // else over capacity
  // retained lists (hdr_w set): valid for the next iteration's containment test
  if (hdr_w && gt == 0 && ok) hdr_w->lists_valid = 1;
  // a P-frame updates only the selected Gaussians (the others keep params, m, v)
  const bool on = i < n && (!select || select[i]);
  float a[kPartials], gr[9];
  // (atomic sums are read and cleared for every Gaussian: an unselected one
  // of a rendered tile has sums too)
  const bool any = acc ? gather_acc(acc, offs, i, i < n && ok, sub, a) && on
                       : gather_partials(partial, offs, i, on && ok, sub, a);
  // (ok is the same for every thread of the grid)
  const bool act = on && ok;
  // the chain rule at the parameters that were rendered (the fake-quantised
  // ones of quantisation-aware fitting; the same array otherwise)
  if (act && any)
    chain_grads(params_eval ? params_eval : params, n, i, a, gr);
  else
    for (int r = 0; r < 9; r++) gr[r] = 0.0f;
  __syncwarp();  // every lane of the group has read the parameters
  if (i >= n) return;
  const float ibc1 = 1.0f / hdr->bc1, ibc2 = 1.0f / hdr->bc2;
  const float lr_now = hdr->lr_now;  // lr * lr_decay^(step - 1)
#pragma unroll
  for (int r = sub; r < 9; r += kRL) {
    const size_t k = (size_t)r * n + i;
    float p = params[k];
    if (act) {
      const float lr = lr_now * (r < 2 ? lr_rows.x : (r < 5 ? lr_rows.y : (r < 8 ? lr_rows.z
                                                                              : lr_rows.w)));
      const float g = gr[r];
      const float mm = fmaf(b1, m[k], (1.0f - b1) * g);
      const float vv = fmaf(b2, v[k], (1.0f - b2) * g * g);
      m[k] = mm;
      v[k] = vv;
      p -= lr * (mm * ibc1) / (sqrtf(vv * ibc2) + eps);
      params[k] = p;
    }
    if (host_out) host_out[k] = p;
  }
}

// Sum of the per-tile loss partials (each already divided by 3 W H of its
// clip): the plan's loss (the sum of the clips' mean squared errors).
__global__ void __launch_bounds__(1024)
k_loss_reduce(int num_tiles, const float2* __restrict__ loss_part, WsHeader* __restrict__ hdr,
              float* __restrict__ out) {
  pdl_begin();
  __shared__ double s_a[32], s_b[32];
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < num_tiles; t += blockDim.x) {
    a += loss_part[t].x;
    b += loss_part[t].y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_a[wid] = a;
    s_b[wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      sa += s_a[w];
      sb += s_b[w];
    }
    hdr->loss[0] = (float)sa;
    hdr->loss[1] = (float)sb;
    if (out) {
      out[0] = hdr->loss[0];
      out[1] = hdr->loss[1];
    }
  }
}

// Per-clip losses: block c sums the tiles of clip c.
__global__ void __launch_bounds__(1024)
k_clip_loss(ClipSet cs, const float2* __restrict__ loss_part, float2* __restrict__ clip_loss) {
  pdl_begin();
  const int c = blockIdx.x;
  const gs2d_clip cl = cs.count == 1 ? cs.one : cs.table[c];
  __shared__ double s_a[32], s_b[32];
  double a = 0.0, b = 0.0;
  const int t0 = cl.tile_off, nt = cl.tiles_x * cl.tiles_y;
  for (int t = t0 + threadIdx.x; t < t0 + nt; t += blockDim.x) {
    a += loss_part[t].x;
    b += loss_part[t].y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_a[wid] = a;
    s_b[wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      sa += s_a[w];
      sb += s_b[w];
    }
    clip_loss[c] = make_float2((float)sa, (float)sb);
  }
}

// ---------------------------------------------------------------------------
cudaError_t opt_in_smem(const void* kernel, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> done;  // (kernel, device) -> bytes
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find({kernel, dev});
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done[{kernel, dev}] = bytes;
  return e;
}

int persistent_grid(const void* kernel, int threads, int work) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;  // (kernel, device) -> blocks
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  int blocks = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find({kernel, dev});
    if (it != cache.end()) {
      blocks = it->second;
    } else {
      int per_sm = 0, sms = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) !=
              cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
      blocks = std::max(1, per_sm) * sms;
      cache[{kernel, dev}] = blocks;
    }
  }
  return std::max(1, std::min(work, blocks));
}

static float4 lr_rows(const gs2d_config& c) {
  return make_float4(c.lr_mu, c.lr_shape, c.lr_color, c.lr_weight);
}

// The per-Gaussian sums of GS2D_REDUCE_ATOMIC, or NULL (per-pair records).
static float* atomic_sums(const gs2d_plan& p, void* ws) {
  return p.cfg.reduce == GS2D_REDUCE_ATOMIC ? ws_ptr<float>(ws, p, kOffAcc) : nullptr;
}

static RenderArgs render_args(const gs2d_plan& p, void* ws) {
  RenderArgs a;
  a.clips = clip_set(p, ws);
  a.n = p.n;
  a.num_tiles = p.num_tiles;
  a.ranges = ws_ptr<int2>(ws, p, kOffRanges);
  a.list = ws_ptr<uint32_t>(ws, p, kOffList);
  a.rec = ws_ptr<float4>(ws, p, kOffRec);
  a.rect = ws_ptr<int4>(ws, p, kOffRect);
  a.offs = ws_ptr<int>(ws, p, kOffCount);
  a.order = ws_ptr<int>(ws, p, kOffOrder);
  a.hdr = ws_ptr<WsHeader>(ws, p, kOffHeader);
  a.img = nullptr;
  a.target = nullptr;
  a.dimg = nullptr;
  a.partial = ws_ptr<float>(ws, p, kOffPartial);
  a.loss_part = ws_ptr<float2>(ws, p, kOffLossPart);
  a.active = nullptr;
  a.ref = nullptr;
  a.frame = nullptr;
  a.threshold = 0.0f;
  a.selected = nullptr;
  a.acc = atomic_sums(p, ws);
  return a;
}

static cudaError_t launch_render(const gs2d_plan& p, RenderMode mode, const RenderArgs& a,
                                 cudaStream_t s) {
  switch (p.tile) {
    case 8: return launch_render_t8(p.stage, p.cfg.launch, mode, a, s);
    case 16: return launch_render_t16(p.stage, p.cfg.launch, mode, a, s);
    case 32: return launch_render_t32(p.stage, p.cfg.launch, mode, a, s);
  }
  return cudaErrorInvalidValue;
}

static cudaError_t launch_reduce(const gs2d_plan& p, void* ws, const float* params, float* grads,
                                 cudaStream_t s) {
  if (p.n == 0) return cudaSuccess;
  return launch_pdl(k_reduce_chain, (p.n * kRL + 255) / 256, 256, 0, s, p.n, params,
                    ws_ptr<int>(ws, p, kOffCount),
                    reinterpret_cast<const float4*>(ws_ptr<float>(ws, p, kOffPartial)),
                    ws_ptr<WsHeader>(ws, p, kOffHeader), grads, atomic_sums(p, ws));
}

cudaError_t launch_render_fwd(const gs2d_plan& p, void* ws, float* img, cudaStream_t s) {
  RenderArgs a = render_args(p, ws);
  a.img = img;
  return launch_render(p, kModeFwd, a, s);
}

cudaError_t launch_render_bwd(const gs2d_plan& p, void* ws, const float* params,
                              const float* dimg, float* grads, cudaStream_t s) {
  RenderArgs a = render_args(p, ws);
  a.dimg = dimg;
  cudaError_t e = launch_render(p, kModeBwd, a, s);
  if (e != cudaSuccess) return e;
  return launch_reduce(p, ws, params, grads, s);
}

cudaError_t launch_loss_reduce(const gs2d_plan& p, void* ws, float* loss, cudaStream_t s) {
  return launch_pdl(k_loss_reduce, 1, 1024, 0, s, p.num_tiles,
                    ws_ptr<float2>(ws, p, kOffLossPart), ws_ptr<WsHeader>(ws, p, kOffHeader), loss);
}

cudaError_t launch_clip_losses(const gs2d_plan& p, void* ws, cudaStream_t s) {
  return launch_pdl(k_clip_loss, p.num_clips, 1024, 0, s, clip_set(p, ws),
                    ws_ptr<float2>(ws, p, kOffLossPart), ws_ptr<float2>(ws, p, kOffClipLoss));
}

cudaError_t launch_render_l2(const gs2d_plan& p, void* ws, const float* params,
                             const float* target, float* grads, float* img, float* loss,
                             cudaStream_t s) {
  RenderArgs a = render_args(p, ws);
  a.target = target;
  a.img = img;
  cudaError_t e = launch_render(p, kModeL2, a, s);
  if (e == cudaSuccess) e = launch_reduce(p, ws, params, grads, s);
  if (e == cudaSuccess && loss) e = launch_loss_reduce(p, ws, loss, s);
  return e;
}

cudaError_t launch_count_pairs(const gs2d_plan& p, void* ws, cudaStream_t s) {
  WsHeader* hdr = ws_ptr<WsHeader>(ws, p, kOffHeader);
  cudaError_t e = cudaMemsetAsync(&hdr->pairs, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  return launch_render(p, kModeCount, render_args(p, ws), s);
}

// One fit iteration after projection and binning (which advanced the Adam
// step counter): fused render + loss + backward, then reduction + chain + Adam.
cudaError_t launch_fit_step(const gs2d_plan& p, void* ws, const float* target, float* params,
                            float* m, float* v, cudaStream_t s, const float* params_eval,
                            float* host_out) {
  RenderArgs a = render_args(p, ws);
  a.target = target;
  cudaError_t e = launch_render(p, kModeL2, a, s);
  if (e != cudaSuccess || p.n == 0) return e;
  WsHeader* hdr = ws_ptr<WsHeader>(ws, p, kOffHeader);
  return launch_pdl(k_reduce_chain_adam, (p.n * kRL + 255) / 256, 256, 0, s, p.n, params,
                    ws_ptr<int>(ws, p, kOffCount),
                    reinterpret_cast<const float4*>(ws_ptr<float>(ws, p, kOffPartial)),
                    (const WsHeader*)hdr, m, v, lr_rows(p.cfg), p.cfg.beta1, p.cfg.beta2,
                    p.cfg.eps, (const uint8_t*)nullptr, params_eval,
                    fit_lists_retained(p.cfg) ? hdr : (WsHeader*)nullptr, atomic_sums(p, ws),
                    host_out);
}

// ---------------------------------------------------------------------------
// P-frames (Sec. 3.2 C, selective Gaussian optimisation): the Gaussians that
// contribute to pixels changed since the reference are selected; each fit
// iteration renders only the tiles those Gaussians' rectangles cover (which
// hold every pixel a selected Gaussian reaches, so their gradients are the
// full-frame ones) and updates only them.

// Tiles of every selected Gaussian's rectangle; block 0 also zeroes the count
// of the active-tile list (its last reader, the previous render, is done).
__global__ void __launch_bounds__(256)
k_active_mark(int n, const uint8_t* __restrict__ select, const int4* __restrict__ rect,
              uint8_t* __restrict__ active, int* __restrict__ act_count) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *act_count = 0;
  if (i >= n || !select[i]) return;
  const int4 rc = rect[i];  // (first tile, row stride, width, height)
  for (int dy = 0; dy < rc.w; dy++)
    for (int dx = 0; dx < rc.z; dx++) active[rc.x + dy * rc.y + dx] = 1;
}

// Active tiles into a list (any order: tiles are independent); clears the marks.
__global__ void __launch_bounds__(256)
k_active_compact(int num_tiles, uint8_t* __restrict__ active, int* __restrict__ act_order,
                 int* __restrict__ act_count) {
  pdl_begin();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= num_tiles || !active[t]) return;
  active[t] = 0;
  act_order[atomicAdd(act_count, 1)] = t;
}

__global__ void __launch_bounds__(256)
k_count_flags(int n, const uint8_t* __restrict__ flags, int* __restrict__ out) {
  __shared__ int s_c;
  if (threadIdx.x == 0) s_c = 0;
  __syncthreads();
  int c = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    c += flags[i] != 0;
  atomicAdd(&s_c, c);
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(out, s_c);
}

cudaError_t launch_count_flags(int n, const uint8_t* flags, int* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int), s);
  if (e != cudaSuccess || n == 0) return e;
  k_count_flags<<<std::min(152 * 4, (n + 255) / 256), 256, 0, s>>>(n, flags, out);
  return cudaGetLastError();
}

cudaError_t launch_select_changed(const gs2d_plan& p, void* ws, const float* ref,
                                  const float* frame, float threshold, uint8_t* selected,
                                  cudaStream_t s) {
  RenderArgs a = render_args(p, ws);
  a.ref = ref;
  a.frame = frame;
  a.threshold = threshold;
  a.selected = selected;
  return launch_render(p, kModeSelect, a, s);
}

// One P-frame iteration after projection and binning: active tiles, the fused
// render over them, reduction + Adam of the selected Gaussians.
cudaError_t launch_pframe_step(const gs2d_plan& p, void* ws, const float* target,
                               float* params, float* m, float* v, const uint8_t* select,
                               cudaStream_t s) {
  if (p.n == 0) return cudaSuccess;
  uint8_t* active = ws_ptr<uint8_t>(ws, p, kOffActive);
  int* act_order = ws_ptr<int>(ws, p, kOffActOrder);
  int* act_count = act_order + p.num_tiles;
  cudaError_t e = launch_pdl(k_active_mark, (p.n + 255) / 256, 256, 0, s, p.n, select,
                             ws_ptr<int4>(ws, p, kOffRect), active, act_count);
  if (e == cudaSuccess)
    e = launch_pdl(k_active_compact, (p.num_tiles + 255) / 256, 256, 0, s, p.num_tiles, active,
                   act_order, act_count);
  if (e != cudaSuccess) return e;
  RenderArgs a = render_args(p, ws);
  a.target = target;
  a.order = act_order;
  a.active = act_count;
  e = launch_render(p, kModeL2, a, s);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_reduce_chain_adam, (p.n * kRL + 255) / 256, 256, 0, s, p.n, params,
                    ws_ptr<int>(ws, p, kOffCount),
                    reinterpret_cast<const float4*>(ws_ptr<float>(ws, p, kOffPartial)),
                    ws_ptr<WsHeader>(ws, p, kOffHeader), m, v, lr_rows(p.cfg), p.cfg.beta1,
                    p.cfg.beta2, p.cfg.eps, select, (const float*)nullptr, (WsHeader*)nullptr,
                    atomic_sums(p, ws), (float*)nullptr);
}

// Runs the one-time per-device queries of the fit loop's launches (occupancy
// of the persistent render, shared-memory opt-in of the long-list sort) so that
// a following stream capture records launches only.
cudaError_t prime_fit_launches(const gs2d_plan& p) {
  cudaError_t e = prime_binning();
  if (e != cudaSuccess) return e;
  switch (p.tile) {
    case 8: return prime_render_t8(p.stage, p.cfg.launch);
    case 16: return prime_render_t16(p.stage, p.cfg.launch);
    case 32: return prime_render_t32(p.stage, p.cfg.launch);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gs2d
