// Forward render for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they need a render: a real-time pipeline that must not stall on the
// allocator mid-stream, a host application or plugin that owns the device
// memory budget and forbids allocations by libraries, or code running where a
// CUDA graph is being captured, where allocation calls are not allowed.
// gs2d_render_fwd_noalloc serves them: the caller passes only the parameters
// and the output image; every intermediate buffer (projected records, tile
// rectangles and counts, the scans' offsets, the per-tile Gaussian lists, the
// tile ranges and the render queue) lives in one file-scope device array of
// fixed size that the library reserves when it is loaded.  The paper has no counterpart; this is an
// integration convenience.
#include <mutex>
#include <stdio.h>

#include "gs2d_internal.cuh"

using namespace gs2d;

namespace {

// Maximum scratch: 16 MiB.  Every GPU that loads the library holds this array
// until the process exits.
constexpr uint64_t kNoallocBytes = uint64_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name stands for a host-side shadow, not a device address, so the
// address is asked from the runtime: once per device, on the first call made
// with that device current, and cached.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__global__ void k_noalloc_status(const WsHeader* __restrict__ hdr, int32_t* __restrict__ out) {
  *out = hdr->status;
}

}  // namespace

extern "C" gs2d_status gs2d_render_fwd_noalloc(const float* params, int32_t n, int32_t width,
                                               int32_t height, const gs2d_config* cfg,
                                               float* img, int32_t* status, void* stream) {
  char msg[256];
  if (!img) return set_error(GS2D_ERR_INVALID_ARG, "gs2d_render_fwd_noalloc: img is NULL");
  if (n > 0 && !params)
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_render_fwd_noalloc: params is NULL");
  // Lay out a workspace with the largest entry capacity that fits the array:
  // the workspace size grows with max_entries (monotonically, in 256-byte
  // steps), so bisect on it.
  gs2d_plan plan;
  const int64_t min_entries = 1024;
  gs2d_status st = gs2d_plan_init(&plan, width, height, n, min_entries, cfg);
  if (st != GS2D_OK) return st;
  if (plan.ws_bytes > kNoallocBytes) {
    snprintf(msg, sizeof(msg),
             "gs2d_render_fwd_noalloc: %d Gaussians on a %d x %d frame need more than the "
             "%llu-byte static scratch; use a caller-allocated workspace (gs2d_plan_init)",
             n, width, height, (unsigned long long)kNoallocBytes);
    return set_error(GS2D_ERR_INVALID_ARG, msg);
  }
  int64_t lo = min_entries, hi = (int64_t)(kNoallocBytes / sizeof(uint32_t)) + 1;  // lo fits
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    st = gs2d_plan_init(&plan, width, height, n, mid, cfg);
    if (st == GS2D_OK && plan.ws_bytes <= kNoallocBytes) lo = mid; else hi = mid;
  }
  st = gs2d_plan_init(&plan, width, height, n, lo, cfg);
  if (st != GS2D_OK) return st;
  void* ws = nullptr;
  cudaError_t e = scratch_address(&ws);
  cudaStream_t s = (cudaStream_t)stream;
  // The array keeps the previous call's contents, laid out for whatever frame
  // that call had.  The header (status word and counters) and the per-tile
  // entry counters and the render-queue class counters must start at zero;
  // every other section is written before it is read within one call.
  if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(ws_ptr<int>(ws, plan, kOffTileCnt), 0,
                        (size_t)plan.num_tiles * sizeof(int), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(ws_ptr<int>(ws, plan, kOffBucket), 0, 2 * kBuckets * sizeof(int), s);
  if (e == cudaSuccess) e = launch_project(plan, ws, params, s);
  if (e == cudaSuccess) e = launch_bin_sort(plan, ws, s);
  if (e == cudaSuccess) e = launch_render_fwd(plan, ws, img, s);
  if (e == cudaSuccess && status) {
    k_noalloc_status<<<1, 1, 0, s>>>(ws_ptr<WsHeader>(ws, plan, kOffHeader), status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "gs2d_render_fwd_noalloc: %s", cudaGetErrorString(e));
    return set_error(GS2D_ERR_CUDA, msg);
  }
  return set_error(GS2D_OK, "");
}
