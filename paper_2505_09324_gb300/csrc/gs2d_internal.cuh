// Internal definitions shared by the gs2d CUDA translation units (not part of
// the C ABI).  Workspace layout, the per-Gaussian render record, status codes
// and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs2d.h"

namespace gs2d {

constexpr uint64_t kPlanMagic = 0x67733264706c616eull;  // "gs2dplan"
constexpr int kTile = 16;                               // tile edge (pixels)
constexpr int kTilePix = kTile * kTile;                 // 256 pixels per tile
constexpr int kBatch = 256;                             // Gaussians staged per smem batch
constexpr int kRadixBits = 8;
constexpr int kRadixBuckets = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;  // per thread in the count scan
constexpr int kPartials = 8;   // backward accumulators per (tile, Gaussian)

// log2(e) / 2: scales the Cholesky-form coordinates so that
// q = u1^2 + u2^2 = sigma * log2(e), and exp(-sigma) = 2^-q.
constexpr float kSc2 = 0.72134752044448170368f;  // log2(e)/2
constexpr float kLn2 = 0.69314718055994530942f;

// Workspace sections (byte offsets stored in gs2d_plan::off).
enum WsSection {
  kOffHeader = 0,   // WsHeader
  kOffRec,          // float4[3][n]  render records (SoA of float4 rows)
  kOffRect,         // int4[n]       tile rectangle [tx0, ty0, tx1, ty1)
  kOffCount,        // int32[n + 1]  tile counts, then exclusive offsets
  kOffBlockSum,     // int32[...]    scan block sums
  kOffKeysA,        // uint32[max_entries]
  kOffKeysB,        // uint32[max_entries]
  kOffValsA,        // uint32[max_entries]
  kOffValsB,        // uint32[max_entries]
  kOffHist,         // uint32[kRadixBuckets * sort_blocks]
  kOffRanges,       // int2[num_tiles]
  kOffPartial,      // float[kPartials][max_entries] (SoA rows) backward partials
  kOffLossPart,     // float2[num_tiles]  per-tile (sum sq err, sum sq err clamped)
  kOffGrad,         // float[9 n] gradient scratch of the fit loop
  kNumSections
};

struct WsHeader {
  int32_t status;       // first device-detected error (gs2d_status), 0 if none
  int32_t n_entries;    // entries in the sorted list (0 when over capacity)
  int64_t entries_raw;  // total entries requested by the tile counts
  int32_t step;         // Adam step counter of the fit loop
  float bc1, bc2;       // Adam bias corrections for that step
  int32_t pad0;
  float loss[2];        // last reduced {loss, clamped mse}
  unsigned long long pairs, hits;  // gs2d_count_pairs results
  int32_t pad[50];
};
static_assert(sizeof(WsHeader) == 256, "header is one 256-byte block");

// Per-Gaussian render record, three float4 rows.
//   r0 = (mu_x, mu_y, a1, a2)      a1 = s/l1, a2 = s/l3, s = sqrt(log2(e)/2)
//   r1 = (k, tau2, c'_r, c'_g)     k = -l2/l3, tau2 = tau * log2(e), c' = w c
//   r2 = (c'_b, hx, hy, 0)         half extents of the tau-ellipse (+ slack)
// With dx = px - mu_x, dy = py - mu_y:
//   u1 = a1 dx, u2 = a2 dy + k u1, q = u1^2 + u2^2 = sigma log2(e),
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

__device__ __forceinline__ void set_status(WsHeader* h, int code) {
  atomicCAS(&h->status, 0, code);
}

// ---- launchers implemented in the .cu files (return cudaGetLastError) ----
cudaError_t launch_project(const gs2d_plan& p, void* ws, const float* params, cudaStream_t s);
cudaError_t launch_bin_sort(const gs2d_plan& p, void* ws, cudaStream_t s);
cudaError_t launch_render_fwd(const gs2d_plan& p, void* ws, float* img, cudaStream_t s);
cudaError_t launch_render_bwd(const gs2d_plan& p, void* ws, const float* params,
                              const float* dimg, float* grads, cudaStream_t s);
cudaError_t launch_render_l2(const gs2d_plan& p, void* ws, const float* params,
                             const float* target, float* grads, float* img, float* loss,
                             cudaStream_t s);
cudaError_t launch_fit_step(const gs2d_plan& p, void* ws, const float* target, float* params,
                            float* m, float* v, cudaStream_t s);
cudaError_t launch_adam(float* params, const float* grads, float* m, float* v, int64_t count,
                        int32_t step, const uint8_t* mask, const gs2d_config& cfg,
                        cudaStream_t s);
cudaError_t launch_loss_reduce(const gs2d_plan& p, void* ws, float* loss, cudaStream_t s);
cudaError_t launch_adam_tick(const gs2d_plan& p, void* ws, cudaStream_t s);
cudaError_t launch_count_pairs(const gs2d_plan& p, void* ws, cudaStream_t s);

// Records msg as the calling thread's last error (gs2d_last_error); returns st.
gs2d_status set_error(gs2d_status st, const char* msg);

}  // namespace gs2d
