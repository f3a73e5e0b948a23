// Throughput probes of the two pipes the render kernels are bound by: FP32
// fused multiply-adds (the FMA pipe) and the MUFU base-2 exponential.  They
// are not part of the paper's method: they measure, on the running device and
// at its current clock, the denominators the render kernels' roofline
// fractions are quoted against (issue-limited peaks are below the nominal
// lane count times the clock).
//
// Each thread runs 8 independent dependency chains (enough to cover the pipe
// latency at full occupancy), 16 unrolled steps per loop iteration; thread 0
// of each block stores the block's sum so that no chain is dead code.
#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kProbeThreads) k_probe_ffma(int iters, float* __restrict__ sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = 1.0f + 1e-3f * (float)(threadIdx.x + k);
  const float b = 0.999f, c = 1e-3f;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < kUnroll; u++)
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  if (threadIdx.x == 0) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_ex2(int iters, float* __restrict__ sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = 1e-3f * (float)(threadIdx.x + k);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < kUnroll; u++)
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = ex2_approx(-a[k]);  // stays in [1/2, 1]
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  if (threadIdx.x == 0) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace gs2d

using namespace gs2d;

extern "C" int64_t gs2d_probe_ops(int32_t blocks, int32_t iters) {
  if (blocks < 1 || iters < 1) return 0;
  return (int64_t)blocks * kProbeThreads * iters * kUnroll * kChains;
}

extern "C" gs2d_status gs2d_probe_peak(int32_t kind, int32_t blocks, int32_t iters, float* sink,
                                       void* stream) {
  if ((kind != GS2D_PROBE_FFMA && kind != GS2D_PROBE_EX2) || blocks < 1 || iters < 1 || !sink)
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_probe_peak: invalid kind, size or sink");
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == GS2D_PROBE_FFMA)
    k_probe_ffma<<<blocks, kProbeThreads, 0, s>>>(iters, sink);
  else
    k_probe_ex2<<<blocks, kProbeThreads, 0, s>>>(iters, sink);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GS2D_ERR_CUDA, cudaGetErrorString(e));
  return set_error(GS2D_OK, "");
}
