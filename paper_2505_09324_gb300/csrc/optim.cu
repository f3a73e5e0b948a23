// Adam over a flat parameter array (the fitting "optimization steps" of
// Sec. 4.1; Adam with bias correction and a constant learning rate is the
// project's reading, the paper names no optimiser).  Vectorised float4 path
// when count is a multiple of 4 and the arrays are 16-byte aligned.
#include "gs2d_internal.cuh"

namespace gs2d {

__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float lr, float b1,
                                      float b2, float eps, float ibc1, float ibc2) {
  m = fmaf(b1, m, (1.0f - b1) * g);
  v = fmaf(b2, v, (1.0f - b2) * g * g);
  p -= lr * (m * ibc1) / (sqrtf(v * ibc2) + eps);
}

__global__ void __launch_bounds__(256)
k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
       float* __restrict__ v, int64_t count, int64_t per_row, const uint8_t* __restrict__ mask,
       float lr, float b1, float b2, float eps, float ibc1, float ibc2) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (mask && !mask[k % per_row]) continue;
    float pp = p[k], mm = m[k], vv = v[k];
    adam1(pp, g[k], mm, vv, lr, b1, b2, eps, ibc1, ibc2);
    p[k] = pp;
    m[k] = mm;
    v[k] = vv;
  }
}

__global__ void __launch_bounds__(256)
k_adam4(float4* __restrict__ p, const float4* __restrict__ g, float4* __restrict__ m,
        float4* __restrict__ v, int64_t count4, float lr, float b1, float b2, float eps,
        float ibc1, float ibc2) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count4;
       k += (int64_t)gridDim.x * blockDim.x) {
    float4 pp = p[k], mm = m[k], vv = v[k];
    const float4 gg = g[k];
    adam1(pp.x, gg.x, mm.x, vv.x, lr, b1, b2, eps, ibc1, ibc2);
    adam1(pp.y, gg.y, mm.y, vv.y, lr, b1, b2, eps, ibc1, ibc2);
    adam1(pp.z, gg.z, mm.z, vv.z, lr, b1, b2, eps, ibc1, ibc2);
    adam1(pp.w, gg.w, mm.w, vv.w, lr, b1, b2, eps, ibc1, ibc2);
    p[k] = pp;
    m[k] = mm;
    v[k] = vv;
  }
}

cudaError_t launch_adam(float* params, const float* grads, float* m, float* v, int64_t count,
                        int32_t step, const uint8_t* mask, const gs2d_config& cfg,
                        cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const float ibc1 = (float)(1.0 / (1.0 - pow((double)cfg.beta1, (double)step)));
  const float ibc2 = (float)(1.0 / (1.0 - pow((double)cfg.beta2, (double)step)));
  const bool aligned =
      ((uintptr_t)params | (uintptr_t)grads | (uintptr_t)m | (uintptr_t)v) % 16 == 0;
  if (!mask && aligned && count % 4 == 0) {
    const int64_t c4 = count / 4;
    int64_t blocks = (c4 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_adam4<<<(int)blocks, 256, 0, s>>>((float4*)params, (const float4*)grads, (float4*)m,
                                        (float4*)v, c4, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps,
                                        ibc1, ibc2);
  } else {
    int64_t blocks = (count + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_adam<<<(int)blocks, 256, 0, s>>>(params, grads, m, v, count, count / 9 > 0 ? count / 9 : 1,
                                       mask, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps, ibc1, ibc2);
  }
  return cudaGetLastError();
}

}  // namespace gs2d
