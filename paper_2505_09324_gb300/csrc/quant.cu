// Quantisation of Gaussian parameters (Sec. 3.3 A): IEEE half or uniform
// scalar quantisers per parameter row; post-training quantisation and the
// fake quantisation of quantisation-aware fitting (QAT).
#include <cooperative_groups.h>
#include <cuda_fp16.h>
#include <math.h>

#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

struct QuantArgs {
  int bits[9];
  float lo[9], hi[9], scale[9], step[9];
};

// One parameter: code and dequantised value.
__device__ __forceinline__ void quant_one(float x, int b, float lo, float scale, float step,
                                          uint16_t& c, float& y) {
  c = 0;
  y = x;
  if (b < 0) {  // IEEE half, round to nearest even; NaN as 0x7E00
    const __half h = __float2half_rn(x);
    c = isnan(x) ? (uint16_t)0x7E00 : __half_as_ushort(h);
    y = __half2float(h);
  } else if (b > 0) {
    const float top = (float)((1 << b) - 1);
    float k = isfinite(x) ? rintf(__fmul_rn(__fsub_rn(x, lo), scale)) : 0.0f;
    k = fminf(fmaxf(k, 0.0f), top);
    c = (uint16_t)k;
    y = __fadd_rn(lo, __fmul_rn(k, step));
  }
}

// Caller-given ranges: grid-stride over all 9 n parameters.
__global__ void __launch_bounds__(256)
k_quantize(const float* __restrict__ params, int n, QuantArgs q, uint16_t* __restrict__ codes,
           float* __restrict__ dequant, float* __restrict__ ranges) {
  pdl_begin();
  if (ranges && blockIdx.x == 0 && threadIdx.x < 9) {
    const int r = threadIdx.x;
    ranges[r] = q.bits[r] > 0 ? q.lo[r] : 0.0f;
    ranges[9 + r] = q.bits[r] > 0 ? q.hi[r] : 0.0f;
  }
  const size_t total = (size_t)9 * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / n);
    uint16_t c;
    float y;
    quant_one(params[t], q.bits[r], q.lo[r], q.scale[r], q.step[r], c, y);
    if (codes) codes[t] = c;
    if (dequant) dequant[t] = y;
  }
}

// Refined ranges: a cluster of kRefineCluster blocks takes one row (blockIdx.y);
// each block reduces [min, max] of the finite values of its chunk, the
// cluster combines the partial ranges through distributed shared memory
// (min and max are order-independent, so every block derives the same range),
// then each block quantises its chunk.
constexpr int kRefineCluster = 8;
constexpr int kRefineThreads = 256;

__global__ void __cluster_dims__(kRefineCluster, 1, 1) __launch_bounds__(kRefineThreads)
k_quantize_refine(const float* __restrict__ params, int n, QuantArgs q,
                  uint16_t* __restrict__ codes, float* __restrict__ dequant,
                  float* __restrict__ ranges) {
  pdl_begin();
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ float s_lo[kRefineThreads / 32], s_hi[kRefineThreads / 32];
  __shared__ float s_part[2];
  __shared__ float s_q[3];
  const int r = blockIdx.y;
  const int b = q.bits[r];
  const int chunk = (n + kRefineCluster - 1) / kRefineCluster;
  const int i0 = min(n, (int)blockIdx.x * chunk), i1 = min(n, i0 + chunk);
  const float* row = params + (size_t)r * n;
  float lo = INFINITY, hi = -INFINITY;
  if (b > 0)
    for (int i = i0 + threadIdx.x; i < i1; i += kRefineThreads) {
      const float x = row[i];
      if (isfinite(x)) {
        lo = fminf(lo, x);
        hi = fmaxf(hi, x);
      }
    }
  for (int o = 16; o; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    s_lo[threadIdx.x >> 5] = lo;
    s_hi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kRefineThreads / 32; w++) {
      lo = fminf(lo, s_lo[w]);
      hi = fmaxf(hi, s_hi[w]);
    }
    s_part[0] = lo;
    s_part[1] = hi;
  }
  cluster.sync();  // every block's partial range is visible cluster-wide
  if (threadIdx.x == 0) {
    for (int k = 0; k < kRefineCluster; k++) {
      const float* part = cluster.map_shared_rank(s_part, k);
      lo = fminf(lo, part[0]);
      hi = fmaxf(hi, part[1]);
    }
    if (!(lo <= hi)) lo = hi = 0.0f;  // no finite value (or not a uniform row)
    float scale = 0.0f, step = 0.0f;
    if (b > 0 && hi > lo) {
      const double levels = (double)((1 << b) - 1);
      const double d = (double)hi - (double)lo;
      scale = __double2float_rn(levels / d);
      step = __double2float_rn(d / levels);
    }
    s_q[0] = b > 0 ? lo : 0.0f;
    s_q[1] = scale;
    s_q[2] = step;
    if (ranges && blockIdx.x == 0) {
      ranges[r] = b > 0 ? lo : 0.0f;
      ranges[9 + r] = b > 0 ? hi : 0.0f;
    }
  }
  __syncthreads();
  const float qlo = s_q[0], scale = s_q[1], step = s_q[2];
  for (int i = i0 + threadIdx.x; i < i1; i += kRefineThreads) {
    uint16_t c;
    float y;
    quant_one(row[i], b, qlo, scale, step, c, y);
    if (codes) codes[(size_t)r * n + i] = c;
    if (dequant) dequant[(size_t)r * n + i] = y;
  }
  cluster.sync();  // no block leaves while a peer may still read its s_part
}

}  // namespace

cudaError_t launch_quantize(const float* params, int n, const gs2d_quant& q, uint16_t* codes,
                            float* dequant, float* ranges, cudaStream_t s) {
  QuantArgs a;
  for (int r = 0; r < 9; r++) {
    a.bits[r] = q.bits[r];
    // refined ranges of an empty set are [0, 0]
    a.lo[r] = q.refine ? 0.0f : q.lo[r];
    a.hi[r] = q.refine ? 0.0f : q.hi[r];
    a.scale[r] = q.scale[r];
    a.step[r] = q.step[r];
  }
  if (n > 0 && q.refine) {
    return launch_pdl(k_quantize_refine, dim3(kRefineCluster, 9), kRefineThreads, 0, s, params,
                      n, a, codes, dequant, ranges);
  }
  const size_t want = ((size_t)9 * (n > 0 ? n : 0) + 255) / 256;
  const int blocks = (int)(want < 1 ? 1 : (want < 152 * 8 ? want : 152 * 8));
  return launch_pdl(k_quantize, blocks, 256, 0, s, params, n > 0 ? n : 0, a, codes, dequant,
                    ranges);
}

}  // namespace gs2d

using namespace gs2d;

static bool quant_valid(const gs2d_quant* q) {
  if (!q) return false;
  for (int r = 0; r < 9; r++) {
    const int b = q->bits[r];
    if (!(b == -16 || (b >= 0 && b <= 16))) return false;
    if (b > 0 && !q->refine &&
        !(isfinite(q->lo[r]) && isfinite(q->scale[r]) && isfinite(q->step[r]) &&
          q->scale[r] > 0.0f && q->step[r] > 0.0f))
      return false;
  }
  return true;
}

extern "C" gs2d_status gs2d_quantize(const float* params, int32_t n, const gs2d_quant* q,
                                     uint16_t* codes, float* dequant, float* ranges,
                                     void* stream) {
  if (n < 0 || !quant_valid(q) || (n > 0 && (!params || (!codes && !dequant))))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_quantize: arguments");
  const cudaError_t e =
      launch_quantize(params, n, *q, codes, dequant, ranges, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(GS2D_ERR_CUDA, cudaGetErrorString(e));
  return set_error(GS2D_OK, "");
}

extern "C" gs2d_status gs2d_fit_step_qat(const gs2d_plan* plan, void* ws, const float* target,
                                         float* params, float* adam_m, float* adam_v,
                                         const gs2d_quant* q, void* stream) {
  if (!plan || plan->magic != kPlanMagic || !ws || ((uintptr_t)ws % 256) || !target ||
      !quant_valid(q) || (plan->n > 0 && (!params || !adam_m || !adam_v)))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_fit_step_qat: arguments");
  const gs2d_plan& p = *plan;
  cudaStream_t s = (cudaStream_t)stream;
  float* pq = ws_ptr<float>(ws, p, kOffQuant);
  cudaError_t e = launch_quantize(params, p.n, *q, nullptr, pq, nullptr, s);
  if (e == cudaSuccess) e = launch_prepare_fit(p, ws, pq, s);
  if (e == cudaSuccess) e = launch_fit_step(p, ws, target, params, adam_m, adam_v, s, pq);
  if (e != cudaSuccess) return set_error(GS2D_ERR_CUDA, cudaGetErrorString(e));
  return set_error(GS2D_OK, "");
}

// ---------------------------------------------------------------------------
// Post-training calibration (Sec. 3.3 A: the quantisation parameters are
// fixed from representative fitted frames): order statistics of every row's
// finite values by a radix select on order-preserving 32-bit keys.
namespace gs2d {
namespace {

constexpr int kCalSlots = 4;  // ranks per row: floor and ceiling of two positions

__device__ __forceinline__ uint32_t order_key(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_value(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Finite values per row (block r).
__global__ void __launch_bounds__(256)
k_cal_count(const float* __restrict__ params, int n, long long* __restrict__ count) {
  __shared__ long long s_c[8];
  long long c = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) c += isfinite(params[(size_t)blockIdx.x * n + i]);
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < 8; w++) t += s_c[w];
    count[blockIdx.x] = t;
  }
}

// Block (r, slot): the rank[r][slot]-th smallest (0-based) finite value of
// row r, found digit by digit (8 bits at a time, most significant first):
// each pass histograms the keys that match the digits found so far and keeps
// the bucket holding the rank.  rank < 0: no value (NaN out).
__global__ void __launch_bounds__(512)
k_cal_select(const float* __restrict__ params, int n, const long long* __restrict__ rank,
             float* __restrict__ out) {
  __shared__ unsigned hist[256];
  __shared__ uint32_t s_prefix, s_mask;
  __shared__ long long s_k;
  const int r = blockIdx.x / kCalSlots;
  const long long k0 = rank[blockIdx.x];
  if (k0 < 0) {
    if (threadIdx.x == 0) out[blockIdx.x] = __int_as_float(0x7fc00000);
    return;
  }
  if (threadIdx.x == 0) {
    s_prefix = 0u;
    s_mask = 0u;
    s_k = k0;
  }
  const float* row = params + (size_t)r * n;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    const uint32_t prefix = s_prefix, mask = s_mask;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float x = row[i];
      if (!isfinite(x)) continue;
      const uint32_t key = order_key(x);
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long k = s_k;
      int b = 0;
      while (b < 255 && k >= (long long)hist[b]) k -= hist[b++];
      s_k = k;
      s_prefix = prefix | ((uint32_t)b << shift);
      s_mask = mask | (255u << shift);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = key_value(s_prefix);
}

}  // namespace
}  // namespace gs2d

// numpy's linear quantile interpolation between order statistics a and b.
static double lerp_quantile(double a, double b, double t) {
  const double d = b - a;
  return t >= 0.5 ? b - d * (1.0 - t) : a + d * t;
}

extern "C" gs2d_status gs2d_quant_calibrate(const float* params, int32_t n, const int32_t* bits,
                                            double coverage, void* scratch, size_t scratch_bytes,
                                            float* lo, float* hi, void* stream) {
  if (n < 0 || !bits || !lo || !hi || !scratch || scratch_bytes < gs2d_quant_calibrate_scratch_bytes() ||
      (n > 0 && !params) || !(coverage > 0.0 && coverage <= 1.0))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_quant_calibrate: arguments");
  for (int r = 0; r < 9; r++)
    if (!(bits[r] == -16 || (bits[r] >= 0 && bits[r] <= 16)))
      return set_error(GS2D_ERR_INVALID_ARG, "gs2d_quant_calibrate: bits");
  cudaStream_t s = (cudaStream_t)stream;
  long long* d_count = static_cast<long long*>(scratch);
  long long* d_rank = d_count + 16;
  float* d_val = reinterpret_cast<float*>(d_rank + 9 * kCalSlots);
  long long count[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  cudaError_t e = cudaSuccess;
  if (n > 0) {
    k_cal_count<<<9, 256, 0, s>>>(params, n, d_count);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(count, d_count, sizeof(count), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  // positions of the central `coverage` interval (numpy's default method)
  const double q = (1.0 - coverage) / 2.0;
  long long rank[9 * kCalSlots];
  double frac[9][2];
  for (int r = 0; r < 9; r++) {
    const long long N = bits[r] > 0 ? count[r] : 0;
    for (int j = 0; j < 2; j++) {
      const double h = (double)(N - 1) * (j == 0 ? q : 1.0 - q);
      const long long f = N > 0 ? (long long)floor(h) : -1;
      rank[r * kCalSlots + 2 * j] = f;
      rank[r * kCalSlots + 2 * j + 1] = N > 0 ? (f + 1 < N ? f + 1 : N - 1) : -1;
      frac[r][j] = N > 0 ? h - (double)f : 0.0;
    }
  }
  float val[9 * kCalSlots];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_rank, rank, sizeof(rank), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n > 0) {
    k_cal_select<<<9 * kCalSlots, 512, 0, s>>>(params, n, d_rank, d_val);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n > 0)
    e = cudaMemcpyAsync(val, d_val, sizeof(val), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(GS2D_ERR_CUDA, cudaGetErrorString(e));
  for (int r = 0; r < 9; r++) {
    double a = 0.0, b = 1.0;
    if (bits[r] > 0 && n > 0 && count[r] > 0) {
      a = lerp_quantile(val[r * kCalSlots], val[r * kCalSlots + 1], frac[r][0]);
      b = lerp_quantile(val[r * kCalSlots + 2], val[r * kCalSlots + 3], frac[r][1]);
      if (!(b > a)) b = a + 1.0;
    }
    lo[r] = (float)a;
    hi[r] = (float)b;
  }
  return set_error(GS2D_OK, "");
}

extern "C" size_t gs2d_quant_calibrate_scratch_bytes(void) {
  return 16 * sizeof(long long) + 9 * kCalSlots * (sizeof(long long) + sizeof(float));
}
