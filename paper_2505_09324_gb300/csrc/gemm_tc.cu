// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05), the dense
// contraction of the learned initialiser's convolutions (forward, weight
// gradient and input gradient are each one GEMM over an im2col operand):
//
//   C[M][N] = A[M][K] . B[N][K]^T      A, B bf16, both K-contiguous (K-major);
//                                       FP32 accumulation in tensor memory.
//
// One CTA computes a 128 x BN tile (BN = 32 ... 256) over a range of K:
//   warp 0, one lane   TMA producer: 128 x 64 A and BN x 64 B boxes per stage
//                      into 128-byte-swizzled shared memory, ST deep (2 for
//                      short K, so that more blocks share an SM; else 4);
//   warp 1, one lane   MMA issuer: four 128 x BN x 16 tcgen05.mma per stage,
//                      a tcgen05.commit per stage frees the stage, one more
//                      signals the finished accumulator;
//   warps 0-3          epilogue: tcgen05.ld of the warp's 32 accumulator rows
//                      (TMEM lanes), bias, ReLU, store as FP32 or BF16.
// Long K is split over gridDim.z (split-K): each split writes an FP32 partial
// tile and k_splitk_reduce sums the splits in a fixed order (deterministic).
//
// Every wait on an mbarrier is bounded in time (%globaltimer, 1 s unless the
// launch asks for less): on a timeout the kernel records GS2D_ERR_TIMEOUT in
// the caller's status word, skips the rest of its work, still frees its tensor
// memory and returns.  gs2d_gemm_wait_check exercises that path: its launch
// withholds every load, so the first wait on a stage runs out while no TMA
// copy or MMA is in flight.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdio.h>

#include <mutex>

#include "gs2d_internal.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace gs2d {
namespace {

template <int BN, int ST>
struct GemmShape {
  static constexpr int kTmemCols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  static constexpr int kABytes = kBM * kBK * 2;  // 16 KB
  static constexpr int kBBytes = BN * kBK * 2;
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kSmem = ST * kStageBytes + 1024;  // + alignment slack
};

// Epilogue of one 128 x BN accumulator tile: warp w (0 ... 3) reads TMEM lanes
// 32 w ... 32 w + 31 (its accumulator rows), adds the bias, applies ReLU and
// stores FP32 or BF16 (16-byte vectors where the row allows).
template <int BN>
__device__ __forceinline__ void store_tile(const TcGemmArgs& g, uint32_t tmem, int warp, int lane,
                                           int m0, int n0, int z) {
  const int row = m0 + warp * 32 + lane;
  const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
  float* out32 = g.out_f32 ? g.out_f32 + (size_t)z * g.split_stride : nullptr;
  // rows of 16-byte aligned, full 16-column chunks take vector stores
  const void* obase = g.out_bf16 ? (const void*)g.out_bf16 : (const void*)out32;
  const bool vec_ok = (g.ldc % 8) == 0 && (reinterpret_cast<uintptr_t>(obase) & 15) == 0;
#pragma unroll 1
  for (int c = 0; c < BN; c += 16) {
    float v[16];
    tmem_ld16(tbase + (uint32_t)c, v);
    if (row < g.M) {
      const int n = n0 + c;
#pragma unroll
      for (int j = 0; j < 16; j++) {
        float x = v[j];
        if (g.bias && n + j < g.N) x += g.bias[n + j];
        if (g.relu) x = fmaxf(x, 0.0f);
        v[j] = x;
      }
      const size_t o = (size_t)row * g.ldc + n;
      if (vec_ok && n + 16 <= g.N) {
        if (g.out_bf16) {
          __align__(16) __nv_bfloat162 h[8];
#pragma unroll
          for (int j = 0; j < 8; j++) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
          uint4* dst = reinterpret_cast<uint4*>(g.out_bf16 + o);
          dst[0] = reinterpret_cast<const uint4*>(h)[0];
          dst[1] = reinterpret_cast<const uint4*>(h)[1];
        } else {
          float4* dst = reinterpret_cast<float4*>(out32 + o);
#pragma unroll
          for (int j = 0; j < 4; j++)
            dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; j++) {
          if (n + j < g.N) {
            if (g.out_bf16)
              g.out_bf16[o + j] = __float2bfloat16_rn(v[j]);
            else
              out32[o + j] = v[j];
          }
        }
      }
    }
  }
}

template <int BN, int ST>
__global__ void __launch_bounds__(128, 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
            TcGemmArgs g) {
  constexpr int kStages = ST;
  using Sh = GemmShape<BN, ST>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accum;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int kt0 = blockIdx.z * g.kt_per_split;
  const int nk = min(g.num_kt, kt0 + g.kt_per_split) - kt0;  // >= 1 (host)

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accum, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(Sh::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0 && lane == 0) {
    // producer (a failure-detection launch withholds every load)
    for (int i = 0; i < nk && !g.withhold_loads; i++) {
      const int s = i % kStages;
      const uint32_t ph = (uint32_t)(i / kStages) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u, g.wait_ns)) {  // the preceding phase: free at first
        s_fail = 1;
        break;
      }
      uint8_t* a_s = smem + s * Sh::kStageBytes;
      uint8_t* b_s = a_s + Sh::kABytes;
      mbar_expect_tx(&full[s], (uint32_t)Sh::kStageBytes);
      tma_load_2d(a_s, &ta, &full[s], (kt0 + i) * kBK, m0);
      tma_load_2d(b_s, &tb, &full[s], (kt0 + i) * kBK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);
    for (int i = 0; i < nk; i++) {
      const int s = i % kStages;
      const uint32_t ph = (uint32_t)(i / kStages) & 1u;
      if (!mbar_wait(&full[s], ph, g.wait_ns)) {
        s_fail = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a_s = smem_u32(smem + s * Sh::kStageBytes);
      const uint32_t b_s = a_s + Sh::kABytes;
      const uint64_t ad = sw128_desc(a_s), bd = sw128_desc(b_s);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; kk++)  // 16 bf16 = 32 bytes = 2 descriptor units
        mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(&accum);
  }
  __syncwarp();

  // epilogue: warp w holds accumulator rows 32 w ... 32 w + 31
  const bool ready = mbar_wait(&accum, 0, g.wait_ns);
  tc_fence_after();
  if (!ready) s_fail = 1;
  __syncthreads();
  if (!s_fail) store_tile<BN>(g, tmem, warp, lane, m0, n0, blockIdx.z);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Sh::kTmemCols));
  if (threadIdx.x == 0 && s_fail && g.status) atomicCAS(g.status, 0, (int)GS2D_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Implicit-GEMM convolution: the same product with A = col(X) never written
// out.  Warps 0-3 (one output pixel per thread) gather each k-tile's A rows
// from the NHWC input (eight 16-byte chunks per row: a tap's 8 channels, the
// bias column of ones, or zeros) straight into the 128-byte-swizzled layout a
// TMA box would have, fence them for the async proxy and arrive on the
// stage's barrier; thread 0 also brings the weights' B box by TMA.  Warp 4,
// one lane, issues the MMAs; warps 0-3 run the epilogue.
struct ConvGeom {
  const __nv_bfloat16* x;  // [B][Hi][Wi][C]
  int Hi, Wi, C, Ho, Wo, ks, stride, pad;
};

template <int BN, int ST>
__global__ void __launch_bounds__(160, 1)
k_conv_bf16(const __grid_constant__ CUtensorMap tb, ConvGeom cg, TcGemmArgs g) {
  constexpr int kStages = ST;
  using Sh = GemmShape<BN, ST>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accum;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int nk = g.num_kt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&full[s], kBM + 1);  // one arrival per A row + the B box's
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accum, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(Sh::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp < 4) {
    // producers: row r = output pixel m0 + r.  Each k-tile's chunks go out as
    // 16-byte cp.async copies (zero-filled outside the image), one commit
    // group per k-tile; a k-tile's rows are announced on its barrier once
    // its group has landed (cp.async.wait_group), kLag k-tiles later: kLag + 1
    // k-tiles of gathers in flight per thread, while the announcement of a
    // k-tile never waits for the MMA of the one before it.
    constexpr int kLag = kStages > 2 ? kStages - 2 : 1;
    const int r = threadIdx.x, p = m0 + r;
    const bool row_ok = p < g.M;
    const int hw = cg.Ho * cg.Wo;
    const int b = row_ok ? p / hw : 0, rem = row_ok ? p - b * hw : 0;
    const int oy = rem / cg.Wo, ox = rem - (rem / cg.Wo) * cg.Wo;
    const int taps = cg.ks * cg.ks;
    const __nv_bfloat16* xb = cg.x + (size_t)b * cg.Hi * cg.Wi * cg.C;
    const int iy0 = oy * cg.stride - cg.pad, ix0 = ox * cg.stride - cg.pad;
    // position of the next chunk in k = (ky ks + kx) C + ci, advanced chunk by
    // chunk (no divisions in the loop)
    int ky = 0, kx = 0, tap = 0, ci = 0;
    int announced = 0;  // k-tiles whose rows have been announced
    for (int i = 0; i < nk; i++) {
      const int s = i % kStages;
      const uint32_t ph = (uint32_t)(i / kStages) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        s_fail = 1;
        break;
      }
      uint8_t* a_s = smem + s * Sh::kStageBytes;
      if (r == 0) {  // the weights' box: its own arrival on the stage barrier
        mbar_expect_tx(&full[s], (uint32_t)Sh::kBBytes);
        tma_load_2d(a_s + Sh::kABytes, &tb, &full[s], i * kBK, n0);
      }
#pragma unroll
      for (int q = 0; q < 8; q++) {
        uint8_t* dst = a_s + r * 128 + ((q ^ (r & 7)) << 4);
        if (row_ok && tap < taps) {
          const int iy = iy0 + ky, ix = ix0 + kx;
          const bool in = iy >= 0 && iy < cg.Hi && ix >= 0 && ix < cg.Wi;
          const __nv_bfloat16* src = in ? xb + ((size_t)iy * cg.Wi + ix) * cg.C + ci : cg.x;
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)),
                       "l"(src), "r"(in ? 16 : 0)
                       : "memory");
        } else {
          // the bias column of ones (bf16 1.0 in the first element), else zeros
          const bool one = row_ok && tap == taps && ci == 0;
          *reinterpret_cast<uint4*>(dst) = make_uint4(one ? 0x3F80u : 0u, 0u, 0u, 0u);
        }
        ci += 8;
        if (ci == cg.C) {
          ci = 0;
          tap++;
          if (++kx == cg.ks) {
            kx = 0;
            ky++;
          }
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      if (i >= kLag) {
        asm volatile("cp.async.wait_group %0;" ::"n"(kLag) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&full[announced % kStages]);
        announced++;
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!s_fail)
      for (; announced < nk; announced++) mbar_arrive(&full[announced % kStages]);
  } else if (lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);
    for (int i = 0; i < nk; i++) {
      const int s = i % kStages;
      const uint32_t ph = (uint32_t)(i / kStages) & 1u;
      if (!mbar_wait(&full[s], ph)) {
        s_fail = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a_s = smem_u32(smem + s * Sh::kStageBytes);
      const uint32_t b_s = a_s + Sh::kABytes;
      const uint64_t ad = sw128_desc(a_s), bd = sw128_desc(b_s);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; kk++)
        mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(&accum);
  }
  __syncwarp();

  const bool ready = warp < 4 ? mbar_wait(&accum, 0) : true;
  tc_fence_after();
  if (!ready) s_fail = 1;
  __syncthreads();
  if (!s_fail && warp < 4) store_tile<BN>(g, tmem, warp, lane, m0, n0, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Sh::kTmemCols));
  if (threadIdx.x == 0 && s_fail && g.status) atomicCAS(g.status, 0, (int)GS2D_ERR_TIMEOUT);
}

// Sum of the split-K partials in split order, then bias, ReLU and the store.
__global__ void __launch_bounds__(256)
k_splitk_reduce(TcGemmArgs g, int splits, const float* __restrict__ partial) {
  const size_t total = (size_t)g.M * g.N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(i / g.N), n = (int)(i % g.N);
    const size_t o = (size_t)m * g.ldc + n;
    float x = 0.0f;
    for (int z = 0; z < splits; z++) x += partial[(size_t)z * g.split_stride + o];
    if (g.bias) x += g.bias[n];
    if (g.relu) x = fmaxf(x, 0.0f);
    if (g.out_bf16)
      g.out_bf16[o] = __float2bfloat16_rn(x);
    else
      g.out_f32[o] = x;
  }
}

template <int BN, int ST>
cudaError_t launch_bn_st(const CUtensorMap& ta, const CUtensorMap& tb, const TcGemmArgs& g,
                         dim3 grid, cudaStream_t s) {
  const cudaError_t attr = opt_in_smem((const void*)k_gemm_bf16<BN, ST>, GemmShape<BN, ST>::kSmem);
  if (attr != cudaSuccess) return attr;
  k_gemm_bf16<BN, ST><<<grid, 128, GemmShape<BN, ST>::kSmem, s>>>(ta, tb, g);
  return cudaGetLastError();
}

template <int BN, int ST>
cudaError_t launch_conv_st(const CUtensorMap& tb, const ConvGeom& cg, const TcGemmArgs& g,
                           dim3 grid, cudaStream_t s) {
  const cudaError_t attr = opt_in_smem((const void*)k_conv_bf16<BN, ST>, GemmShape<BN, ST>::kSmem);
  if (attr != cudaSuccess) return attr;
  k_conv_bf16<BN, ST><<<grid, 160, GemmShape<BN, ST>::kSmem, s>>>(tb, cg, g);
  return cudaGetLastError();
}

// Two stages up to 16 k-tiles, three beyond: shared memory for more CTAs per
// SM hides more latency than a deeper pipeline per CTA.
template <int BN>
cudaError_t launch_conv(const CUtensorMap& tb, const ConvGeom& cg, const TcGemmArgs& g,
                        dim3 grid, cudaStream_t s) {
  return g.num_kt <= 16 ? launch_conv_st<BN, 2>(tb, cg, g, grid, s)
                        : launch_conv_st<BN, 3>(tb, cg, g, grid, s);
}

// Two stages when every block runs few k-tiles (more blocks per SM hide the
// per-block latency), four otherwise.
template <int BN>
cudaError_t launch_bn(const CUtensorMap& ta, const CUtensorMap& tb, const TcGemmArgs& g,
                      dim3 grid, cudaStream_t s) {
  return g.kt_per_split <= 8 ? launch_bn_st<BN, 2>(ta, tb, g, grid, s)
                             : launch_bn_st<BN, 4>(ta, tb, g, grid, s);
}

}  // namespace

EncodeTiled tensor_map_encoder() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// 2D bf16 tensor map of a rows x cols (K-contiguous) matrix with leading
// dimension ld (elements), box 64 (K) x box_rows, 128-byte swizzle,
// out-of-range elements read as zero.
bool make_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows) {
  EncodeTiled fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Tile width for N columns: one tile up to 256, else the fewest tiles of a
// multiple of 16 columns.
int tc_gemm_bn(int n) {
  if (n <= 32) return 32;
  if (n <= 64) return 64;
  if (n <= 96) return 96;
  if (n <= 128) return 128;
  if (n <= 192) return 192;
  if (n <= 256) return 256;
  const int tiles = (n + 255) / 256;
  const int per = (n + tiles - 1) / tiles;
  return per <= 192 ? 192 : 256;
}

cudaError_t tc_gemm(const TcGemmProblem& pr, cudaStream_t s) {
  if (pr.M <= 0 || pr.N <= 0 || pr.K <= 0) return cudaSuccess;
  if (pr.lda % 8 || pr.ldb % 8 || (reinterpret_cast<uintptr_t>(pr.A) & 15) ||
      (reinterpret_cast<uintptr_t>(pr.B) & 15))
    return cudaErrorInvalidValue;  // TMA: 16-byte aligned rows
  const int bn = tc_gemm_bn(pr.N);
  CUtensorMap ta, tb;
  if (!make_map(&ta, pr.A, pr.M, pr.K, pr.lda, kBM) ||
      !make_map(&tb, pr.B, pr.N, pr.K, pr.ldb, bn))
    return cudaErrorInvalidValue;
  const int num_kt = (pr.K + kBK - 1) / kBK;
  int splits = pr.splits < 1 ? 1 : pr.splits;
  if (splits > num_kt) splits = num_kt;
  const int per = (num_kt + splits - 1) / splits;
  splits = (num_kt + per - 1) / per;  // every split gets at least one k-tile
  TcGemmArgs g;
  g.M = pr.M;
  g.N = pr.N;
  g.num_kt = num_kt;
  g.kt_per_split = per;
  g.ldc = pr.ldc;
  g.bias = pr.bias;
  g.relu = pr.relu;
  g.status = pr.status;
  g.wait_ns = pr.wait_ns;
  g.withhold_loads = pr.withhold_loads;
  g.split_stride = (size_t)pr.M * pr.ldc;
  if (splits == 1) {
    g.out_f32 = pr.out_f32;
    g.out_bf16 = pr.out_bf16;
  } else {
    if (!pr.partial) return cudaErrorInvalidValue;
    g.out_f32 = pr.partial;  // FP32 partials, epilogue in the reduction
    g.out_bf16 = nullptr;
    g.bias = nullptr;
    g.relu = 0;
  }
  const dim3 grid((pr.M + kBM - 1) / kBM, (pr.N + bn - 1) / bn, splits);
  cudaError_t e;
  switch (bn) {
    case 32: e = launch_bn<32>(ta, tb, g, grid, s); break;
    case 64: e = launch_bn<64>(ta, tb, g, grid, s); break;
    case 96: e = launch_bn<96>(ta, tb, g, grid, s); break;
    case 128: e = launch_bn<128>(ta, tb, g, grid, s); break;
    case 192: e = launch_bn<192>(ta, tb, g, grid, s); break;
    default: e = launch_bn<256>(ta, tb, g, grid, s); break;
  }
  if (e != cudaSuccess || splits == 1) return e;
  TcGemmArgs r = g;
  r.out_f32 = pr.out_f32;
  r.out_bf16 = pr.out_bf16;
  r.bias = pr.bias;
  r.relu = pr.relu;
  const size_t total = (size_t)pr.M * pr.N;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
  k_splitk_reduce<<<blocks, 256, 0, s>>>(r, splits, pr.partial);
  return cudaGetLastError();
}

cudaError_t tc_conv(const TcConvProblem& pr, cudaStream_t s) {
  const int Ho = (pr.Hi + 2 * pr.pad - pr.ks) / pr.stride + 1;
  const int Wo = (pr.Wi + 2 * pr.pad - pr.ks) / pr.stride + 1;
  const int M = pr.B * Ho * Wo;
  if (M <= 0 || pr.N <= 0) return cudaSuccess;
  if (pr.C % 8 || pr.ldk % 8 || pr.ldk < pr.ks * pr.ks * pr.C + 1 ||
      (reinterpret_cast<uintptr_t>(pr.x) & 15) || (reinterpret_cast<uintptr_t>(pr.W) & 15))
    return cudaErrorInvalidValue;
  // wide output rows: the persistent kernels with TMA row or tap loads
  // (same result)
  if (rows_conv_supported(pr)) return rows_conv(pr, s);
  if (tap_conv_supported(pr)) return tap_conv(pr, s);
  const int bn = tc_gemm_bn(pr.N);
  CUtensorMap tb;
  if (!make_map(&tb, pr.W, pr.N, pr.ldk, pr.ldk, bn)) return cudaErrorInvalidValue;
  ConvGeom cg;
  cg.x = pr.x;
  cg.Hi = pr.Hi;
  cg.Wi = pr.Wi;
  cg.C = pr.C;
  cg.Ho = Ho;
  cg.Wo = Wo;
  cg.ks = pr.ks;
  cg.stride = pr.stride;
  cg.pad = pr.pad;
  TcGemmArgs g;
  g.M = M;
  g.N = pr.N;
  g.num_kt = (pr.ldk + kBK - 1) / kBK;
  g.kt_per_split = g.num_kt;
  g.ldc = pr.ldc;
  g.split_stride = 0;
  g.out_f32 = pr.out_f32;
  g.out_bf16 = pr.out_bf16;
  g.bias = nullptr;
  g.relu = pr.relu;
  g.status = pr.status;
  g.wait_ns = 0;
  g.withhold_loads = 0;
  const dim3 grid((M + kBM - 1) / kBM, (pr.N + bn - 1) / bn, 1);
  switch (bn) {
    case 32: return launch_conv<32>(tb, cg, g, grid, s);
    case 64: return launch_conv<64>(tb, cg, g, grid, s);
    case 96: return launch_conv<96>(tb, cg, g, grid, s);
    case 128: return launch_conv<128>(tb, cg, g, grid, s);
    case 192: return launch_conv<192>(tb, cg, g, grid, s);
    default: return launch_conv<256>(tb, cg, g, grid, s);
  }
}

size_t tc_gemm_partial_floats(int M, int N, int ldc, int K, int splits) {
  const int num_kt = (K + kBK - 1) / kBK;
  if (splits > num_kt) splits = num_kt;
  if (splits <= 1) return 0;
  (void)N;
  return (size_t)splits * M * ldc;
}

}  // namespace gs2d
