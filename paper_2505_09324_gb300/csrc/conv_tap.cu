// Implicit-GEMM convolution fed by TMA tap loads: the learned initialiser's
// wide 3 x 3 stride-2 layers (paper section 3.2 B) as a persistent tcgen05
// kernel, one CTA per SM.  At 1080p it runs layer 4 (C = 128); the 3 x 3,
// stride-2, pad-1 layers with C = 32 or 64 and an even width go to the
// row-box kernel of csrc/conv_rows.cu (fewer, larger TMA boxes), and this
// kernel keeps every other supported shape.
//
//   Z[p][n] = sum_k col(X)[p][k] W[n][k],   k = (ky ks + kx) C + ci,
//   a column of ones at k = ks^2 C carrying the bias, zeros beyond.
//
// A tile is 128 consecutive output pixels of one output row.  For a fixed
// tap (ky, kx) and a chunk of cw channels, the tile's im2col rows are the
// input pixels x0 + kx, x0 + kx + stride, ... of input row y0 + ky: one TMA
// box of the NHWC input with traversal stride `stride` along W (out-of-image
// pixels read as zero), 128 rows x cw channels, which lands in shared memory
// in the K-major layout the MMA reads:
//   cw = 16  32-byte rows, 32-byte swizzle;
//   cw = 32  64-byte rows, 64-byte swizzle;
//   cw = 64  128-byte rows, 128-byte swizzle (C = 64 j: j chunks per tap).
// A k-tile is 64 K (16 KB of A, like one 128-byte swizzle row); the MMA
// sequence, K = 16 slice by K = 16 slice, is the one the GEMM over an im2col
// operand issues, so the output equals im2col + GEMM bit for bit.  The bias
// slice and the zero slice past it come from a constant block (unswizzled,
// 16-byte rows, its two core-matrix columns 2 KB apart).  C = 8 (16-byte rows,
// which TMA moves slowly with a traversal stride) stays with the gathering
// kernel of csrc/gemm_tc.cu.
//
// Roles: warp 0 (one lane) issues the TMA loads into an ST-deep ring of
// k-tile stages; warp 1 (one lane) issues the MMAs into TMEM accumulators
// (two or four); warps 2-5 read a finished accumulator (tcgen05.ld), apply
// ReLU, convert and store while the next tile accumulates.  The weights stay
// in shared memory when they fit (the narrow early layers); else each stage
// also brings the k-tile's weight box, and serves two of the CTA's tiles
// with it (their A boxes side by side, one accumulator each), which halves
// the weight traffic out of L2.  The producer and the MMA issuer are lone
// threads whose every dependent instruction costs about ten cycles, so they
// keep the launch's fields in registers, advance stage and tap counters by
// increments and add precomputed descriptor offsets.  Every mbarrier wait is
// bounded in time; a timeout records GS2D_ERR_TIMEOUT in the caller's status
// word.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "gs2d_internal.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace gs2d {
namespace {

constexpr int kTapThreads = 192;    // warps 0-1 producer / MMA, 2-5 epilogue
constexpr int kMaxStages = 8;
constexpr int kABytes = kBM * kBK * 2;  // one k-tile of A: 16 KB
constexpr int kCstBytes = 6144;     // bias block (2 KB) + zero block (4 KB)
// The constant block comes first, so that the reach of its unswizzled
// descriptors (16 row groups, two core-matrix columns) stays inside the
// allocation whichever of their two offsets the hardware steps along the rows.
constexpr int kCstRegion = 8192;
constexpr int kSmemBudget = 227 * 1024;

struct TapArgs {
  int Ho, Wo, ks, stride, pad;
  int N, ldc, relu;
  int segs, tiles, nk;
  int cw, cpt, blocks_real, kbias;  // channels per block, blocks per tap, tap blocks, bias k
  int stages, resident_b;
  int per;                          // output tiles per weight load (2 when streamed)
  int stage_bytes;                  // A (+ the weights' box if streamed)
  int b_off;                        // the weights' box within a stage (streamed)
  int ring_off, bres_off;           // offsets of the stage ring and the resident weights
  unsigned long long wait_ns;       // limit of every mbarrier wait (0: one second)
  int withhold;                     // failure-detection check: the producer issues no load
  float* out_f32;
  __nv_bfloat16* out_bf16;
  int* status;
};

template <int BN>
struct TapShape {
  static constexpr int kAcc = BN <= 128 ? 4 : 2;
  static constexpr int kAccStride = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  static constexpr int kCols = kAcc * kAccStride;
  static constexpr int kTmemCols =
      kCols <= 32 ? 32 : kCols <= 64 ? 64 : kCols <= 128 ? 128 : kCols <= 256 ? 256 : 512;
  static constexpr int kBBytes = BN * kBK * 2;  // one k-tile of weights
};

__device__ __forceinline__ bool failed(const int* flag) {
  return *reinterpret_cast<const volatile int*>(flag) != 0;
}

// Descriptor of the A operand's K = 16 slice kk (0..3) of a k-tile held in
// the stage at a_s, for k-blocks of cw channels.
__device__ __forceinline__ uint64_t tap_desc(uint32_t a_s, int kk, int cw) {
  switch (cw) {
    case 16: return kmajor_desc(a_s + 4096u * kk, 16u, 256u, 6u);
    case 32: return kmajor_desc(a_s + 8192u * (kk >> 1) + 32u * (kk & 1), 16u, 512u, 4u);
    default: return kmajor_desc(a_s + 32u * kk, 16u, 1024u, 2u);
  }
}

template <int BN, int PER>
__global__ void __launch_bounds__(kTapThreads, 1)
k_conv_tap(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
           TapArgs g) {
  using Sh = TapShape<BN>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
  __shared__ __align__(8) uint64_t acc_full[Sh::kAcc], acc_empty[Sh::kAcc], bres_full;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ST = g.stages;
  uint8_t* cst = smem;  // constant block at the start
  uint8_t* ring = smem + g.ring_off;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < Sh::kAcc; a++) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);  // one arrival per epilogue warp
    }
    mbar_init(&bres_full, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // constant block: 128 rows of 16 bytes with bf16 1.0 first (the bias
  // column), then 4 KB of zeros
  for (int i = threadIdx.x; i < kCstBytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(cst)[i] = make_uint4(i < kBM ? 0x3F80u : 0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

  if (warp == 0) {
    if (lane == 0 && !g.withhold) {  // a failure-detection launch issues no load
      // producer: the launch's fields held in registers, the stage and the
      // tap position advanced incrementally (a lone thread: every
      // instruction of its loop is on the pipeline's critical path)
      const int nk = g.nk, tiles = g.tiles, cw = g.cw, cpt = g.cpt, ks = g.ks;
      const int blocks_real = g.blocks_real, stage_bytes = g.stage_bytes;
      const bool resident = g.resident_b != 0;
      const unsigned long long wait_ns = g.wait_ns;
      if (resident) {
        mbar_expect_tx(&bres_full, (uint32_t)(nk * Sh::kBBytes));
        for (int i = 0; i < nk; i++)
          tma_load_2d(smem + g.bres_off + i * Sh::kBBytes, &tb, &bres_full, i * kBK, 0);
      }
      const int bpk = kBK / cw;  // k-blocks per k-tile
      const int block_bytes = kBM * cw * 2;
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      // a unit: this CTA's next PER tiles, which share each weight box
      for (int t0 = blockIdx.x; t0 < tiles && ok && !failed(&s_fail); t0 += PER * gridDim.x) {
        const int nt = PER == 2 && t0 + (int)gridDim.x < tiles ? 2 : 1;
        int ub[2], ux0[2], uy0[2];
        for (int k = 0; k < nt; k++) {
          const int t = t0 + k * (int)gridDim.x;
          const int row = t / g.segs, seg = t - row * g.segs;
          ub[k] = row / g.Ho;
          ux0[k] = seg * kBM * g.stride - g.pad;
          uy0[k] = (row - ub[k] * g.Ho) * g.stride - g.pad;
        }
        int qc = 0, qx = 0, qy = 0;  // chunk and tap (ky, kx) of the k-tile's first block
        for (int i = 0; i < nk; i++) {
          if (!mbar_wait(&empty[s], ph ^ 1u, wait_ns)) {
            ok = false;
            break;
          }
          uint8_t* st = ring + s * stage_bytes;
          const int nl = max(0, min(bpk, blocks_real - i * bpk));
          const uint32_t bytes =
              (uint32_t)(nt * nl * block_bytes) + (resident ? 0u : (uint32_t)Sh::kBBytes);
          if (bytes == 0) {
            mbar_arrive(&full[s]);
          } else {
            mbar_expect_tx(&full[s], bytes);
            for (int k = 0; k < nt; k++) {
              int c = qc, x = qx, y = qy;
              for (int j = 0; j < nl; j++) {
                tma_load_4d(st + k * kABytes + j * block_bytes, &ta, &full[s], c * cw,
                            ux0[k] + x, uy0[k] + y, ub[k]);
                if (++c == cpt) {
                  c = 0;
                  if (++x == ks) {
                    x = 0;
                    ++y;
                  }
                }
              }
            }
            if (!resident) tma_load_2d(st + g.b_off, &tb, &full[s], i * kBK, 0);
          }
          for (int j = 0; j < nl; j++) {
            if (++qc == cpt) {
              qc = 0;
              if (++qx == ks) {
                qx = 0;
                ++qy;
              }
            }
          }
          if (++s == ST) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      if (!ok) s_fail = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: the descriptors of stage 0 built once, each K = 16 slice's
      // as a fixed offset of them (the start address field counts 16 bytes)
      constexpr uint32_t idesc = idesc_bf16(kBM, BN);
      const int nk = g.nk, tiles = g.tiles, kbias = g.kbias, cw = g.cw;
      const bool resident = g.resident_b != 0;
      const unsigned long long wait_ns = g.wait_ns;
      if (resident && !mbar_wait(&bres_full, 0, wait_ns)) s_fail = 1;
      const uint32_t cst_s = smem_u32(cst), ring_s = smem_u32(ring);
      uint64_t adesc[kBK / 16];
#pragma unroll
      for (int kk = 0; kk < kBK / 16; kk++) adesc[kk] = tap_desc(ring_s, kk, cw);
      const uint64_t bdesc0 =
          sw128_desc(resident ? smem_u32(smem + g.bres_off) : ring_s + (uint32_t)g.b_off);
      const uint64_t bias_d = kmajor_desc(cst_s, 2048u, 128u, 0u);
      const uint64_t zero_d = kmajor_desc(cst_s + 2048u, 2048u, 128u, 0u);
      const uint64_t stage_d = (uint64_t)(g.stage_bytes >> 4);
      constexpr uint64_t tile_d = kABytes >> 4, bk_d = Sh::kBBytes >> 4;
      const int kfull = kbias / kBK;  // k-tiles of tap slices only
      int s = 0;
      uint32_t ph = 0, at = 0;  // stage, its phase; accumulators used so far
      bool ok = true;
      for (int t0 = blockIdx.x; t0 < tiles && ok && !failed(&s_fail); t0 += PER * gridDim.x) {
        const int nt = PER == 2 && t0 + (int)gridDim.x < tiles ? 2 : 1;
        uint32_t d[2];
        for (int k = 0; k < nt && ok; k++) {
          const uint32_t ak = at + (uint32_t)k;
          const int a = (int)(ak % (uint32_t)Sh::kAcc);
          ok = mbar_wait(&acc_empty[a], ((ak / (uint32_t)Sh::kAcc) & 1u) ^ 1u, wait_ns);
          d[k] = tmem + (uint32_t)(a * Sh::kAccStride);
        }
        if (!ok) break;
        tc_fence_after();
        for (int i = 0; i < nk; i++) {
          if (!mbar_wait(&full[s], ph, wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t so = (uint64_t)s * stage_d;
          const uint64_t bd = bdesc0 + (resident ? (uint64_t)i * bk_d : so);
          if (i < kfull) {
            for (int k = 0; k < nt; k++) {
              const uint64_t ko = so + (uint64_t)k * tile_d;
#pragma unroll
              for (int kk = 0; kk < kBK / 16; kk++)
                mma_bf16(d[k], adesc[kk] + ko, bd + 2 * kk, idesc, (i | kk) ? 1u : 0u);
            }
          } else {  // the k-tile of the bias slice: taps, bias, zeros
            for (int k = 0; k < nt; k++) {
              const uint64_t ko = so + (uint64_t)k * tile_d;
#pragma unroll
              for (int kk = 0; kk < kBK / 16; kk++) {
                const int kq = i * kBK + kk * 16;
                const uint64_t ad = kq < kbias ? adesc[kk] + ko : kq == kbias ? bias_d : zero_d;
                mma_bf16(d[k], ad, bd + 2 * kk, idesc, (i | kk) ? 1u : 0u);
              }
            }
          }
          mma_commit(&empty[s]);
          if (++s == ST) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        for (int k = 0; k < nt; k++)
          mma_commit(&acc_full[(at + (uint32_t)k) % (uint32_t)Sh::kAcc]);
        at += (uint32_t)nt;
      }
      if (!ok) s_fail = 1;
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) ... (its accumulator rows)
    const int quarter = warp & 3, r = quarter * 32 + lane;
    const bool vec_ok =
        (g.ldc % 8) == 0 &&
        ((reinterpret_cast<uintptr_t>(g.out_bf16 ? (const void*)g.out_bf16
                                                 : (const void*)g.out_f32) &
          15) == 0);
    uint32_t at = 0;
    bool ok = true;
    for (int t0 = blockIdx.x; t0 < g.tiles && ok; t0 += PER * gridDim.x) {
      const int nt = PER == 2 && t0 + (int)gridDim.x < g.tiles ? 2 : 1;
      for (int k = 0; k < nt; k++, at++) {
        const int t = t0 + k * (int)gridDim.x;
        const int a = (int)(at % (uint32_t)Sh::kAcc);
        const uint32_t aph = (at / (uint32_t)Sh::kAcc) & 1u;
        // tcgen05.ld is warp-collective: the warp goes on only if every lane
        // saw the accumulator complete
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[a], aph, g.wait_ns))) {
          s_fail = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const int row = t / g.segs, seg = t - row * g.segs;
        const int ox = seg * kBM + r;
        const bool valid = ox < g.Wo;
        const size_t o = ((size_t)row * g.Wo + ox) * g.ldc;
        const uint32_t taddr =
            tmem + (uint32_t)(a * Sh::kAccStride) + ((uint32_t)(quarter * 32) << 16);
        store_acc_row<BN>(taddr, valid, o, g.N, g.relu, vec_ok, g.out_f32, g.out_bf16);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[a]);
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Sh::kTmemCols));
  if (threadIdx.x == 0 && s_fail && g.status) atomicCAS(g.status, 0, (int)GS2D_ERR_TIMEOUT);
}

// 4D bf16 tensor map of an NHWC activation [B][Hi][Wi][C] for the tap loads:
// box cw channels x 128 pixels, traversal stride `stride` along W (so the
// box spans 128 stride pixels), one row, one image; the swizzle matches the
// block's row width; zeros out of range.
bool make_tap_map(CUtensorMap* map, const void* x, int B, int Hi, int Wi, int C, int cw,
                  int stride) {
  EncodeTiled fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)Wi, (cuuint64_t)Hi, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)Wi * C * 2,
                                 (cuuint64_t)Hi * Wi * C * 2};
  const cuuint32_t box[4] = {(cuuint32_t)cw, (cuuint32_t)(kBM * stride), 1, 1};
  const cuuint32_t estr[4] = {1, (cuuint32_t)stride, 1, 1};
  const CUtensorMapSwizzle swz = cw == 16   ? CU_TENSOR_MAP_SWIZZLE_32B
                                 : cw == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                            : CU_TENSOR_MAP_SWIZZLE_128B;
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

// Shared-memory plan of one launch: the constant block, the stage ring and
// the resident weights (when all k-tiles of them fit in 64 KB); the ring as
// deep as the budget allows (2 ... 8 stages).
// Returns the dynamic shared-memory bytes, 0 when even two stages do not fit.
int tap_plan(int bn, int nk, TapArgs* g) {
  const int kb = bn * kBK * 2;
  g->resident_b = nk * kb <= 64 * 1024 ? 1 : 0;
  g->per = g->resident_b ? 1 : 2;  // streamed weights: each box serves two tiles
  g->b_off = g->per * kABytes;
  g->stage_bytes = g->b_off + (g->resident_b ? 0 : kb);
  const int bres = g->resident_b ? nk * kb : 0;
  const int fixed = kCstRegion + bres + 1024;  // + alignment slack
  const int stages = std::min(kMaxStages, (kSmemBudget - fixed) / g->stage_bytes);
  if (stages < 2) return 0;
  g->stages = stages;
  g->ring_off = kCstRegion;
  g->bres_off = g->ring_off + stages * g->stage_bytes;
  return g->bres_off + bres + 1024;
}

template <int BN, int PER>
cudaError_t launch_tap_per(const CUtensorMap& ta, const CUtensorMap& tb, const TapArgs& g,
                           int smem, cudaStream_t s) {
  const cudaError_t attr = opt_in_smem((const void*)k_conv_tap<BN, PER>, smem);
  if (attr != cudaSuccess) return attr;
  const int sms = sm_count();
  const int grid = std::max(1, std::min(g.tiles, sms > 0 ? sms : 1));
  k_conv_tap<BN, PER><<<grid, kTapThreads, smem, s>>>(ta, tb, g);
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_tap(const CUtensorMap& ta, const CUtensorMap& tb, const TapArgs& g, int smem,
                       cudaStream_t s) {
  return g.per == 2 ? launch_tap_per<BN, 2>(ta, tb, g, smem, s)
                    : launch_tap_per<BN, 1>(ta, tb, g, smem, s);
}

}  // namespace

bool tap_conv_supported(const TcConvProblem& pr) {
  const int Wo = (pr.Wi + 2 * pr.pad - pr.ks) / pr.stride + 1;
  const bool cw_ok = pr.C == 16 || pr.C == 32 || pr.C % 64 == 0;
  return cw_ok && (pr.stride == 1 || pr.stride == 2) && pr.N >= 1 && pr.N <= 256 &&
         Wo >= 64 && pr.pad < pr.ks;
}

cudaError_t tap_conv(const TcConvProblem& pr, cudaStream_t s) {
  const int Ho = (pr.Hi + 2 * pr.pad - pr.ks) / pr.stride + 1;
  const int Wo = (pr.Wi + 2 * pr.pad - pr.ks) / pr.stride + 1;
  if (pr.B <= 0 || Ho <= 0 || Wo <= 0 || pr.N <= 0) return cudaSuccess;
  if (!tap_conv_supported(pr)) return cudaErrorInvalidValue;
  const int bn = tc_gemm_bn(pr.N);
  TapArgs g;
  g.Ho = Ho;
  g.Wo = Wo;
  g.ks = pr.ks;
  g.stride = pr.stride;
  g.pad = pr.pad;
  g.N = pr.N;
  g.ldc = pr.ldc;
  g.relu = pr.relu;
  g.segs = (Wo + kBM - 1) / kBM;
  g.tiles = pr.B * Ho * g.segs;
  g.nk = (pr.ldk + kBK - 1) / kBK;
  g.cw = pr.C < 64 ? pr.C : 64;
  g.cpt = pr.C / g.cw;
  g.blocks_real = pr.ks * pr.ks * g.cpt;
  g.kbias = pr.ks * pr.ks * pr.C;
  g.out_f32 = pr.out_f32;
  g.out_bf16 = pr.out_bf16;
  g.status = pr.status;
  g.wait_ns = pr.wait_ns;
  g.withhold = pr.withhold_loads;
  const int smem = tap_plan(bn, g.nk, &g);
  if (smem <= 0) return cudaErrorInvalidValue;
  CUtensorMap ta, tb;
  if (!make_tap_map(&ta, pr.x, pr.B, pr.Hi, pr.Wi, pr.C, g.cw, pr.stride) ||
      !make_map(&tb, pr.W, pr.N, pr.ldk, pr.ldk, bn))
    return cudaErrorInvalidValue;
  switch (bn) {
    case 32: return launch_tap<32>(ta, tb, g, smem, s);
    case 64: return launch_tap<64>(ta, tb, g, smem, s);
    case 96: return launch_tap<96>(ta, tb, g, smem, s);
    case 128: return launch_tap<128>(ta, tb, g, smem, s);
    case 192: return launch_tap<192>(ta, tb, g, smem, s);
    default: return launch_tap<256>(ta, tb, g, smem, s);
  }
}

}  // namespace gs2d
