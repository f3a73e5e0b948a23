// Implicit-GEMM convolution fed by one TMA box per input row: the learned
// initialiser's 3 x 3, stride-2, pad-1 layers (paper section 3.2 B) with an
// even input width and C = 32 or 64, as a persistent tcgen05
// kernel, one CTA per SM.
//
//   Z[p][n] = sum_k col(X)[p][k] W[n][k],   k = (3 ky + kx) C + ci,
//   a column of ones at k = 9 C carrying the bias, zeros beyond.
//
// A tile is 128 consecutive output pixels x0 ... x0 + 127 of one output row.
// Output pixel x0 + m reads input pixels 2 (x0 + m) - 1 + kx, i.e. with the
// input row seen as pixel pairs (2 j, 2 j + 1):
//   kx = 0: odd pixel of pair x0 - 1 + m,
//   kx = 1: even pixel of pair x0 + m,
//   kx = 2: odd pixel of pair x0 + m.
// So for one input row the three taps are served by the 129 pairs
// x0 - 1 ... x0 + 127, read once (out-of-image pairs and rows read as zero):
//   C = 32    one box of 129 rows x 128 bytes (the two pixels of a pair side
//             by side); kx = 1 reads its left half, kx = 0 and 2 its right;
//   C = 64    two boxes of 129 rows x 128 bytes, the even and the odd
//             pixels of the pairs.
// The boxes land in the 128-byte swizzle; a tap's K-major operand starts at
// row 0 (kx = 0) or row 1 (kx = 1, 2) of its box.  The MMA applies the
// swizzle to the absolute shared-memory address (the descriptor's base offset
// stays 0), so a start one 128-byte row into an 8-row atom reads the rows the
// TMA wrote there.  The TMA engine of an SM moves large boxes faster than
// small ones (with about four boxes in flight, 8 KB boxes reach some 28 GB/s
// per SM and 16 KB boxes 46 GB/s), and one box per tap would be 8 KB for
// C = 32: here each tile reads three (C = 32) or 6 C / 64 boxes of 16.5 KB,
// every input pixel once per input row (the tap kernel reads 9 boxes of
// 8 KB or 16 KB per tile).
//
// The MMA sequence, K = 16 slice by K = 16 slice in k order (the bias slice
// and the zero slices past it from a constant block), is the one the GEMM
// over an im2col operand issues, so the output equals im2col + GEMM bit for
// bit.  Roles as in the tap kernel of csrc/conv_tap.cu: warp 0 (one lane)
// issues the TMA loads, the A boxes of (tile, input row) into a ring of
// slots and, when the weights do not fit in 64 KB, the weight k-tiles into a
// second ring (each then serving two of the CTA's tiles); warp 1 (one lane)
// issues the MMAs; warps 2-5 drain the accumulators.  Every mbarrier wait is
// bounded in time; a timeout records GS2D_ERR_TIMEOUT in the status word.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "gs2d_internal.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace gs2d {
namespace {

constexpr int kThreads = 192;        // warps 0-1 producer / MMA, 2-5 epilogue
constexpr int kBoxRows = kBM + 1;    // 129 pairs
constexpr int kBoxBytes = kBoxRows * 128;
constexpr int kBoxSlot = 17 * 1024;  // a box, 1024-byte aligned
constexpr int kMaxA = 12, kMaxB = 8;
constexpr int kCstBytes = 6144;      // bias block (2 KB) + zero block (4 KB)
constexpr int kCstRegion = 8192;
constexpr int kSmemBudget = 227 * 1024;

struct RowsArgs {
  int C, Ho, Wo;
  int N, ldc, relu;
  int segs, tiles, nk;
  int sa, sb;                   // A slots; weight slots (streamed weights)
  int resident_b;
  int a_off, b_off;             // the A ring; the weight ring or the resident weights
  unsigned long long wait_ns;   // limit of every mbarrier wait (0: one second)
  int withhold;                 // failure-detection check: the producer issues no load
  float* out_f32;
  __nv_bfloat16* out_bf16;
  int* status;
};

template <int BN>
struct RowsShape {
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


// PER tiles share each weight k-tile (PER = 2 streams the weights, PER = 1
// keeps them resident); C = 32 or 64 fixes the order of the tile's
// K = 16 slices at compile time, so the MMA issuer's whole tile unrolls into
// descriptor additions and MMAs: the lone issuing thread runs about ten SM
// cycles per dependent instruction, and every instruction between two MMAs
// delays the tensor pipe.
template <int BN, int PER, int C>
__global__ void __launch_bounds__(kThreads, 1)
k_conv_rows(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
            RowsArgs g) {
  using Sh = RowsShape<BN>;
  constexpr bool kRes = PER == 1;                 // weights resident
  constexpr int kBoxes = C == 32 ? 1 : C / 32;    // boxes per A slot
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t a_full[kMaxA], a_empty[kMaxA], b_full[kMaxB], b_empty[kMaxB];
  __shared__ __align__(8) uint64_t acc_full[Sh::kAcc], acc_empty[Sh::kAcc], bres_full;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int SA = g.sa, SB = g.sb;
  uint8_t* cst = smem;  // constant block at the start
  uint8_t* aring = smem + g.a_off;
  uint8_t* bmem = smem + g.b_off;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; s++) {
      mbar_init(&a_full[s], 1);
      mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < SB; s++) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
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
      // producer, in the order the MMA issuer consumes: per unit of PER
      // tiles and input row ky, the tiles' A slots, then the weight k-tiles
      // that start within the row's K range (after the last row, the rest)
      const int nk = g.nk, tiles = g.tiles;
      const unsigned long long wait_ns = g.wait_ns;
      if (kRes) {
        mbar_expect_tx(&bres_full, (uint32_t)(nk * Sh::kBBytes));
        for (int i = 0; i < nk; i++)
          tma_load_2d(bmem + i * Sh::kBBytes, &tb, &bres_full, i * kBK, 0);
      }
      int sa = 0, sb = 0;
      uint32_t pa = 0, pb = 0;
      for (int t0 = blockIdx.x; t0 < tiles && !failed(&s_fail); t0 += PER * gridDim.x) {
        const int nt = PER == 2 && t0 + (int)gridDim.x < tiles ? 2 : 1;
        int ub[2], px[2], iy[2];
        for (int k = 0; k < nt; k++) {
          const int t = t0 + k * (int)gridDim.x;
          const int row = t / g.segs, seg = t - row * g.segs;
          ub[k] = row / g.Ho;
          px[k] = seg * kBM - 1;                  // first pair of the box
          iy[k] = (row - ub[k] * g.Ho) * 2 - 1;   // input row of ky = 0
        }
        int kt = 0;  // next weight k-tile (streamed weights)
        for (int ky = 0; ky < 3; ky++) {
          for (int k = 0; k < nt; k++) {
            if (!mbar_wait(&a_empty[sa], pa ^ 1u, wait_ns)) goto producer_failed;
            mbar_expect_tx(&a_full[sa], (uint32_t)(kBoxes * kBoxBytes));
            {
              uint8_t* dst = aring + sa * (kBoxes * kBoxSlot);
              if (C == 32) {
                tma_load_4d(dst, &ta, &a_full[sa], 0, px[k], iy[k] + ky, ub[k]);
              } else {
#pragma unroll
                for (int b = 0; b < kBoxes; b++)  // chunk b / 2, even (b even) or odd pixels
                  tma_load_5d(dst + b * kBoxSlot, &ta, &a_full[sa], (b >> 1) * 64, b & 1, px[k],
                              iy[k] + ky, ub[k]);
              }
            }
            if (++sa == SA) {
              sa = 0;
              pa ^= 1u;
            }
          }
          if constexpr (!kRes) {
            for (const int kend = ky == 2 ? nk * kBK : (ky + 1) * 3 * C; kt * kBK < kend; kt++) {
              if (!mbar_wait(&b_empty[sb], pb ^ 1u, wait_ns)) goto producer_failed;
              mbar_expect_tx(&b_full[sb], (uint32_t)Sh::kBBytes);
              tma_load_2d(bmem + sb * Sh::kBBytes, &tb, &b_full[sb], kt * kBK, 0);
              if (++sb == SB) {
                sb = 0;
                pb ^= 1u;
              }
            }
          }
        }
      }
      if (false) {
      producer_failed:
        s_fail = 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer.  Descriptors as 32-bit words: the rings' first slots and
      // compile-time offsets (16-byte units) of each slice.
      constexpr uint32_t idesc = idesc_bf16(kBM, BN);
      constexpr int kCh = C == 32 ? 1 : C / 64;     // 64-channel chunks per tap
      constexpr int kQ = C == 32 ? 2 : 4;           // K = 16 slices per chunk
      constexpr uint32_t kBox = kBoxSlot >> 4;
      constexpr uint32_t kOdd = C == 32 ? 4u : kBox;  // the odd pixels: right half or next box
      constexpr uint32_t kSlot = kBoxes * kBox;
      constexpr uint32_t kBk = Sh::kBBytes >> 4;
      const int nk = g.nk, tiles = g.tiles;
      const unsigned long long wait_ns = g.wait_ns;
      if (kRes && !mbar_wait(&bres_full, 0, wait_ns)) s_fail = 1;
      const uint64_t a0 = sw128_desc(smem_u32(aring)), b0 = sw128_desc(smem_u32(bmem));
      const uint64_t c0 = kmajor_desc(smem_u32(cst), 2048u, 128u, 0u);
      const uint32_t a_lo0 = (uint32_t)a0, b_lo0 = (uint32_t)b0, sw_hi = (uint32_t)(a0 >> 32);
      const uint32_t bias_lo = (uint32_t)c0, zero_lo = bias_lo + (2048u >> 4);
      const uint32_t c_hi = (uint32_t)(c0 >> 32);
      int sa = 0, sb = 0;
      uint32_t pa = 0, pb = 0, at = 0;  // ring slots, phases; accumulators used so far
      for (int t0 = blockIdx.x; t0 < tiles && !failed(&s_fail); t0 += PER * gridDim.x) {
        const int nt = PER == 2 && t0 + (int)gridDim.x < tiles ? 2 : 1;
        uint32_t d[2];
        for (int k = 0; k < nt; k++) {
          const uint32_t ak = at + (uint32_t)k;
          const int a = (int)(ak % (uint32_t)Sh::kAcc);
          if (!mbar_wait(&acc_empty[a], ((ak / (uint32_t)Sh::kAcc) & 1u) ^ 1u, wait_ns))
            goto mma_failed;
          d[k] = tmem + (uint32_t)(a * Sh::kAccStride);
        }
        tc_fence_after();
        {
          uint32_t b_lo = b_lo0;  // the current weight k-tile (streamed: its slot)
#pragma unroll
          for (int ky = 0; ky < 3; ky++) {
            uint32_t al[2];
            {
              int s2 = sa;
              uint32_t p2 = pa;
              for (int k = 0; k < nt; k++) {
                if (!mbar_wait(&a_full[s2], p2, wait_ns)) goto mma_failed;
                al[k] = a_lo0 + (uint32_t)s2 * kSlot;
                if (++s2 == SA) {
                  s2 = 0;
                  p2 ^= 1u;
                }
              }
            }
            tc_fence_after();
#pragma unroll
            for (int kx = 0; kx < 3; kx++) {
#pragma unroll
              for (int ch = 0; ch < kCh; ch++) {
#pragma unroll
                for (int q = 0; q < kQ; q++) {
                  const int kq = (3 * ky + kx) * C + ch * 64 + q * 16;
                  if (!kRes && (kq & 63) == 0) {  // a new weight k-tile
                    if (!mbar_wait(&b_full[sb], pb, wait_ns)) goto mma_failed;
                    tc_fence_after();
                    b_lo = b_lo0 + (uint32_t)sb * kBk;
                  }
                  // tap kx: one 128-byte row down for kx = 1, 2; odd pixels for kx = 0, 2
                  const uint32_t off = (kx > 0 ? 8u : 0u) + (kx != 1 ? kOdd : 0u) +
                                       (uint32_t)ch * 2u * kBox + 2u * (uint32_t)q;
                  const uint32_t bq =
                      (kRes ? b_lo0 + (uint32_t)(kq >> 6) * kBk : b_lo) + 2u * ((kq & 63) >> 4);
                  mma_bf16_w(d[0], al[0] + off, sw_hi, bq, sw_hi, idesc, kq > 0 ? 1u : 0u);
                  if (PER == 2 && nt == 2)
                    mma_bf16_w(d[1], al[1] + off, sw_hi, bq, sw_hi, idesc, kq > 0 ? 1u : 0u);
                  if (!kRes && (kq & 63) == 48) {  // the k-tile's last slice
                    mma_commit(&b_empty[sb]);
                    if (++sb == SB) {
                      sb = 0;
                      pb ^= 1u;
                    }
                  }
                }
              }
            }
            for (int k = 0; k < nt; k++) {
              mma_commit(&a_empty[sa]);
              if (++sa == SA) {
                sa = 0;
                pa ^= 1u;
              }
            }
          }
          // the bias slice, then the zero slices up to the last k-tile's end
          for (int kq = 9 * C; kq < nk * kBK; kq += 16) {
            if (!kRes && (kq & 63) == 0) {
              if (!mbar_wait(&b_full[sb], pb, wait_ns)) goto mma_failed;
              tc_fence_after();
              b_lo = b_lo0 + (uint32_t)sb * kBk;
            }
            const uint32_t bq =
                (kRes ? b_lo0 + (uint32_t)(kq >> 6) * kBk : b_lo) + 2u * (uint32_t)((kq & 63) >> 4);
            const uint32_t al_ = kq == 9 * C ? bias_lo : zero_lo;
            mma_bf16_w(d[0], al_, c_hi, bq, sw_hi, idesc, 1u);
            if (PER == 2 && nt == 2) mma_bf16_w(d[1], al_, c_hi, bq, sw_hi, idesc, 1u);
            if (!kRes && (kq & 63) == 48) {
              mma_commit(&b_empty[sb]);
              if (++sb == SB) {
                sb = 0;
                pb ^= 1u;
              }
            }
          }
        }
        for (int k = 0; k < nt; k++)
          mma_commit(&acc_full[(at + (uint32_t)k) % (uint32_t)Sh::kAcc]);
        at += (uint32_t)nt;
      }
      if (false) {
      mma_failed:
        s_fail = 1;
      }
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

// bf16 tensor map of an NHWC activation [B][Hi][Wi][C] (Wi even) as pixel
// pairs, boxes of 129 pairs x 128 bytes in the 128-byte swizzle, zeros out
// of range:
//   C = 32    4D {2 C, Wi / 2, Hi, B}: both pixels of a pair in one row;
//   C = 64    5D {C, 2, Wi / 2, Hi, B}: the even or the odd pixels (the
//             channel coordinate selects a 64-channel chunk).
bool make_rows_map(CUtensorMap* map, const void* x, int B, int Hi, int Wi, int C) {
  EncodeTiled fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint64_t row = (cuuint64_t)Wi * C * 2, img = row * Hi;
  if (C == 32) {
    const cuuint64_t dims[4] = {64, (cuuint64_t)Wi / 2, (cuuint64_t)Hi, (cuuint64_t)B};
    const cuuint64_t strides[3] = {128, row, img};
    const cuuint32_t box[4] = {64, (cuuint32_t)kBoxRows, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides,
              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  const cuuint64_t dims[5] = {(cuuint64_t)C, 2, (cuuint64_t)Wi / 2, (cuuint64_t)Hi,
                              (cuuint64_t)B};
  const cuuint64_t strides[4] = {(cuuint64_t)C * 2, (cuuint64_t)C * 4, row, img};
  const cuuint32_t box[5] = {64, 1, (cuuint32_t)kBoxRows, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(x), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Shared-memory plan: the constant block, the A ring, then the resident
// weights (all k-tiles within 64 KB; one tile per unit) or a ring of weight
// k-tiles (two tiles per unit, A slots for two input rows of the unit when
// they fit, else one).  Returns the dynamic shared-memory bytes, 0 when the
// shape does not fit.
int rows_plan(int bn, int nk, int nbox, RowsArgs* g) {
  const int kb = bn * kBK * 2, aslot = nbox * kBoxSlot;
  const int budget = kSmemBudget - 2048;  // alignment slack of the base, static shared memory
  g->resident_b = nk * kb <= 64 * 1024 ? 1 : 0;
  g->a_off = kCstRegion;
  if (g->resident_b) {
    g->sb = 0;
    g->sa = std::min(kMaxA, (budget - kCstRegion - nk * kb) / aslot);
    if (g->sa < 2) return 0;
    g->b_off = g->a_off + g->sa * aslot;
    return g->b_off + nk * kb + 1024;
  }
  for (int sa = 4; sa >= 2; sa -= 2) {
    const int sb = std::min(kMaxB, (budget - kCstRegion - sa * aslot) / kb);
    if (sb >= 2) {
      g->sa = sa;
      g->sb = sb;
      g->b_off = g->a_off + sa * aslot;
      return g->b_off + sb * kb + 1024;
    }
  }
  return 0;
}

template <int BN, int PER, int C>
cudaError_t launch_rows_per(const CUtensorMap& ta, const CUtensorMap& tb, const RowsArgs& g,
                            int smem, cudaStream_t s) {
  const cudaError_t attr = opt_in_smem((const void*)k_conv_rows<BN, PER, C>, smem);
  if (attr != cudaSuccess) return attr;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  const int grid = std::max(1, std::min(g.tiles, sms));
  k_conv_rows<BN, PER, C><<<grid, kThreads, smem, s>>>(ta, tb, g);
  return cudaGetLastError();
}

// Whether the weights of a C-channel layer with BN-column tiles stay
// resident: all k-tiles of the smallest ldk (9 C + 8) within 64 KB.
constexpr bool rows_resident(int c, int bn) {
  return ((9 * c + 8 + kBK - 1) / kBK) * bn * kBK * 2 <= 64 * 1024;
}

template <int BN, int C>
cudaError_t launch_rows_c(const CUtensorMap& ta, const CUtensorMap& tb, const RowsArgs& g,
                          int smem, cudaStream_t s) {
  return launch_rows_per<BN, rows_resident(C, BN) ? 1 : 2, C>(ta, tb, g, smem, s);
}

template <int BN>
cudaError_t launch_rows(const CUtensorMap& ta, const CUtensorMap& tb, const RowsArgs& g,
                        int smem, cudaStream_t s) {
  return g.C == 32 ? launch_rows_c<BN, 32>(ta, tb, g, smem, s)
                   : launch_rows_c<BN, 64>(ta, tb, g, smem, s);
}

// Fills the shape fields of g and plans shared memory; 0 when unsupported.
int rows_setup(const TcConvProblem& pr, RowsArgs* g) {
  if (pr.ks != 3 || pr.stride != 2 || pr.pad != 1 || pr.Wi % 2 != 0 || pr.Wi <= 0) return 0;
  // C = 128 (four 16.5 KB boxes per input row and tile) leaves room for one
  // row per unit in flight; the tap kernel of csrc/conv_tap.cu is faster there
  if (pr.C != 32 && pr.C != 64) return 0;
  if (pr.N < 1 || pr.N > 256 || pr.B <= 0 || pr.Hi <= 0) return 0;
  g->C = pr.C;
  g->Ho = (pr.Hi - 1) / 2 + 1;
  g->Wo = (pr.Wi - 1) / 2 + 1;
  if (g->Wo < 64) return 0;
  g->N = pr.N;
  g->ldc = pr.ldc;
  g->relu = pr.relu;
  g->segs = (g->Wo + kBM - 1) / kBM;
  g->tiles = pr.B * g->Ho * g->segs;
  g->nk = (pr.ldk + kBK - 1) / kBK;
  const int nbox = pr.C == 32 ? 1 : 2;  // boxes per A slot
  const int bn = tc_gemm_bn(pr.N);
  const int smem = rows_plan(bn, g->nk, nbox, g);
  // the kernels are built for the weights' placement of the smallest ldk
  return g->resident_b == (rows_resident(pr.C, bn) ? 1 : 0) ? smem : 0;
}

}  // namespace

bool rows_conv_supported(const TcConvProblem& pr) {
  RowsArgs g;
  return rows_setup(pr, &g) > 0;
}

cudaError_t rows_conv(const TcConvProblem& pr, cudaStream_t s) {
  RowsArgs g;
  const int smem = rows_setup(pr, &g);
  if (smem <= 0) return cudaErrorInvalidValue;
  g.out_f32 = pr.out_f32;
  g.out_bf16 = pr.out_bf16;
  g.status = pr.status;
  g.wait_ns = pr.wait_ns;
  g.withhold = pr.withhold_loads;
  const int bn = tc_gemm_bn(pr.N);
  CUtensorMap ta, tb;
  if (!make_rows_map(&ta, pr.x, pr.B, pr.Hi, pr.Wi, pr.C) ||
      !make_map(&tb, pr.W, pr.N, pr.ldk, pr.ldk, bn))
    return cudaErrorInvalidValue;
  switch (bn) {
    case 32: return launch_rows<32>(ta, tb, g, smem, s);
    case 64: return launch_rows<64>(ta, tb, g, smem, s);
    case 96: return launch_rows<96>(ta, tb, g, smem, s);
    case 128: return launch_rows<128>(ta, tb, g, smem, s);
    case 192: return launch_rows<192>(ta, tb, g, smem, s);
    default: return launch_rows<256>(ta, tb, g, smem, s);
  }
}

}  // namespace gs2d
