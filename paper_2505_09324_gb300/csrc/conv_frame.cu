// The learned initialiser's first convolution straight from the float frame
// and its ROI mask (paper section 3.2 B): gs2d_cnn_input (8-channel BF16 NHWC:
// R, G, B, mask, four zeros) followed by gs2d_conv_bf16 in one persistent
// tcgen05 kernel, so the 8-channel image is never written out or read back.
//
// A tile is 128 (120 for 3 x 3 at stride 2) consecutive output pixels of
// one output row; the CTA takes tiles j = 0, 1, ... of its share in turn.
// Per tile:
//   warp 0, one lane   TMA loads of the tile's three input rows into a ring of
//                      raw stages: the colour planes (256 floats per row and
//                      plane from a 16-byte boundary, for 128-pixel tiles 8
//                      more in a second box) and the mask (256 bytes, and 16
//                      more);
//   warps 10-27        three groups of six warps, group j % 3, build the
//                      tile's operand in shared memory, then the group's
//                      first thread issues the tile's MMAs (128 x BN x 16 per
//                      K slice, weights resident) into TMEM accumulator j % 4:
//                      3 x 3 at stride 2: each window pixel converted once to
//                      a 16-byte record (R, G, B, mask as BF16, four zeros)
//                      in arrays of the odd and even pixels of each input
//                      row, the taps joined by the MMA descriptors (see the
//                      record-mode group below);
//                      else: one thread per (row, input row ky) writes its
//                      taps' records into the 128-byte-swizzled K-major
//                      layout a TMA box of the im2col operand would have, the
//                      tile's k-tiles (64 K each) in consecutive stages of a
//                      second ring whose bias and zero chunks are written once;
//   warps 2-9          two groups of four warps, group j % 2, run the
//                      epilogue (tcgen05.ld, ReLU, BF16 stores).
// Three tiles are built and two drained at a time: a single warp per role
// left each tile's work waiting on its own instruction latency.
// The operands and the MMA sequence are those of gs2d_im2col + gs2d_gemm_bf16
// on gs2d_cnn_input's output, so the result is the same bit for bit.  Every
// mbarrier wait is bounded in time (GS2D_ERR_TIMEOUT in the status word); a
// group leaves its loop only together, after its barrier.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "gs2d_internal.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace gs2d {
namespace {

constexpr int kEpiWarp0 = 2;           // warps 2-9: two epilogue groups of four
constexpr int kEpiGroups = 2;
constexpr int kXfWarp0 = 10;           // warps 10-27: three im2col groups of six
constexpr int kXfGroups = 3;
constexpr int kXfGroupWarps = 6;
constexpr int kFrThreads = (kXfWarp0 + kXfGroups * kXfGroupWarps) * 32;  // 896
constexpr int kRawStages = 6;
constexpr int kAStages = 6;
constexpr int kAcc = 4;
constexpr int kRawRows = 3;            // input rows per tile (ks <= 3)
// raw stage: floats [plane][row][256] + [plane][row][8], mask [row][256] +
// [row][16], each box at a 128-byte boundary
constexpr int kRawTail = 9 * 256 * 4;                // 9216
constexpr int kRawMask = kRawTail + 512;             // 9728
constexpr int kRawMaskTail = kRawMask + 3 * 256;     // 10496
constexpr int kRawBytes = 11264;
constexpr int kStageA = kBM * kBK * 2;  // 16 KB
// 3 x 3 at stride 2 (the network's first layer): a tile's operand as six
// arrays of 16-byte pixel records, the even and the odd window pixels of
// each input row (129 records each), two buffers per group
// Arrays of 129 records, 2112 bytes apart: an odd and an even record of the
// same index (stored by adjacent lanes) then fall 64 bytes apart in the
// banks, so a quarter-warp's 16-byte stores do not conflict (at 2064 bytes
// apart half of the build's shared-memory wavefronts were conflicts).
constexpr int kParArr = 2112;
constexpr int kParBuf = 6 * kParArr + 32;  // 12704
constexpr int kCstBytes = 6144;            // bias rows (2 KB), then 4 KB of zeros

struct FrameArgs {
  int B, H, W, Ho, Wo, ks, stride, pad;
  int N, ldc, relu, has_mask;
  int segs, tiles, nk;
  unsigned long long wait_ns;       // limit of every mbarrier wait (0: one second)
  int withhold;                     // failure-detection check: the producer issues no load
  float* out_f32;
  __nv_bfloat16* out_bf16;
  int* status;
};

__device__ __forceinline__ bool failed(const int* flag) {
  return *reinterpret_cast<const volatile int*>(flag) != 0;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Barrier of one im2col group (named barriers 1-3; 0 is __syncthreads)
// that returns the OR of every participating thread's v.
__device__ __forceinline__ bool group_sync_or(int grp, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n"
      " bar.red.or.pred p, %2, %3, q;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + grp), "n"(kXfGroupWarps * 32)
      : "memory");
  return r != 0;
}

// Shared-memory offsets (from the 1024-aligned base): A ring (or the
// groups' record buffers and the constant block), raw ring, resident weights.
template <bool PAR>
struct FrameSmem {
  static constexpr int kA = 0;
  static constexpr int kCst = PAR ? (kXfGroups * 2 * kParBuf + 1023) / 1024 * 1024 : 0;
  static constexpr int kRaw = PAR ? kCst + 8192 : kAStages * kStageA;
  static constexpr int kB = kRaw + kRawStages * kRawBytes;
};

template <int BN, bool PAR>
__global__ void __launch_bounds__(kFrThreads, 1)
k_conv_frame(const __grid_constant__ CUtensorMap tf256, const __grid_constant__ CUtensorMap tf8,
             const __grid_constant__ CUtensorMap tm256, const __grid_constant__ CUtensorMap tm16,
             const __grid_constant__ CUtensorMap tb, FrameArgs g) {
  constexpr int kAccStride = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  constexpr int kCols = kAcc * kAccStride;
  constexpr int kTmemCols = kCols <= 128 ? 128 : kCols <= 256 ? 256 : 512;
  constexpr int kBBytes = BN * kBK * 2;
  // output pixels per tile: 120 in record mode, so that the 241 input pixels
  // of a row, from a 16-byte boundary, fit one 256-element TMA box (colour
  // planes and mask alike); 128 otherwise
  constexpr int kTW = PAR ? 120 : kBM;
  using Sm = FrameSmem<PAR>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t raw_full[kRawStages], raw_empty[kRawStages];
  __shared__ __align__(8) uint64_t a_empty[kAStages];
  __shared__ __align__(8) uint64_t acc_full[kAcc], acc_empty[kAcc], bres_full;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  // 1024-aligned, and kept in the shared window so that accesses compile to
  // shared-memory instructions
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = g.nk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kRawStages; s++) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], kXfGroupWarps);
    }
    for (int s = 0; s < kAStages; s++) mbar_init(&a_empty[s], 1);
    for (int a = 0; a < kAcc; a++) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);
    }
    mbar_init(&bres_full, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if constexpr (PAR) {
    // constant block: 128 rows of 16 bytes with bf16 1.0 first (the bias
    // column), then 4 KB of zeros
    for (int i = threadIdx.x; i < kCstBytes / 16; i += blockDim.x)
      reinterpret_cast<uint4*>(smem + Sm::kCst)[i] =
          make_uint4(i < kBM ? 0x3F80u : 0u, 0u, 0u, 0u);
  } else {
  // the chunks past the taps (the bias column's 1, then zeros): stage s
  // always holds k-tile s % nk (nk divides the ring), so they are written once
  for (int q = threadIdx.x; q < kAStages * 8 * kBM; q += blockDim.x) {
    const int st = q / (8 * kBM), c = (q / kBM) & 7, r = q % kBM;
    const int tap = (st % nk) * 8 + c;
    if (tap >= g.ks * g.ks)
      *reinterpret_cast<uint4*>(smem + Sm::kA + st * kStageA + r * 128 +
                                ((c ^ (r & 7)) << 4)) =
          make_uint4(tap == g.ks * g.ks ? 0x3F80u : 0u, 0u, 0u, 0u);
  }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0 && !g.withhold) {  // a failure-detection launch issues no load
      // producer: the weights once, then each tile's raw input rows
      mbar_expect_tx(&bres_full, (uint32_t)(nk * kBBytes));
      for (int i = 0; i < nk; i++)
        tma_load_2d(smem + Sm::kB + i * kBBytes, &tb, &bres_full, i * kBK, 0);
      const uint32_t bytes =
          PAR ? (uint32_t)(kRawRows * (3 * 256 * 4 + (g.has_mask ? 256 : 0)))
              : (uint32_t)(kRawRows * (3 * (256 + 8) * 4 + (g.has_mask ? 256 + 16 : 0)));
      uint32_t j = 0;
      for (int t = blockIdx.x; t < g.tiles && !failed(&s_fail); t += gridDim.x, j++) {
        const int row = t / g.segs, seg = t - row * g.segs;
        const int b = row / g.Ho, oy = row - b * g.Ho;
        const int x0 = seg * kTW * g.stride - g.pad, y0 = oy * g.stride - g.pad;
        const int xa = x0 & ~3, xm = x0 & ~15;  // 16-byte boundaries (floor)
        const int s = (int)(j % kRawStages);
        if (!mbar_wait(&raw_empty[s], ((j / kRawStages) & 1u) ^ 1u, g.wait_ns)) {
          s_fail = 1;
          break;
        }
        uint8_t* st = smem + Sm::kRaw + s * kRawBytes;
        mbar_expect_tx(&raw_full[s], bytes);
        tma_load_4d(st, &tf256, &raw_full[s], xa, y0, 0, b);
        if (!PAR) tma_load_4d(st + kRawTail, &tf8, &raw_full[s], xa + 256, y0, 0, b);
        if (g.has_mask) {
          tma_load_3d(st + kRawMask, &tm256, &raw_full[s], xm, y0, b);
          if (!PAR) tma_load_3d(st + kRawMaskTail, &tm16, &raw_full[s], xm + 256, y0, b);
        }
      }
    }
  } else if (warp >= kEpiWarp0 && warp < kXfWarp0) {
    // epilogue group e takes tiles j = e, e + 2, ...; warp w reads TMEM lanes
    // 32 (w % 4) ... (its accumulator rows)
    const int e = (warp - kEpiWarp0) >> 2;
    const int quarter = warp & 3, r = quarter * 32 + lane;
    const bool vec_ok =
        (g.ldc % 8) == 0 &&
        ((reinterpret_cast<uintptr_t>(g.out_bf16 ? (const void*)g.out_bf16
                                                 : (const void*)g.out_f32) &
          15) == 0);
    uint32_t j = (uint32_t)e;
    for (int t = blockIdx.x + e * gridDim.x; t < g.tiles;
         t += kEpiGroups * gridDim.x, j += kEpiGroups) {
      const int a = (int)(j % kAcc);
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[a], (j / kAcc) & 1u, g.wait_ns))) {
        s_fail = 1;
        break;
      }
      tc_fence_after();
      const int row = t / g.segs, seg = t - row * g.segs;
      const int ox = seg * kTW + r;
      const size_t o = ((size_t)row * g.Wo + ox) * g.ldc;
      const uint32_t taddr =
          tmem + (uint32_t)(a * kAccStride) + ((uint32_t)(quarter * 32) << 16);
      store_acc_row<BN>(taddr, r < kTW && ox < g.Wo, o, g.N, g.relu, vec_ok, g.out_f32,
                        g.out_bf16);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[a]);
    }
  } else if (PAR && warp >= kXfWarp0) {
    // 3 x 3, stride 2.  Group x takes tiles j = x, x + 3, ... into its two
    // record buffers in turn.  Window pixel d (input x0 + d, d = 0 ... 240) of
    // input row ky is converted once, to a 16-byte record (R, G, B, mask as
    // BF16, four zeros), stored in O_ky[d / 2] (d even) or E_ky[d / 2] (d odd).
    // Output pixel m reads window pixels 2m + kx, so its taps are O_ky[m],
    // E_ky[m], O_ky[m + 1]: each tap's operand is an array (or one record
    // further), 128 consecutive 16-byte rows (the last 8 unused: a tile has
    // 120 output pixels), the unswizzled K-major layout
    // (8-row groups 128 bytes apart).  A K = 16 slice joins two taps (the
    // second 8 channels at the descriptor's leading-dimension offset from
    // the first); the arrays lie in the order O_0, E_0, E_1, O_1, O_2, E_2
    // and the constant block above them, so that every such offset is
    // positive.  Slice 4 joins tap (2, 2) and the bias row, the slices past
    // it are zeros: the MMA sequence of the GEMM over the im2col operand.
    const int x = (warp - kXfWarp0) / kXfGroupWarps;
    const int xt = threadIdx.x - (kXfWarp0 + x * kXfGroupWarps) * 32;  // 0 ... 191
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);
    constexpr uint32_t S = kParArr;
    const uint32_t cst_s = smem_u32(smem + Sm::kCst);
    if (xt == 0 && !mbar_wait(&bres_full, 0, g.wait_ns)) s_fail = 1;
    uint32_t j = (uint32_t)x, jj = 0;  // CTA tile index; the group's own count
    for (int t = blockIdx.x + x * gridDim.x; t < g.tiles;
         t += kXfGroups * gridDim.x, j += kXfGroups, jj++) {
      const int rs = (int)(j % kRawStages);
      const int ab = x * 2 + (int)(jj & 1u);  // the record buffer, its barrier
      uint8_t* buf = smem + Sm::kA + ab * kParBuf;
      bool ok =
          __all_sync(0xffffffffu, mbar_wait(&raw_full[rs], (j / kRawStages) & 1u, g.wait_ns));
      // the buffer's last MMAs (the group's tile jj - 2) have completed
      ok = ok && __all_sync(0xffffffffu,
                            mbar_wait(&a_empty[ab], ((jj >> 1) & 1u) ^ 1u, g.wait_ns));
      if (ok) {
        const int row = t / g.segs, seg = t - row * g.segs;
        const int x0 = seg * kTW * 2 - g.pad;
        const int fa = x0 - (x0 & ~3), fm = x0 - (x0 & ~15);  // x0 within the raw rows
        const uint8_t* raw = smem + Sm::kRaw + rs * kRawBytes;
        const float* rf = reinterpret_cast<const float*>(raw);
        constexpr int kWin = 2 * kTW + 1;  // window pixels per input row
        for (int q = xt; q < 3 * kWin; q += kXfGroupWarps * 32) {
          const int ky = q >= 2 * kWin ? 2 : q >= kWin ? 1 : 0;
          const int d = q - ky * kWin, f = fa + d, h = fm + d;  // f, h < 256
          const float* p = rf + ky * 256 + f;  // planes 768 floats apart
          const float c0 = p[0], c1 = p[768], c2 = p[2 * 768];
          const uint8_t mb = g.has_mask ? raw[kRawMask + ky * 256 + h] : 0;
          const __nv_bfloat162 rg = __floats2bfloat162_rn(c0, c1);
          const __nv_bfloat162 bm = __floats2bfloat162_rn(c2, mb ? 1.0f : 0.0f);
          const int arr = ky * 2 + ((d & 1) ^ (ky == 1 ? 1 : 0));  // O_0 E_0 | E_1 O_1 | O_2 E_2
          *reinterpret_cast<uint4*>(buf + arr * kParArr + (d >> 1) * 16) =
              make_uint4(*reinterpret_cast<const uint32_t*>(&rg),
                         *reinterpret_cast<const uint32_t*>(&bm), 0u, 0u);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&raw_empty[rs]);
      // the whole group stops together: the barrier ORs every thread's view
      if (group_sync_or(x, !ok || failed(&s_fail))) {
        s_fail = 1;
        break;
      }
      if (xt == 0) {
        const int a = (int)(j % kAcc);
        if (!mbar_wait(&acc_empty[a], ((j / kAcc) & 1u) ^ 1u, g.wait_ns)) {
          s_fail = 1;
        } else {
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(a * kAccStride);
          const uint32_t bs = smem_u32(buf);
          // the weights' K = 16 slice q: k-tile q / 4, 32 bytes per slice
          const uint64_t bd0 = sw128_desc(smem_u32(smem + Sm::kB));
          auto bq = [&](int q) {
            return bd0 + (uint64_t)((q >> 2) * (kBBytes >> 4)) + 2u * (uint32_t)(q & 3);
          };
          // slices 0 ... 4: (start, leading-dimension offset) as above
          mma_bf16(d, kmajor_desc(bs, S, 128u, 0u), bq(0), idesc, 0u);
          mma_bf16(d, kmajor_desc(bs + 16u, 3u * S - 16u, 128u, 0u), bq(1), idesc, 1u);
          mma_bf16(d, kmajor_desc(bs + 2u * S, S + 16u, 128u, 0u), bq(2), idesc, 1u);
          mma_bf16(d, kmajor_desc(bs + 4u * S, S, 128u, 0u), bq(3), idesc, 1u);
          mma_bf16(d, kmajor_desc(bs + 4u * S + 16u, cst_s - (bs + 4u * S + 16u), 128u, 0u),
                   bq(4), idesc, 1u);
          const uint64_t zd = kmajor_desc(cst_s + 2048u, 2048u, 128u, 0u);
          for (int q = 5; q < 4 * nk; q++) mma_bf16(d, zd, bq(q), idesc, 1u);
          mma_commit(&a_empty[ab]);
          mma_commit(&acc_full[a]);
        }
      }
    }
  } else if (!PAR && warp >= kXfWarp0) {
    // im2col group x takes tiles j = x, x + 3, ...: one thread per (tile row
    // r, input row ky) writes the ks chunks of taps (ky, 0 ... ks - 1) of row
    // r (consecutive threads take consecutive rows: stride-apart words on the
    // loads, the 16-byte stores spread over the swizzle); then the group's
    // first thread issues the tile's MMAs
    const int x = (warp - kXfWarp0) / kXfGroupWarps;
    const int xt = threadIdx.x - (kXfWarp0 + x * kXfGroupWarps) * 32;  // 0 ... 191
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);
    if (xt == 0 && !mbar_wait(&bres_full, 0, g.wait_ns)) s_fail = 1;
    uint32_t j = (uint32_t)x;
    for (int t = blockIdx.x + x * gridDim.x; t < g.tiles;
         t += kXfGroups * gridDim.x, j += kXfGroups) {
      const uint32_t aj = j * (uint32_t)nk;  // the tile's k-tiles: stages aj, aj + 1, ...
      const int rs = (int)(j % kRawStages);
      bool ok =
          __all_sync(0xffffffffu, mbar_wait(&raw_full[rs], (j / kRawStages) & 1u, g.wait_ns));
      for (int i = 0; i < nk && ok; i++) {
        const uint32_t q = aj + (uint32_t)i;
        ok = __all_sync(0xffffffffu, mbar_wait(&a_empty[q % kAStages],
                                               ((q / kAStages) & 1u) ^ 1u, g.wait_ns));
      }
      if (ok) {
        const int row = t / g.segs, seg = t - row * g.segs;
        const int x0 = seg * kBM * g.stride - g.pad;
        const int fa = x0 - (x0 & ~3), fm = x0 - (x0 & ~15);  // x0 within the raw rows
        const uint8_t* raw = smem + Sm::kRaw + rs * kRawBytes;
        const float* rf = reinterpret_cast<const float*>(raw);
        const float* rt = reinterpret_cast<const float*>(raw + kRawTail);
        // the 16-byte chunk of window pixel d of input row ky: R, G, B, mask
        // as BF16, four zeros
        auto chunk = [&](int ky, int d) {
          const int f = fa + d, h = fm + d;
          const float* fr = rf + ky * 256;
          const float* ft = rt + ky * 8;
          float c3[3];
#pragma unroll
          for (int p = 0; p < 3; p++) c3[p] = f < 256 ? fr[p * 768 + f] : ft[p * 24 + f - 256];
          const uint8_t mb = !g.has_mask                ? 0
                             : h < 256                   ? raw[kRawMask + ky * 256 + h]
                                                         : raw[kRawMaskTail + ky * 16 + h - 256];
          const __nv_bfloat162 rg = __floats2bfloat162_rn(c3[0], c3[1]);
          const __nv_bfloat162 bm = __floats2bfloat162_rn(c3[2], mb ? 1.0f : 0.0f);
          return make_uint2(*reinterpret_cast<const uint32_t*>(&rg),
                            *reinterpret_cast<const uint32_t*>(&bm));
        };
        auto store = [&](int ky, int kx, int r, uint2 v) {
          const int tap = ky * g.ks + kx, c = tap & 7;
          uint8_t* A = smem + Sm::kA + ((aj + (uint32_t)(tap >> 3)) % kAStages) * kStageA;
          *reinterpret_cast<uint4*>(A + r * 128 + ((c ^ (r & 7)) << 4)) =
              make_uint4(v.x, v.y, 0u, 0u);
        };
        if (g.stride == 2 && g.ks == 3) {
          // 3 x 3, stride 2: the kx = 2 pixel of row r is the kx = 0 pixel of
          // row r + 1, taken from the next lane (a warp's lanes hold
          // consecutive rows of one ky); each pixel is converted once
          for (int q = xt; q < 3 * kBM; q += kXfGroupWarps * 32) {
            const int ky = q >> 7, r = q & (kBM - 1);
            const uint2 v0 = chunk(ky, 2 * r), v1 = chunk(ky, 2 * r + 1);
            uint2 v2;
            v2.x = __shfl_down_sync(0xffffffffu, v0.x, 1);
            v2.y = __shfl_down_sync(0xffffffffu, v0.y, 1);
            if (lane == 31) v2 = chunk(ky, 2 * r + 2);
            store(ky, 0, r, v0);
            store(ky, 1, r, v1);
            store(ky, 2, r, v2);
          }
        } else {
          for (int q = xt; q < g.ks * kBM; q += kXfGroupWarps * 32) {
            const int ky = q >> 7, r = q & (kBM - 1);
            for (int kx = 0; kx < g.ks; kx++) store(ky, kx, r, chunk(ky, r * g.stride + kx));
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&raw_empty[rs]);
      // the whole group stops together: the barrier ORs every thread's view
      if (group_sync_or(x, !ok || failed(&s_fail))) {
        s_fail = 1;
        break;
      }
      if (xt == 0) {
        const int a = (int)(j % kAcc);
        if (!mbar_wait(&acc_empty[a], ((j / kAcc) & 1u) ^ 1u, g.wait_ns)) {
          s_fail = 1;
        } else {
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(a * kAccStride);
          for (int i = 0; i < nk; i++) {
            const int s = (int)((aj + (uint32_t)i) % kAStages);
            const uint64_t ad = sw128_desc(smem_u32(smem + Sm::kA + s * kStageA));
            const uint64_t bd = sw128_desc(smem_u32(smem + Sm::kB + i * kBBytes));
#pragma unroll
            for (int kk = 0; kk < kBK / 16; kk++)
              mma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&a_empty[s]);
          }
          mma_commit(&acc_full[a]);
        }
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  if (threadIdx.x == 0 && s_fail && g.status) atomicCAS(g.status, 0, (int)GS2D_ERR_TIMEOUT);
}

// Tensor map of a dim-4 float tensor [B][3][H][W] (box w pixels x 3 rows x 3
// planes) or of a dim-3 byte tensor [B][H][W] (box w pixels x 3 rows); zeros
// out of range.
bool make_row_map(CUtensorMap* map, const void* base, bool bytes, int B, int H, int W, int w) {
  EncodeTiled fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint64_t es = bytes ? 1 : 4;
  const cuuint64_t dims4[4] = {(cuuint64_t)W, (cuuint64_t)H, 3, (cuuint64_t)B};
  const cuuint64_t str4[3] = {W * es, (cuuint64_t)H * W * es, (cuuint64_t)3 * H * W * es};
  const cuuint64_t dims3[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t str3[2] = {W * es, (cuuint64_t)H * W * es};
  const cuuint32_t box[4] = {(cuuint32_t)w, kRawRows, bytes ? 1u : 3u, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(map, bytes ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
            bytes ? 3 : 4, const_cast<void*>(base), bytes ? dims3 : dims4, bytes ? str3 : str4,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, bool PAR>
cudaError_t launch_frame(const CUtensorMap (&maps)[5], const FrameArgs& g, int smem,
                         cudaStream_t s) {
  const cudaError_t attr = opt_in_smem((const void*)k_conv_frame<BN, PAR>, smem);
  if (attr != cudaSuccess) return attr;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  const int grid = std::max(1, std::min(g.tiles, sms));
  k_conv_frame<BN, PAR><<<grid, kFrThreads, smem, s>>>(maps[0], maps[1], maps[2], maps[3],
                                                        maps[4], g);
  return cudaGetLastError();
}

}  // namespace

bool frame_conv_supported(int W, int ks, int stride, int N) {
  return W % 16 == 0 && ks >= 1 && ks <= kRawRows && stride >= 1 &&
         kBM * stride - stride + ks <= 257 && N >= 1 && N <= 128;
}

cudaError_t tc_conv_frame(const TcFrameConvProblem& pr, cudaStream_t s) {
  const int Ho = (pr.H + 2 * pr.pad - pr.ks) / pr.stride + 1;
  const int Wo = (pr.W + 2 * pr.pad - pr.ks) / pr.stride + 1;
  if (pr.B <= 0 || Ho <= 0 || Wo <= 0 || pr.N <= 0) return cudaSuccess;
  if (!frame_conv_supported(pr.W, pr.ks, pr.stride, pr.N) || pr.ldk % 8 ||
      pr.ldk < pr.ks * pr.ks * 8 + 1 || (reinterpret_cast<uintptr_t>(pr.frames) & 15) ||
      (reinterpret_cast<uintptr_t>(pr.masks) & 15) || (reinterpret_cast<uintptr_t>(pr.W_) & 15))
    return cudaErrorInvalidValue;
  const int bn = tc_gemm_bn(pr.N);
  FrameArgs g;
  g.B = pr.B;
  g.H = pr.H;
  g.W = pr.W;
  g.Ho = Ho;
  g.Wo = Wo;
  g.ks = pr.ks;
  g.stride = pr.stride;
  g.pad = pr.pad;
  g.N = pr.N;
  g.ldc = pr.ldc;
  g.relu = pr.relu;
  g.has_mask = pr.masks ? 1 : 0;
  // 3 x 3 at stride 2: the record layout, 120-pixel tiles; else im2col rows
  // in a ring whose stage s always holds k-tile s % nk, 128-pixel tiles
  const bool par = pr.ks == 3 && pr.stride == 2;
  const int tw = par ? 120 : kBM;
  g.segs = (Wo + tw - 1) / tw;
  g.tiles = pr.B * Ho * g.segs;
  g.nk = (pr.ldk + kBK - 1) / kBK;
  g.out_f32 = pr.out_f32;
  g.out_bf16 = pr.out_bf16;
  g.status = pr.status;
  g.wait_ns = pr.wait_ns;
  g.withhold = pr.withhold_loads;
  if (!par && kAStages % g.nk != 0) return cudaErrorInvalidValue;
  const int smem = (par ? FrameSmem<true>::kB : FrameSmem<false>::kB) + g.nk * bn * kBK * 2 + 1024;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  CUtensorMap maps[5];
  // without a mask the mask maps are never used: encode them over the frames
  const void* mbase = pr.masks ? (const void*)pr.masks : (const void*)pr.frames;
  if (!make_row_map(&maps[0], pr.frames, false, pr.B, pr.H, pr.W, 256) ||
      !make_row_map(&maps[1], pr.frames, false, pr.B, pr.H, pr.W, 8) ||
      !make_row_map(&maps[2], mbase, true, pr.B, pr.H, pr.W, 256) ||
      !make_row_map(&maps[3], mbase, true, pr.B, pr.H, pr.W, 16) ||
      !make_map(&maps[4], pr.W_, pr.N, pr.ldk, pr.ldk, bn))
    return cudaErrorInvalidValue;
  if (par) {
    switch (bn) {
      case 32: return launch_frame<32, true>(maps, g, smem, s);
      case 64: return launch_frame<64, true>(maps, g, smem, s);
      case 96: return launch_frame<96, true>(maps, g, smem, s);
      default: return launch_frame<128, true>(maps, g, smem, s);
    }
  }
  switch (bn) {
    case 32: return launch_frame<32, false>(maps, g, smem, s);
    case 64: return launch_frame<64, false>(maps, g, smem, s);
    case 96: return launch_frame<96, false>(maps, g, smem, s);
    default: return launch_frame<128, false>(maps, g, smem, s);
  }
}

}  // namespace gs2d
