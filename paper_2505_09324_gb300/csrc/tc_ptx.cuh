// Inline-PTX building blocks of the tcgen05 kernels (csrc/gemm_tc.cu,
// csrc/conv_tap.cu, csrc/conv_rows.cu, csrc/conv_frame.cu): mbarriers with
// time-bounded waits, TMA tensor loads, shared-memory matrix descriptors,
// tcgen05.mma / commit / ld and the
// tcgen05 thread-sync fences.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace gs2d {
namespace {

constexpr int kBM = 128;    // accumulator rows (TMEM lanes)
constexpr int kBK = 64;     // K per stage: one 128-byte swizzle row of bf16
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One test of the phase; a thread whose phase is not complete may be
// suspended for up to 20 us (the suspend-time hint) and is resumed when it
// completes, so that waiting warps do not spin on the issue slots of the
// working ones.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 20000;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for the phase of the given parity to complete; false after limit_ns
// (kWaitNs when 0).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          uint64_t limit_ns = 0) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t limit = limit_ns ? limit_ns : kWaitNs;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; i++)
      if (mbar_test(bar, parity)) return true;
    if (global_ns() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// 4D tiled TMA load (coordinates innermost first) completing on a barrier.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2),
      "r"(c3)
      : "memory");
}

// 5D tiled TMA load (coordinates innermost first) completing on a barrier.
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2),
      "r"(c3), "r"(c4)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand, descriptor version 1:
// start address, leading byte offset (between the 16-byte core-matrix
// columns along K; used by the unswizzled layout only), stride byte offset
// (between 8-row groups) and the layout: 0 none, 6 32-byte, 4 64-byte,
// 2 128-byte swizzle.
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t addr, uint32_t lbo, uint32_t sbo,
                                                uint32_t layout) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)layout << 61);
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle
// layout (8-row atoms of 1024 bytes; stride between atoms 1024 bytes; the
// leading-dimension offset is unused for this layout), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// The same with each descriptor as its two 32-bit words: a K-major
// descriptor's start address sits in the low word (14 bits, in 16-byte units,
// no carry out of it below 256 KB of shared memory), so operand offsets are
// 32-bit additions.
__device__ __forceinline__ void mma_bf16_w(uint32_t d_tmem, uint32_t a_lo, uint32_t a_hi,
                                           uint32_t b_lo, uint32_t b_hi, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b64 da, db;\n setp.ne.b32 p, %6, 0;\n"
      " mov.b64 da, {%1, %2};\n mov.b64 db, {%3, %4};\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n}" ::"r"(d_tmem),
      "r"(a_lo), "r"(a_hi), "r"(b_lo), "r"(b_hi), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// tcgen05.ld of 16 or 32 consecutive accumulator columns of the warp's 32
// TMEM lanes, with the wait in the same statement so that no use of the
// registers can be scheduled before the data has arrived.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {"
      "%0, %1, %2, %3, %4, %5, %6, %7, "
      "%8, %9, %10, %11, %12, %13, %14, %15"
      "}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {"
      "%0, %1, %2, %3, %4, %5, %6, %7, "
      "%8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, "
      "%24, %25, %26, %27, %28, %29, %30, %31"
      "}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Epilogue of one accumulator row (TMEM lane) of a 128-row tile: BN FP32
// columns read 16 at a time with tcgen05.ld (warp-collective: every lane of
// the warp calls this), ReLU when asked, then stored as BF16 or FP32 at
// out + o, columns below N only, when the row is valid (16-byte vectors when
// vec_ok and the 16 columns are all below N).
template <int BN>
__device__ __forceinline__ void store_acc_row(uint32_t taddr, bool valid, size_t o, int N,
                                              int relu, bool vec_ok, float* out_f32,
                                              __nv_bfloat16* out_bf16) {
  // 32 columns per load where the tile allows (one wait per 32 columns)
  constexpr int kW = BN % 32 == 0 ? 32 : 16;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += kW) {
    float w[kW];
    if constexpr (kW == 32)
      tmem_ld32(taddr + (uint32_t)c0, w);
    else
      tmem_ld16(taddr + (uint32_t)c0, w);
    if (!valid) continue;
#pragma unroll
    for (int j = 0; j < kW; j++)
      if (relu) w[j] = fmaxf(w[j], 0.0f);
#pragma unroll
    for (int q = 0; q < kW; q += 16) {
      const int c = c0 + q;
      const float* v = w + q;
      if (vec_ok && c + 16 <= N) {
        if (out_bf16) {
          __align__(16) __nv_bfloat162 hv[8];
#pragma unroll
          for (int j = 0; j < 8; j++) hv[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
          uint4* dst = reinterpret_cast<uint4*>(out_bf16 + o + c);
          dst[0] = reinterpret_cast<const uint4*>(hv)[0];
          dst[1] = reinterpret_cast<const uint4*>(hv)[1];
        } else {
          float4* dst = reinterpret_cast<float4*>(out_f32 + o + c);
#pragma unroll
          for (int j = 0; j < 4; j++)
            dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; j++) {
          if (c + j < N) {
            if (out_bf16)
              out_bf16[o + c + j] = __float2bfloat16_rn(v[j]);
            else
              out_f32[o + c + j] = v[j];
          }
        }
      }
    }
  }
}

}  // namespace

// cuTensorMapEncodeTiled, found once through the runtime's driver entry
// points (NULL when the driver lacks it); defined in csrc/gemm_tc.cu.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled tensor_map_encoder();

// 2D bf16 tensor map of a rows x cols (K-contiguous) matrix with leading
// dimension ld (elements): box 64 (K) x box_rows, 128-byte swizzle, zeros out
// of range; defined in csrc/gemm_tc.cu.
bool make_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows);

}  // namespace gs2d
