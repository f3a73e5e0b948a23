// BF16 tcgen05 GEMM (csrc/gemm_tc.cu): C[M][N] = A[M][K] . B[N][K]^T with
// optional split-K, bias and ReLU; FP32 or BF16 output.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace gs2d {

struct TcGemmArgs {
  int M, N, num_kt, kt_per_split, ldc;
  size_t split_stride;     // floats between split partials
  float* out_f32;          // FP32 output (or the split partials)
  __nv_bfloat16* out_bf16; // BF16 output (one split only)
  const float* bias;       // [N] or NULL
  int relu;
  int* status;             // device status word (GS2D_ERR_TIMEOUT) or NULL
  unsigned long long wait_ns;  // limit of every mbarrier wait
  int withhold_loads;      // failure-detection check: the producer issues no load
};

struct TcGemmProblem {
  const __nv_bfloat16* A;  // [M][lda], K-contiguous, 16-byte aligned rows
  int lda;
  const __nv_bfloat16* B;  // [N][ldb], K-contiguous
  int ldb;
  int M, N, K;
  float* out_f32;          // [M][ldc] or NULL
  __nv_bfloat16* out_bf16; // [M][ldc] or NULL (exactly one output)
  int ldc;
  const float* bias;
  int relu;
  int splits;              // split-K factor (1: none)
  float* partial;          // splits x M x ldc floats when splits > 1
  int* status;
  unsigned long long wait_ns = 0;  // mbarrier wait limit (0: one second)
  int withhold_loads = 0;  // failure-detection check only (see gs2d_gemm_wait_check)
};

// Implicit-GEMM convolution: Z[p][n] = sum_k col(X)[p][k] W[n][k] with col the
// im2col operand of an NHWC BF16 input (k = tap C + ci, a ones column at
// k = ks^2 C for the bias), never materialised.
struct TcConvProblem {
  const __nv_bfloat16* x;  // [B][Hi][Wi][C], C a multiple of 8, 16-byte aligned
  int B, Hi, Wi, C, ks, stride, pad;
  const __nv_bfloat16* W;  // [N][ldk], ldk a multiple of 8, >= ks^2 C + 1
  int ldk, N;
  int relu;
  float* out_f32;          // [M][ldc] or NULL (exactly one output)
  __nv_bfloat16* out_bf16;
  int ldc;
  int* status;
  unsigned long long wait_ns = 0;  // mbarrier wait limit (0: one second)
  int withhold_loads = 0;  // failure-detection check only (see gs2d_conv_wait_check)
};

// The first convolution straight from float frames [B][3][H][W] and masks
// [B][H][W] (or NULL): im2col of the 8-channel BF16 input (R, G, B, mask != 0,
// zeros) formed on the fly; csrc/conv_frame.cu.
struct TcFrameConvProblem {
  const float* frames;
  const uint8_t* masks;
  int B, H, W, ks, stride, pad;
  const __nv_bfloat16* W_;  // [N][ldk], ldk >= ks^2 8 + 1
  int ldk, N;
  int relu;
  float* out_f32;
  __nv_bfloat16* out_bf16;
  int ldc;
  int* status;
  unsigned long long wait_ns = 0;  // mbarrier wait limit (0: one second)
  int withhold_loads = 0;  // failure-detection check only (see gs2d_conv_wait_check)
};

cudaError_t tc_gemm(const TcGemmProblem& pr, cudaStream_t s);
cudaError_t tc_conv(const TcConvProblem& pr, cudaStream_t s);
// The persistent TMA-tap convolution (csrc/conv_tap.cu): C of 16, 32 or a
// multiple of 64, stride 1 or 2, N <= 256, output rows of 64 pixels or more.
bool tap_conv_supported(const TcConvProblem& pr);
cudaError_t tap_conv(const TcConvProblem& pr, cudaStream_t s);
// The persistent row-box convolution (csrc/conv_rows.cu): 3 x 3, stride 2,
// pad 1, an even input width, C of 32 or 64, N <= 256, output rows of 64
// pixels or more, within its shared-memory plan.
bool rows_conv_supported(const TcConvProblem& pr);
cudaError_t rows_conv(const TcConvProblem& pr, cudaStream_t s);
// W a multiple of 16, ks <= 3, the 128-pixel window within 257 input pixels,
// N <= 128.
bool frame_conv_supported(int W, int ks, int stride, int N);
cudaError_t tc_conv_frame(const TcFrameConvProblem& pr, cudaStream_t s);
int tc_gemm_bn(int n);
size_t tc_gemm_partial_floats(int M, int N, int ldc, int K, int splits);

}  // namespace gs2d
