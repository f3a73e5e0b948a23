// C ABI of the learned initialiser's building blocks (include/gs2d.h): the
// BF16 tensor-core GEMM and the convolution helpers around it.
#include <cuda_bf16.h>
#include <stdio.h>

#include "gs2d_internal.cuh"
#include "tc_gemm.cuh"

using namespace gs2d;

extern "C" uint64_t gs2d_gemm_partial_bytes(int32_t M, int32_t N, int32_t ldc, int32_t K,
                                            int32_t splits) {
  if (M < 0 || N < 0 || K < 0 || ldc < N) return 0;
  return (uint64_t)tc_gemm_partial_floats(M, N, ldc, K, splits) * sizeof(float);
}

extern "C" gs2d_status gs2d_gemm_bf16(const void* A, int32_t lda, const void* B, int32_t ldb,
                                      int32_t M, int32_t N, int32_t K, const float* bias,
                                      int32_t relu, float* out_f32, void* out_bf16, int32_t ldc,
                                      int32_t splits, float* partial, int32_t* status,
                                      void* stream) {
  if (M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldc < N || (lda % 8) || (ldb % 8))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_gemm_bf16: sizes / leading dimensions");
  if (M == 0 || N == 0) return set_error(GS2D_OK, "");
  if (!A || !B || ((out_f32 == nullptr) == (out_bf16 == nullptr)))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_gemm_bf16: NULL operand or not one output");
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_gemm_bf16: operands not 16-byte aligned");
  if (splits > 1 && tc_gemm_partial_floats(M, N, ldc, K, splits) > 0 && !partial)
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_gemm_bf16: split-K needs the partial buffer");
  TcGemmProblem pr;
  pr.A = static_cast<const __nv_bfloat16*>(A);
  pr.lda = lda;
  pr.B = static_cast<const __nv_bfloat16*>(B);
  pr.ldb = ldb;
  pr.M = M;
  pr.N = N;
  pr.K = K;
  pr.out_f32 = out_f32;
  pr.out_bf16 = static_cast<__nv_bfloat16*>(out_bf16);
  pr.ldc = ldc;
  pr.bias = bias;
  pr.relu = relu;
  pr.splits = splits;
  pr.partial = partial;
  pr.status = status;
  const cudaError_t e = tc_gemm(pr, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof(msg), "gs2d_gemm_bf16: %s", cudaGetErrorString(e));
    return set_error(GS2D_ERR_CUDA, msg);
  }
  return set_error(GS2D_OK, "");
}
