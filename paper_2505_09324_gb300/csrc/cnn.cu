// C ABI of the learned initialiser's building blocks (include/gs2d.h): the
// BF16 tensor-core GEMM and the convolution helpers around it.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <stdio.h>

#include <algorithm>

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

extern "C" gs2d_status gs2d_gemm_wait_check(const void* A, const void* B, float* out,
                                            int32_t* status, uint64_t wait_ns, void* stream) {
  if (!A || !B || !out || !status || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_gemm_wait_check: NULL or misaligned pointer");
  if (wait_ns < 1000000ull || wait_ns > 1000000000ull)
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_gemm_wait_check: wait_ns outside [1 ms, 1 s]");
  TcGemmProblem pr;
  pr.A = static_cast<const __nv_bfloat16*>(A);
  pr.lda = 64;
  pr.B = static_cast<const __nv_bfloat16*>(B);
  pr.ldb = 64;
  pr.M = 128;
  pr.N = 32;
  pr.K = 64;
  pr.out_f32 = out;
  pr.out_bf16 = nullptr;
  pr.ldc = 32;
  pr.bias = nullptr;
  pr.relu = 0;
  pr.splits = 1;
  pr.partial = nullptr;
  pr.status = status;
  pr.wait_ns = wait_ns;
  pr.withhold_loads = 1;
  const cudaError_t e = tc_gemm(pr, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof(msg), "gs2d_gemm_wait_check: %s", cudaGetErrorString(e));
    return set_error(GS2D_ERR_CUDA, msg);
  }
  return set_error(GS2D_OK, "");
}

extern "C" gs2d_status gs2d_conv_wait_check(int32_t kernel, const void* x, const void* W,
                                            void* out, int32_t* status, uint64_t wait_ns,
                                            void* stream) {
  if ((kernel != GS2D_CHECK_CONV_FRAME && kernel != GS2D_CHECK_CONV_TAP &&
       kernel != GS2D_CHECK_CONV_ROWS) || !x || !W || !out ||
      !status || ((uintptr_t)x & 15) || ((uintptr_t)W & 15) || ((uintptr_t)out & 15))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_conv_wait_check: kernel, NULL or misaligned");
  if (wait_ns < 1000000ull || wait_ns > 1000000000ull)
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_conv_wait_check: wait_ns outside [1 ms, 1 s]");
  cudaError_t e;
  if (kernel == GS2D_CHECK_CONV_FRAME) {  // 1 x 3 x 16 x 256 frame -> 8 x 128 x 32
    TcFrameConvProblem pr;
    pr.frames = static_cast<const float*>(x);
    pr.masks = nullptr;
    pr.B = 1;
    pr.H = 16;
    pr.W = 256;
    pr.ks = 3;
    pr.stride = 2;
    pr.pad = 1;
    pr.W_ = static_cast<const __nv_bfloat16*>(W);
    pr.ldk = 80;
    pr.N = 32;
    pr.relu = 1;
    pr.out_f32 = nullptr;
    pr.out_bf16 = static_cast<__nv_bfloat16*>(out);
    pr.ldc = 32;
    pr.status = status;
    pr.wait_ns = wait_ns;
    pr.withhold_loads = 1;
    e = tc_conv_frame(pr, (cudaStream_t)stream);
  } else {  // 1 x 16 x 256 x 32 activation -> 8 x 128 x 64
    TcConvProblem pr;
    pr.x = static_cast<const __nv_bfloat16*>(x);
    pr.B = 1;
    pr.Hi = 16;
    pr.Wi = 256;
    pr.C = 32;
    pr.ks = 3;
    pr.stride = 2;
    pr.pad = 1;
    pr.W = static_cast<const __nv_bfloat16*>(W);
    pr.ldk = 296;
    pr.N = 64;
    pr.relu = 1;
    pr.out_f32 = nullptr;
    pr.out_bf16 = static_cast<__nv_bfloat16*>(out);
    pr.ldc = 64;
    pr.status = status;
    pr.wait_ns = wait_ns;
    pr.withhold_loads = 1;
    e = kernel == GS2D_CHECK_CONV_TAP ? tap_conv(pr, (cudaStream_t)stream)
                                      : rows_conv(pr, (cudaStream_t)stream);
  }
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof(msg), "gs2d_conv_wait_check: %s", cudaGetErrorString(e));
    return set_error(GS2D_ERR_CUDA, msg);
  }
  return set_error(GS2D_OK, "");
}

extern "C" gs2d_status gs2d_conv_bf16(const void* x, int32_t B, int32_t Hi, int32_t Wi,
                                      int32_t C, int32_t ks, int32_t stride, int32_t pad,
                                      const void* W, int32_t ldk, int32_t N, int32_t relu,
                                      float* out_f32, void* out_bf16, int32_t ldc,
                                      int32_t* status, void* stream) {
  if (B < 0 || Hi < 1 || Wi < 1 || C < 8 || (C % 8) || ks < 1 || stride < 1 || pad < 0 ||
      N < 0 || ldk % 8 || ldk < ks * ks * C + 1 || ldc < N)
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_conv_bf16: sizes");
  const int Ho = (Hi + 2 * pad - ks) / stride + 1, Wo = (Wi + 2 * pad - ks) / stride + 1;
  if (Ho < 1 || Wo < 1) return set_error(GS2D_ERR_INVALID_ARG, "gs2d_conv_bf16: empty output");
  if (B == 0 || N == 0) return set_error(GS2D_OK, "");
  if (!x || !W || ((out_f32 == nullptr) == (out_bf16 == nullptr)) || ((uintptr_t)x & 15) ||
      ((uintptr_t)W & 15))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_conv_bf16: operands");
  TcConvProblem pr;
  pr.x = static_cast<const __nv_bfloat16*>(x);
  pr.B = B;
  pr.Hi = Hi;
  pr.Wi = Wi;
  pr.C = C;
  pr.ks = ks;
  pr.stride = stride;
  pr.pad = pad;
  pr.W = static_cast<const __nv_bfloat16*>(W);
  pr.ldk = ldk;
  pr.N = N;
  pr.relu = relu;
  pr.out_f32 = out_f32;
  pr.out_bf16 = static_cast<__nv_bfloat16*>(out_bf16);
  pr.ldc = ldc;
  pr.status = status;
  const cudaError_t e = tc_conv(pr, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof(msg), "gs2d_conv_bf16: %s", cudaGetErrorString(e));
    return set_error(GS2D_ERR_CUDA, msg);
  }
  return set_error(GS2D_OK, "");
}

extern "C" gs2d_status gs2d_conv_frame_bf16(const float* frames, const uint8_t* masks,
                                            int32_t B, int32_t H, int32_t W, int32_t ks,
                                            int32_t stride, int32_t pad, const void* Wt,
                                            int32_t ldk, int32_t N, int32_t relu, float* out_f32,
                                            void* out_bf16, int32_t ldc, int32_t* status,
                                            void* stream) {
  if (B < 0 || H < 1 || W < 1 || ks < 1 || stride < 1 || pad < 0 || N < 0 || ldk % 8 ||
      ldk < ks * ks * 8 + 1 || ldk > 192 || ldc < N)
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_conv_frame_bf16: sizes");
  const int Ho = (H + 2 * pad - ks) / stride + 1, Wo = (W + 2 * pad - ks) / stride + 1;
  if (Ho < 1 || Wo < 1) return set_error(GS2D_ERR_INVALID_ARG, "gs2d_conv_frame_bf16: empty output");
  if (B == 0 || N == 0) return set_error(GS2D_OK, "");
  if (!frame_conv_supported(W, ks, stride, N))
    return set_error(GS2D_ERR_INVALID_ARG,
                     "gs2d_conv_frame_bf16: W a multiple of 16, ks <= 3, stride <= 2, N <= 128");
  if (!frames || !Wt || ((out_f32 == nullptr) == (out_bf16 == nullptr)) ||
      ((uintptr_t)frames & 15) || ((uintptr_t)masks & 15) || ((uintptr_t)Wt & 15))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_conv_frame_bf16: operands");
  TcFrameConvProblem pr;
  pr.frames = frames;
  pr.masks = masks;
  pr.B = B;
  pr.H = H;
  pr.W = W;
  pr.ks = ks;
  pr.stride = stride;
  pr.pad = pad;
  pr.W_ = static_cast<const __nv_bfloat16*>(Wt);
  pr.ldk = ldk;
  pr.N = N;
  pr.relu = relu;
  pr.out_f32 = out_f32;
  pr.out_bf16 = static_cast<__nv_bfloat16*>(out_bf16);
  pr.ldc = ldc;
  pr.status = status;
  const cudaError_t e = tc_conv_frame(pr, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof(msg), "gs2d_conv_frame_bf16: %s", cudaGetErrorString(e));
    return set_error(GS2D_ERR_CUDA, msg);
  }
  return set_error(GS2D_OK, "");
}

// ---------------------------------------------------------------------------
// Convolution helpers.  Activations are NHWC BF16 ([B][H][W][C], C a multiple
// of 8); a ks x ks convolution is the GEMM  Z = col(X) . W^T  with
// col(X)[p][k], k = (ky ks + kx) C + ci, and one extra column of ones at
// k = ks^2 C that carries the bias (the weight row's last used entry).

namespace {

using bf16 = __nv_bfloat16;

__global__ void k_cnn_input(int B, int H, int W, const float* __restrict__ frames,
                            const uint8_t* __restrict__ masks, bf16* __restrict__ x) {
  const size_t HW = (size_t)H * W, total = (size_t)B * HW;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total;
       p += (size_t)gridDim.x * blockDim.x) {
    const size_t b = p / HW, q = p % HW;
    const float* f = frames + b * 3 * HW;
    __align__(16) bf16 v[8];
    v[0] = __float2bfloat16_rn(f[q]);
    v[1] = __float2bfloat16_rn(f[HW + q]);
    v[2] = __float2bfloat16_rn(f[2 * HW + q]);
    v[3] = __float2bfloat16_rn(masks && masks[p] ? 1.0f : 0.0f);
    for (int i = 4; i < 8; i++) v[i] = __float2bfloat16_rn(0.0f);
    reinterpret_cast<uint4*>(x)[p] = *reinterpret_cast<const uint4*>(v);
  }
}

// One thread per (output pixel, 8-wide chunk of k).
// One thread per 16-byte chunk of col (consecutive threads, consecutive
// chunks of a row: coalesced stores).  I is the index type: 32-bit whenever
// the chunk count fits, since 64-bit divisions are long emulated sequences
// and this kernel is a few divisions per 16 bytes moved.
template <typename I>
__global__ void k_im2col(int B, int Hi, int Wi, int C, int Ho, int Wo, int ks, int stride,
                         int pad, int ldk, const bf16* __restrict__ x, bf16* __restrict__ col) {
  const I chunks = (I)(ldk / 8), hw = (I)Ho * (I)Wo;
  const int kk = ks * ks * C;
  const I total = (I)B * hw * chunks;
  for (I t = (I)blockIdx.x * (I)blockDim.x + (I)threadIdx.x; t < total;
       t += (I)gridDim.x * (I)blockDim.x) {
    const I p = t / chunks;
    const int c = (int)(t - p * chunks), k0 = 8 * c;
    const int b = (int)(p / hw);
    const int r = (int)(p - (I)b * hw);
    const int oy = r / Wo, ox = r - oy * Wo;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (k0 < kk) {
      const int tap = k0 / C, ci = k0 - tap * C;
      const int ky = tap / ks, kx = tap - ky * ks;
      const int iy = oy * stride + ky - pad, ix = ox * stride + kx - pad;
      if (iy >= 0 && iy < Hi && ix >= 0 && ix < Wi)
        v = *reinterpret_cast<const uint4*>(x + (((size_t)b * Hi + iy) * Wi + ix) * C + ci);
    } else if (k0 == kk) {
      v.x = 0x3F80u;  // bf16 1.0 in the low half: element k0
    }
    *reinterpret_cast<uint4*>(col + (size_t)p * ldk + k0) = v;
  }
}

// One thread per (input pixel, channel): the taps that read it.
// I: the index type, 32-bit whenever the element count fits (as k_im2col).
template <typename I>
__global__ void k_col2im(const float* __restrict__ dcol, int ldk, int B, int Hi, int Wi, int C,
                         int Ho, int Wo, int ks, int stride, int pad,
                         const bf16* __restrict__ act, bf16* __restrict__ dx) {
  const I hw = (I)Hi * (I)Wi;
  const I total = (I)B * hw * (I)C;
  for (I t = (I)blockIdx.x * (I)blockDim.x + (I)threadIdx.x; t < total;
       t += (I)gridDim.x * (I)blockDim.x) {
    const I pin = t / (I)C;
    const int ci = (int)(t - pin * (I)C);
    const int b = (int)(pin / hw);
    const int r = (int)(pin - (I)b * hw);
    const int iy = r / Wi, ix = r - iy * Wi;
    float s = 0.0f;
    for (int ky = 0; ky < ks; ky++) {
      const int ny = iy + pad - ky;
      if (ny < 0 || ny % stride) continue;
      const int oy = ny / stride;
      if (oy >= Ho) continue;
      for (int kx = 0; kx < ks; kx++) {
        const int nx = ix + pad - kx;
        if (nx < 0 || nx % stride) continue;
        const int ox = nx / stride;
        if (ox >= Wo) continue;
        s += dcol[(((size_t)b * Ho + oy) * Wo + ox) * ldk + (ky * ks + kx) * C + ci];
      }
    }
    if (act && !(__bfloat162float(act[t]) > 0.0f)) s = 0.0f;
    dx[t] = __float2bfloat16_rn(s);
  }
}

// out[c][r] = in[r][c], 32 x 32 tiles through shared memory (row tiles on
// the grid's x dimension, which allows 2^31 - 1 of them).
__global__ void k_transpose(const bf16* __restrict__ in, int R, int C, int ld_in,
                            bf16* __restrict__ out, int ld_out) {
  __shared__ bf16 tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < C) tile[i][threadIdx.x] = in[(size_t)r * ld_in + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < R && c < C) out[(size_t)c * ld_out + r] = tile[threadIdx.x][i];
  }
}

__global__ void k_relu_bwd(const float* __restrict__ dx, int rows, int cols, int ldx,
                           const bf16* __restrict__ act, int lda, bf16* __restrict__ dz, int ldz) {
  const size_t total = (size_t)rows * cols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t r = t / cols;
    const int c = (int)(t % cols);
    const float a = __bfloat162float(act[r * lda + c]);
    dz[r * ldz + c] = __float2bfloat16_rn(a > 0.0f ? dx[r * ldx + c] : 0.0f);
  }
}

__global__ void k_cast_weights(const float* __restrict__ w, int co, int ldk, bf16* __restrict__ wb,
                               bf16* __restrict__ wt) {
  const size_t total = (size_t)co * ldk;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(t / ldk), k = (int)(t % ldk);
    const bf16 v = __float2bfloat16_rn(w[t]);
    if (wb) wb[t] = v;
    if (wt) wt[(size_t)k * co + o] = v;
  }
}

int grid_for(size_t work, int threads) {
  const size_t b = (work + threads - 1) / threads;
  return (int)std::min<size_t>(std::max<size_t>(b, 1), 152 * 32);
}

gs2d_status launched(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
    return set_error(GS2D_ERR_CUDA, msg);
  }
  return set_error(GS2D_OK, "");
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

extern "C" gs2d_status gs2d_cnn_input(const float* frames, const uint8_t* masks, int32_t B,
                                      int32_t H, int32_t W, void* x, void* stream) {
  if (B < 0 || H < 1 || W < 1 || (B > 0 && (!frames || !x)) || !aligned16(x))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_cnn_input: arguments");
  const size_t total = (size_t)B * H * W;
  if (total == 0) return set_error(GS2D_OK, "");
  k_cnn_input<<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(
      B, H, W, frames, masks, static_cast<bf16*>(x));
  return launched("gs2d_cnn_input");
}

extern "C" gs2d_status gs2d_im2col(const void* x, int32_t B, int32_t Hi, int32_t Wi, int32_t C,
                                   int32_t ks, int32_t stride, int32_t pad, void* col,
                                   int32_t ldk, void* stream) {
  if (B < 0 || Hi < 1 || Wi < 1 || C < 8 || C % 8 || ks < 1 || stride < 1 || pad < 0 ||
      ldk % 8 || ldk <= ks * ks * C || !x || !col || !aligned16(x) || !aligned16(col))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_im2col: arguments");
  const int Ho = (Hi + 2 * pad - ks) / stride + 1, Wo = (Wi + 2 * pad - ks) / stride + 1;
  if (Ho < 1 || Wo < 1) return set_error(GS2D_ERR_INVALID_ARG, "gs2d_im2col: empty output");
  const size_t total = (size_t)B * Ho * Wo * (ldk / 8);
  if (total == 0) return set_error(GS2D_OK, "");
  if (total < (size_t)INT32_MAX)
    k_im2col<uint32_t><<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(
        B, Hi, Wi, C, Ho, Wo, ks, stride, pad, ldk, static_cast<const bf16*>(x),
        static_cast<bf16*>(col));
  else
    k_im2col<size_t><<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(
        B, Hi, Wi, C, Ho, Wo, ks, stride, pad, ldk, static_cast<const bf16*>(x),
        static_cast<bf16*>(col));
  return launched("gs2d_im2col");
}

extern "C" gs2d_status gs2d_col2im(const float* dcol, int32_t ldk, int32_t B, int32_t Hi,
                                   int32_t Wi, int32_t C, int32_t ks, int32_t stride, int32_t pad,
                                   const void* act, void* dx, void* stream) {
  if (B < 0 || Hi < 1 || Wi < 1 || C < 1 || ks < 1 || stride < 1 || pad < 0 ||
      ldk < ks * ks * C || !dcol || !dx)
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_col2im: arguments");
  const int Ho = (Hi + 2 * pad - ks) / stride + 1, Wo = (Wi + 2 * pad - ks) / stride + 1;
  const size_t total = (size_t)B * Hi * Wi * C;
  if (total == 0) return set_error(GS2D_OK, "");
  if (total < (size_t)INT32_MAX)
    k_col2im<uint32_t><<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(
        dcol, ldk, B, Hi, Wi, C, Ho, Wo, ks, stride, pad, static_cast<const bf16*>(act),
        static_cast<bf16*>(dx));
  else
    k_col2im<size_t><<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(
        dcol, ldk, B, Hi, Wi, C, Ho, Wo, ks, stride, pad, static_cast<const bf16*>(act),
        static_cast<bf16*>(dx));
  return launched("gs2d_col2im");
}

extern "C" gs2d_status gs2d_transpose_bf16(const void* in, int32_t R, int32_t C, int32_t ld_in,
                                           void* out, int32_t ld_out, void* stream) {
  if (R < 0 || C < 0 || ld_in < C || ld_out < R || (R * C > 0 && (!in || !out)))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_transpose_bf16: arguments");
  if (R == 0 || C == 0) return set_error(GS2D_OK, "");
  if ((C + 31) / 32 > 65535) return set_error(GS2D_ERR_INVALID_ARG, "gs2d_transpose_bf16: C");
  const dim3 grid((R + 31) / 32, (C + 31) / 32), block(32, 8);
  k_transpose<<<grid, block, 0, (cudaStream_t)stream>>>(static_cast<const bf16*>(in), R, C, ld_in,
                                                        static_cast<bf16*>(out), ld_out);
  return launched("gs2d_transpose_bf16");
}

extern "C" gs2d_status gs2d_relu_bwd(const float* dx, int32_t rows, int32_t cols, int32_t ldx,
                                     const void* act, int32_t lda, void* dz, int32_t ldz,
                                     void* stream) {
  if (rows < 0 || cols < 0 || ldx < cols || lda < cols || ldz < cols ||
      (rows * cols > 0 && (!dx || !act || !dz)))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_relu_bwd: arguments");
  const size_t total = (size_t)rows * cols;
  if (total == 0) return set_error(GS2D_OK, "");
  k_relu_bwd<<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(
      dx, rows, cols, ldx, static_cast<const bf16*>(act), lda, static_cast<bf16*>(dz), ldz);
  return launched("gs2d_relu_bwd");
}

extern "C" gs2d_status gs2d_cast_weights(const float* w, int32_t co, int32_t ldk, void* wb,
                                         void* wt, void* stream) {
  if (co < 0 || ldk < 0 || (co * ldk > 0 && (!w || (!wb && !wt))))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_cast_weights: arguments");
  const size_t total = (size_t)co * ldk;
  if (total == 0) return set_error(GS2D_OK, "");
  k_cast_weights<<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(
      w, co, ldk, static_cast<bf16*>(wb), static_cast<bf16*>(wt));
  return launched("gs2d_cast_weights");
}

// ---------------------------------------------------------------------------
// Head: the network's last layer gives, per cell of a gh x gw grid of cell_px
// pixel cells and per slot s of `slots`, nine numbers o0 .. o8 (columns
// 9 s ... 9 s + 8 of the cell's row) that decode into one Gaussian:
//   mu    = cell origin + anchor(s) + (cell_px / 2) tanh(o0, o1)
//           anchor(s) = cell_px ((s mod q + 1/2) / q, (s div q + 1/2) / r),
//           q = ceil(sqrt(slots)) columns, r = ceil(slots / q) rows
//   l1    = scale exp(clamp(o2, -4, 3)),  l2 = scale o3,  l3 = scale exp(clamp(o4, -4, 3))
//   c     = 0.5 + (o5, o6, o7),           w  = 0.25 + o8
// Each frame keeps the n slots with the largest |w| (ties: lower slot index),
// in slot order.

namespace {

constexpr float kExpLo = -4.0f, kExpHi = 3.0f;

__host__ __device__ inline int anchor_cols(int slots) {
  int q = 1;
  while (q * q < slots) q++;
  return q;
}

__device__ __forceinline__ void decode_slot(const float* __restrict__ o, int cell, int gw, int s,
                                            int slots, int cell_px, float scale, float g[9]) {
  const float half = 0.5f * (float)cell_px;
  const int cy = cell / gw, cx = cell % gw;
  const int q = anchor_cols(slots), r = (slots + q - 1) / q;
  const float ax = ((float)(s % q) + 0.5f) / (float)q, ay = ((float)(s / q) + 0.5f) / (float)r;
  g[0] = ((float)cx + ax) * (float)cell_px + half * tanhf(o[0]);
  g[1] = ((float)cy + ay) * (float)cell_px + half * tanhf(o[1]);
  g[2] = scale * expf(fminf(fmaxf(o[2], kExpLo), kExpHi));
  g[3] = scale * o[3];
  g[4] = scale * expf(fminf(fmaxf(o[4], kExpLo), kExpHi));
  g[5] = 0.5f + o[5];
  g[6] = 0.5f + o[6];
  g[7] = 0.5f + o[7];
  g[8] = 0.25f + o[8];
}

// Block-wide exclusive prefix of a 0/1 flag over the block's threads (in
// thread order) by ballots; returns the prefix and leaves the total in *tot.
__device__ __forceinline__ int block_flag_prefix(bool f, int* s_w, int* tot) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if (lane == 0) s_w[wid] = __popc(bal);
  __syncthreads();
  if (wid == 0) {
    const int c = lane < nw ? s_w[lane] : 0;
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane < nw) s_w[lane] = inc - c;
    if (lane == 31) s_w[32] = inc;
  }
  __syncthreads();
  const int pre = s_w[wid] + __popc(bal & ((1u << lane) - 1u));
  *tot = s_w[32];
  __syncthreads();  // s_w is reused by the next call
  return pre;
}

// Selection of the n largest |w| keys of a frame (ties: lowest slot first),
// in slot order, by a cluster of kSelCluster CTAs per frame: CTA k holds
// slots [k C, (k + 1) C); an MSB-first radix select, a byte per pass, sums
// the CTAs' histograms through distributed shared memory (every CTA reads all
// of them and takes the same decision); the compaction offsets each CTA by
// the counts of the CTAs before it.  Writes the selected slot of every output
// position to sel.
constexpr int kSelCluster = 8;

__global__ void __cluster_dims__(kSelCluster, 1, 1) __launch_bounds__(512)
k_head_select_cluster(const float* __restrict__ out, int ldo, int gh, int gw, int slots, int n,
                      int* __restrict__ sel) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ uint32_t s_key[];
  __shared__ int s_hist[2][256];   // this CTA's histogram, double-buffered over passes
  __shared__ int s_tot[256];       // the cluster's
  __shared__ int s_w[33];
  __shared__ int s_cnt[2];         // this CTA's keys above T, equal to T
  __shared__ uint32_t s_prefix;
  __shared__ int s_need;
  const int b = blockIdx.x / kSelCluster, rank = (int)cluster.block_rank();
  const int t = threadIdx.x, nt = blockDim.x;
  const int cells = gh * gw, S = cells * slots;
  const int C = (S + kSelCluster - 1) / kSelCluster;
  const int i0 = min(S, rank * C), i1 = min(S, i0 + C), len = i1 - i0;
  const float* ob = out + (size_t)b * cells * ldo;
  for (int i = t; i < len; i += nt) {
    const int g = i0 + i, cell = g / slots, sl = g % slots;
    s_key[i] = __float_as_uint(fabsf(0.25f + ob[(size_t)cell * ldo + 9 * sl + 8]));
  }
  if (t == 0) {
    s_prefix = 0;
    s_need = n;
  }
  __syncthreads();
  int buf = 0;
  for (int shift = 24; shift >= 0; shift -= 8, buf ^= 1) {
    for (int i = t; i < 256; i += nt) s_hist[buf][i] = 0;
    __syncthreads();
    const uint32_t hi_mask = shift == 24 ? 0u : (0xFFFFFFFFu << (shift + 8));
    const uint32_t prefix = s_prefix;
    for (int i = t; i < len; i += nt) {
      const uint32_t k = s_key[i];
      if ((k & hi_mask) == (prefix & hi_mask)) atomicAdd(&s_hist[buf][(k >> shift) & 255u], 1);
    }
    cluster.sync();  // every CTA's histogram of this pass is complete
    for (int i = t; i < 256; i += nt) {
      int c = 0;
      for (int r = 0; r < kSelCluster; r++) c += cluster.map_shared_rank(&s_hist[buf][0], r)[i];
      s_tot[i] = c;
    }
    __syncthreads();
    if (t < 32) {
      const int lane = t;
      int c[8], sum = 0;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        c[k] = s_tot[255 - (8 * lane + k)];
        sum += c[k];
      }
      int inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      const int need = s_need, exc = inc - sum;
      if (exc < need && need <= inc) {
        int acc = exc;
#pragma unroll
        for (int k = 0; k < 8; k++) {
          if (acc + c[k] >= need) {
            s_need = need - acc;
            s_prefix = prefix | ((uint32_t)(255 - (8 * lane + k)) << shift);
            break;
          }
          acc += c[k];
        }
      } else if (lane == 31 && need > inc) {
        s_need = need - (inc - c[7]);
        s_prefix = prefix;
      }
    }
    __syncthreads();
    // the other buffer is zeroed next pass; no CTA rereads it before then
  }
  const uint32_t T = s_prefix;
  const int need_eq = s_need;
  // this CTA's counts above and at T, then the offsets from the CTAs before it
  if (t == 0) s_cnt[0] = s_cnt[1] = 0;
  __syncthreads();
  int above = 0, at = 0;
  for (int i = t; i < len; i += nt) {
    above += s_key[i] > T;
    at += s_key[i] == T;
  }
  for (int o = 16; o; o >>= 1) {
    above += __shfl_xor_sync(0xffffffffu, above, o);
    at += __shfl_xor_sync(0xffffffffu, at, o);
  }
  if ((t & 31) == 0) {
    atomicAdd(&s_cnt[0], above);
    atomicAdd(&s_cnt[1], at);
  }
  cluster.sync();
  int eq_before = 0, taken_before = 0;
  {
    // keys of lower CTAs taken: all above T, and the first need_eq equal ones
    int eq_lower = 0, above_lower = 0;
    for (int r = 0; r < rank; r++) {
      const int* cr = cluster.map_shared_rank(&s_cnt[0], r);
      above_lower += cr[0];
      eq_lower += cr[1];
    }
    eq_before = eq_lower;
    taken_before = above_lower + min(eq_lower, need_eq);
  }
  cluster.sync();  // no CTA leaves while a peer may still read its counts
  for (int base = 0; base < len; base += nt) {
    const int i = base + t;
    const uint32_t k = i < len ? s_key[i] : 0u;
    const bool eq = i < len && k == T;
    int eq_total, take_total;
    const int eq_rank = eq_before + block_flag_prefix(eq, s_w, &eq_total);
    const bool take = i < len && (k > T || (eq && eq_rank < need_eq));
    const int j = taken_before + block_flag_prefix(take, s_w, &take_total);
    if (take && j < n) sel[(size_t)b * n + j] = i0 + i;
    taken_before += take_total;
    eq_before += eq_total;
  }
}

// Decoding of the selected slots into Gaussians, one thread per output.
__global__ void __launch_bounds__(256)
k_head_decode(const float* __restrict__ out, int ldo, int B, int gh, int gw, int slots,
              int cell_px, float scale, int n, float* __restrict__ params, int ldp,
              const int* __restrict__ sel) {
  const int cells = gh * gw;
  const size_t total = (size_t)B * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / n), j = (int)(t % n);
    const int i = sel[t];
    const int cell = i / slots, s = i % slots;
    float g[9];
    decode_slot(out + ((size_t)b * cells + cell) * ldo + 9 * s, cell, gw, s, slots, cell_px,
                scale, g);
    float* pb = params + (size_t)b * n;
#pragma unroll
    for (int r = 0; r < 9; r++) pb[(size_t)r * ldp + j] = g[r];
  }
}

// dout[row][9 s + r] = d(loss)/d(o_r) of selected slot (cell, s); dout was
// zeroed by the caller.
__global__ void k_head_decode_bwd(const float* __restrict__ out, int ldo, int B, int gh, int gw,
                                  int slots, int cell_px, float scale, int n,
                                  const int* __restrict__ sel, const float* __restrict__ dparams,
                                  int ldp, bf16* __restrict__ dout) {
  const int cells = gh * gw;
  const size_t total = (size_t)B * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / n), j = (int)(t % n);
    const int slot = sel[t];
    const int cell = slot / slots, s = slot % slots;
    const size_t row = (size_t)b * cells + cell;
    const float* o = out + row * ldo + 9 * s;
    const float* dp = dparams + (size_t)b * n;
    float d[9];
#pragma unroll
    for (int r = 0; r < 9; r++) d[r] = dp[(size_t)r * ldp + j];
    const float half = 0.5f * (float)cell_px;
    float g[9];
    const float t0 = tanhf(o[0]), t1 = tanhf(o[1]);
    g[0] = d[0] * half * (1.0f - t0 * t0);
    g[1] = d[1] * half * (1.0f - t1 * t1);
    g[2] = (o[2] >= kExpLo && o[2] <= kExpHi) ? d[2] * scale * expf(o[2]) : 0.0f;
    g[3] = d[3] * scale;
    g[4] = (o[4] >= kExpLo && o[4] <= kExpHi) ? d[4] * scale * expf(o[4]) : 0.0f;
    g[5] = d[5];
    g[6] = d[6];
    g[7] = d[7];
    g[8] = d[8];
    bf16* db = dout + row * ldo + 9 * s;
#pragma unroll
    for (int r = 0; r < 9; r++) db[r] = __float2bfloat16_rn(g[r]);
  }
}

// Nearest neighbour of every point of P among Q (per frame): points are rows
// 0, 1 of [9][count] parameter blocks.
__global__ void __launch_bounds__(256)
k_nearest(const float* __restrict__ P, int np, int ldp, const float* __restrict__ Q, int nq,
          int ldq, int* __restrict__ nn, float* __restrict__ dist) {
  __shared__ float2 s_q[1024];
  const int b = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float* pb = P + (size_t)b * np;
  const float* qb = Q + (size_t)b * nq;
  const float px = i < np ? pb[i] : 0.0f, py = i < np ? pb[ldp + i] : 0.0f;
  float best = INFINITY;
  int arg = 0;
  for (int j0 = 0; j0 < nq; j0 += 1024) {
    const int cnt = min(1024, nq - j0);
    __syncthreads();
    for (int k = threadIdx.x; k < cnt; k += blockDim.x)
      s_q[k] = make_float2(qb[j0 + k], qb[(size_t)ldq + j0 + k]);
    __syncthreads();
    for (int k = 0; k < cnt; k++) {
      const float dx = px - s_q[k].x, dy = py - s_q[k].y;
      const float d = fmaf(dx, dx, dy * dy);
      if (d < best) {
        best = d;
        arg = j0 + k;
      }
    }
  }
  if (i < np) {
    nn[(size_t)b * np + i] = arg;
    dist[(size_t)b * np + i] = best;
  }
}

// Gradient of the Chamfer term with respect to the predicted means: each
// predicted point towards its nearest target, each target pulling its
// nearest predicted point (accumulated with atomics).  Also the per-frame
// loss (a fixed-order sum).
__global__ void __launch_bounds__(256)
k_chamfer_grad(const float* __restrict__ P, int np, int ldp, const float* __restrict__ Q, int nq,
               int ldq, const int* __restrict__ nn1, const int* __restrict__ nn2, float lambda,
               float* __restrict__ dP) {
  const int b = blockIdx.y;
  const float* pb = P + (size_t)b * np;
  const float* qb = Q + (size_t)b * nq;
  float* db = dP + (size_t)b * np;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np) {
    const int j = nn1[(size_t)b * np + i];
    atomicAdd(&db[i], lambda * 2.0f * (pb[i] - qb[j]) / (float)np);
    atomicAdd(&db[ldp + i], lambda * 2.0f * (pb[ldp + i] - qb[ldq + j]) / (float)np);
  }
  if (i < nq) {
    const int k = nn2[(size_t)b * nq + i];
    atomicAdd(&db[k], lambda * 2.0f * (pb[k] - qb[i]) / (float)nq);
    atomicAdd(&db[ldp + k], lambda * 2.0f * (pb[ldp + k] - qb[ldq + i]) / (float)nq);
  }
}

__global__ void __launch_bounds__(1024)
k_chamfer_loss(const float* __restrict__ d1, int np, const float* __restrict__ d2, int nq,
               float* __restrict__ loss) {
  __shared__ double s[32];
  const int b = blockIdx.x;
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) a += d1[(size_t)b * np + i];
  for (int i = threadIdx.x; i < nq; i += blockDim.x) c += d2[(size_t)b * nq + i];
  double v = a / np + c / nq;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += s[w];
    loss[b] = (float)tot;
  }
}

}  // namespace

extern "C" uint64_t gs2d_head_smem_bytes(int32_t gh, int32_t gw, int32_t slots) {
  return (uint64_t)gh * gw * slots * sizeof(uint32_t);
}

extern "C" gs2d_status gs2d_head_decode(const float* out, int32_t ldo, int32_t B, int32_t gh,
                                        int32_t gw, int32_t slots, int32_t cell_px, float scale,
                                        int32_t n, float* params, int32_t ldp, int32_t* sel,
                                        void* stream) {
  const uint64_t smem = gs2d_head_smem_bytes(gh, gw, slots);
  if (B < 0 || gh < 1 || gw < 1 || slots < 1 || ldo < 9 * slots || cell_px < 1 || n < 0 ||
      (int64_t)ldp < (int64_t)B * n ||
      (int64_t)n > (int64_t)gh * gw * slots || smem > 200 * 1024 ||
      (B > 0 && (!out || !params || !sel)))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_head_decode: arguments");
  if (B == 0 || n == 0) return set_error(GS2D_OK, "");
  cudaStream_t s = (cudaStream_t)stream;
  k_head_select_cluster<<<B * kSelCluster, 512,
                          (size_t)((gh * gw * slots + kSelCluster - 1) / kSelCluster) * 4, s>>>(
      out, ldo, gh, gw, slots, n, sel);
  const size_t total = (size_t)B * n;
  const size_t want = (total + 255) / 256;
  k_head_decode<<<(int)(want < 152 * 8 ? want : 152 * 8), 256, 0, s>>>(
      out, ldo, B, gh, gw, slots, cell_px, scale, n, params, ldp, sel);
  return launched("gs2d_head_decode");
}

extern "C" gs2d_status gs2d_head_decode_bwd(const float* out, int32_t ldo, int32_t B, int32_t gh,
                                            int32_t gw, int32_t slots, int32_t cell_px,
                                            float scale, int32_t n, const int32_t* sel,
                                            const float* dparams, int32_t ldp, void* dout,
                                            void* stream) {
  if (B < 0 || gh < 1 || gw < 1 || slots < 1 || ldo < 9 * slots || n < 0 ||
      (int64_t)ldp < (int64_t)B * n ||
      (B > 0 && (!out || !sel || !dparams || !dout)))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_head_decode_bwd: arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t rows = (size_t)B * gh * gw;
  if (cudaMemsetAsync(dout, 0, rows * ldo * sizeof(bf16), s) != cudaSuccess)
    return launched("gs2d_head_decode_bwd");
  const size_t total = (size_t)B * n;
  if (total == 0) return set_error(GS2D_OK, "");
  k_head_decode_bwd<<<grid_for(total, 256), 256, 0, s>>>(out, ldo, B, gh, gw, slots, cell_px,
                                                         scale, n, sel, dparams, ldp,
                                                         static_cast<bf16*>(dout));
  return launched("gs2d_head_decode_bwd");
}

extern "C" uint64_t gs2d_chamfer_scratch_bytes(int32_t n, int32_t m, int32_t B) {
  return (uint64_t)B * ((uint64_t)n + m) * (sizeof(int) + sizeof(float)) + 64;
}

extern "C" gs2d_status gs2d_chamfer(const float* params, int32_t n, int32_t ldp,
                                    const float* targets, int32_t m, int32_t ldq, int32_t B,
                                    float lambda, float* dparams, float* loss, void* scratch,
                                    void* stream) {
  if (n < 1 || m < 1 || B < 1 || !params || !targets || !scratch ||
      (int64_t)ldp < (int64_t)B * n || (int64_t)ldq < (int64_t)B * m)
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_chamfer: arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int* nn1 = static_cast<int*>(scratch);
  int* nn2 = nn1 + (size_t)B * n;
  float* d1 = reinterpret_cast<float*>(nn2 + (size_t)B * m);
  float* d2 = d1 + (size_t)B * n;
  k_nearest<<<dim3((n + 255) / 256, B), 256, 0, s>>>(params, n, ldp, targets, m, ldq, nn1, d1);
  k_nearest<<<dim3((m + 255) / 256, B), 256, 0, s>>>(targets, m, ldq, params, n, ldp, nn2, d2);
  if (dparams)
    k_chamfer_grad<<<dim3((std::max(n, m) + 255) / 256, B), 256, 0, s>>>(
        params, n, ldp, targets, m, ldq, nn1, nn2, lambda, dparams);
  if (loss) k_chamfer_loss<<<B, 1024, 0, s>>>(d1, n, d2, m, loss);
  return launched("gs2d_chamfer");
}
