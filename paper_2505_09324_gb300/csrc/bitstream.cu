// Bitstream accounting of a coded sequence (Sec. 3.3 B, Eq. 3-4): the ideal
// order-0 code length of quantised Gaussians (per-row histograms and their
// entropy, on the device) and the bits-back totals of a sequence (host).
#include <math.h>

#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr int kBins = 1 << 16;  // per row: every 16-bit symbol
constexpr int kEntropyThreads = 1024;

struct RowBits {
  int bits[9];
};

__device__ __forceinline__ int symbol_bits(int b) { return b < 0 ? 16 : b; }

// Histogram of the (selected) codes of every row that is coded (bits != 0);
// codes are masked to the row's width, so any input stays in bounds.  The
// last scratch word counts the selected columns.
__global__ void __launch_bounds__(256)
k_code_hist(const uint16_t* __restrict__ codes, int n, RowBits rb,
            const uint8_t* __restrict__ select, uint32_t* __restrict__ hist) {
  const size_t total = (size_t)9 * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / n);
    const int i = (int)(t - (size_t)r * n);
    if (select && !select[i]) continue;
    if (r == 0) atomicAdd(&hist[(size_t)9 * kBins], 1u);
    const int b = rb.bits[r];
    if (b == 0) continue;
    const uint32_t mask = (1u << symbol_bits(b)) - 1u;
    atomicAdd(&hist[(size_t)r * kBins + (codes[t] & mask)], 1u);
  }
}

// Block r: code length of row r = T log2 T - sum_s c_s log2 c_s, summed in a
// fixed order (per-thread strided sums, then a fixed reduction tree), so the
// result is reproducible.
__global__ void __launch_bounds__(kEntropyThreads)
k_code_entropy(const uint32_t* __restrict__ hist, RowBits rb, double* __restrict__ out) {
  __shared__ double s_acc[kEntropyThreads / 32];
  const int r = blockIdx.x;
  const int b = rb.bits[r];
  const double total = (double)hist[(size_t)9 * kBins];
  if (b == 0) {
    if (threadIdx.x == 0) out[r] = 32.0 * total;
    return;
  }
  const int nb = 1 << symbol_bits(b);
  double acc = 0.0;
  for (int j = threadIdx.x; j < nb; j += kEntropyThreads) {
    const uint32_t c = hist[(size_t)r * kBins + j];
    if (c > 1) acc += (double)c * log2((double)c);
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_acc[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < kEntropyThreads / 32; w++) sum += s_acc[w];
    out[r] = total > 1.0 ? total * log2(total) - sum : 0.0;
  }
}

}  // namespace
}  // namespace gs2d

using namespace gs2d;

extern "C" size_t gs2d_code_entropy_scratch_bytes(void) {
  return ((size_t)9 * kBins + 1) * sizeof(uint32_t);
}

extern "C" gs2d_status gs2d_code_entropy(const uint16_t* codes, int32_t n, const int32_t* bits,
                                         const uint8_t* select, void* scratch,
                                         size_t scratch_bytes, double* out_bits,
                                         void* stream) {
  if (n < 0 || !bits || !out_bits || !scratch ||
      scratch_bytes < gs2d_code_entropy_scratch_bytes() || (n > 0 && !codes))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_code_entropy: arguments");
  RowBits rb;
  for (int r = 0; r < 9; r++) {
    const int b = bits[r];
    if (!(b == -16 || (b >= 0 && b <= 16)))
      return set_error(GS2D_ERR_INVALID_ARG, "gs2d_code_entropy: bits");
    rb.bits[r] = b;
  }
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* hist = (uint32_t*)scratch;
  cudaError_t e = cudaMemsetAsync(hist, 0, gs2d_code_entropy_scratch_bytes(), s);
  if (e == cudaSuccess && n > 0) {
    const size_t want = ((size_t)9 * n + 255) / 256;
    const int blocks = (int)(want < 152 * 8 ? want : 152 * 8);
    k_code_hist<<<blocks, 256, 0, s>>>(codes, n, rb, select, hist);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_code_entropy<<<9, kEntropyThreads, 0, s>>>(hist, rb, out_bits);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return set_error(GS2D_ERR_CUDA, cudaGetErrorString(e));
  return set_error(GS2D_OK, "");
}

// Eq. 3: log2(m!) - log2(m), through lgamma (0 for m <= 1).
static double bitsback_saving(int32_t m) {
  if (m <= 1) return 0.0;
  return (lgamma((double)m + 1.0) - log((double)m)) / log(2.0);
}

extern "C" gs2d_status gs2d_sequence_bits(const int32_t* counts, const double* payload_bits,
                                          int32_t frames, int32_t gop, gs2d_seq_bits* out) {
  if (frames < 0 || gop < 1 || !out || (frames > 0 && (!counts || !payload_bits)))
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_sequence_bits: arguments");
  gs2d_seq_bits r = {0.0, 0.0, 0.0, 0.0, 0, 0};
  for (int32_t k = 0; k < frames; k++) {
    if (counts[k] < 0 || !isfinite(payload_bits[k]) || payload_bits[k] < 0.0)
      return set_error(GS2D_ERR_INVALID_ARG, "gs2d_sequence_bits: frame entry");
    if (k % gop == 0) {
      r.i_bits += payload_bits[k];
      r.i_frames++;
    } else {
      r.p_bits += payload_bits[k];
      r.savings += bitsback_saving(counts[k]);
      r.p_frames++;
    }
  }
  r.total_bits = r.i_bits + r.p_bits - r.savings;
  *out = r;
  return set_error(GS2D_OK, "");
}

// ---------------------------------------------------------------------------
// Coded size of one frame (Sec. 3.3 B): the rows' ideal code lengths, plus
// for a P-frame the index of every selected Gaussian (ceil(log2 n) bits),
// plus the per-frame ranges of a quantiser that refines them per frame
// (two float32 per uniform row).
namespace gs2d {
namespace {

__global__ void k_frame_bits(const double* __restrict__ rows, const uint32_t* __restrict__ hist,
                             int index_bits, int range_bits, double* __restrict__ out) {
  double t = 0.0;
  for (int r = 0; r < 9; r++) t += rows[r];
  const double m = (double)hist[(size_t)9 * kBins];  // selected columns
  out[0] = t + m * (double)index_bits + (double)range_bits;
}

}  // namespace
}  // namespace gs2d

extern "C" size_t gs2d_frame_bits_scratch_bytes(void) {
  return gs2d_code_entropy_scratch_bytes() + 16 * sizeof(double);
}

extern "C" gs2d_status gs2d_frame_bits(const uint16_t* codes, int32_t n, const int32_t* bits,
                                       const uint8_t* select, int32_t refine, void* scratch,
                                       size_t scratch_bytes, double* out_bits, void* stream) {
  if (!scratch || scratch_bytes < gs2d_frame_bits_scratch_bytes() || !out_bits || !bits)
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_frame_bits: arguments");
  const size_t eb = gs2d_code_entropy_scratch_bytes();
  double* rows = reinterpret_cast<double*>(static_cast<char*>(scratch) +
                                           ((eb + 15) & ~size_t(15)));
  gs2d_status st = gs2d_code_entropy(codes, n, bits, select, scratch, eb, rows, stream);
  if (st != GS2D_OK) return st;
  int index_bits = 0;
  if (select) {
    int64_t span = 1;
    while (span < (int64_t)(n > 2 ? n : 2)) {
      span <<= 1;
      index_bits++;
    }
  }
  int uniform = 0;
  for (int r = 0; r < 9; r++) uniform += bits[r] > 0;
  const int range_bits = refine ? 64 * uniform : 0;
  k_frame_bits<<<1, 1, 0, (cudaStream_t)stream>>>(
      rows, static_cast<const uint32_t*>(scratch), index_bits, range_bits, out_bits);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GS2D_ERR_CUDA, cudaGetErrorString(e));
  return set_error(GS2D_OK, "");
}
