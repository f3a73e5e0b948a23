// Region-of-interest superpixel initialiser (Sec. 3.2 A): K-means superpixels
// of the ROI mask, one Gaussian per segment (mean = segment centre, Cholesky
// factor of the segment covariance, colour = mean segment colour), plus
// isotropic Gaussians for the rest of the frame at caller-supplied positions.
//
// Readings (the paper leaves them open): seeds on a grid of step
// S = sqrt(A_roi / K) at ((i + 1/2) S, (j + 1/2) S) inside the mask; 10
// iterations of assignment (D = |col_p - col_c|^2 + (m/S)^2 |p - c|^2, m = 0.2,
// among centres within S of the pixel on both axes; ties to the lower index)
// and update (mean colour and position, clamped to within S of the seed, so the
// candidates of a pixel are the seeds of the 5 x 5 grid cells around it);
// Sigma = 4 (pixel-centre covariance + I/12) (the segment's second moment of
// area, widened so that the accumulated sum over a tiling of segments is flat),
// weight = A / (2 pi sqrt(det Sigma)) (the Gaussian's integral equals the area);
// background Gaussians: variance 4 a / (2 pi), weight 1/4 (integral a).
// Arithmetic: the assignment decides in single precision (explicitly rounded
// FP32 operations, centres kept as float); every segment sum is an exact
// integer (pixel centres as 2 x + 1 - 2 floor(seed), colours as
// rint(c 2^20)), accumulated by warp-aggregated 64-bit atomics in any order;
// means and covariances follow in a fixed sequence of double operations, so
// the result is reproducible bit for bit.
#include <math.h>
#include <stdio.h>

#include <vector>

#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr double kCompactness = 0.2;
constexpr int kIterations = 10;
constexpr double kKappa = 4.0;  // covariance scale: keeps the blend of a tiling flat
constexpr double kColourScale = 1048576.0;  // 2^20
constexpr double kColourLimit = 32.0;
constexpr int kSums = 9;  // n, u, v, uu, uv, vv, r, g, b

struct SpArgs {
  int W, H, M, gx, gy;
  double S;
  float S32, lam32;
  const float* frame;
  const uint8_t* mask;
  const int* cell_of;          // [gy][gx] seed index or -1
  const double* seed_xy;       // [2][M]
  float* cen;                  // [5][M]: r, g, b, x, y
  int* label;                  // [H][W]
  unsigned long long* acc;     // [kSums][M] exact segment sums (two's complement)
};

// Assignment + segment sums: each ROI pixel joins the nearest candidate
// centre (FP32 decisions), then adds its integer moments to the centre's sums
// (one 64-bit atomic per sum and group of lanes with the same centre).
__global__ void __launch_bounds__(256) k_sp_assign(SpArgs a) {
  pdl_begin();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.W * a.H) return;
  const int x = idx % a.W, y = idx / a.W;
  if (!a.mask[idx]) {
    a.label[idx] = -1;
    return;
  }
  const size_t HW = (size_t)a.W * a.H;
  const float pr = a.frame[idx], pg = a.frame[HW + idx], pb = a.frame[2 * HW + idx];
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const int pcx = (int)floor((double)px / a.S), pcy = (int)floor((double)py / a.S);
  // candidates of the 5 x 5 cells, visited in ascending centre index
  int cand[25];
  int nc = 0;
  for (int dj = -2; dj <= 2; dj++)
    for (int di = -2; di <= 2; di++) {
      const int cx = pcx + di, cy = pcy + dj;
      if (cx < 0 || cx >= a.gx || cy < 0 || cy >= a.gy) continue;
      const int c = a.cell_of[cy * a.gx + cx];
      if (c < 0) continue;
      int k = nc++;
      while (k > 0 && cand[k - 1] > c) {  // insertion sort (25 at most)
        cand[k] = cand[k - 1];
        k--;
      }
      cand[k] = c;
    }
  const int M = a.M;
  float best = INFINITY;
  int lab = -1;
  for (int k = 0; k < nc; k++) {
    const int c = cand[k];
    const float dx = __fsub_rn(px, a.cen[3 * M + c]);
    const float dy = __fsub_rn(py, a.cen[4 * M + c]);
    if (!(fabsf(dx) <= a.S32 && fabsf(dy) <= a.S32)) continue;
    const float dr = __fsub_rn(pr, a.cen[c]), dg = __fsub_rn(pg, a.cen[M + c]),
                db = __fsub_rn(pb, a.cen[2 * M + c]);
    const float dc = __fadd_rn(__fadd_rn(__fmul_rn(dr, dr), __fmul_rn(dg, dg)), __fmul_rn(db, db));
    const float d =
        __fadd_rn(dc, __fmul_rn(a.lam32, __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy))));
    if (d < best) {
      best = d;
      lab = c;
    }
  }
  a.label[idx] = lab;
  // exact moments: |u|, |v| <= 4 S + 2 and |q| <= 2^25, so a group sum of up
  // to 32 lanes stays within int32 for S < 2000
  int val[kSums] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (lab >= 0) {
    const int u = 2 * x + 1 - 2 * (int)floor(a.seed_xy[lab]);
    const int v = 2 * y + 1 - 2 * (int)floor(a.seed_xy[M + lab]);
    val[0] = 1;
    val[1] = u;
    val[2] = v;
    val[3] = u * u;
    val[4] = u * v;
    val[5] = v * v;
    const float col[3] = {pr, pg, pb};
#pragma unroll
    for (int ch = 0; ch < 3; ch++)
      val[6 + ch] = (int)__double2ll_rn(
          fmin(fmax((double)col[ch], -kColourLimit), kColourLimit) * kColourScale);
  }
  const unsigned peers = __match_any_sync(__activemask(), lab);
  const int leader = __ffs(peers) - 1;
#pragma unroll
  for (int k = 0; k < kSums; k++) val[k] = __reduce_add_sync(peers, val[k]);
  if (lab >= 0 && (int)(threadIdx.x & 31) == leader)
#pragma unroll
    for (int k = 0; k < kSums; k++)
      atomicAdd(&a.acc[(size_t)k * M + lab], (unsigned long long)(long long)val[k]);
}

__device__ __forceinline__ long long acc_get(const SpArgs& a, int k, int c) {
  return (long long)a.acc[(size_t)k * a.M + c];
}

// Update: each centre moves to its segment's mean (clamped to within S of the
// seed) and mean colour; the sums are cleared for the next assignment.
__global__ void __launch_bounds__(128) k_sp_update(SpArgs a) {
  pdl_begin();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.M) return;
  const int M = a.M;
  const long long n = acc_get(a, 0, c);
  if (n > 0) {
    const double qx = a.seed_xy[c], qy = a.seed_xy[M + c];
    const double mx = __dadd_rn(__ddiv_rn((double)acc_get(a, 1, c), (double)(2 * n)), floor(qx));
    const double my = __dadd_rn(__ddiv_rn((double)acc_get(a, 2, c), (double)(2 * n)), floor(qy));
    a.cen[3 * M + c] = (float)fmin(fmax(mx, __dsub_rn(qx, a.S)), __dadd_rn(qx, a.S));
    a.cen[4 * M + c] = (float)fmin(fmax(my, __dsub_rn(qy, a.S)), __dadd_rn(qy, a.S));
    const double den = __dmul_rn((double)n, kColourScale);
#pragma unroll
    for (int ch = 0; ch < 3; ch++)
      a.cen[ch * M + c] = (float)__ddiv_rn((double)acc_get(a, 6 + ch, c), den);
  }
#pragma unroll
  for (int k = 0; k < kSums; k++) a.acc[(size_t)k * M + c] = 0ull;
}

__global__ void __launch_bounds__(128) k_sp_init_centres(SpArgs a) {
  pdl_begin();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.M) return;
  const int M = a.M;
  const double sx = a.seed_xy[c], sy = a.seed_xy[M + c];
  const int xi = min(max((int)floor(sx), 0), a.W - 1), yi = min(max((int)floor(sy), 0), a.H - 1);
  const size_t HW = (size_t)a.W * a.H, idx = (size_t)yi * a.W + xi;
  a.cen[c] = a.frame[idx];
  a.cen[M + c] = a.frame[HW + idx];
  a.cen[2 * M + c] = a.frame[2 * HW + idx];
  a.cen[3 * M + c] = (float)sx;
  a.cen[4 * M + c] = (float)sy;
#pragma unroll
  for (int k = 0; k < kSums; k++) a.acc[(size_t)k * M + c] = 0ull;
}

// Final segments -> Gaussians, from the exact sums of the last assignment.
__global__ void __launch_bounds__(128) k_sp_gaussians(SpArgs a, int n_total,
                                                      float* __restrict__ params) {
  pdl_begin();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.M) return;
  const size_t HW = (size_t)a.W * a.H;
  const long long cnt = acc_get(a, 0, c);
  const double qx = a.seed_xy[c], qy = a.seed_xy[a.M + c];
  const int n = n_total;
  float out[9];
  if (cnt == 0) {
    const int xi = min(max((int)floor(qx), 0), a.W - 1), yi = min(max((int)floor(qy), 0), a.H - 1);
    const size_t idx = (size_t)yi * a.W + xi;
    const double s = __dmul_rn(2.0, __ddiv_rn(a.S, sqrt(12.0)));
    out[0] = (float)qx;
    out[1] = (float)qy;
    out[2] = (float)s;
    out[3] = 0.0f;
    out[4] = (float)s;
    out[5] = a.frame[idx];
    out[6] = a.frame[HW + idx];
    out[7] = a.frame[2 * HW + idx];
    out[8] = 1.0f;
  } else {
    const double fn = (double)cnt;
    const double au = __ddiv_rn((double)acc_get(a, 1, c), fn);
    const double av = __ddiv_rn((double)acc_get(a, 2, c), fn);
    const double cxx = __ddiv_rn(__dsub_rn(__ddiv_rn((double)acc_get(a, 3, c), fn), __dmul_rn(au, au)), 4.0);
    const double cxy = __ddiv_rn(__dsub_rn(__ddiv_rn((double)acc_get(a, 4, c), fn), __dmul_rn(au, av)), 4.0);
    const double cyy = __ddiv_rn(__dsub_rn(__ddiv_rn((double)acc_get(a, 5, c), fn), __dmul_rn(av, av)), 4.0);
    const double twelfth = __ddiv_rn(1.0, 12.0);
    const double vxx = __dadd_rn(cxx, twelfth);
    const double vyy = __dadd_rn(cyy, twelfth);
    const double c1 = __dsqrt_rn(vxx);
    const double c2 = __ddiv_rn(cxy, c1);
    const double c3 = __dsqrt_rn(__dsub_rn(vyy, __dmul_rn(c2, c2)));
    // Sigma = kappa (cov + I/12), kappa = 4: the factor 2 on L is exact
    const double l1 = 2.0 * c1, l2 = 2.0 * c2, l3 = 2.0 * c3;
    const double two_pi = 6.283185307179586;  // 2.0 * math.pi in double
    out[0] = (float)__dadd_rn(__ddiv_rn((double)acc_get(a, 1, c), (double)(2 * cnt)), floor(qx));
    out[1] = (float)__dadd_rn(__ddiv_rn((double)acc_get(a, 2, c), (double)(2 * cnt)), floor(qy));
    out[2] = (float)l1;
    out[3] = (float)l2;
    out[4] = (float)l3;
    const double den = __dmul_rn(fn, kColourScale);
#pragma unroll
    for (int ch = 0; ch < 3; ch++) out[5 + ch] = (float)__ddiv_rn((double)acc_get(a, 6 + ch, c), den);
    out[8] = (float)__ddiv_rn(fn, __dmul_rn(__dmul_rn(two_pi, l1), l3));
  }
#pragma unroll
  for (int r = 0; r < 9; r++) params[(size_t)r * n + c] = out[r];
}

// Isotropic background Gaussians at bg_xy[0 .. nbg).
__global__ void __launch_bounds__(256) k_sp_background(int W, int H, int M, int nbg, int n,
                                                       double s, const float* __restrict__ frame,
                                                       const float* __restrict__ bg_xy,
                                                       float* __restrict__ params) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nbg) return;
  const double x = bg_xy[k], y = bg_xy[n + k];
  const int xi = min(max((int)floor(x), 0), W - 1), yi = min(max((int)floor(y), 0), H - 1);
  const size_t HW = (size_t)W * H, idx = (size_t)yi * W + xi;
  const int c = M + k;
  params[c] = (float)x;
  params[n + c] = (float)y;
  params[2 * n + c] = (float)s;
  params[3 * n + c] = 0.0f;
  params[4 * n + c] = (float)s;
  params[5 * n + c] = frame[idx];
  params[6 * n + c] = frame[HW + idx];
  params[7 * n + c] = frame[2 * HW + idx];
  params[8 * n + c] = (float)(1.0 / kKappa);
}

uint64_t a256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

}  // namespace

// Scratch layout for a W x H frame with n Gaussians: labels int[H W], centres
// float[5][n], seeds double[2][n], cell map int[(W+1) (H+1)] (the grid has at
// most one cell per pixel), segment sums int64[9][n].
uint64_t roi_init_scratch_bytes(int W, int H, int n) {
  const uint64_t hw = (uint64_t)W * H;
  return a256(hw * 4) + a256(5ull * n * 4) + a256(2ull * n * 8) +
         a256((uint64_t)(W + 1) * (H + 1) * 4) + a256((uint64_t)kSums * n * 8) + 256;
}

gs2d_status roi_init(const float* frame, const uint8_t* mask, int W, int H, int n, float roi_frac,
                     const float* bg_xy, float* params, int32_t* n_roi, void* scratch,
                     uint64_t scratch_bytes, cudaStream_t s, char* err, size_t err_len) {
  if (scratch_bytes < roi_init_scratch_bytes(W, H, n)) {
    snprintf(err, err_len, "gs2d_roi_init: scratch too small");
    return GS2D_ERR_INVALID_ARG;
  }
  const uint64_t hw = (uint64_t)W * H;
  char* base = static_cast<char*>(scratch);
  int* label = reinterpret_cast<int*>(base);
  float* cen = reinterpret_cast<float*>(base + a256(hw * 4));
  double* seed_xy = reinterpret_cast<double*>(base + a256(hw * 4) + a256(5ull * n * 4));
  int* cell_of =
      reinterpret_cast<int*>(base + a256(hw * 4) + a256(5ull * n * 4) + a256(2ull * n * 8));
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(
      base + a256(hw * 4) + a256(5ull * n * 4) + a256(2ull * n * 8) +
      a256((uint64_t)(W + 1) * (H + 1) * 4));
  // seeds on the host (the mask comes back once)
  std::vector<uint8_t> hmask(hw);
  cudaError_t e = cudaMemcpyAsync(hmask.data(), mask, hw, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(err, err_len, "gs2d_roi_init: %s", cudaGetErrorString(e));
    return GS2D_ERR_CUDA;
  }
  uint64_t area = 0;
  for (uint64_t i = 0; i < hw; i++) area += hmask[i] != 0;
  const int k_target = (int)llround((double)roi_frac * n);
  int M = 0, gx = 1, gy = 1;
  double S = 1.0;
  std::vector<double> sx, sy;
  std::vector<int> cells;
  if (area > 0 && k_target > 0) {
    S = sqrt((double)area / (double)k_target);
    gx = (int)ceil((double)W / S);
    gy = (int)ceil((double)H / S);
    cells.assign((size_t)gx * gy, -1);
    for (int j = 0; j < gy; j++)
      for (int i = 0; i < gx; i++) {
        const double x = (i + 0.5) * S, y = (j + 0.5) * S;
        const int xi = (int)floor(x), yi = (int)floor(y);
        if (xi < W && yi < H && hmask[(size_t)yi * W + xi] && M < n) {
          cells[(size_t)j * gx + i] = M++;
          sx.push_back(x);
          sy.push_back(y);
        }
      }
  }
  if (n_roi) *n_roi = M;
  std::vector<double> sxy(sx);
  sxy.insert(sxy.end(), sy.begin(), sy.end());
  SpArgs a;
  a.W = W;
  a.H = H;
  a.M = M;
  a.gx = gx;
  a.gy = gy;
  a.S = S;
  a.S32 = (float)S;
  a.lam32 = (float)((kCompactness / S) * (kCompactness / S));
  a.frame = frame;
  a.mask = mask;
  a.cell_of = cell_of;
  a.seed_xy = seed_xy;
  a.cen = cen;
  a.label = label;
  a.acc = acc;
  if (M > 0) {
    e = cudaMemcpyAsync(seed_xy, sxy.data(), sxy.size() * sizeof(double),
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cell_of, cells.data(), cells.size() * sizeof(int),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      const int pb = (int)((hw + 255) / 256), cb = (M + 127) / 128;
      e = launch_pdl(k_sp_init_centres, cb, 128, 0, s, a);
      // the last assignment's sums make the Gaussians
      for (int it = 0; it < kIterations && e == cudaSuccess; it++) {
        e = launch_pdl(k_sp_assign, pb, 256, 0, s, a);
        if (e == cudaSuccess && it + 1 < kIterations)
          e = launch_pdl(k_sp_update, cb, 128, 0, s, a);
      }
      if (e == cudaSuccess) e = launch_pdl(k_sp_gaussians, cb, 128, 0, s, a, n, params);
    }
  }
  const int nbg = n - M;
  if (e == cudaSuccess && nbg > 0) {
    const double abg = (double)(hw - area) / (double)nbg;
    const double sd = sqrt(kKappa * (abg > 1.0 ? abg : 1.0) / (2.0 * 3.141592653589793));
    k_sp_background<<<(nbg + 255) / 256, 256, 0, s>>>(W, H, M, nbg, n, sd, frame, bg_xy, params);
    e = cudaGetLastError();
  }
  // the host vectors above are read by the copies: wait for them
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(err, err_len, "gs2d_roi_init: %s", cudaGetErrorString(e));
    return GS2D_ERR_CUDA;
  }
  return GS2D_OK;
}

}  // namespace gs2d
