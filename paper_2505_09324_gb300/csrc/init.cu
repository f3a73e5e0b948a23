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
// All clustering arithmetic is double precision with explicitly rounded
// operations and raster-order sums, so the result is reproducible bit for bit.
#include <math.h>
#include <stdio.h>

#include <vector>

#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr double kCompactness = 0.2;
constexpr int kIterations = 10;
constexpr double kKappa = 4.0;  // covariance scale: keeps the blend of a tiling flat

struct SpArgs {
  int W, H, M, gx, gy;
  double S, lam;
  const float* frame;
  const uint8_t* mask;
  const int* cell_of;     // [gy][gx] seed index or -1
  const double* seed_xy;  // [2][M]
  double* cen;            // [5][M]: r, g, b, x, y
  int* label;             // [H][W]
};

__device__ __forceinline__ double sq(double a) { return __dmul_rn(a, a); }

// Assignment: each ROI pixel joins the nearest candidate centre.
__global__ void __launch_bounds__(256) k_sp_assign(SpArgs a) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.W * a.H) return;
  const int x = idx % a.W, y = idx / a.W;
  if (!a.mask[idx]) {
    a.label[idx] = -1;
    return;
  }
  const size_t HW = (size_t)a.W * a.H;
  const double pr = a.frame[idx], pg = a.frame[HW + idx], pb = a.frame[2 * HW + idx];
  const double px = (double)x + 0.5, py = (double)y + 0.5;
  const int pcx = (int)floor(px / a.S), pcy = (int)floor(py / a.S);
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
  double best = INFINITY;
  int lab = -1;
  for (int k = 0; k < nc; k++) {
    const int c = cand[k];
    const double dx = __dsub_rn(px, a.cen[3 * M + c]);
    const double dy = __dsub_rn(py, a.cen[4 * M + c]);
    if (!(fabs(dx) <= a.S && fabs(dy) <= a.S)) continue;
    const double dc = __dadd_rn(__dadd_rn(sq(__dsub_rn(pr, a.cen[c])),
                                          sq(__dsub_rn(pg, a.cen[M + c]))),
                                sq(__dsub_rn(pb, a.cen[2 * M + c])));
    const double d = __dadd_rn(dc, __dmul_rn(a.lam, __dadd_rn(sq(dx), sq(dy))));
    if (d < best) {
      best = d;
      lab = c;
    }
  }
  a.label[idx] = lab;
}

// Window [seed - 2S, seed + 2S] of pixel indices that may belong to centre c.
__device__ __forceinline__ void sp_window(const SpArgs& a, int c, int* x0, int* x1, int* y0,
                                          int* y1) {
  const double sx = a.seed_xy[c], sy = a.seed_xy[a.M + c];
  *x0 = max(0, (int)floor(sx - 2.0 * a.S) - 1);
  *x1 = min(a.W - 1, (int)ceil(sx + 2.0 * a.S) + 1);
  *y0 = max(0, (int)floor(sy - 2.0 * a.S) - 1);
  *y1 = min(a.H - 1, (int)ceil(sy + 2.0 * a.S) + 1);
}

// Update: one thread per centre sums its pixels in raster order.
__global__ void __launch_bounds__(128) k_sp_update(SpArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.M) return;
  int x0, x1, y0, y1;
  sp_window(a, c, &x0, &x1, &y0, &y1);
  const size_t HW = (size_t)a.W * a.H;
  double n = 0, sx = 0, sy = 0, sr = 0, sg = 0, sb = 0;
  for (int y = y0; y <= y1; y++)
    for (int x = x0; x <= x1; x++) {
      const int idx = y * a.W + x;
      if (a.label[idx] != c) continue;
      n = __dadd_rn(n, 1.0);
      sx = __dadd_rn(sx, (double)x + 0.5);
      sy = __dadd_rn(sy, (double)y + 0.5);
      sr = __dadd_rn(sr, (double)a.frame[idx]);
      sg = __dadd_rn(sg, (double)a.frame[HW + idx]);
      sb = __dadd_rn(sb, (double)a.frame[2 * HW + idx]);
    }
  if (n > 0) {
    const int M = a.M;
    const double qx = a.seed_xy[c], qy = a.seed_xy[M + c];
    a.cen[c] = __ddiv_rn(sr, n);
    a.cen[M + c] = __ddiv_rn(sg, n);
    a.cen[2 * M + c] = __ddiv_rn(sb, n);
    a.cen[3 * M + c] = fmin(fmax(__ddiv_rn(sx, n), __dsub_rn(qx, a.S)), __dadd_rn(qx, a.S));
    a.cen[4 * M + c] = fmin(fmax(__ddiv_rn(sy, n), __dsub_rn(qy, a.S)), __dadd_rn(qy, a.S));
  }
}

__global__ void __launch_bounds__(128) k_sp_init_centres(SpArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.M) return;
  const int M = a.M;
  const double sx = a.seed_xy[c], sy = a.seed_xy[M + c];
  const int xi = min(max((int)floor(sx), 0), a.W - 1), yi = min(max((int)floor(sy), 0), a.H - 1);
  const size_t HW = (size_t)a.W * a.H, idx = (size_t)yi * a.W + xi;
  a.cen[c] = a.frame[idx];
  a.cen[M + c] = a.frame[HW + idx];
  a.cen[2 * M + c] = a.frame[2 * HW + idx];
  a.cen[3 * M + c] = sx;
  a.cen[4 * M + c] = sy;
}

// Final segments -> Gaussians (two raster-order passes: sums, centred moments).
__global__ void __launch_bounds__(128) k_sp_gaussians(SpArgs a, int n_total,
                                                      float* __restrict__ params) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.M) return;
  int x0, x1, y0, y1;
  sp_window(a, c, &x0, &x1, &y0, &y1);
  const size_t HW = (size_t)a.W * a.H;
  double cnt = 0, sx = 0, sy = 0, sr = 0, sg = 0, sb = 0;
  for (int y = y0; y <= y1; y++)
    for (int x = x0; x <= x1; x++) {
      const int idx = y * a.W + x;
      if (a.label[idx] != c) continue;
      cnt = __dadd_rn(cnt, 1.0);
      sx = __dadd_rn(sx, (double)x + 0.5);
      sy = __dadd_rn(sy, (double)y + 0.5);
      sr = __dadd_rn(sr, (double)a.frame[idx]);
      sg = __dadd_rn(sg, (double)a.frame[HW + idx]);
      sb = __dadd_rn(sb, (double)a.frame[2 * HW + idx]);
    }
  const int n = n_total;
  float out[9];
  if (cnt == 0) {
    const double qx = a.seed_xy[c], qy = a.seed_xy[a.M + c];
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
    const double mx = __ddiv_rn(sx, cnt), my = __ddiv_rn(sy, cnt);
    double sxx = 0, sxy = 0, syy = 0;
    for (int y = y0; y <= y1; y++)
      for (int x = x0; x <= x1; x++) {
        if (a.label[y * a.W + x] != c) continue;
        const double dx = __dsub_rn((double)x + 0.5, mx), dy = __dsub_rn((double)y + 0.5, my);
        sxx = __dadd_rn(sxx, __dmul_rn(dx, dx));
        sxy = __dadd_rn(sxy, __dmul_rn(dx, dy));
        syy = __dadd_rn(syy, __dmul_rn(dy, dy));
      }
    const double twelfth = __ddiv_rn(1.0, 12.0);
    const double vxx = __dadd_rn(__ddiv_rn(sxx, cnt), twelfth);
    const double vxy = __ddiv_rn(sxy, cnt);
    const double vyy = __dadd_rn(__ddiv_rn(syy, cnt), twelfth);
    const double c1 = __dsqrt_rn(vxx);
    const double c2 = __ddiv_rn(vxy, c1);
    const double c3 = __dsqrt_rn(__dsub_rn(vyy, __dmul_rn(c2, c2)));
    // Sigma = kappa (cov + I/12), kappa = 4: the factor 2 on L is exact
    const double l1 = 2.0 * c1, l2 = 2.0 * c2, l3 = 2.0 * c3;
    const double two_pi = 6.283185307179586;  // 2.0 * math.pi in double
    out[0] = (float)mx;
    out[1] = (float)my;
    out[2] = (float)l1;
    out[3] = (float)l2;
    out[4] = (float)l3;
    out[5] = (float)__ddiv_rn(sr, cnt);
    out[6] = (float)__ddiv_rn(sg, cnt);
    out[7] = (float)__ddiv_rn(sb, cnt);
    out[8] = (float)__ddiv_rn(cnt, __dmul_rn(__dmul_rn(two_pi, l1), l3));
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
// double[5][n], seeds double[2][n], cell map int[(W+1) (H+1)] (the grid has at
// most one cell per pixel).
uint64_t roi_init_scratch_bytes(int W, int H, int n) {
  const uint64_t hw = (uint64_t)W * H;
  return a256(hw * 4) + a256(5ull * n * 8) + a256(2ull * n * 8) +
         a256((uint64_t)(W + 1) * (H + 1) * 4) + 256;
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
  double* cen = reinterpret_cast<double*>(base + a256(hw * 4));
  double* seed_xy = reinterpret_cast<double*>(base + a256(hw * 4) + a256(5ull * n * 8));
  int* cell_of =
      reinterpret_cast<int*>(base + a256(hw * 4) + a256(5ull * n * 8) + a256(2ull * n * 8));
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
  a.lam = (kCompactness / S) * (kCompactness / S);
  a.frame = frame;
  a.mask = mask;
  a.cell_of = cell_of;
  a.seed_xy = seed_xy;
  a.cen = cen;
  a.label = label;
  if (M > 0) {
    e = cudaMemcpyAsync(seed_xy, sxy.data(), sxy.size() * sizeof(double),
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cell_of, cells.data(), cells.size() * sizeof(int),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      const int pb = (int)((hw + 255) / 256), cb = (M + 127) / 128;
      k_sp_init_centres<<<cb, 128, 0, s>>>(a);
      for (int it = 0; it < kIterations; it++) {
        k_sp_assign<<<pb, 256, 0, s>>>(a);
        k_sp_update<<<cb, 128, 0, s>>>(a);
      }
      k_sp_gaussians<<<cb, 128, 0, s>>>(a, n, params);
      e = cudaGetLastError();
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
