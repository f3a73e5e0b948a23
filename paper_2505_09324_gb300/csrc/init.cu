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


#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr double kCompactness = 0.2;
constexpr int kIterations = kRoiIterations;
constexpr double kKappa = 4.0;  // covariance scale: keeps the blend of a tiling flat
constexpr double kColourScale = 1048576.0;  // 2^20
constexpr double kColourLimit = 32.0;
constexpr int kSums = 9;  // n, u, v, uu, uv, vv, r, g, b

// Seed grid, derived on the device from the mask's area.
struct SpGeom {
  int M, gx, gy, ncell;
  double S, area;
  float S32, lam32;
};

struct SpArgs {
  int W, H, n, k_target;
  const float* frame;
  const uint8_t* mask;
  int* cell_of;                // [gy][gx] seed index or -1
  double* seed_xy;             // [2][n] (the first M used)
  float* cen;                  // [5][n]: r, g, b, x, y
  int* label;                  // [H][W]
  unsigned long long* acc;     // [kSums][n] exact segment sums (two's complement)
  SpGeom* geo;
  unsigned long long* area;    // mask pixel count
  int* blk;                    // per-block seed counts (the grid compaction)
};

// Assignment + segment sums: each ROI pixel joins the nearest candidate
// centre (FP32 decisions), then adds its integer moments to the centre's sums
// (one 64-bit atomic per sum and group of lanes with the same centre).
__global__ void __launch_bounds__(256) k_sp_assign(SpArgs a) {
  pdl_begin();
  const SpGeom g = *a.geo;
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
  const int pcx = (int)floor((double)px / g.S), pcy = (int)floor((double)py / g.S);
  // candidates: the seeds of the 5 x 5 cells around the pixel's, visited in
  // raster order of the cells, which is ascending seed index (seeds are
  // numbered in raster order of the grid)
  const int M = a.n;  // array stride
  float best = INFINITY;
  int lab = -1;
  for (int dj = -2; dj <= 2; dj++) {
    const int cy = pcy + dj;
    if (cy < 0 || cy >= g.gy) continue;
    for (int di = -2; di <= 2; di++) {
      const int cx = pcx + di;
      if (cx < 0 || cx >= g.gx) continue;
      const int c = a.cell_of[cy * g.gx + cx];
      if (c < 0) continue;
      const float dx = __fsub_rn(px, a.cen[3 * M + c]);
      const float dy = __fsub_rn(py, a.cen[4 * M + c]);
      if (!(fabsf(dx) <= g.S32 && fabsf(dy) <= g.S32)) continue;
      const float dr = __fsub_rn(pr, a.cen[c]), dg = __fsub_rn(pg, a.cen[M + c]),
                  db = __fsub_rn(pb, a.cen[2 * M + c]);
      const float dc =
          __fadd_rn(__fadd_rn(__fmul_rn(dr, dr), __fmul_rn(dg, dg)), __fmul_rn(db, db));
      const float d =
          __fadd_rn(dc, __fmul_rn(g.lam32, __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy))));
      if (d < best) {
        best = d;
        lab = c;
      }
    }
  }
  a.label[idx] = lab;
  // exact moments: |u|, |v| <= 4 S + 2 and |q| <= 2^25, so a group sum of up
  // to 32 lanes stays within int32 for S < 2000
  int val[kSums] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (lab >= 0) {
    const int u = 2 * x + 1 - 2 * (int)floor(a.seed_xy[lab]);
    const int v = 2 * y + 1 - 2 * (int)floor(a.seed_xy[a.n + lab]);
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
  return (long long)a.acc[(size_t)k * a.n + c];
}

// Update: each centre moves to its segment's mean (clamped to within S of the
// seed) and mean colour; the sums are cleared for the next assignment.
__global__ void __launch_bounds__(128) k_sp_update(SpArgs a) {
  pdl_begin();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const SpGeom g = *a.geo;
  if (c >= g.M) return;
  const int M = a.n;  // array stride
  const long long n = acc_get(a, 0, c);
  if (n > 0) {
    const double qx = a.seed_xy[c], qy = a.seed_xy[a.n + c];
    const double mx = __dadd_rn(__ddiv_rn((double)acc_get(a, 1, c), (double)(2 * n)), floor(qx));
    const double my = __dadd_rn(__ddiv_rn((double)acc_get(a, 2, c), (double)(2 * n)), floor(qy));
    a.cen[3 * M + c] = (float)fmin(fmax(mx, __dsub_rn(qx, g.S)), __dadd_rn(qx, g.S));
    a.cen[4 * M + c] = (float)fmin(fmax(my, __dsub_rn(qy, g.S)), __dadd_rn(qy, g.S));
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
  if (c >= a.geo->M) return;
  const int M = a.n;  // array stride
  const double sx = a.seed_xy[c], sy = a.seed_xy[a.n + c];
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
  const SpGeom g = *a.geo;
  if (c >= g.M) return;
  const size_t HW = (size_t)a.W * a.H;
  const long long cnt = acc_get(a, 0, c);
  const double qx = a.seed_xy[c], qy = a.seed_xy[a.n + c];
  const int n = n_total;
  float out[9];
  if (cnt == 0) {
    const int xi = min(max((int)floor(qx), 0), a.W - 1), yi = min(max((int)floor(qy), 0), a.H - 1);
    const size_t idx = (size_t)yi * a.W + xi;
    const double s = __dmul_rn(2.0, __ddiv_rn(g.S, sqrt(12.0)));
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

// Mask area (pixel count).
__global__ void __launch_bounds__(256) k_sp_area(SpArgs a) {
  pdl_begin();
  const size_t hw = (size_t)a.W * a.H;
  unsigned c = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < hw;
       i += (size_t)gridDim.x * blockDim.x)
    c += a.mask[i] != 0;
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(a.area, (unsigned long long)c);
}

// The seed grid from the area: step S = max(1, sqrt(A / K)), cells of the
// gx x gy grid in raster order; a cell holds a seed when its centre's pixel is
// in the mask.  Every thread derives the same geometry.
__device__ __forceinline__ SpGeom seed_geometry(const SpArgs& a) {
  SpGeom g;
  g.area = (double)*a.area;
  g.M = 0;
  g.S = 1.0;
  g.gx = 1;
  g.gy = 1;
  if (g.area > 0.0 && a.k_target > 0) {
    g.S = fmax(1.0, __dsqrt_rn(__ddiv_rn(g.area, (double)a.k_target)));
    g.gx = (int)ceil(__ddiv_rn((double)a.W, g.S));
    g.gy = (int)ceil(__ddiv_rn((double)a.H, g.S));
  }
  g.ncell = g.gx * g.gy;
  g.S32 = (float)g.S;
  const double q = __ddiv_rn(kCompactness, g.S);
  g.lam32 = (float)__dmul_rn(q, q);
  return g;
}

__device__ __forceinline__ bool seed_cell(const SpArgs& a, const SpGeom& g, int cell, double* x,
                                          double* y) {
  if (g.area <= 0.0 || a.k_target <= 0 || cell >= g.ncell) return false;
  const int j = cell / g.gx, i = cell - j * g.gx;
  *x = __dmul_rn((double)i + 0.5, g.S);
  *y = __dmul_rn((double)j + 0.5, g.S);
  const int xi = (int)floor(*x), yi = (int)floor(*y);
  return xi < a.W && yi < a.H && a.mask[(size_t)yi * a.W + xi];
}

constexpr int kSeedBlocks = 152 * 4;

// Cells [b C, (b + 1) C) of block b, C = ceil(cells / blocks): the seed count.
__global__ void __launch_bounds__(256) k_sp_seed_count(SpArgs a) {
  pdl_begin();
  const SpGeom g = seed_geometry(a);
  const int chunk = (g.ncell + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * chunk, c1 = min(g.ncell, c0 + chunk);
  int cnt = 0;
  for (int cell = c0 + threadIdx.x; cell < c1; cell += blockDim.x) {
    double x, y;
    cnt += seed_cell(a, g, cell, &x, &y);
  }
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  __shared__ int s_w[8];
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_w[w];
    a.blk[blockIdx.x] = t;
  }
}

// Seeds numbered in raster order of the grid (at most n): each block adds the
// counts of the blocks before it, then numbers its cells by ballots.
__global__ void __launch_bounds__(256) k_sp_seed_write(SpArgs a) {
  pdl_begin();
  const SpGeom g = seed_geometry(a);
  __shared__ int s_base, s_w[9];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  {
    // this block's base (counts of the blocks before it) and the total
    int b = 0, tot = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
      const int c = a.blk[k];
      b += k < (int)blockIdx.x ? c : 0;
      tot += c;
    }
    for (int o = 16; o; o >>= 1) {
      b += __shfl_xor_sync(0xffffffffu, b, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    __shared__ int s_b[8], s_t[8];
    if (lane == 0) {
      s_b[wid] = b;
      s_t[wid] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int bb = 0, tt = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
        bb += s_b[w];
        tt += s_t[w];
      }
      s_base = bb;
      if (blockIdx.x == 0) {
        SpGeom out = g;
        out.M = min(tt, a.n);
        *a.geo = out;
      }
    }
    __syncthreads();
  }
  const int chunk = (g.ncell + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * chunk, c1 = min(g.ncell, c0 + chunk);
  int run = s_base;
  for (int base = c0; base < c1; base += blockDim.x) {
    const int cell = base + threadIdx.x;
    double x = 0.0, y = 0.0;
    const bool f = cell < c1 && seed_cell(a, g, cell, &x, &y);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) s_w[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
        const int c = s_w[w];
        s_w[w] = t;
        t += c;
      }
      s_w[8] = t;
    }
    __syncthreads();
    const int idx = run + s_w[wid] + __popc(bal & ((1u << lane) - 1u));
    if (cell < c1) {
      const bool take = f && idx < a.n;
      a.cell_of[cell] = take ? idx : -1;
      if (take) {
        a.seed_xy[idx] = x;
        a.seed_xy[a.n + idx] = y;
      }
    }
    run += s_w[8];
    __syncthreads();
  }
}

// Isotropic background Gaussians at bg_xy[0 .. nbg).
__global__ void __launch_bounds__(256) k_sp_background(SpArgs a, const float* __restrict__ bg_xy,
                                                       float* __restrict__ params) {
  pdl_begin();
  const SpGeom g = *a.geo;
  const int M = g.M, n = a.n, nbg = n - M;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nbg) return;
  const double hw = (double)a.W * (double)a.H;
  const double abg = __ddiv_rn(__dsub_rn(hw, g.area), (double)nbg);
  const double s = __dsqrt_rn(__ddiv_rn(__dmul_rn(kKappa, abg > 1.0 ? abg : 1.0),
                                        __dmul_rn(2.0, 3.141592653589793)));
  const double x = bg_xy[k], y = bg_xy[n + k];
  const int xi = min(max((int)floor(x), 0), a.W - 1), yi = min(max((int)floor(y), 0), a.H - 1);
  const size_t HW = (size_t)a.W * a.H, idx = (size_t)yi * a.W + xi;
  const int c = M + k;
  params[c] = (float)x;
  params[n + c] = (float)y;
  params[2 * n + c] = (float)s;
  params[3 * n + c] = 0.0f;
  params[4 * n + c] = (float)s;
  params[5 * n + c] = a.frame[idx];
  params[6 * n + c] = a.frame[HW + idx];
  params[7 * n + c] = a.frame[2 * HW + idx];
  params[8 * n + c] = (float)(1.0 / kKappa);
}

uint64_t a256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

}  // namespace

// Scratch layout for a W x H frame with n Gaussians: labels int[H W], centres
// float[5][n], seeds double[2][n], cell map int[(W+1) (H+1)] (the grid step
// is at least one pixel), segment sums int64[9][n], the area, the geometry and
// the per-block seed counts.
uint64_t roi_init_scratch_bytes(int W, int H, int n) {
  const uint64_t hw = (uint64_t)W * H;
  return a256(hw * 4) + a256(5ull * n * 4) + a256(2ull * n * 8) +
         a256((uint64_t)(W + 1) * (H + 1) * 4) + a256((uint64_t)kSums * n * 8) + a256(8) +
         a256(sizeof(SpGeom)) + a256(kSeedBlocks * 4) + 256;
}

gs2d_status roi_init(const float* frame, const uint8_t* mask, int W, int H, int n, float roi_frac,
                     const float* bg_xy, float* params, int32_t* n_roi, void* scratch,
                     uint64_t scratch_bytes, cudaStream_t s, char* err, size_t err_len,
                     float* cen_trace, int32_t* label_trace) {
  if (scratch_bytes < roi_init_scratch_bytes(W, H, n)) {
    snprintf(err, err_len, "gs2d_roi_init: scratch too small");
    return GS2D_ERR_INVALID_ARG;
  }
  const uint64_t hw = (uint64_t)W * H;
  char* p = static_cast<char*>(scratch);
  auto take = [&p](uint64_t bytes) {
    char* q = p;
    p += a256(bytes);
    return q;
  };
  SpArgs a;
  a.W = W;
  a.H = H;
  a.n = n;
  a.k_target = (int)llround((double)roi_frac * n);
  a.frame = frame;
  a.mask = mask;
  a.label = reinterpret_cast<int*>(take(hw * 4));
  a.cen = reinterpret_cast<float*>(take(5ull * n * 4));
  a.seed_xy = reinterpret_cast<double*>(take(2ull * n * 8));
  a.cell_of = reinterpret_cast<int*>(take((uint64_t)(W + 1) * (H + 1) * 4));
  a.acc = reinterpret_cast<unsigned long long*>(take((uint64_t)kSums * n * 8));
  a.area = reinterpret_cast<unsigned long long*>(take(8));
  a.geo = reinterpret_cast<SpGeom*>(take(sizeof(SpGeom)));
  a.blk = reinterpret_cast<int*>(take(kSeedBlocks * 4));
  // everything on the device; the region count comes back at the end
  const int pb = (int)((hw + 255) / 256), cb = (n + 127) / 128;
  cudaError_t e = cudaMemsetAsync(a.area, 0, 8, s);
  if (e == cudaSuccess) e = launch_pdl(k_sp_area, 152 * 8, 256, 0, s, a);
  if (e == cudaSuccess) e = launch_pdl(k_sp_seed_count, kSeedBlocks, 256, 0, s, a);
  if (e == cudaSuccess) e = launch_pdl(k_sp_seed_write, kSeedBlocks, 256, 0, s, a);
  if (e == cudaSuccess && n > 0) {
    e = launch_pdl(k_sp_init_centres, cb, 128, 0, s, a);
    // the last assignment's sums make the Gaussians
    for (int it = 0; it < kIterations && e == cudaSuccess; it++) {
      // optional trace: the centres this assignment uses, the labels it makes
      if (cen_trace)
        e = cudaMemcpyAsync(cen_trace + (size_t)it * 5 * n, a.cen, 5ull * n * sizeof(float),
                            cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = launch_pdl(k_sp_assign, pb, 256, 0, s, a);
      if (e == cudaSuccess && label_trace)
        e = cudaMemcpyAsync(label_trace + (size_t)it * hw, a.label, hw * sizeof(int32_t),
                            cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess && it + 1 < kIterations) e = launch_pdl(k_sp_update, cb, 128, 0, s, a);
    }
    if (e == cudaSuccess) e = launch_pdl(k_sp_gaussians, cb, 128, 0, s, a, n, params);
    if (e == cudaSuccess)
      e = launch_pdl(k_sp_background, (n + 255) / 256, 256, 0, s, a, bg_xy, params);
  }
  SpGeom g;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&g, a.geo, sizeof(g), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(err, err_len, "gs2d_roi_init: %s", cudaGetErrorString(e));
    return GS2D_ERR_CUDA;
  }
  if (n_roi) *n_roi = g.M;
  return GS2D_OK;
}

}  // namespace gs2d
