// Forward and backward rasterization of the accumulated-sum blend (Eq. 2).
//
// One 64-thread CTA per 16x16 tile (many CTAs per SM, independent barriers).
// The tile's sorted list [start, end) is staged into shared memory in batches
// of kStage Gaussians; the staging thread also computes each Gaussian's pixel
// box inside the tile, a 2-bit mask of the 8-row halves that box touches, and
// the slot where the backward pass writes this (tile, Gaussian) pair's sums.
//
// sigma in Cholesky form (Eq. 1): with s = sqrt(log2(e)/2),
//   u1 = s dx / l1,  u2 = s (dy - l2 dx / l1) / l3 = a2 dy + k u1,
//   q = u1^2 + u2^2 = sigma log2(e),  contribution c' 2^-q if q <= tau log2(e).
// For a fixed column dx, u1 and k u1 are constant, so each further pixel of
// that column costs one FADD (dy), one FFMA (u2) and one FFMA (q).
//
// Forward: thread <-> one column x 4-row strip; warp <-> 16 x 8 half-tile,
// which skips Gaussians whose box misses its rows (warp-uniform test).
// Accumulation is in ascending Gaussian index (the list order).
//
// Backward: the blend is recomputed from the saved lists (no per-pixel state
// is stored by the forward pass).  A 16-lane half-warp takes one Gaussian;
// lane = column of its box, looping over the box rows.  Per lane it keeps
// sum g e (3), sum S, sum S u2, sum S u2^2 with S = (g . c') e; the moments
// in u1 follow by multiplying with the lane's constant u1.  The half-warp
// reduces the eight sums with a transposing shuffle tree (8 shuffles) and
// writes one 32-byte record to the pair's slot.  k_reduce_chain sums each
// Gaussian's slots in a fixed order (deterministic, no float atomics) and
// applies the chain rule to (mu, l, c, w).
#include "gs2d_internal.cuh"

namespace gs2d {

constexpr int kRT = 64;      // threads per render CTA
constexpr int kStage = 64;   // Gaussians staged per batch

struct TileSmem {
  float4 r0[kStage], r1[kStage];
  float cb[kStage];
  int4 bb[kStage];      // local box (x0, x1, y0, y1); x0 > x1 when empty
  int slot[kStage];     // partial slot of the pair
  uint32_t half[kStage];  // bit h: box touches rows [8h, 8h + 8)
};

struct TileCtx {
  int W, H, TX, n;
  const int2* ranges;
  const uint32_t* vals;
  const float4* rec;
  const int4* rect;
  const int* offs;
};

// Stage entries [b, b + cnt) of the tile's list (cnt <= kStage).
__device__ __forceinline__ void stage_batch(TileSmem& sm, const TileCtx& c, int b, int cnt,
                                            int tile) {
  const int t = threadIdx.x;
  if (t < cnt) {
    const int g = (int)c.vals[b + t];
    const float4 r0 = c.rec[g], r1 = c.rec[c.n + g], r2 = c.rec[2 * c.n + g];
    const int4 rc = c.rect[g];
    const int off = c.offs[g];
    const int tx = tile % c.TX, ty = tile / c.TX;
    const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
    // pixel lx contributes only if |ox + lx + 0.5 - mu_x| <= hx
    float fx0 = ceilf(r0.x - r2.y - 0.5f - ox), fx1 = floorf(r0.x + r2.y - 0.5f - ox);
    float fy0 = ceilf(r0.y - r2.z - 0.5f - oy), fy1 = floorf(r0.y + r2.z - 0.5f - oy);
    fx0 = fmaxf(fx0, 0.0f);
    fy0 = fmaxf(fy0, 0.0f);
    fx1 = fminf(fx1, fminf((float)(kTile - 1), (float)(c.W - 1) - ox));
    fy1 = fminf(fy1, fminf((float)(kTile - 1), (float)(c.H - 1) - oy));
    int4 bb = make_int4(1, 0, 1, 0);
    uint32_t half = 0;
    if (fx0 <= fx1 && fy0 <= fy1) {
      bb = make_int4((int)fx0, (int)fx1, (int)fy0, (int)fy1);
      half = (bb.z <= 7 ? 1u : 0u) | (bb.w >= 8 ? 2u : 0u);
    }
    sm.r0[t] = r0;
    sm.r1[t] = r1;
    sm.cb[t] = r2.x;
    sm.bb[t] = bb;
    sm.half[t] = half;
    sm.slot[t] = off + (ty - rc.y) * (rc.z - rc.x) + (tx - rc.x);
  }
}

// Forward accumulation over staged Gaussians [0, cnt) for this thread's column
// px and rows py[0..3].
__device__ __forceinline__ void fwd_batch(const TileSmem& sm, int cnt, float px, const float py[4],
                                          int wid, float acc[4][3]) {
  for (int j = 0; j < cnt; j++) {
    if (!((sm.half[j] >> wid) & 1u)) continue;  // warp-uniform
    const float4 r0 = sm.r0[j], r1 = sm.r1[j];
    const float cb = sm.cb[j];
    const float u1 = r0.z * (px - r0.x);
    const float c0 = r1.x * u1;
    const float u1sq = u1 * u1;
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const float u2 = fmaf(r0.w, py[r] - r0.y, c0);
      const float q = fmaf(u2, u2, u1sq);
      if (q <= r1.y) {
        const float e = ex2_approx(-q);
        acc[r][0] = fmaf(r1.z, e, acc[r][0]);
        acc[r][1] = fmaf(r1.w, e, acc[r][1]);
        acc[r][2] = fmaf(cb, e, acc[r][2]);
      }
    }
  }
}

// Sum of eight per-lane values over the 16 lanes of each half-warp; afterwards
// lane j (even) of the half holds the total of value j / 2.
__device__ __forceinline__ float half_warp_transpose_sum(const float v[8], int j) {
  const bool b8 = j & 8, b4 = j & 4, b2 = j & 2;
  float w[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const float send = b8 ? v[k] : v[k + 4];
    const float keep = b8 ? v[k + 4] : v[k];
    w[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float x[2];
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const float send = b4 ? w[k] : w[k + 2];
    const float keep = b4 ? w[k + 2] : w[k];
    x[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  float y = (b2 ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, b2 ? x[0] : x[1], 2);
  y += __shfl_xor_sync(0xffffffffu, y, 1);
  return y;
}

// Backward over staged Gaussians [0, cnt); g (dL/dC) of the tile in s_g.
__device__ __forceinline__ void bwd_batch(const TileSmem& sm, const float4* __restrict__ s_g,
                                          int cnt, float ox, float oy,
                                          float* __restrict__ partial) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int h = lane >> 4, j = lane & 15;
  const float px = ox + (float)j + 0.5f;
  constexpr int kHalves = kRT / 16;
  for (int base = 2 * wid; base < cnt; base += kHalves) {  // warp-uniform
    const int gi = base + h;
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = 0.0f;
    if (gi < cnt) {
      const int4 bb = sm.bb[gi];
      if (j >= bb.x && j <= bb.y) {
        const float4 r0 = sm.r0[gi], r1 = sm.r1[gi];
        const float cr = r1.z, cg = r1.w, cb = sm.cb[gi];
        const float u1 = r0.z * (px - r0.x);
        const float c0 = r1.x * u1;
        const float u1sq = u1 * u1;
        float dy = (oy + (float)bb.z + 0.5f) - r0.y;
        float ge0 = 0.f, ge1 = 0.f, ge2 = 0.f, ss = 0.f, s2 = 0.f, s22 = 0.f;
        for (int y = bb.z; y <= bb.w; y++, dy += 1.0f) {
          const float u2 = fmaf(r0.w, dy, c0);
          const float q = fmaf(u2, u2, u1sq);
          if (q <= r1.y) {
            const float e = ex2_approx(-q);
            const float4 g = s_g[y * kTile + j];
            ge0 = fmaf(g.x, e, ge0);
            ge1 = fmaf(g.y, e, ge1);
            ge2 = fmaf(g.z, e, ge2);
            const float S = fmaf(g.x, cr, fmaf(g.y, cg, g.z * cb)) * e;
            const float su2 = S * u2;
            ss += S;
            s2 += su2;
            s22 = fmaf(su2, u2, s22);
          }
        }
        const float a1 = u1 * ss;
        v[0] = ge0;
        v[1] = ge1;
        v[2] = ge2;
        v[3] = a1;
        v[4] = s2;
        v[5] = u1 * a1;
        v[6] = u1 * s2;
        v[7] = s22;
      }
    }
    const float tot = half_warp_transpose_sum(v, j);
    if (gi < cnt && !(j & 1)) partial[8 * sm.slot[gi] + (j >> 1)] = tot;
  }
}

__device__ __forceinline__ void thread_pixels(int tile, int TX, float* px, float py[4], int* x,
                                              int* y0) {
  const int t = threadIdx.x;
  const int tx = tile % TX, ty = tile / TX;
  *x = tx * kTile + (t & 15);
  *y0 = ty * kTile + 4 * (t >> 4);
  *px = (float)*x + 0.5f;
#pragma unroll
  for (int r = 0; r < 4; r++) py[r] = (float)(*y0 + r) + 0.5f;
}

__global__ void __launch_bounds__(kRT)
k_render_fwd(TileCtx c, float* __restrict__ img) {
  __shared__ TileSmem sm;
  const int tile = blockIdx.x, wid = threadIdx.x >> 5;
  float px, py[4];
  int x, y0;
  thread_pixels(tile, c.TX, &px, py, &x, &y0);
  const int2 rg = c.ranges[tile];
  float acc[4][3] = {};
  for (int b = rg.x; b < rg.y; b += kStage) {
    const int cnt = min(kStage, rg.y - b);
    if (b != rg.x) __syncthreads();
    stage_batch(sm, c, b, cnt, tile);
    __syncthreads();
    fwd_batch(sm, cnt, px, py, wid, acc);
  }
  if (x < c.W) {
    const size_t HW = (size_t)c.W * c.H;
#pragma unroll
    for (int r = 0; r < 4; r++) {
      if (y0 + r < c.H) {
        const size_t o = (size_t)(y0 + r) * c.W + x;
        img[o] = acc[r][0];
        img[HW + o] = acc[r][1];
        img[2 * HW + o] = acc[r][2];
      }
    }
  }
}

__global__ void __launch_bounds__(kRT)
k_render_bwd(TileCtx c, const float* __restrict__ dimg, float* __restrict__ partial) {
  __shared__ TileSmem sm;
  __shared__ float4 s_g[kTilePix];
  const int tile = blockIdx.x;
  const int tx = tile % c.TX, ty = tile / c.TX;
  {
    float px, py[4];
    int x, y0;
    thread_pixels(tile, c.TX, &px, py, &x, &y0);
    const size_t HW = (size_t)c.W * c.H;
#pragma unroll
    for (int r = 0; r < 4; r++) {
      float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
      if (x < c.W && y0 + r < c.H) {
        const size_t o = (size_t)(y0 + r) * c.W + x;
        g = make_float4(dimg[o], dimg[HW + o], dimg[2 * HW + o], 0.f);
      }
      s_g[(y0 - ty * kTile + r) * kTile + (x - tx * kTile)] = g;
    }
  }
  const int2 rg = c.ranges[tile];
  const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
  for (int b = rg.x; b < rg.y; b += kStage) {
    const int cnt = min(kStage, rg.y - b);
    __syncthreads();
    stage_batch(sm, c, b, cnt, tile);
    __syncthreads();
    bwd_batch(sm, s_g, cnt, ox, oy, partial);
  }
}

// Fused forward + L2 loss + backward.  loss_part[tile] = (sum (C-T)^2,
// sum (clamp(C,0,1)-T)^2) over the tile's valid pixels.
__global__ void __launch_bounds__(kRT)
k_render_l2(TileCtx c, const float* __restrict__ target, float gscale, float* __restrict__ img,
            float* __restrict__ partial, float2* __restrict__ loss_part) {
  __shared__ TileSmem sm;
  __shared__ float4 s_g[kTilePix];
  __shared__ float2 s_red[kRT / 32];
  const int tile = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int tx = tile % c.TX, ty = tile / c.TX;
  float px, py[4];
  int x, y0;
  thread_pixels(tile, c.TX, &px, py, &x, &y0);
  const int2 rg = c.ranges[tile];
  float acc[4][3] = {};
  int staged = -1;
  for (int b = rg.x; b < rg.y; b += kStage) {
    const int cnt = min(kStage, rg.y - b);
    if (b != rg.x) __syncthreads();
    stage_batch(sm, c, b, cnt, tile);
    __syncthreads();
    fwd_batch(sm, cnt, px, py, wid, acc);
    staged = b;
  }
  // loss and dL/dC of this thread's four pixels
  float2 l = make_float2(0.f, 0.f);
  const size_t HW = (size_t)c.W * c.H;
#pragma unroll
  for (int r = 0; r < 4; r++) {
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (x < c.W && y0 + r < c.H) {
      const size_t o = (size_t)(y0 + r) * c.W + x;
      const float t0 = target[o], t1 = target[HW + o], t2 = target[2 * HW + o];
      const float d0 = acc[r][0] - t0, d1 = acc[r][1] - t1, d2 = acc[r][2] - t2;
      const float e0 = __saturatef(acc[r][0]) - t0, e1 = __saturatef(acc[r][1]) - t1,
                  e2 = __saturatef(acc[r][2]) - t2;
      l.x += fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
      l.y += fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
      g = make_float4(gscale * d0, gscale * d1, gscale * d2, 0.f);
      if (img) {
        img[o] = acc[r][0];
        img[HW + o] = acc[r][1];
        img[2 * HW + o] = acc[r][2];
      }
    }
    s_g[(y0 - ty * kTile + r) * kTile + (x - tx * kTile)] = g;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l.x += __shfl_xor_sync(0xffffffffu, l.x, o);
    l.y += __shfl_xor_sync(0xffffffffu, l.y, o);
  }
  if (lane == 0) s_red[wid] = l;
  __syncthreads();
  if (t == 0) loss_part[tile] = make_float2(s_red[0].x + s_red[1].x, s_red[0].y + s_red[1].y);
  const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
  // backward; the last forward batch is still staged
  for (int b = rg.x; b < rg.y; b += kStage) {
    const int cnt = min(kStage, rg.y - b);
    if (b != staged) {
      __syncthreads();
      stage_batch(sm, c, b, cnt, tile);
      __syncthreads();
      staged = b;
    }
    bwd_batch(sm, s_g, cnt, ox, oy, partial);
  }
}

// ---------------------------------------------------------------------------
// Per-Gaussian reduction of the slot partials (fixed order) and the chain rule
// from the eight sums to (mu, l, c, w):
//   e = 2^-q, q = u1^2 + u2^2, u1 = s dx / l1, u2 = s (dy - l2 dx / l1) / l3,
//   dL/dq = -ln2 S, S = (g . c') e; sums G = sum g e, A1 = sum S u1,
//   A2 = sum S u2, A11 = sum S u1^2, A12 = sum S u1 u2, A22 = sum S u2^2.
__device__ __forceinline__ void chain_grads(const float* __restrict__ params, int n, int i,
                                            const float a[kPartials], float gr[9]) {
  const float l1 = params[2 * n + i], l2 = params[3 * n + i], l3 = params[4 * n + i];
  const float cr = params[5 * n + i], cg = params[6 * n + i], cb = params[7 * n + i];
  const float w = params[8 * n + i];
  const float k2 = 1.17741002251547469101f;  // 2 ln2 s = sqrt(2 ln 2)
  const float c2 = 2.0f * kLn2;
  const float il1 = 1.0f / l1, il3 = 1.0f / l3, r = l2 * il3;
  gr[0] = k2 * (a[3] - r * a[4]) * il1;
  gr[1] = k2 * a[4] * il3;
  gr[2] = c2 * (a[5] - r * a[6]) * il1;
  gr[3] = c2 * a[6] * il3;
  gr[4] = c2 * a[7] * il3;
  gr[5] = w * a[0];
  gr[6] = w * a[1];
  gr[7] = w * a[2];
  gr[8] = fmaf(cr, a[0], fmaf(cg, a[1], cb * a[2]));
}

// kRL lanes share one Gaussian: lane `sub` sums slots s0 + sub, s0 + sub + kRL,
// ..., then the group adds its kRL partial sums (a fixed order: deterministic).
constexpr int kRL = 4;

__device__ __forceinline__ bool gather_partials(const float4* __restrict__ partial,
                                                const int* __restrict__ offs, int i, bool valid,
                                                int sub, float a[kPartials]) {
  int s0 = 0, s1 = 0;
  if (valid) {
    s0 = offs[i];
    s1 = offs[i + 1];
  }
#pragma unroll
  for (int k = 0; k < kPartials; k++) a[k] = 0.0f;
  for (int sl = s0 + sub; sl < s1; sl += kRL) {
    const float4 p = partial[2 * sl], q = partial[2 * sl + 1];
    a[0] += p.x;
    a[1] += p.y;
    a[2] += p.z;
    a[3] += p.w;
    a[4] += q.x;
    a[5] += q.y;
    a[6] += q.z;
    a[7] += q.w;
  }
#pragma unroll
  for (int o = 1; o < kRL; o <<= 1)
#pragma unroll
    for (int k = 0; k < kPartials; k++) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
  return s1 > s0;
}

__global__ void __launch_bounds__(256)
k_reduce_chain(int n, const float* __restrict__ params, const int* __restrict__ offs,
               const float4* __restrict__ partial, const WsHeader* __restrict__ hdr,
               float* __restrict__ grads) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gt / kRL, sub = gt % kRL;
  const bool valid = i < n && hdr->entries_raw == (int64_t)hdr->n_entries;
  float a[kPartials], gr[9];
  const bool any = gather_partials(partial, offs, i, valid, sub, a);
  if (i >= n) return;
  if (any) chain_grads(params, n, i, a, gr);
#pragma unroll
  for (int r = sub; r < 9; r += kRL) grads[(size_t)r * n + i] = any ? gr[r] : 0.0f;
}

// Fit loop: reduction + chain + Adam on the Gaussian's nine parameters (lane
// `sub` of the group updates rows sub, sub + kRL, ...).
__global__ void __launch_bounds__(256)
k_reduce_chain_adam(int n, float* __restrict__ params, const int* __restrict__ offs,
                    const float4* __restrict__ partial, const WsHeader* __restrict__ hdr,
                    float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                    float eps) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gt / kRL, sub = gt % kRL;
  const bool ok = hdr->entries_raw == (int64_t)hdr->n_entries;  // else over capacity
  float a[kPartials], gr[9];
  const bool any = gather_partials(partial, offs, i, i < n && ok, sub, a);
  if (!ok) return;  // the same for every thread of the grid
  const bool act = i < n;
  if (act && any)
    chain_grads(params, n, i, a, gr);
  else
    for (int r = 0; r < 9; r++) gr[r] = 0.0f;
  __syncwarp();  // every lane of the group has read the parameters
  if (!act) return;
  const float ibc1 = 1.0f / hdr->bc1, ibc2 = 1.0f / hdr->bc2;
#pragma unroll
  for (int r = sub; r < 9; r += kRL) {
    const size_t k = (size_t)r * n + i;
    const float g = gr[r];
    const float mm = fmaf(b1, m[k], (1.0f - b1) * g);
    const float vv = fmaf(b2, v[k], (1.0f - b2) * g * g);
    m[k] = mm;
    v[k] = vv;
    params[k] -= lr * (mm * ibc1) / (sqrtf(vv * ibc2) + eps);
  }
}

__global__ void __launch_bounds__(1024)
k_loss_reduce(int num_tiles, const float2* __restrict__ loss_part, double inv_count,
              WsHeader* __restrict__ hdr, float* __restrict__ out) {
  __shared__ double s_a[32], s_b[32];
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < num_tiles; t += blockDim.x) {
    a += loss_part[t].x;
    b += loss_part[t].y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_a[wid] = a;
    s_b[wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      sa += s_a[w];
      sb += s_b[w];
    }
    hdr->loss[0] = (float)(sa * inv_count);
    hdr->loss[1] = (float)(sb * inv_count);
    if (out) {
      out[0] = hdr->loss[0];
      out[1] = hdr->loss[1];
    }
  }
}

// Work statistics: listed pairs and contributing pairs (same predicate and
// arithmetic as the render kernels).  Diagnostic only.
__global__ void __launch_bounds__(kRT)
k_count_pairs(TileCtx c, WsHeader* __restrict__ hdr) {
  __shared__ TileSmem sm;
  __shared__ unsigned s_hits;
  const int tile = blockIdx.x, t = threadIdx.x;
  const int tx = tile % c.TX, ty = tile / c.TX;
  float px, py[4];
  int x, y0;
  thread_pixels(tile, c.TX, &px, py, &x, &y0);
  if (t == 0) s_hits = 0;
  const int2 rg = c.ranges[tile];
  unsigned hits = 0;
  for (int b = rg.x; b < rg.y; b += kStage) {
    const int cnt = min(kStage, rg.y - b);
    __syncthreads();
    stage_batch(sm, c, b, cnt, tile);
    __syncthreads();
    for (int j = 0; j < cnt && x < c.W; j++) {
      const float4 r0 = sm.r0[j], r1 = sm.r1[j];
      const float u1 = r0.z * (px - r0.x);
      const float c0 = r1.x * u1;
      for (int r = 0; r < 4; r++) {
        const float u2 = fmaf(r0.w, py[r] - r0.y, c0);
        hits += (y0 + r < c.H) && fmaf(u2, u2, u1 * u1) <= r1.y;
      }
    }
  }
  __syncthreads();
  atomicAdd(&s_hits, hits);
  __syncthreads();
  if (t == 0) {
    const int vw = min(kTile, c.W - tx * kTile), vh = min(kTile, c.H - ty * kTile);
    atomicAdd(&hdr->pairs, (unsigned long long)(vw * vh) * (unsigned long long)(rg.y - rg.x));
    atomicAdd(&hdr->hits, (unsigned long long)s_hits);
  }
}

// ---------------------------------------------------------------------------
static TileCtx make_ctx(const gs2d_plan& p, void* ws) {
  TileCtx c;
  c.W = p.width;
  c.H = p.height;
  c.TX = p.tiles_x;
  c.n = p.n;
  c.ranges = ws_ptr<int2>(ws, p, kOffRanges);
  c.vals = ws_ptr<uint32_t>(ws, p, kOffList);
  c.rec = ws_ptr<float4>(ws, p, kOffRec);
  c.rect = ws_ptr<int4>(ws, p, kOffRect);
  c.offs = ws_ptr<int>(ws, p, kOffCount);
  return c;
}

cudaError_t launch_render_fwd(const gs2d_plan& p, void* ws, float* img, cudaStream_t s) {
  k_render_fwd<<<p.num_tiles, kRT, 0, s>>>(make_ctx(p, ws), img);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const gs2d_plan& p, void* ws, const float* params,
                              const float* dimg, float* grads, cudaStream_t s) {
  float* partial = ws_ptr<float>(ws, p, kOffPartial);
  k_render_bwd<<<p.num_tiles, kRT, 0, s>>>(make_ctx(p, ws), dimg, partial);
  if (p.n > 0)
    k_reduce_chain<<<(p.n * kRL + 255) / 256, 256, 0, s>>>(
        p.n, params, ws_ptr<int>(ws, p, kOffCount), reinterpret_cast<const float4*>(partial),
        ws_ptr<WsHeader>(ws, p, kOffHeader), grads);
  return cudaGetLastError();
}

static float grad_scale(const gs2d_plan& p) {
  return (float)(2.0 / (3.0 * (double)p.width * (double)p.height));
}

cudaError_t launch_loss_reduce(const gs2d_plan& p, void* ws, float* loss, cudaStream_t s) {
  k_loss_reduce<<<1, 1024, 0, s>>>(p.num_tiles, ws_ptr<float2>(ws, p, kOffLossPart),
                                   1.0 / (3.0 * (double)p.width * (double)p.height),
                                   ws_ptr<WsHeader>(ws, p, kOffHeader), loss);
  return cudaGetLastError();
}

cudaError_t launch_render_l2(const gs2d_plan& p, void* ws, const float* params,
                             const float* target, float* grads, float* img, float* loss,
                             cudaStream_t s) {
  float* partial = ws_ptr<float>(ws, p, kOffPartial);
  k_render_l2<<<p.num_tiles, kRT, 0, s>>>(make_ctx(p, ws), target, grad_scale(p), img, partial,
                                          ws_ptr<float2>(ws, p, kOffLossPart));
  if (p.n > 0)
    k_reduce_chain<<<(p.n * kRL + 255) / 256, 256, 0, s>>>(
        p.n, params, ws_ptr<int>(ws, p, kOffCount), reinterpret_cast<const float4*>(partial),
        ws_ptr<WsHeader>(ws, p, kOffHeader), grads);
  if (loss) return launch_loss_reduce(p, ws, loss, s);
  return cudaGetLastError();
}

cudaError_t launch_count_pairs(const gs2d_plan& p, void* ws, cudaStream_t s) {
  WsHeader* hdr = ws_ptr<WsHeader>(ws, p, kOffHeader);
  cudaError_t e = cudaMemsetAsync(&hdr->pairs, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_count_pairs<<<p.num_tiles, kRT, 0, s>>>(make_ctx(p, ws), hdr);
  return cudaGetLastError();
}

// One fit iteration after projection and binning (which advanced the Adam
// step counter): fused render + loss + backward, then reduction + chain + Adam.
cudaError_t launch_fit_step(const gs2d_plan& p, void* ws, const float* target, float* params,
                            float* m, float* v, cudaStream_t s) {
  float* partial = ws_ptr<float>(ws, p, kOffPartial);
  k_render_l2<<<p.num_tiles, kRT, 0, s>>>(make_ctx(p, ws), target, grad_scale(p), nullptr,
                                          partial, ws_ptr<float2>(ws, p, kOffLossPart));
  if (p.n > 0)
    k_reduce_chain_adam<<<(p.n * kRL + 255) / 256, 256, 0, s>>>(
        p.n, params, ws_ptr<int>(ws, p, kOffCount), reinterpret_cast<const float4*>(partial),
        ws_ptr<WsHeader>(ws, p, kOffHeader), m, v, p.cfg.lr, p.cfg.beta1, p.cfg.beta2, p.cfg.eps);
  return cudaGetLastError();
}

}  // namespace gs2d
