// Forward and backward rasterization of the accumulated-sum blend (Eq. 2).
//
// One CTA per 16x16 tile.  The tile's list (sorted entries [start, end)) is
// staged into shared memory in batches of kBatch Gaussians; for each staged
// Gaussian the staging thread also computes its pixel bounding box inside the
// tile, an 8-bit mask of the warp regions that box touches, and the slot where
// the backward pass writes this (tile, Gaussian) pair's partial sums.
//
// Forward: thread <-> pixel (warp <-> 8x4 region).  Each warp skips Gaussians
// whose box misses its region (a warp-uniform test), then every lane evaluates
// sigma in Cholesky form and accumulates c' 2^-q in ascending index order.
//
// Backward: the blend is recomputed from the saved lists (no per-pixel state).
// Thread group <-> Gaussian: s lanes (a power of two, about 256 / list length)
// share one Gaussian and stride over the pixels of its box, accumulating eight
// sums (dL/dc' direction and the quadratic-form moments); the group reduces
// them with shuffles and one lane writes them to the pair's slot.  A second
// kernel sums each Gaussian's slots in a fixed order (deterministic, no float
// atomics) and applies the chain rule to (mu, l, c, w).
#include "gs2d_internal.cuh"

namespace gs2d {

struct TileSmem {
  float4 r0[kBatch], r1[kBatch], r2[kBatch];
  int4 bb[kBatch];      // local box (x0, x1, y0, y1); x0 > x1 when empty
  int slot[kBatch];     // partial slot of the pair
  uint32_t hit[kBatch]; // bit w: box touches warp region w
};

__device__ __forceinline__ int tile_region_x(int w) { return (w & 1) * 8; }
__device__ __forceinline__ int tile_region_y(int w) { return (w >> 1) * 4; }

// Stage entries [b, b + cnt) of the tile's list.
__device__ __forceinline__ void stage_batch(TileSmem& sm, int b, int cnt, int tile, int TX, int W,
                                            int H, int n, const uint32_t* __restrict__ vals,
                                            const float4* __restrict__ rec,
                                            const int4* __restrict__ rect,
                                            const int* __restrict__ offs) {
  const int t = threadIdx.x;
  if (t < cnt) {
    const int g = (int)vals[b + t];
    const float4 r0 = rec[g], r1 = rec[n + g], r2 = rec[2 * n + g];
    const int tx = tile % TX, ty = tile / TX;
    const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
    // pixel lx contributes only if |ox + lx + 0.5 - mu_x| <= hx
    float fx0 = ceilf(r0.x - r2.y - 0.5f - ox), fx1 = floorf(r0.x + r2.y - 0.5f - ox);
    float fy0 = ceilf(r0.y - r2.z - 0.5f - oy), fy1 = floorf(r0.y + r2.z - 0.5f - oy);
    const float xmax = fminf((float)(kTile - 1), (float)(W - 1) - ox);
    const float ymax = fminf((float)(kTile - 1), (float)(H - 1) - oy);
    fx0 = fmaxf(fx0, 0.0f);
    fy0 = fmaxf(fy0, 0.0f);
    fx1 = fminf(fx1, xmax);
    fy1 = fminf(fy1, ymax);
    int4 bb = make_int4(1, 0, 1, 0);
    uint32_t hit = 0;
    if (fx0 <= fx1 && fy0 <= fy1) {
      bb = make_int4((int)fx0, (int)fx1, (int)fy0, (int)fy1);
#pragma unroll
      for (int w = 0; w < 8; w++) {
        const int rx = tile_region_x(w), ry = tile_region_y(w);
        if (bb.x <= rx + 7 && bb.y >= rx && bb.z <= ry + 3 && bb.w >= ry) hit |= 1u << w;
      }
    }
    const int4 rc = rect[g];
    sm.r0[t] = r0;
    sm.r1[t] = r1;
    sm.r2[t] = r2;
    sm.bb[t] = bb;
    sm.hit[t] = hit;
    sm.slot[t] = offs[g] + (ty - rc.y) * (rc.z - rc.x) + (tx - rc.x);
  }
}

// Forward accumulation of staged Gaussians [0, cnt) for this thread's pixel.
__device__ __forceinline__ void fwd_batch(const TileSmem& sm, int cnt, float px, float py,
                                          int wid, float3& acc) {
  for (int j = 0; j < cnt; j++) {
    if (!((sm.hit[j] >> wid) & 1u)) continue;  // warp-uniform
    const float4 r0 = sm.r0[j], r1 = sm.r1[j];
    const float cb = sm.r2[j].x;
    const float dx = px - r0.x, dy = py - r0.y;
    const float u1 = r0.z * dx;
    const float u2 = fmaf(r1.x, u1, r0.w * dy);
    const float q = fmaf(u2, u2, u1 * u1);
    if (q <= r1.y) {
      const float e = ex2_approx(-q);
      acc.x = fmaf(r1.z, e, acc.x);
      acc.y = fmaf(r1.w, e, acc.y);
      acc.z = fmaf(cb, e, acc.z);
    }
  }
}

// Backward over staged Gaussians [0, cnt) with g (dL/dC) of the tile in s_g.
__device__ __forceinline__ void bwd_batch(const TileSmem& sm, const float4* __restrict__ s_g,
                                          int cnt, float ox, float oy,
                                          float4* __restrict__ partial) {
  const int t = threadIdx.x;
  // lanes per Gaussian: power of two ~ 256 / cnt, within [1, 32]
  int s = 32;
  while (s > 1 && s * cnt > kTilePix) s >>= 1;
  const int lg = __ffs(s) - 1;
  const int grp = t >> lg, j = t & (s - 1);
  const int per_round = kTilePix >> lg;
  for (int base = 0; base < cnt; base += per_round) {
    const int gi = base + grp;
    float a[kPartials];
#pragma unroll
    for (int k = 0; k < kPartials; k++) a[k] = 0.0f;
    if (gi < cnt) {
      const int4 bb = sm.bb[gi];
      const int bw = bb.y - bb.x + 1, bh = bb.w - bb.z + 1;
      const int npx = (bw > 0 && bh > 0) ? bw * bh : 0;
      if (npx > 0) {
        const float4 r0 = sm.r0[gi], r1 = sm.r1[gi];
        const float cb = sm.r2[gi].x;
        const int ystep = s / bw, xstep = s - ystep * bw;
        int yy = j / bw, xx = j - yy * bw;
        for (int k = j; k < npx; k += s) {
          const int lx = bb.x + xx, ly = bb.z + yy;
          const float dx = (ox + (float)lx + 0.5f) - r0.x;
          const float dy = (oy + (float)ly + 0.5f) - r0.y;
          const float u1 = r0.z * dx;
          const float u2 = fmaf(r1.x, u1, r0.w * dy);
          const float q = fmaf(u2, u2, u1 * u1);
          if (q <= r1.y) {
            const float e = ex2_approx(-q);
            const float4 g = s_g[ly * kTile + lx];
            a[0] = fmaf(g.x, e, a[0]);
            a[1] = fmaf(g.y, e, a[1]);
            a[2] = fmaf(g.z, e, a[2]);
            const float S = fmaf(g.x, r1.z, fmaf(g.y, r1.w, g.z * cb)) * e;
            const float su1 = S * u1, su2 = S * u2;
            a[3] += su1;
            a[4] += su2;
            a[5] = fmaf(su1, u1, a[5]);
            a[6] = fmaf(su1, u2, a[6]);
            a[7] = fmaf(su2, u2, a[7]);
          }
          xx += xstep;
          yy += ystep;
          if (xx >= bw) {
            xx -= bw;
            yy++;
          }
        }
      }
    }
    for (int o = s >> 1; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < kPartials; k++) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
    }
    if (gi < cnt && j == 0) {
      const int slot = sm.slot[gi];
      partial[2 * slot] = make_float4(a[0], a[1], a[2], a[3]);
      partial[2 * slot + 1] = make_float4(a[4], a[5], a[6], a[7]);
    }
  }
}

struct TileCtx {
  int W, H, TX, n;
  const int2* ranges;
  const uint32_t* vals;
  const float4* rec;
  const int4* rect;
  const int* offs;
};

__global__ void __launch_bounds__(kTilePix)
k_render_fwd(TileCtx c, float* __restrict__ img) {
  __shared__ TileSmem sm;
  const int tile = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tx = tile % c.TX, ty = tile / c.TX;
  const int lx = tile_region_x(wid) + (lane & 7), ly = tile_region_y(wid) + (lane >> 3);
  const int x = tx * kTile + lx, y = ty * kTile + ly;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const int2 rg = c.ranges[tile];
  float3 acc = make_float3(0.f, 0.f, 0.f);
  for (int b = rg.x; b < rg.y; b += kBatch) {
    const int cnt = min(kBatch, rg.y - b);
    stage_batch(sm, b, cnt, tile, c.TX, c.W, c.H, c.n, c.vals, c.rec, c.rect, c.offs);
    __syncthreads();
    fwd_batch(sm, cnt, px, py, wid, acc);
    __syncthreads();
  }
  if (x < c.W && y < c.H) {
    const size_t HW = (size_t)c.W * c.H, o = (size_t)y * c.W + x;
    img[o] = acc.x;
    img[HW + o] = acc.y;
    img[2 * HW + o] = acc.z;
  }
}

__global__ void __launch_bounds__(kTilePix)
k_render_bwd(TileCtx c, const float* __restrict__ dimg, float4* __restrict__ partial) {
  __shared__ TileSmem sm;
  __shared__ float4 s_g[kTilePix];
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int tx = tile % c.TX, ty = tile / c.TX;
  {
    const int lx = tid & (kTile - 1), ly = tid >> 4;
    const int x = tx * kTile + lx, y = ty * kTile + ly;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (x < c.W && y < c.H) {
      const size_t HW = (size_t)c.W * c.H, o = (size_t)y * c.W + x;
      g = make_float4(dimg[o], dimg[HW + o], dimg[2 * HW + o], 0.f);
    }
    s_g[tid] = g;
  }
  const int2 rg = c.ranges[tile];
  const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
  for (int b = rg.x; b < rg.y; b += kBatch) {
    const int cnt = min(kBatch, rg.y - b);
    stage_batch(sm, b, cnt, tile, c.TX, c.W, c.H, c.n, c.vals, c.rec, c.rect, c.offs);
    __syncthreads();
    bwd_batch(sm, s_g, cnt, ox, oy, partial);
    __syncthreads();
  }
}

// Fused forward + L2 loss + backward.  loss_part[tile] = (sum (C-T)^2,
// sum (clamp(C,0,1)-T)^2) over the tile's valid pixels.
__global__ void __launch_bounds__(kTilePix)
k_render_l2(TileCtx c, const float* __restrict__ target, float gscale, float* __restrict__ img,
            float4* __restrict__ partial, float2* __restrict__ loss_part) {
  __shared__ TileSmem sm;
  __shared__ float4 s_g[kTilePix];
  __shared__ float2 s_red[kTilePix / 32];
  const int tile = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tx = tile % c.TX, ty = tile / c.TX;
  const int lx = tile_region_x(wid) + (lane & 7), ly = tile_region_y(wid) + (lane >> 3);
  const int x = tx * kTile + lx, y = ty * kTile + ly;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const int2 rg = c.ranges[tile];
  float3 acc = make_float3(0.f, 0.f, 0.f);
  int staged_b = -1;
  for (int b = rg.x; b < rg.y; b += kBatch) {
    const int cnt = min(kBatch, rg.y - b);
    stage_batch(sm, b, cnt, tile, c.TX, c.W, c.H, c.n, c.vals, c.rec, c.rect, c.offs);
    __syncthreads();
    fwd_batch(sm, cnt, px, py, wid, acc);
    __syncthreads();
    staged_b = b;
  }
  // loss and dL/dC
  float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 l = make_float2(0.f, 0.f);
  if (x < c.W && y < c.H) {
    const size_t HW = (size_t)c.W * c.H, o = (size_t)y * c.W + x;
    const float t0 = target[o], t1 = target[HW + o], t2 = target[2 * HW + o];
    const float d0 = acc.x - t0, d1 = acc.y - t1, d2 = acc.z - t2;
    const float e0 = __saturatef(acc.x) - t0, e1 = __saturatef(acc.y) - t1,
                e2 = __saturatef(acc.z) - t2;
    l.x = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
    l.y = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
    g = make_float4(gscale * d0, gscale * d1, gscale * d2, 0.f);
    if (img) {
      img[o] = acc.x;
      img[HW + o] = acc.y;
      img[2 * HW + o] = acc.z;
    }
  }
  s_g[ly * kTile + lx] = g;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l.x += __shfl_xor_sync(0xffffffffu, l.x, o);
    l.y += __shfl_xor_sync(0xffffffffu, l.y, o);
  }
  if (lane == 0) s_red[wid] = l;
  __syncthreads();
  if (tid == 0) {
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int w = 0; w < kTilePix / 32; w++) {
      s.x += s_red[w].x;
      s.y += s_red[w].y;
    }
    loss_part[tile] = s;
  }
  const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
  // backward; the last forward batch is still staged
  for (int b = rg.x; b < rg.y; b += kBatch) {
    const int cnt = min(kBatch, rg.y - b);
    if (b != staged_b) {
      __syncthreads();
      stage_batch(sm, b, cnt, tile, c.TX, c.W, c.H, c.n, c.vals, c.rec, c.rect, c.offs);
      staged_b = b;
    }
    __syncthreads();
    bwd_batch(sm, s_g, cnt, ox, oy, partial);
  }
}

// ---------------------------------------------------------------------------
// Per-Gaussian reduction of the slot partials (fixed order) and the chain rule
// from (sum g e, moments of S u) to (mu, l, c, w):
//   e = 2^-q, q = u1^2 + u2^2, u1 = s dx / l1, u2 = s (dy - l2 dx / l1) / l3,
//   dL/dq = -ln2 S, S = (g . c') e, accumulated A1 = sum S u1, A2 = sum S u2,
//   A11 = sum S u1^2, A12 = sum S u1 u2, A22 = sum S u2^2, G = sum g e.
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

__device__ __forceinline__ bool gather_partials(const float4* __restrict__ partial,
                                                const int* __restrict__ offs, int i,
                                                float a[kPartials]) {
  const int s0 = offs[i], s1 = offs[i + 1];
#pragma unroll
  for (int k = 0; k < kPartials; k++) a[k] = 0.0f;
  for (int sl = s0; sl < s1; sl++) {
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
  return s1 > s0;
}

__global__ void __launch_bounds__(256)
k_reduce_chain(int n, const float* __restrict__ params, const int* __restrict__ offs,
               const float4* __restrict__ partial, const WsHeader* __restrict__ hdr,
               float* __restrict__ grads) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool ok = hdr->entries_raw == (int64_t)hdr->n_entries;
  float a[kPartials], gr[9];
  const bool any = ok && gather_partials(partial, offs, i, a);
  if (any) chain_grads(params, n, i, a, gr);
#pragma unroll
  for (int r = 0; r < 9; r++) grads[(size_t)r * n + i] = any ? gr[r] : 0.0f;
}

// Fit loop: reduction + chain + Adam on the Gaussian's nine parameters.
__global__ void __launch_bounds__(256)
k_reduce_chain_adam(int n, float* __restrict__ params, const int* __restrict__ offs,
                    const float4* __restrict__ partial, const WsHeader* __restrict__ hdr,
                    float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                    float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (hdr->entries_raw != (int64_t)hdr->n_entries) return;  // over capacity: no update
  float a[kPartials], gr[9];
  const bool any = gather_partials(partial, offs, i, a);
  if (any)
    chain_grads(params, n, i, a, gr);
  else
    for (int r = 0; r < 9; r++) gr[r] = 0.0f;
  const float ibc1 = 1.0f / hdr->bc1, ibc2 = 1.0f / hdr->bc2;
#pragma unroll
  for (int r = 0; r < 9; r++) {
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

// Work statistics: listed pairs and contributing pairs (same predicate as the
// render kernels).  Diagnostic only.
__global__ void __launch_bounds__(kTilePix)
k_count_pairs(TileCtx c, WsHeader* __restrict__ hdr) {
  __shared__ TileSmem sm;
  __shared__ unsigned s_hits;
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int tx = tile % c.TX, ty = tile / c.TX;
  const int lx = tid & (kTile - 1), ly = tid >> 4;
  const int x = tx * kTile + lx, y = ty * kTile + ly;
  const bool valid = x < c.W && y < c.H;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  if (tid == 0) s_hits = 0;
  const int2 rg = c.ranges[tile];
  unsigned hits = 0;
  for (int b = rg.x; b < rg.y; b += kBatch) {
    const int cnt = min(kBatch, rg.y - b);
    __syncthreads();
    stage_batch(sm, b, cnt, tile, c.TX, c.W, c.H, c.n, c.vals, c.rec, c.rect, c.offs);
    __syncthreads();
    for (int j = 0; j < cnt && valid; j++) {
      const float4 r0 = sm.r0[j], r1 = sm.r1[j];
      const float dx = px - r0.x, dy = py - r0.y;
      const float u1 = r0.z * dx;
      const float u2 = fmaf(r1.x, u1, r0.w * dy);
      hits += fmaf(u2, u2, u1 * u1) <= r1.y;
    }
  }
  __syncthreads();
  atomicAdd(&s_hits, hits);
  __syncthreads();
  if (tid == 0) {
    const int vw = min(kTile, c.W - tx * kTile), vh = min(kTile, c.H - ty * kTile);
    atomicAdd(&hdr->pairs, (unsigned long long)(vw * vh) * (unsigned long long)(rg.y - rg.x));
    atomicAdd(&hdr->hits, (unsigned long long)s_hits);
  }
}

__global__ void k_adam_tick(WsHeader* __restrict__ hdr, float b1, float b2) {
  const int t = ++hdr->step;
  hdr->bc1 = (float)(1.0 - pow((double)b1, (double)t));
  hdr->bc2 = (float)(1.0 - pow((double)b2, (double)t));
}

// ---------------------------------------------------------------------------
static TileCtx make_ctx(const gs2d_plan& p, void* ws) {
  TileCtx c;
  c.W = p.width;
  c.H = p.height;
  c.TX = p.tiles_x;
  c.n = p.n;
  c.ranges = ws_ptr<int2>(ws, p, kOffRanges);
  c.vals = ws_ptr<uint32_t>(ws, p, (p.sort_passes & 1) ? kOffValsB : kOffValsA);
  c.rec = ws_ptr<float4>(ws, p, kOffRec);
  c.rect = ws_ptr<int4>(ws, p, kOffRect);
  c.offs = ws_ptr<int>(ws, p, kOffCount);
  return c;
}

cudaError_t launch_render_fwd(const gs2d_plan& p, void* ws, float* img, cudaStream_t s) {
  k_render_fwd<<<p.num_tiles, kTilePix, 0, s>>>(make_ctx(p, ws), img);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const gs2d_plan& p, void* ws, const float* params,
                              const float* dimg, float* grads, cudaStream_t s) {
  float4* partial = ws_ptr<float4>(ws, p, kOffPartial);
  k_render_bwd<<<p.num_tiles, kTilePix, 0, s>>>(make_ctx(p, ws), dimg, partial);
  if (p.n > 0)
    k_reduce_chain<<<(p.n + 255) / 256, 256, 0, s>>>(p.n, params, ws_ptr<int>(ws, p, kOffCount),
                                                     partial, ws_ptr<WsHeader>(ws, p, kOffHeader),
                                                     grads);
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
  float4* partial = ws_ptr<float4>(ws, p, kOffPartial);
  k_render_l2<<<p.num_tiles, kTilePix, 0, s>>>(make_ctx(p, ws), target, grad_scale(p), img,
                                               partial, ws_ptr<float2>(ws, p, kOffLossPart));
  if (p.n > 0)
    k_reduce_chain<<<(p.n + 255) / 256, 256, 0, s>>>(p.n, params, ws_ptr<int>(ws, p, kOffCount),
                                                     partial, ws_ptr<WsHeader>(ws, p, kOffHeader),
                                                     grads);
  if (loss) return launch_loss_reduce(p, ws, loss, s);
  return cudaGetLastError();
}

cudaError_t launch_adam_tick(const gs2d_plan& p, void* ws, cudaStream_t s) {
  k_adam_tick<<<1, 1, 0, s>>>(ws_ptr<WsHeader>(ws, p, kOffHeader), p.cfg.beta1, p.cfg.beta2);
  return cudaGetLastError();
}

cudaError_t launch_count_pairs(const gs2d_plan& p, void* ws, cudaStream_t s) {
  WsHeader* hdr = ws_ptr<WsHeader>(ws, p, kOffHeader);
  cudaError_t e = cudaMemsetAsync(&hdr->pairs, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_count_pairs<<<p.num_tiles, kTilePix, 0, s>>>(make_ctx(p, ws), hdr);
  return cudaGetLastError();
}

// One fit iteration after projection and binning: fused render + loss +
// backward, then reduction + chain + Adam.
cudaError_t launch_fit_step(const gs2d_plan& p, void* ws, const float* target, float* params,
                            float* m, float* v, cudaStream_t s) {
  float4* partial = ws_ptr<float4>(ws, p, kOffPartial);
  k_render_l2<<<p.num_tiles, kTilePix, 0, s>>>(make_ctx(p, ws), target, grad_scale(p), nullptr,
                                               partial, ws_ptr<float2>(ws, p, kOffLossPart));
  k_adam_tick<<<1, 1, 0, s>>>(ws_ptr<WsHeader>(ws, p, kOffHeader), p.cfg.beta1, p.cfg.beta2);
  if (p.n > 0)
    k_reduce_chain_adam<<<(p.n + 255) / 256, 256, 0, s>>>(
        p.n, params, ws_ptr<int>(ws, p, kOffCount), partial, ws_ptr<WsHeader>(ws, p, kOffHeader),
        m, v, p.cfg.lr, p.cfg.beta1, p.cfg.beta2, p.cfg.eps);
  return cudaGetLastError();
}

}  // namespace gs2d
