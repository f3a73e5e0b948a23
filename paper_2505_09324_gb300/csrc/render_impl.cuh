// Forward and backward rasterization of the accumulated-sum blend (Eq. 2),
// templated on the tile edge T (8, 16, 32) and the shared-memory batch S
// (Gaussians staged at a time: 32, 64, 128).  Included by render_t8.cu,
// render_t16.cu and render_t32.cu, one instantiation set each.
//
// Work order: gs2d_bin_sort leaves the tiles in the order section, longest
// list first, so that the longest tiles do not end up in the tail of the
// launch.  Two launch forms (gs2d_config::launch):
//  * persistent: one wave of thread blocks (resident blocks per SM x SMs)
//    takes tiles from a queue (a ticket counter in the workspace header); a
//    block takes its next ticket while it renders the current tile, so the
//    atomic's latency is hidden; the last block to leave the queue resets the
//    counter for the next launch;
//  * grid: one block per tile, block b rendering the b-th tile of the order;
//    the hardware block scheduler hands them out in that order.
// A tile of any clip of a batch is processed in that clip's frame (size,
// image offset, loss scale).
//
// Each tile's sorted list [start, end) is staged into shared memory in batches
// of S Gaussians; the staging thread also computes each Gaussian's pixel box
// inside the tile, a mask of the warps whose rows that box touches, and the
// slot where the backward pass writes this (tile, Gaussian) pair's sums.
//
// sigma in Cholesky form (Eq. 1): with s = sqrt(log2(e)/2) and tile-local
// offsets dx = px - mu_x, dy = py - mu_y,
//   u1 = a1 dx,  u2 = a2 dy + kappa dx  (a1 = s / l1, a2 = s / l3,
//   kappa = -(l2 / l3) a1),  q = u1^2 + u2^2 = sigma log2(e),
//   contribution c' 2^-q if q <= tau log2(e).
// For a fixed column, u1 is constant and u2 advances by a2 per row, so each
// further pixel of that column costs one FADD (u2) and one FFMA (q).
//
// Forward: thread <-> one column x R-row strip (R = 2 for T = 8, else 4);
// a warp covers a band of rows.  After each batch is staged every warp
// compacts (by ballot) the batch's Gaussians whose box meets its band into
// its own ascending list; each list entry carries the Gaussian's staged
// position and the row term a2 dy of the band's first row, so a thread's
// setup per Gaussian is four FP32 operations.  Accumulation is in ascending
// Gaussian index (the list order).
//
// Backward: the blend is recomputed from the saved lists (no per-pixel state
// is stored by the forward pass).  A group of T lanes takes one Gaussian and
// lays itself over the Gaussian's box inside the tile: box columns rounded up
// to a power of two c, T / c rows per step, each lane one column and every
// (T / c)-th row of the box.  Per lane it keeps
// sum g e (3), sum S, sum S u2, sum S u2^2 with S = (g . c') e; the moments
// in u1 follow by multiplying with the lane's constant u1.  The group reduces
// the eight sums with a transposing shuffle tree and writes one 32-byte
// record to the pair's slot.  k_reduce_chain sums each Gaussian's slots in a
// fixed order (deterministic, no float atomics) and applies the chain rule to
// (mu, l, c, w).
#pragma once

#include "gs2d_internal.cuh"

namespace gs2d {

template <int T>
struct TileGeom {
  static constexpr int R = T == 8 ? 2 : 4;  // rows per thread
  static constexpr int NT = T * T / R;      // threads per block: 32, 64, 256
  static constexpr int NW = NT / 32;        // warps: 1, 2, 8
  static constexpr int RW = 32 / T * R;     // rows per warp band: 8, 8, 4
  static constexpr int GPW = 32 / T;        // Gaussians per warp in the backward pass
  static constexpr int Q = T / 8;           // lanes per reduced value
};

template <int S>
struct TileSmem {
  float4 fa[S];      // (mu_x - ox, a1, kappa, a2): tile-local
  float4 fb[S];      // (tau2, c'_r, c'_g, c'_b)
  float my[S];       // mu_y - oy
  int4 bb[S];        // local box (x0, x1, y0, y1); x0 > x1 when empty
  int slot[S];       // partial slot of the pair
  uint32_t wmask[S]; // bit w: box touches the rows of warp w
  int next;          // the backward's next Gaussian (warps take them in turn)
};

// The tile a block works on, in its clip's frame.
struct TileFrame {
  int tile;       // global tile id
  int W, H;       // clip size
  int tx, ty;     // tile column and row in the clip
  int ox, oy;     // pixel origin of the tile in the clip
  int64_t pix;    // first float of the clip's image
  int2 rg;        // list range
};

template <int T>
__device__ __forceinline__ TileFrame tile_frame(const RenderArgs& a, int tile) {
  const gs2d_clip cl = clip_of_tile(a.clips, tile);
  const int lt = tile - cl.tile_off;
  const int ty = lt / cl.tiles_x, tx = lt - ty * cl.tiles_x;
  TileFrame f;
  f.tile = tile;
  f.W = cl.width;
  f.H = cl.height;
  f.tx = tx;
  f.ty = ty;
  f.ox = tx * T;
  f.oy = ty * T;
  f.pix = cl.pix_off;
  f.rg = a.ranges[tile];
  return f;
}

// Stage entries [b, b + cnt) of the tile's list (cnt <= S).
template <int T, int S>
__device__ __forceinline__ void stage_batch(TileSmem<S>& sm, const RenderArgs& a,
                                            const TileFrame& f, int b, int cnt) {
  using G = TileGeom<T>;
  if (threadIdx.x == 0) sm.next = 0;
  for (int k = threadIdx.x; k < cnt; k += G::NT) {
    const int g = (int)a.list[b + k];
    const float4 r0 = a.rec[g], r1 = a.rec[a.n + g], r2 = a.rec[2 * a.n + g];
    const int4 rc = a.rect[g];
    const int off = a.offs[g];
    const float ox = (float)f.ox, oy = (float)f.oy;
    // pixel lx contributes only if |ox + lx + 0.5 - mu_x| <= hx
    float fx0 = ceilf(r0.x - r2.y - 0.5f - ox), fx1 = floorf(r0.x + r2.y - 0.5f - ox);
    float fy0 = ceilf(r0.y - r2.z - 0.5f - oy), fy1 = floorf(r0.y + r2.z - 0.5f - oy);
    fx0 = fmaxf(fx0, 0.0f);
    fy0 = fmaxf(fy0, 0.0f);
    fx1 = fminf(fx1, fminf((float)(T - 1), (float)(f.W - 1) - ox));
    fy1 = fminf(fy1, fminf((float)(T - 1), (float)(f.H - 1) - oy));
    // slot: position of this tile inside the Gaussian's (tight) rectangle.
    // Lists kept across fit iterations may hold Gaussians whose rectangle no
    // longer covers the tile: such a pair is empty and has no slot (-1).
    int dx = -1, dy = -1;
    if (rc.z > 0) {
      const int first = rc.x - (f.tile - f.ty * rc.y - f.tx);  // y0 * stride + x0 in the clip
      const int y0 = first / rc.y;
      dx = f.tx - (first - y0 * rc.y);
      dy = f.ty - y0;
    }
    const bool covered = (unsigned)dx < (unsigned)rc.z && (unsigned)dy < (unsigned)rc.w;
    int4 bb = make_int4(1, 0, 1, 0);
    uint32_t wm = 0;
    if (covered && fx0 <= fx1 && fy0 <= fy1) {
      bb = make_int4((int)fx0, (int)fx1, (int)fy0, (int)fy1);
      const int w0 = bb.z / G::RW, w1 = bb.w / G::RW;
      wm = ((2u << w1) - 1u) & ~((1u << w0) - 1u);
    }
    sm.fa[k] = make_float4(r0.x - ox, r0.z, r1.x, r0.w);
    sm.fb[k] = make_float4(r1.y, r1.z, r1.w, r2.x);
    sm.my[k] = r0.y - oy;
    sm.bb[k] = bb;
    sm.wmask[k] = wm;
    sm.slot[k] = covered ? off + dy * rc.z + dx : -1;
  }
}

// One entry of a warp's list of staged Gaussians: the row term a2 (y - mu_y)
// at the first row of the warp's band (float bits) and the byte offset of
// the Gaussian in the staged arrays.
struct WarpEntry {
  uint32_t t;
  uint32_t off;
};

// Forward accumulation over the warp's list for this thread's column
// (tile-local centre pxl) and rows; drow = rows between the band's first row
// and this thread's first row.
template <int T, int S>
__device__ __forceinline__ void fwd_batch(const TileSmem<S>& sm, const WarpEntry* __restrict__ wl,
                                          int wn, float pxl, float drow,
                                          float (&acc)[TileGeom<T>::R][3]) {
  constexpr int R = TileGeom<T>::R;
  const char* fa_base = reinterpret_cast<const char*>(sm.fa);
  const char* fb_base = reinterpret_cast<const char*>(sm.fb);
  for (int i = 0; i < wn; i++) {
    const WarpEntry we = wl[i];
    const float4 fa = *reinterpret_cast<const float4*>(fa_base + we.off);
    const float4 fb = *reinterpret_cast<const float4*>(fb_base + we.off);
    const float dx = pxl - fa.x;
    const float u1 = fa.y * dx;
    const float u1sq = u1 * u1;
    float u2 = fmaf(fa.z, dx, __uint_as_float(we.t));
    if constexpr (T != 32) u2 = fmaf(fa.w, drow, u2);
#pragma unroll
    for (int r = 0; r < R; r++) {
      if (r) u2 += fa.w;
      const float q = fmaf(u2, u2, u1sq);
      if (q <= fb.x) {
        const float e = ex2_approx(-q);
        acc[r][0] = fmaf(fb.y, e, acc[r][0]);
        acc[r][1] = fmaf(fb.z, e, acc[r][1]);
        acc[r][2] = fmaf(fb.w, e, acc[r][2]);
      }
    }
  }
}

// Sum of eight per-lane values over each aligned group of G lanes (G = 8, 16
// or 32).  Three transposing levels (distances G/2, G/4, G/8) halve the values
// each lane carries; plain levels finish the sum.  Afterwards lane j of the
// group holds the total of value j / (G / 8) (lanes with j % (G / 8) == 0
// hold distinct values).
template <int G>
__device__ __forceinline__ float group_transpose_sum(const float (&v)[8], int j) {
  const bool b1 = j & (G / 2), b2 = j & (G / 4), b3 = j & (G / 8);
  float w[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const float send = b1 ? v[k] : v[k + 4];
    const float keep = b1 ? v[k + 4] : v[k];
    w[k] = keep + __shfl_xor_sync(0xffffffffu, send, G / 2);
  }
  float x[2];
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const float send = b2 ? w[k] : w[k + 2];
    const float keep = b2 ? w[k + 2] : w[k];
    x[k] = keep + __shfl_xor_sync(0xffffffffu, send, G / 4);
  }
  float y = (b3 ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, b3 ? x[0] : x[1], G / 8);
#pragma unroll
  for (int d = G / 16; d >= 1; d >>= 1) y += __shfl_xor_sync(0xffffffffu, y, d);
  return y;
}

// Backward over staged Gaussians [0, cnt) (entries batch[0 .. cnt) of the
// tile's list); g (dL/dC) of the tile in s_g.  Each pair's eight sums go to
// its slot of `partial`, or with `acc` (GS2D_REDUCE_ATOMIC) are added to the
// Gaussian's sums by float atomics (pairs whose box misses the tile add
// nothing).
template <int T, int S>
__device__ __forceinline__ void bwd_batch(TileSmem<S>& sm, const float4* __restrict__ s_g,
                                          int cnt, const RenderArgs& a, int b) {
  using G = TileGeom<T>;
  float* __restrict__ partial = a.partial;
  const int lane = threadIdx.x & 31;
  const int h = lane / T, j = lane % T;
  for (;;) {  // warps take the next GPW Gaussians as they finish (balance)
    int base = 0;
    if (lane == 0) base = atomicAdd(&sm.next, G::GPW);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= cnt) break;
    const int gi = base + h;
    // Gaussians whose box misses the tile: a zero record, no reduction
    const bool empty = gi >= cnt || sm.bb[gi].x > sm.bb[gi].y;
    if (__all_sync(0xffffffffu, empty)) {
      if (!a.acc && gi < cnt && j < 8 && sm.slot[gi] >= 0) partial[8 * sm.slot[gi] + j] = 0.0f;
      continue;
    }
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = 0.0f;
    if (gi < cnt) {
      const int4 bb = sm.bb[gi];
      // c = box width rounded up to a power of two; lane j: column j % c,
      // rows bb.z + j / c, + T / c, ...
      const int bw = bb.y - bb.x + 1;
      const int lc = bw <= 1 ? 0 : 32 - __clz(bw - 1);  // log2 c
      const int col = bb.x + (j & ((1 << lc) - 1));
      const int rstep = T >> lc;
      const int y0 = bb.z + (j >> lc);
      if (bw > 0 && col <= bb.y && y0 <= bb.w) {
        const float4 fa = sm.fa[gi], fb = sm.fb[gi];
        const float dx = ((float)col + 0.5f) - fa.x;
        const float u1 = fa.y * dx;
        const float u1sq = u1 * u1;
        const float ustep = fa.w * (float)rstep;
        float u2 = fmaf(fa.w, ((float)y0 + 0.5f) - sm.my[gi], fa.z * dx);
        float ge0 = 0.f, ge1 = 0.f, ge2 = 0.f, ss = 0.f, s2 = 0.f, s22 = 0.f;
        const float4* gp = s_g + y0 * T + col;
        const float4* const gend = s_g + bb.w * T + col;
        const int gstep = rstep * T;
        // branch-free: a pixel outside the cut-off adds exact zeros
#pragma unroll 2
        for (; gp <= gend; gp += gstep, u2 += ustep) {
          const float q = fmaf(u2, u2, u1sq);
          const float e = q <= fb.x ? ex2_approx(-q) : 0.0f;
          const float4 g = *gp;
          ge0 = fmaf(g.x, e, ge0);
          ge1 = fmaf(g.y, e, ge1);
          ge2 = fmaf(g.z, e, ge2);
          const float Sv = fmaf(g.x, fb.y, fmaf(g.y, fb.z, g.z * fb.w)) * e;
          const float su2 = Sv * u2;
          ss += Sv;
          s2 += su2;
          s22 = fmaf(su2, u2, s22);
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
    const float tot = group_transpose_sum<T>(v, j);
    if (gi < cnt && (j % G::Q) == 0 && sm.slot[gi] >= 0) {
      if (!a.acc)
        partial[8 * sm.slot[gi] + j / G::Q] = tot;
      else if (sm.bb[gi].x <= sm.bb[gi].y)
        atomicAdd(&a.acc[(size_t)kPartials * a.list[b + gi] + j / G::Q], tot);
    }
  }
}

// Per-mode shared memory beyond the staged batch.
template <int T, int S, int MODE>
struct ModeSmem {
  static constexpr int kGrad = (MODE == kModeBwd || MODE == kModeL2) ? T * T : 1;
  static constexpr int kList = (MODE == kModeFwd || MODE == kModeL2) ? S : 1;
  float4 g[kGrad];                       // dL/dC of the tile
  WarpEntry wl[TileGeom<T>::NW][kList];  // per-warp lists of the staged batch
  float2 red[TileGeom<T>::NW];         // loss partials per warp
  unsigned hits;                       // kModeCount
};

// Warp wid's list of the staged Gaussians [0, cnt) whose box touches its
// rows, in ascending order; returns its length.  pyw: tile-local centre of
// the band's first row.
template <int T, int S>
__device__ __forceinline__ int warp_list(const TileSmem<S>& sm, int cnt, int wid, int lane,
                                         float pyw, WarpEntry* __restrict__ wl) {
  int m = 0;
  for (int base = 0; base < cnt; base += 32) {
    const int k = base + lane;
    const bool on = k < cnt && ((sm.wmask[k] >> wid) & 1u);
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    if (on) {
      WarpEntry e;
      e.t = __float_as_uint(sm.fa[k].w * (pyw - sm.my[k]));
      e.off = (uint32_t)(k * sizeof(float4));
      wl[m + __popc(bal & ((1u << lane) - 1u))] = e;
    }
    m += __popc(bal);
  }
  __syncwarp();
  return m;
}

template <int T, int S, int MODE>
__device__ __forceinline__ void process_tile(const RenderArgs& a, const TileFrame& f,
                                             TileSmem<S>& sm, ModeSmem<T, S, MODE>& ms) {
  using G = TileGeom<T>;
  constexpr int R = G::R;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int x = f.ox + t % T, y0 = f.oy + R * (t / T);
  // tile-local pixel centres of this thread's column and first row
  const float pxl = (float)(t % T) + 0.5f, pyl = (float)(R * (t / T)) + 0.5f;
  const size_t HW = (size_t)f.W * f.H;
  const int2 rg = f.rg;

  if constexpr (MODE == kModeBwd) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
      if (x < f.W && y0 + r < f.H) {
        const size_t o = f.pix + (size_t)(y0 + r) * f.W + x;
        g = make_float4(a.dimg[o], a.dimg[HW + o], a.dimg[2 * HW + o], 0.f);
      }
      ms.g[(R * (t / T) + r) * T + t % T] = g;
    }
    for (int b = rg.x; b < rg.y; b += S) {
      const int cnt = min(S, rg.y - b);
      __syncthreads();
      stage_batch<T, S>(sm, a, f, b, cnt);
      __syncthreads();
      bwd_batch<T, S>(sm, ms.g, cnt, a, b);
    }
    return;
  }

  if constexpr (MODE == kModeSelect) {
    // Gaussians that contribute to a changed pixel of this tile (the
    // renderer's predicate); a pixel changed if max_c |ref - frame| > threshold
    bool changed[R];
    bool any = false;
#pragma unroll
    for (int r = 0; r < R; r++) {
      changed[r] = false;
      if (x < f.W && y0 + r < f.H) {
        const size_t o = f.pix + (size_t)(y0 + r) * f.W + x;
        float d = fabsf(a.ref[o] - a.frame[o]);
        d = fmaxf(d, fabsf(a.ref[HW + o] - a.frame[HW + o]));
        d = fmaxf(d, fabsf(a.ref[2 * HW + o] - a.frame[2 * HW + o]));
        changed[r] = d > a.threshold;
        any |= changed[r];
      }
    }
    if (!__syncthreads_or(any)) return;  // the whole tile unchanged
    for (int b = rg.x; b < rg.y; b += S) {
      const int cnt = min(S, rg.y - b);
      __syncthreads();
      stage_batch<T, S>(sm, a, f, b, cnt);
      __syncthreads();
      if (!any) continue;
      for (int j = 0; j < cnt; j++) {
        const float4 fa = sm.fa[j];
        const float dx = pxl - fa.x, dy = pyl - sm.my[j], tau2 = sm.fb[j].x;
        const float u1 = fa.y * dx;
        bool hit = false;
#pragma unroll
        for (int r = 0; r < R; r++) {
          const float u2 = fmaf(fa.w, dy + (float)r, fa.z * dx);
          hit |= changed[r] && fmaf(u2, u2, u1 * u1) <= tau2;
        }
        if (hit) a.selected[a.list[b + j]] = 1;  // every writer stores 1
      }
    }
    return;
  }

  if constexpr (MODE == kModeCount) {
    if (t == 0) ms.hits = 0;
    unsigned hits = 0;
    for (int b = rg.x; b < rg.y; b += S) {
      const int cnt = min(S, rg.y - b);
      __syncthreads();
      stage_batch<T, S>(sm, a, f, b, cnt);
      __syncthreads();
      for (int j = 0; j < cnt && x < f.W; j++) {
        const float4 fa = sm.fa[j];
        const float dx = pxl - fa.x, dy = pyl - sm.my[j], tau2 = sm.fb[j].x;
        const float u1 = fa.y * dx;
        for (int r = 0; r < R; r++) {
          const float u2 = fmaf(fa.w, dy + (float)r, fa.z * dx);
          hits += (y0 + r < f.H) && fmaf(u2, u2, u1 * u1) <= tau2;
        }
      }
    }
    __syncthreads();
    atomicAdd(&ms.hits, hits);
    __syncthreads();
    if (t == 0) {
      const int vw = min(T, f.W - f.ox), vh = min(T, f.H - f.oy);
      atomicAdd(&a.hdr->pairs, (unsigned long long)(vw * vh) * (unsigned long long)(rg.y - rg.x));
      atomicAdd(&a.hdr->hits, (unsigned long long)ms.hits);
    }
    return;
  }

  if constexpr (MODE == kModeFwd || MODE == kModeL2) {
    // forward (kModeFwd, kModeL2)
    float acc[R][3];
#pragma unroll
    for (int r = 0; r < R; r++) acc[r][0] = acc[r][1] = acc[r][2] = 0.0f;
    int staged = -1;
    for (int b = rg.x; b < rg.y; b += S) {
      const int cnt = min(S, rg.y - b);
      __syncthreads();
      stage_batch<T, S>(sm, a, f, b, cnt);
      __syncthreads();
      const int wn = warp_list<T, S>(sm, cnt, wid, lane, (float)(G::RW * wid) + 0.5f,
                                     ms.wl[wid]);
      fwd_batch<T, S>(sm, ms.wl[wid], wn, pxl, (float)(R * (lane / T)), acc);
      staged = b;
    }
    if constexpr (MODE == kModeFwd) {
      if (x < f.W) {
#pragma unroll
        for (int r = 0; r < R; r++) {
          if (y0 + r < f.H) {
            const size_t o = f.pix + (size_t)(y0 + r) * f.W + x;
            a.img[o] = acc[r][0];
            a.img[HW + o] = acc[r][1];
            a.img[2 * HW + o] = acc[r][2];
          }
        }
      }
      return;
    }

    // L2 loss and dL/dC of this thread's pixels; the clip's own mean
    const double count3 = 3.0 * (double)f.W * (double)f.H;
    const float gscale = (float)(2.0 / count3), lscale = (float)(1.0 / count3);
    float2 l = make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < R; r++) {
      float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
      if (x < f.W && y0 + r < f.H) {
        const size_t o = f.pix + (size_t)(y0 + r) * f.W + x;
        const float t0 = a.target[o], t1 = a.target[HW + o], t2 = a.target[2 * HW + o];
        const float d0 = acc[r][0] - t0, d1 = acc[r][1] - t1, d2 = acc[r][2] - t2;
        const float e0 = __saturatef(acc[r][0]) - t0, e1 = __saturatef(acc[r][1]) - t1,
                    e2 = __saturatef(acc[r][2]) - t2;
        l.x += fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
        l.y += fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
        g = make_float4(gscale * d0, gscale * d1, gscale * d2, 0.f);
        if (a.img) {
          a.img[o] = acc[r][0];
          a.img[HW + o] = acc[r][1];
          a.img[2 * HW + o] = acc[r][2];
        }
      }
      ms.g[(R * (t / T) + r) * T + t % T] = g;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      l.x += __shfl_xor_sync(0xffffffffu, l.x, o);
      l.y += __shfl_xor_sync(0xffffffffu, l.y, o);
    }
    if (lane == 0) ms.red[wid] = l;
    __syncthreads();
    if (t == 0) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int w = 0; w < G::NW; w++) {
        s.x += ms.red[w].x;
        s.y += ms.red[w].y;
      }
      a.loss_part[f.tile] = make_float2(s.x * lscale, s.y * lscale);
    }
    // backward; the last forward batch is still staged
    for (int b = rg.x; b < rg.y; b += S) {
      const int cnt = min(S, rg.y - b);
      if (b != staged) {
        __syncthreads();
        stage_batch<T, S>(sm, a, f, b, cnt);
        __syncthreads();
        staged = b;
      }
      bwd_batch<T, S>(sm, ms.g, cnt, a, b);
    }
  }
}

// Blocks per SM the register budget must allow (about 50 registers per
// thread of the 64 K per SM; 32 blocks at most): 32, 20, 5 for T = 8, 16, 32.
template <int T>
constexpr int kMinBlocks = 65536 / (TileGeom<T>::NT * 50) < 32 ? 65536 / (TileGeom<T>::NT * 50)
                                                                 : 32;

template <int T, int S, int MODE, int LAUNCH>
__global__ void __launch_bounds__(TileGeom<T>::NT, kMinBlocks<T>) k_render(RenderArgs a) {
  pdl_begin();
  __shared__ TileSmem<S> sm;
  __shared__ ModeSmem<T, S, MODE> ms;
  if constexpr (LAUNCH == GS2D_LAUNCH_GRID) {
    if (a.active && (int)blockIdx.x >= *a.active) return;  // a P-frame's subset
    const int tile = a.order[blockIdx.x];
    if ((unsigned)tile >= (unsigned)a.num_tiles) {  // a stale queue: report, skip
      if (threadIdx.x == 0) set_status(a.hdr, GS2D_ERR_BOUNDS);
      return;
    }
    process_tile<T, S, MODE>(a, tile_frame<T>(a, tile), sm, ms);
  } else {
    __shared__ int s_next[2];
    if (threadIdx.x == 0) s_next[0] = atomicAdd(&a.hdr->queue, 1);
    __syncthreads();
    const int limit = a.active ? min(*a.active, a.num_tiles) : a.num_tiles;
    for (int k = 0;; k ^= 1) {
      const int q = s_next[k];
      if (q >= limit) break;
      // next ticket now, stored after the tile: its latency overlaps the work
      int next = 0;
      if (threadIdx.x == 0) next = atomicAdd(&a.hdr->queue, 1);
      const int tile = a.order[q];
      if ((unsigned)tile < (unsigned)a.num_tiles)
        process_tile<T, S, MODE>(a, tile_frame<T>(a, tile), sm, ms);
      else if (threadIdx.x == 0)
        set_status(a.hdr, GS2D_ERR_BOUNDS);  // a stale queue: report, skip
      if (threadIdx.x == 0) s_next[k ^ 1] = next;
      __syncthreads();
    }
    // every block has taken its last ticket once `done` reaches the grid size
    if (threadIdx.x == 0 && atomicAdd(&a.hdr->done, 1) == (int)gridDim.x - 1) {
      atomicExch(&a.hdr->done, 0);
      atomicExch(&a.hdr->queue, 0);
    }
  }
}

template <int T, int S, int MODE, int LAUNCH>
cudaError_t launch_mode(const RenderArgs& a, cudaStream_t s) {
  if (a.num_tiles <= 0) return cudaSuccess;
  int grid = a.num_tiles;
  if (LAUNCH == GS2D_LAUNCH_PERSISTENT)
    grid = persistent_grid((const void*)k_render<T, S, MODE, LAUNCH>, TileGeom<T>::NT,
                           a.num_tiles);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  return launch_pdl(k_render<T, S, MODE, LAUNCH>, grid, TileGeom<T>::NT, 0, s, a);
}

template <int T, int S, int LAUNCH>
cudaError_t launch_form(RenderMode mode, const RenderArgs& a, cudaStream_t s) {
  switch (mode) {
    case kModeFwd: return launch_mode<T, S, kModeFwd, LAUNCH>(a, s);
    case kModeBwd: return launch_mode<T, S, kModeBwd, LAUNCH>(a, s);
    case kModeL2: return launch_mode<T, S, kModeL2, LAUNCH>(a, s);
    case kModeCount: return launch_mode<T, S, kModeCount, LAUNCH>(a, s);
    case kModeSelect: return launch_mode<T, S, kModeSelect, LAUNCH>(a, s);
  }
  return cudaErrorInvalidValue;
}

template <int T, int S>
cudaError_t launch_stage(int launch, RenderMode mode, const RenderArgs& a, cudaStream_t s) {
  return launch == GS2D_LAUNCH_GRID ? launch_form<T, S, GS2D_LAUNCH_GRID>(mode, a, s)
                                    : launch_form<T, S, GS2D_LAUNCH_PERSISTENT>(mode, a, s);
}

template <int T>
cudaError_t launch_tile(int stage, int launch, RenderMode mode, const RenderArgs& a,
                        cudaStream_t s) {
  switch (stage) {
    case 32: return launch_stage<T, 32>(launch, mode, a, s);
    case 64: return launch_stage<T, 64>(launch, mode, a, s);
    case 128: return launch_stage<T, 128>(launch, mode, a, s);
    case 256: return launch_stage<T, 256>(launch, mode, a, s);
  }
  return cudaErrorInvalidValue;
}

// Occupancy query of the fit loop's persistent render kernel (cached by
// persistent_grid); the grid form needs none.
template <int T>
cudaError_t prime_tile(int stage, int launch) {
  if (launch == GS2D_LAUNCH_GRID) return cudaSuccess;
  constexpr int NT = TileGeom<T>::NT, P = GS2D_LAUNCH_PERSISTENT;
  int g = 0;
  switch (stage) {
    case 32: g = persistent_grid((const void*)k_render<T, 32, kModeL2, P>, NT, 1); break;
    case 64: g = persistent_grid((const void*)k_render<T, 64, kModeL2, P>, NT, 1); break;
    case 128: g = persistent_grid((const void*)k_render<T, 128, kModeL2, P>, NT, 1); break;
    case 256: g = persistent_grid((const void*)k_render<T, 256, kModeL2, P>, NT, 1); break;
    default: return cudaErrorInvalidValue;
  }
  return g > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

}  // namespace gs2d
