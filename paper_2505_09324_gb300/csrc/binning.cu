// Projection, tile binning and the sort by tile id.
//
// The method renders with the tile-based rasterizer it inherits (Sec. 3,
// "differentiable tile-based rasterization"); in 2D there is no depth
// (Sec. 3.1, accumulated-sum blending), so within a tile the Gaussians are
// ordered by index: the sorted list is the (tile, index) key order.
//
// The sort is a single-digit radix (counting) sort by tile id over all SMs:
//   1. per-tile entry counts (atomic increments from each Gaussian's tiles)
//      and per-block sums of the per-Gaussian counts;
//   2. exclusive scans: one CTA per block of 256 Gaussians for the offsets
//      (backward slots), one CTA per 1024 tiles for the list ranges; capacity;
//   3. scatter: every entry claims the next slot of its tile's list;
//   4. segment sort: each tile's list is sorted by Gaussian index (a warp
//      bitonic network in registers for lists of up to 512, a CTA bitonic
//      network in shared memory for longer ones), restoring exactly the order
//      a stable sort of the index-ordered entries would give.
// Steps 2 and 4 also build the render queue: tiles grouped by list-length
// class (floor(log2(len)) + 1, 0 for empty tiles), longest class first.  The
// scan gives each tile its rank inside its class (one atomic per class and
// block), the segment sort turns (class, rank) into the queue position once
// every class size is known.
// A batch of clips is binned in one pass: tiles are numbered clip after clip
// and each Gaussian's rectangle is stored in that numbering.
#include "gs2d_internal.cuh"

namespace gs2d {

constexpr int kLongMax = 1 << 15;  // longest list the CTA sort holds (128 KB)
constexpr int kGB = 256;           // Gaussians per counting / scan block

// ---------------------------------------------------------------------------
// Projection (gs2d_project): records, rectangles, per-Gaussian counts.
__global__ void __launch_bounds__(kGB)
k_project(int n, ClipSet cs, int tile_shift, float sigma_cut, float alpha_min, float det_eps,
          const float* __restrict__ params, float4* __restrict__ rec, int4* __restrict__ rect,
          int* __restrict__ count) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  project_one(i, n, clip_of_gaussian(cs, i), tile_shift, sigma_cut, alpha_min, det_eps, params,
              rec, rect, count);
}

// Per-tile entry counts from the rectangles (warp-cooperative: lanes share the
// tiles of one Gaussian at a time; fire-and-forget atomics).
__device__ __forceinline__ void count_tiles_warp(int n, const int4* __restrict__ rect,
                                                 int* __restrict__ tile_cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int4 rc = i < n ? rect[i] : make_int4(0, 0, 0, 0);
  for (int l = 0; l < 32; l++) {
    const int t0 = __shfl_sync(0xffffffffu, rc.x, l);
    const int stride = __shfl_sync(0xffffffffu, rc.y, l);
    const int w = __shfl_sync(0xffffffffu, rc.z, l);
    const int cnt = w * __shfl_sync(0xffffffffu, rc.w, l);
    for (int j = lane; j < cnt; j += 32) {
      const int dy = j / w;
      atomicAdd(&tile_cnt[t0 + dy * stride + (j - dy * w)], 1);
    }
  }
}

// The block's sum of per-Gaussian counts.
__device__ __forceinline__ void block_count_sum(int n, const int* __restrict__ count,
                                                long long* __restrict__ block_sum) {
  __shared__ int s_warp[kGB / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int c = i < n ? count[i] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) s_warp[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int w = 0; w < kGB / 32; w++) s += s_warp[w];
    block_sum[blockIdx.x] = s;
  }
}

__device__ __forceinline__ void count_block(int n, const int4* __restrict__ rect,
                                           const int* __restrict__ count,
                                           int* __restrict__ tile_cnt,
                                           long long* __restrict__ block_sum) {
  count_tiles_warp(n, rect, tile_cnt);
  block_count_sum(n, count, block_sum);
}

// Adam step counter, the powers beta^step and the decayed learning rate of
// the step that begins (thread 0 of the first kernel of a fit iteration).
__device__ __forceinline__ void adam_tick_header(WsHeader* hdr, float b1, float b2, float lr,
                                                 float lr_decay) {
  const int t = ++hdr->step;
  const double p1 = t == 1 ? (double)b1 : hdr->pw1 * b1;
  const double p2 = t == 1 ? (double)b2 : hdr->pw2 * b2;
  hdr->pw1 = p1;
  hdr->pw2 = p2;
  hdr->bc1 = (float)(1.0 - p1);
  hdr->bc2 = (float)(1.0 - p2);
  const double pd = t == 1 ? 1.0 : hdr->pwd * lr_decay;
  hdr->pwd = pd;
  hdr->lr_now = (float)(lr * pd);
}

__global__ void __launch_bounds__(kGB)
k_count_tiles(int n, const int4* __restrict__ rect, const int* __restrict__ count,
              int* __restrict__ tile_cnt, long long* __restrict__ block_sum,
              WsHeader* __restrict__ hdr) {
  pdl_begin();
  if (blockIdx.x == 0 && threadIdx.x == 0) hdr->lists_valid = 0;  // rebuilt from tight boxes
  count_block(n, rect, count, tile_cnt, block_sum);
}

// Fused projection + counts for gs2d_prepare and the fit loop; with adam_tick
// the Adam step counter and the powers beta^step advance here (the first
// kernel of a fit iteration).
__global__ void __launch_bounds__(kGB)
k_project_count(int n, ClipSet cs, int tile_shift, float sigma_cut, float alpha_min,
                float det_eps,
                const float* __restrict__ params, float4* __restrict__ rec,
                int4* __restrict__ rect, int* __restrict__ count, int* __restrict__ tile_cnt,
                long long* __restrict__ block_sum, WsHeader* __restrict__ hdr, int adam_tick,
                float b1, float b2, float lr, float lr_decay) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    if (adam_tick) adam_tick_header(hdr, b1, b2, lr, lr_decay);
    hdr->lists_valid = 0;  // the lists below are built from the tight rectangles
  }
  if (i < n)
    project_one(i, n, clip_of_gaussian(cs, i), tile_shift, sigma_cut, alpha_min, det_eps, params,
                rec, rect, count);
  __syncwarp();
  count_block(n, rect, count, tile_cnt, block_sum);
}

// ---------------------------------------------------------------------------
// Fit loop with retained tile lists.  Within a tile a Gaussian adds nothing
// outside its cut-off box, so a list may hold Gaussians that do not reach the
// tile: the render skips a (tile, Gaussian) pair whose tile lies outside the
// Gaussian's tight rectangle, and the backward slots stay those of the tight
// rectangles, so results are the same as with lists rebuilt every iteration.
// Each Gaussian is listed over its rectangle widened by `margin` pixels; the
// lists are rebuilt only in an iteration where some tight rectangle has left
// its listed one.
//
// k_project_fit: records, tight rectangles and counts (the backward slots),
// block sums of the counts, the containment test against the listed
// rectangle (clears hdr->lists_valid on a miss) and the Adam tick.
__global__ void __launch_bounds__(kGB)
k_project_fit(int n, ClipSet cs, int tile_shift, float sigma_cut, float alpha_min, float det_eps,
              const float* __restrict__ params, float4* __restrict__ rec, int4* __restrict__ rect,
              int* __restrict__ count, long long* __restrict__ block_sum,
              const int4* __restrict__ lrect, WsHeader* __restrict__ hdr, float b1, float b2,
              float lr, float lr_decay) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) adam_tick_header(hdr, b1, b2, lr, lr_decay);
  if (i < n) {
    const gs2d_clip cl = clip_of_gaussian(cs, i);
    int tx0 = 0, ty0 = 0, tx1 = 0, ty1 = 0;
    const bool vis = gaussian_tiles(i, n, cl, tile_shift, sigma_cut, alpha_min, det_eps, params,
                                    0.0f, tx0, ty0, tx1, ty1);
    const int4 rc = vis ? make_int4(cl.tile_off + ty0 * cl.tiles_x + tx0, cl.tiles_x, tx1 - tx0,
                                    ty1 - ty0)
                        : make_int4(0, 0, 0, 0);
    rect[i] = rc;
    count[i] = rc.z * rc.w;
    write_record(i, n, vis, sigma_cut, alpha_min, params, rec);
    if (vis) {
      const int4 lr4 = lrect[i];
      bool inside = lr4.z > 0;
      if (inside) {
        const int rel = lr4.x - cl.tile_off;
        const int ly0 = rel / cl.tiles_x, lx0 = rel - ly0 * cl.tiles_x;
        inside = lx0 <= tx0 && ly0 <= ty0 && tx1 <= lx0 + lr4.z && ty1 <= ly0 + lr4.w;
      }
      if (!inside) hdr->lists_valid = 0;
    }
  }
  block_count_sum(n, count, block_sum);
}

// Rebuild step 1 (only when k_project_fit found a miss): the listed
// rectangles, widened by `margin` pixels, and the per-tile entry counts; the
// tight rectangles are counted too (tile_cnt2), so that the scan can fall
// back to them when the widened lists would overflow max_entries.
__global__ void __launch_bounds__(kGB)
k_rebin_count(int n, ClipSet cs, int tile_shift, float sigma_cut, float alpha_min,
              float det_eps, float margin, const float* __restrict__ params,
              const int4* __restrict__ rect, int4* __restrict__ lrect,
              int* __restrict__ tile_cnt, int* __restrict__ tile_cnt2,
              WsHeader* __restrict__ hdr) {
  pdl_begin();
  if (hdr->lists_valid) return;  // the same for every thread of the grid
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) hdr->rebins++;
  if (i < n) {
    const gs2d_clip cl = clip_of_gaussian(cs, i);
    int tx0 = 0, ty0 = 0, tx1 = 0, ty1 = 0;
    const bool vis = gaussian_tiles(i, n, cl, tile_shift, sigma_cut, alpha_min, det_eps, params,
                                    margin, tx0, ty0, tx1, ty1);
    lrect[i] = vis ? make_int4(cl.tile_off + ty0 * cl.tiles_x + tx0, cl.tiles_x, tx1 - tx0,
                               ty1 - ty0)
                   : make_int4(0, 0, 0, 0);
  }
  __syncwarp();
  count_tiles_warp(n, lrect, tile_cnt);
  count_tiles_warp(n, rect, tile_cnt2);
}

// ---------------------------------------------------------------------------
// Scans.  CTAs 0 .. nbg-1: offsets of their 256 Gaussians (prefix of the block
// sums + in-block exclusive scan).  CTAs nbg ..: per-tile ranges and cursors of
// a chunk of 1024 tiles; the first of them also records the entry total and
// the capacity decision.  Sums are 64-bit so that a pathological input is
// reported as over capacity instead of wrapping around.
__device__ __forceinline__ long long block_scan64(long long v, long long* warp_sum,
                                                  long long* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long t = lane < nw ? warp_sum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_sum[lane] = t;
  }
  __syncthreads();
  const long long ex = (wid > 0 ? warp_sum[wid - 1] : 0) + x - v;
  *total = warp_sum[nw - 1];
  __syncthreads();
  return ex;
}

constexpr int kTileItems = 4;  // tiles per thread of a tile-scan CTA

// Render-queue class of a list of length len: 0 (empty), 1 + floor(log2(len))
// capped at kBuckets - 1.
__device__ __forceinline__ int length_class(int len) {
  return len <= 0 ? 0 : min(kBuckets - 1, 32 - __clz(len));
}

__global__ void __launch_bounds__(kGB)
k_bin_scan(int n, int nbg, int num_tiles, int64_t max_entries, int* __restrict__ count,
           const long long* __restrict__ block_sum, int* __restrict__ tile_cnt,
           int* __restrict__ cursor, int2* __restrict__ ranges, int* __restrict__ bucket,
           uint32_t* __restrict__ rank, WsHeader* __restrict__ hdr, int lazy,
           const int* __restrict__ tile_cnt2) {
  pdl_begin();
  __shared__ long long warp_sum[32];
  __shared__ int s_hist[kBuckets];
  __shared__ int s_base[kBuckets];
  const int t = threadIdx.x;
  if ((int)blockIdx.x < nbg) {
    // total and this block's prefix from the block sums
    long long tot = 0, pre = 0;
    for (int b = t; b < nbg; b += kGB) {
      const long long v = block_sum[b];
      tot += v;
      pre += b < (int)blockIdx.x ? v : 0;
    }
    long long total, prefix;
    block_scan64(tot, warp_sum, &total);
    block_scan64(pre, warp_sum, &prefix);
    const bool over = total > max_entries;
    const int i = blockIdx.x * kGB + t;
    const int c = i < n ? count[i] : 0;
    long long dummy;
    const long long ex = block_scan64(c, warp_sum, &dummy);
    if (i < n) count[i] = over ? 0 : (int)(prefix + ex);
    if (blockIdx.x == 0 && t == 0) count[n] = over ? 0 : (int)total;
    return;
  }
  // retained lists: only the slots (above) change
  if (lazy && hdr->lists_valid) return;  // the same for every thread of the grid
  // tile CTAs: chunk [c0, c0 + kGB * kTileItems) of the tiles; the prefix of the
  // chunk and the total come from a strided pass over all tile counts (the
  // counts are reset later, by k_sort_short, once nothing reads them)
  const int tb = (int)blockIdx.x - nbg;
  const int c0 = tb * kGB * kTileItems;
  long long tot = 0, pre = 0, tot2 = 0, pre2 = 0;
  for (int i = t; i < num_tiles; i += kGB) {
    const int v = tile_cnt[i];
    tot += v;
    pre += i < c0 ? v : 0;
    if (lazy) {
      const int v2 = tile_cnt2[i];
      tot2 += v2;
      pre2 += i < c0 ? v2 : 0;
    }
  }
  long long total, prefix;
  block_scan64(tot, warp_sum, &total);
  block_scan64(pre, warp_sum, &prefix);
  // a rebuild whose widened lists overflow lists the tight rectangles instead
  // (the same decision in every tile CTA: the totals are global)
  bool tight = false;
  if (lazy) {
    long long total2, prefix2;
    block_scan64(tot2, warp_sum, &total2);
    block_scan64(pre2, warp_sum, &prefix2);
    tight = total > max_entries && total2 <= max_entries;
    if (tight) {
      total = total2;
      prefix = prefix2;
      tile_cnt = const_cast<int*>(tile_cnt2);
    }
  }
  const bool over = total > max_entries;
  if (t < kBuckets) s_hist[t] = 0;
  __syncthreads();
  {
    const int base = c0 + t * kTileItems;
    int c[kTileItems];
    long long v = 0;
#pragma unroll
    for (int k = 0; k < kTileItems; k++) {
      c[k] = base + k < num_tiles ? tile_cnt[base + k] : 0;
      v += c[k];
    }
    long long chunk;
    long long run = prefix + block_scan64(v, warp_sum, &chunk);
    int cls[kTileItems], r[kTileItems];
#pragma unroll
    for (int k = 0; k < kTileItems; k++) {
      const int i = base + k;
      cls[k] = length_class(over ? 0 : c[k]);
      r[k] = 0;
      if (i < num_tiles) {
        const int s = over ? 0 : (int)run;
        // an empty tile's range is (0, 0) wherever it sits in the list
        ranges[i] = (over || c[k] == 0) ? make_int2(0, 0) : make_int2(s, s + c[k]);
        cursor[i] = s;
        r[k] = atomicAdd(&s_hist[cls[k]], 1);
      }
      run += c[k];
    }
    __syncthreads();
    // this block's first rank in each class
    if (t < kBuckets) s_base[t] = s_hist[t] ? atomicAdd(&bucket[t], s_hist[t]) : 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTileItems; k++)
      if (base + k < num_tiles)
        rank[base + k] = ((uint32_t)cls[k] << 28) | (uint32_t)(s_base[cls[k]] + r[k]);
  }
  if (tb == 0 && t == 0) {
    hdr->entries_raw = total;
    hdr->n_entries = over ? 0 : (int)total;
    if (over) atomicCAS(&hdr->status, 0, (int)GS2D_ERR_CAPACITY);
    if (nbg == 0) count[n] = 0;
    hdr->long_count = 0;
    hdr->lists_tight = tight ? 1 : 0;
  }
}

// Scatter: every entry claims the next slot of its tile's list.  A warp takes
// 32 Gaussians, flattens their entries, and each lane keeps kInFlight atomics
// in flight before it stores the claimed slots.
constexpr int kInFlight = 4;

__global__ void __launch_bounds__(kGB)
k_bin_scatter(int n, const int4* __restrict__ tight_rect, int4* __restrict__ lrect,
              const WsHeader* __restrict__ hdr, int* __restrict__ cursor,
              uint32_t* __restrict__ list, int lazy) {
  pdl_begin();
  __shared__ int s_start[kGB / 32][33];
  if (hdr->entries_raw != (int64_t)hdr->n_entries) return;  // over capacity
  if (lazy && hdr->lists_valid) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g_base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31;
  const int g = g_base + lane;
  // the rectangles listed: widened ones, or the tight ones (eager binning, or
  // a rebuild whose widened lists overflowed: they become the listed ones)
  const bool use_tight = !lazy || hdr->lists_tight;
  const int4* __restrict__ rect = use_tight ? tight_rect : (const int4*)lrect;
  const int4 rc = g < n ? rect[g] : make_int4(0, 0, 0, 0);
  if (lazy && use_tight && g < n) lrect[g] = rc;
  const int cnt = rc.z * rc.w;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  int* start = s_start[wid];
  start[lane] = incl - cnt;
  const int T = __shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();
  for (int e0 = 0; e0 < T; e0 += 32 * kInFlight) {
    int pos[kInFlight];
    uint32_t gi[kInFlight];
#pragma unroll
    for (int u = 0; u < kInFlight; u++) {
      const int e = e0 + u * 32 + lane;
      pos[u] = -1;
      if (e < T) {
        // owner: the last lane whose start is <= e (binary search over 32)
        // (starts are non-decreasing; 16 + 8 + 4 + 2 + 1 keeps lo + step <= 31)
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (start[lo + step] <= e) lo += step;
        gi[u] = (uint32_t)(g_base + lo);
        const int4 ro = rect[g_base + lo];
        const int j = e - start[lo];
        const int dy = j / ro.z;
        pos[u] = atomicAdd(&cursor[ro.x + dy * ro.y + (j - dy * ro.z)], 1);
      }
    }
#pragma unroll
    for (int u = 0; u < kInFlight; u++)
      if (pos[u] >= 0) list[pos[u]] = gi[u];
  }
}

// Bitonic sort of up to 32 K keys held by one warp, K per lane in blocked
// order (element e = lane * K + r).  Exchange distances j >= K pair lanes
// (shuffles), distances j < K pair registers of the same lane.
template <int K>
__device__ __forceinline__ void warp_bitonic(uint32_t (&v)[K], int lane) {
#pragma unroll
  for (int k = 2; k <= 32 * K; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= K) {
        const int lj = j / K;
        const bool lower = (lane & lj) == 0;
#pragma unroll
        for (int r = 0; r < K; r++) {
          const uint32_t w = __shfl_xor_sync(0xffffffffu, v[r], lj);
          const bool asc = ((lane * K + r) & k) == 0;
          v[r] = (lower == asc) ? min(v[r], w) : max(v[r], w);
        }
      } else {
#pragma unroll
        for (int r = 0; r < K; r++) {
          const int p = r ^ j;
          if (p > r) {
            const bool asc = ((lane * K + r) & k) == 0;
            const uint32_t a = v[r], b = v[p];
            if ((a > b) == asc) {
              v[r] = b;
              v[p] = a;
            }
          }
        }
      }
    }
  }
}

template <int K>
__device__ __forceinline__ void warp_sort_list(uint32_t* __restrict__ seg, int len, int lane) {
  uint32_t v[K];
#pragma unroll
  for (int r = 0; r < K; r++) {
    const int e = lane * K + r;
    v[r] = e < len ? seg[e] : 0xffffffffu;
  }
  warp_bitonic<K>(v, lane);
#pragma unroll
  for (int r = 0; r < K; r++) {
    const int e = lane * K + r;
    if (e < len) seg[e] = v[r];
  }
}

// Segment sort: one warp per tile, bitonic network in registers for lists of
// up to 512; longer lists are queued for k_sort_long.  Also resets the tile's
// entry counter for the next binning (its last reader, the scan, is done) and
// places the tile in the render queue: after all tiles of longer classes, at
// the next free position of its class.
__global__ void __launch_bounds__(256)
k_sort_short(int num_tiles, const int2* __restrict__ ranges, uint32_t* __restrict__ list,
             int* __restrict__ long_tiles, int* __restrict__ tile_cnt,
             const int* __restrict__ bucket, const uint32_t* __restrict__ rank,
             int* __restrict__ order, WsHeader* __restrict__ hdr, int lazy,
             int* __restrict__ tile_cnt2) {
  pdl_begin();
  if (lazy && hdr->lists_valid) return;
  const int lane = threadIdx.x & 31;
  const int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (tile >= num_tiles) return;
  const int2 rg = ranges[tile];
  const int len = rg.y - rg.x;
  {
    // queue position: the tiles of all longer classes, then the rank in its own
    const uint32_t rk = rank[tile];
    const int cls = (int)(rk >> 28);
    int x = lane < kBuckets && lane > cls ? bucket[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) {
      tile_cnt[tile] = 0;
      if (lazy) tile_cnt2[tile] = 0;
      const int q = x + (int)(rk & 0x0fffffffu);
      if (q < num_tiles)
        order[q] = tile;
      else
        set_status(hdr, GS2D_ERR_BOUNDS);  // class sizes out of step with the ranks
    }
  }
  uint32_t* seg = list + rg.x;
  if (len <= 1) return;
  if (len <= 32)
    warp_sort_list<1>(seg, len, lane);
  else if (len <= 64)
    warp_sort_list<2>(seg, len, lane);
  else if (len <= 128)
    warp_sort_list<4>(seg, len, lane);
  else if (len <= 256)
    warp_sort_list<8>(seg, len, lane);
  else if (len <= 512)
    warp_sort_list<16>(seg, len, lane);
  else if (lane == 0)
    long_tiles[atomicAdd(&hdr->long_count, 1)] = tile;
}

// Segment sort, long lists: one CTA per queued tile, bitonic network in shared
// memory over the list padded to a power of two.  A list longer than kLongMax
// is reported as over capacity: its tile is emptied and the entry count is
// zeroed so that no gradient is reduced from this binning.
__global__ void __launch_bounds__(1024)
k_sort_long(int2* __restrict__ ranges, uint32_t* __restrict__ list,
            const int* __restrict__ long_tiles, int* __restrict__ bucket,
            WsHeader* __restrict__ hdr, int lazy) {
  pdl_begin();
  extern __shared__ uint32_t s_keys[];
  if (lazy && hdr->lists_valid) return;
  const int t = threadIdx.x;
  // the queue classes were last read by k_sort_short: clear them for the next binning
  if (blockIdx.x == 0 && t < 2 * kBuckets) bucket[t] = 0;
  const int count = hdr->long_count;
  for (int q = blockIdx.x; q < count; q += gridDim.x) {
    const int tile = long_tiles[q];
    const int2 rg = ranges[tile];
    const int len = rg.y - rg.x;
    if (len > kLongMax) {
      if (t == 0) {
        atomicCAS(&hdr->status, 0, (int)GS2D_ERR_CAPACITY);
        hdr->n_entries = 0;
        ranges[tile] = make_int2(rg.x, rg.x);
      }
      continue;
    }
    int P = 64;
    while (P < len) P <<= 1;
    __syncthreads();
    for (int i = t; i < P; i += blockDim.x) s_keys[i] = i < len ? list[rg.x + i] : 0xffffffffu;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = t; i < P; i += blockDim.x) {
          const int p = i ^ j;
          if (p > i) {
            const uint32_t a = s_keys[i], b = s_keys[p];
            const bool asc = (i & k) == 0;
            if ((a > b) == asc) {
              s_keys[i] = b;
              s_keys[p] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int i = t; i < len; i += blockDim.x) list[rg.x + i] = s_keys[i];
  }
}

// ---------------------------------------------------------------------------
// Every kernel of the chain starts with pdl_begin() and is launched with
// launch_pdl: each one's blocks become resident while its predecessor drains.
cudaError_t launch_project(const gs2d_plan& p, void* ws, const float* params, cudaStream_t s) {
  if (p.n == 0) return cudaSuccess;
  return launch_pdl(k_project, (p.n + kGB - 1) / kGB, kGB, 0, s, p.n, clip_set(p, ws),
                    tile_shift_of(p.tile), p.cfg.sigma_cut, p.cfg.alpha_min, p.cfg.det_eps,
                    params, ws_ptr<float4>(ws, p, kOffRec), ws_ptr<int4>(ws, p, kOffRect),
                    ws_ptr<int>(ws, p, kOffCount));
}

cudaError_t prime_binning() {
  return opt_in_smem((const void*)k_sort_long, kLongMax * (int)sizeof(uint32_t));
}

// Scans, scatter and segment sorts (everything after the counts); `lists`:
// the rectangles the lists are built from; with `lazy` the tile part returns
// at once while hdr->lists_valid is set.
static cudaError_t launch_bin_rest(const gs2d_plan& p, void* ws, cudaStream_t s, int lazy) {
  WsHeader* hdr = ws_ptr<WsHeader>(ws, p, kOffHeader);
  int* count = ws_ptr<int>(ws, p, kOffCount);
  int* tile_cnt = ws_ptr<int>(ws, p, kOffTileCnt);
  int* cursor = ws_ptr<int>(ws, p, kOffCursor);
  int* long_tiles = ws_ptr<int>(ws, p, kOffLong);
  uint32_t* list = ws_ptr<uint32_t>(ws, p, kOffList);
  int2* ranges = ws_ptr<int2>(ws, p, kOffRanges);
  int* bucket = ws_ptr<int>(ws, p, kOffBucket);
  int* order = ws_ptr<int>(ws, p, kOffOrder);
  uint32_t* rank = ws_ptr<uint32_t>(ws, p, kOffRank);
  int* tile_cnt2 = ws_ptr<int>(ws, p, kOffTileCnt2);
  const int nbg = (p.n + kGB - 1) / kGB;
  const int nbt = (p.num_tiles + kGB * kTileItems - 1) / (kGB * kTileItems);
  cudaError_t e = prime_binning();
  if (e == cudaSuccess)
    e = launch_pdl(k_bin_scan, nbg + nbt, kGB, 0, s, p.n, nbg, p.num_tiles, p.max_entries, count,
                   ws_ptr<long long>(ws, p, kOffBlockSum), tile_cnt, cursor, ranges, bucket,
                   rank, hdr, lazy, (const int*)tile_cnt2);
  if (e == cudaSuccess && p.n > 0)
    e = launch_pdl(k_bin_scatter, nbg, kGB, 0, s, p.n, (const int4*)ws_ptr<int4>(ws, p, kOffRect),
                   ws_ptr<int4>(ws, p, kOffLRect), hdr, cursor, list, lazy);
  if (e == cudaSuccess)
    e = launch_pdl(k_sort_short, (p.num_tiles + 7) / 8, 256, 0, s, p.num_tiles, ranges, list,
                   long_tiles, tile_cnt, bucket, rank, order, hdr, lazy, tile_cnt2);
  if (e == cudaSuccess)
    e = launch_pdl(k_sort_long, 152, 1024, kLongMax * sizeof(uint32_t), s, ranges, list,
                   long_tiles, bucket, hdr, lazy);
  return e;
}

cudaError_t launch_bin_sort(const gs2d_plan& p, void* ws, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (p.n > 0)
    e = launch_pdl(k_count_tiles, (p.n + kGB - 1) / kGB, kGB, 0, s, p.n,
                   ws_ptr<int4>(ws, p, kOffRect), ws_ptr<int>(ws, p, kOffCount),
                   ws_ptr<int>(ws, p, kOffTileCnt), ws_ptr<long long>(ws, p, kOffBlockSum),
                   ws_ptr<WsHeader>(ws, p, kOffHeader));
  if (e != cudaSuccess) return e;
  return launch_bin_rest(p, ws, s, 0);
}

cudaError_t launch_prepare(const gs2d_plan& p, void* ws, const float* params, bool adam_tick,
                           cudaStream_t s) {
  const int blocks = (p.n + kGB - 1) / kGB;
  const cudaError_t e = launch_pdl(
      k_project_count, blocks > 0 ? blocks : 1, kGB, 0, s, p.n, clip_set(p, ws),
      tile_shift_of(p.tile), p.cfg.sigma_cut, p.cfg.alpha_min, p.cfg.det_eps, params,
      ws_ptr<float4>(ws, p, kOffRec), ws_ptr<int4>(ws, p, kOffRect), ws_ptr<int>(ws, p, kOffCount),
      ws_ptr<int>(ws, p, kOffTileCnt), ws_ptr<long long>(ws, p, kOffBlockSum),
      ws_ptr<WsHeader>(ws, p, kOffHeader), adam_tick ? 1 : 0, p.cfg.beta1, p.cfg.beta2, p.cfg.lr,
      p.cfg.lr_decay);
  if (e != cudaSuccess) return e;
  return launch_bin_rest(p, ws, s, 0);
}

cudaError_t launch_prepare_fit(const gs2d_plan& p, void* ws, const float* params,
                               cudaStream_t s) {
  if (!fit_lists_retained(p.cfg)) return launch_prepare(p, ws, params, true, s);
  const int blocks = (p.n + kGB - 1) / kGB;
  WsHeader* hdr = ws_ptr<WsHeader>(ws, p, kOffHeader);
  int4* lrect = ws_ptr<int4>(ws, p, kOffLRect);
  const ClipSet cs = clip_set(p, ws);
  const int shift = tile_shift_of(p.tile);
  cudaError_t e = launch_pdl(
      k_project_fit, blocks > 0 ? blocks : 1, kGB, 0, s, p.n, cs, shift, p.cfg.sigma_cut,
      p.cfg.alpha_min, p.cfg.det_eps, params, ws_ptr<float4>(ws, p, kOffRec),
      ws_ptr<int4>(ws, p, kOffRect), ws_ptr<int>(ws, p, kOffCount),
      ws_ptr<long long>(ws, p, kOffBlockSum), (const int4*)lrect, hdr, p.cfg.beta1, p.cfg.beta2,
      p.cfg.lr, p.cfg.lr_decay);
  if (e == cudaSuccess)
    e = launch_pdl(k_rebin_count, blocks > 0 ? blocks : 1, kGB, 0, s, p.n, cs, shift,
                   p.cfg.sigma_cut, p.cfg.alpha_min, p.cfg.det_eps, p.cfg.bin_margin, params,
                   (const int4*)ws_ptr<int4>(ws, p, kOffRect), lrect,
                   ws_ptr<int>(ws, p, kOffTileCnt), ws_ptr<int>(ws, p, kOffTileCnt2), hdr);
  if (e != cudaSuccess) return e;
  return launch_bin_rest(p, ws, s, 1);
}

}  // namespace gs2d
