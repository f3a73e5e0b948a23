// Projection, tile binning and the stable LSD radix sort by tile id.
//
// The method renders with the tile-based rasterizer it inherits (Sec. 3,
// "differentiable tile-based rasterization"); in 2D there is no depth
// (Sec. 3.1, accumulated-sum blending), so within a tile the Gaussians are
// ordered by index.  Emission writes the entries of Gaussian n before those of
// n + 1, so a stable sort by tile id alone yields the (tile, n) order.
#include "gs2d_internal.cuh"

namespace gs2d {

// ---------------------------------------------------------------------------
// Projection: one thread per Gaussian.  The tile rectangle uses only
// single-rounded operations (no FMA contraction) so it is reproducible on the
// host; the rest of the record is ordinary FP32.
__global__ void __launch_bounds__(256)
k_project(int n, int W, int H, int TX, int num_tiles, float sigma_cut, float alpha_min,
          float det_eps, const float* __restrict__ params, float4* __restrict__ rec,
          int4* __restrict__ rect, int* __restrict__ count, int2* __restrict__ ranges) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < num_tiles) ranges[i] = make_int2(0, 0);
  if (i == 0) count[n] = 0;
  if (i >= n) return;
  const float mx = params[i], my = params[n + i];
  const float l1 = params[2 * n + i], l2 = params[3 * n + i], l3 = params[4 * n + i];
  const float cr = params[5 * n + i], cg = params[6 * n + i], cb = params[7 * n + i];
  const float w = params[8 * n + i];
  int4 rc = make_int4(0, 0, 0, 0);
  int cnt = 0;
  const bool finite = isfinite(mx) && isfinite(my) && isfinite(l1) && isfinite(l2) &&
                      isfinite(l3) && isfinite(cr) && isfinite(cg) && isfinite(cb) && isfinite(w);
  // --- bit-reproducible binning arithmetic ---
  const float sxx = __fmul_rn(l1, l1);
  const float syy = __fadd_rn(__fmul_rn(l2, l2), __fmul_rn(l3, l3));
  const float a = __fmul_rn(l1, l3);
  const float det = __fmul_rn(a, a);
  bool live = finite && (det > det_eps) && (fabsf(w) >= alpha_min);
  if (live) {
    const float mid = __fmul_rn(0.5f, __fadd_rn(sxx, syy));
    float disc = __fsub_rn(__fmul_rn(mid, mid), det);
    if (!(disc > 0.1f)) disc = 0.1f;
    const float lam = __fadd_rn(mid, __fsqrt_rn(disc));
    const float r = ceilf(__fmul_rn(3.0f, __fsqrt_rn(lam)));
    float fx0 = floorf(__fsub_rn(mx, r)), fx1 = floorf(__fadd_rn(mx, r));
    float fy0 = floorf(__fsub_rn(my, r)), fy1 = floorf(__fadd_rn(my, r));
    fx0 = fx0 < 0.0f ? 0.0f : fx0;
    fy0 = fy0 < 0.0f ? 0.0f : fy0;
    fx1 = fx1 > (float)(W - 1) ? (float)(W - 1) : fx1;
    fy1 = fy1 > (float)(H - 1) ? (float)(H - 1) : fy1;
    if (fx0 <= fx1 && fy0 <= fy1) {
      rc = make_int4((int)fx0 / kTile, (int)fy0 / kTile, (int)fx1 / kTile + 1, (int)fy1 / kTile + 1);
      cnt = (rc.z - rc.x) * (rc.w - rc.y);
    }
  }
  rect[i] = rc;
  count[i] = cnt;
  // --- render record ---
  float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
  if (cnt > 0) {
    const float s = 0.84932180028801904272f;  // sqrt(log2(e) / 2)
    const float log2e = 1.44269504088896340736f;
    float tau2 = fminf(sigma_cut * log2e, log2f(fabsf(w) / alpha_min));
    tau2 = fmaxf(tau2, 0.0f);
    const float tau = tau2 * kLn2;
    // half extents of {sigma <= tau}: sqrt(2 tau Sxx), sqrt(2 tau Syy), padded so
    // the box stays conservative under FP32 rounding
    const float hx = sqrtf(2.0f * tau * sxx) * 1.001f + 0.0039f;
    const float hy = sqrtf(2.0f * tau * syy) * 1.001f + 0.0039f;
    r0 = make_float4(mx, my, s / l1, s / l3);
    r1 = make_float4(-l2 / l3, tau2, w * cr, w * cg);
    r2 = make_float4(w * cb, hx, hy, 0.0f);
  }
  rec[i] = r0;
  rec[n + i] = r1;
  rec[2 * n + i] = r2;
}

// ---------------------------------------------------------------------------
// Exclusive scan of the tile counts (reduce -> scan block sums -> scan blocks).
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) s_warp[lane] = t;
  }
  __syncthreads();
  const int warp_prefix = wid > 0 ? s_warp[wid - 1] : 0;
  if (total) *total = s_warp[nw - 1];
  const int excl = warp_prefix + x - v;
  __syncthreads();
  return excl;
}

// Block totals are summed in 64 bits: a pathological input (many Gaussians
// covering every tile) must be reported as over capacity, never wrap around.
__device__ __forceinline__ long long block_sum64(long long v, long long* s_warp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s_warp[wid] = v;
  __syncthreads();
  long long t = 0;
  for (int w = 0; w < nw; w++) t += s_warp[w];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(int n, const int* __restrict__ count, long long* __restrict__ block_sum) {
  __shared__ long long s_warp[32];
  const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanItems;
  long long v = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) v += (base + k < n) ? count[base + k] : 0;
  const long long total = block_sum64(v, s_warp);
  if (threadIdx.x == 0) block_sum[blockIdx.x] = total;
}

// Single thread block, sequential over the block sums (there are n / 8192 of
// them): exclusive prefix in 64 bits and the capacity check.  Offsets are only
// used when the total fits max_entries (< 2^30), so they fit 32 bits then.
__global__ void __launch_bounds__(32)
k_scan_top(int nblocks, int n, int64_t max_entries, long long* __restrict__ block_sum,
           int* __restrict__ count, WsHeader* __restrict__ hdr) {
  if (threadIdx.x != 0) return;
  long long carry = 0;
  for (int b = 0; b < nblocks; b++) {
    const long long v = block_sum[b];
    block_sum[b] = carry;
    carry += v;
  }
  const int64_t tot = carry;
  hdr->entries_raw = tot;
  if (tot > max_entries) {
    hdr->n_entries = 0;
    atomicCAS(&hdr->status, 0, (int)GS2D_ERR_CAPACITY);
  } else {
    hdr->n_entries = (int)tot;
  }
  count[n] = (int)(tot > max_entries ? max_entries : tot);
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_down(int n, int* __restrict__ count, const long long* __restrict__ block_sum) {
  __shared__ int s_warp[32];
  const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanItems;
  int c[kScanItems];
  int v = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    c[k] = (base + k < n) ? count[base + k] : 0;
    v += c[k];
  }
  // wraps harmlessly when over capacity (the offsets are then unused)
  int run = (int)((unsigned)block_exclusive_scan(v, s_warp, nullptr) +
                  (unsigned)block_sum[blockIdx.x]);
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    if (base + k < n) count[base + k] = run;
    run += c[k];
  }
}

// ---------------------------------------------------------------------------
// Emission: Gaussian i writes its entries at [offset_i, offset_{i+1}) in
// row-major tile order.  Nothing is written when over capacity.
__global__ void __launch_bounds__(256)
k_emit(int n, int TX, const int4* __restrict__ rect, const int* __restrict__ offs,
       const WsHeader* __restrict__ hdr, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (hdr->n_entries == 0) return;
  const int4 rc = rect[i];
  int o = offs[i];
  for (int ty = rc.y; ty < rc.w; ty++)
    for (int tx = rc.x; tx < rc.z; tx++) {
      keys[o] = (uint32_t)(ty * TX + tx);
      vals[o] = (uint32_t)i;
      o++;
    }
}

// ---------------------------------------------------------------------------
// LSD radix sort by tile id, 8-bit digits, stable.  nb CTAs; CTA b owns the
// chunk [b*C, min(E, (b+1)*C)), C = ceil(E / nb), with E read on the device.
__device__ __forceinline__ void chunk_of(int E, int nb, int b, int* lo, int* hi) {
  const int C = (E + nb - 1) / nb;
  const long long l = (long long)b * C;
  const long long h = l + C;
  *lo = (int)(l < E ? l : E);
  *hi = (int)(h < E ? h : E);
}

__global__ void __launch_bounds__(kSortThreads)
k_radix_upsweep(const uint32_t* __restrict__ keys, const WsHeader* __restrict__ hdr, int nb,
                int shift, uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_cnt[kRadixBuckets];
  for (int d = threadIdx.x; d < kRadixBuckets; d += blockDim.x) s_cnt[d] = 0;
  __syncthreads();
  int lo, hi;
  chunk_of(hdr->n_entries, nb, blockIdx.x, &lo, &hi);
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
    atomicAdd(&s_cnt[(keys[i] >> shift) & (kRadixBuckets - 1)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadixBuckets; d += blockDim.x)
    hist[d * nb + blockIdx.x] = s_cnt[d];
}

// Single block: exclusive scan of hist in digit-major order.
__global__ void __launch_bounds__(kScanThreads)
k_radix_scan(int total, uint32_t* __restrict__ hist) {
  __shared__ int s_warp[32];
  __shared__ uint32_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  constexpr int kItems = 4;
  for (int b0 = 0; b0 < total; b0 += kScanThreads * kItems) {
    const int base = b0 + threadIdx.x * kItems;
    uint32_t c[kItems];
    int v = 0;
#pragma unroll
    for (int k = 0; k < kItems; k++) {
      c[k] = base + k < total ? hist[base + k] : 0u;
      v += (int)c[k];
    }
    int tot;
    uint32_t run = (uint32_t)block_exclusive_scan(v, s_warp, &tot) + s_carry;
#pragma unroll
    for (int k = 0; k < kItems; k++) {
      if (base + k < total) hist[base + k] = run;
      run += c[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry += (uint32_t)tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSortThreads)
k_radix_downsweep(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                  uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                  const WsHeader* __restrict__ hdr, int nb, int shift,
                  const uint32_t* __restrict__ hist) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint32_t s_base[kRadixBuckets];
  __shared__ uint32_t s_wc[kWarps][kRadixBuckets];
  __shared__ uint32_t s_round[kRadixBuckets];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  static_assert(kSortThreads == kRadixBuckets, "one thread per digit");
  s_base[tid] = hist[tid * nb + blockIdx.x];
  int lo, hi;
  chunk_of(hdr->n_entries, nb, blockIdx.x, &lo, &hi);
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int start = lo; start < hi; start += kSortThreads) {
    const int idx = start + tid;
    const bool valid = idx < hi;
    const uint32_t key = valid ? keys_in[idx] : 0u;
    const uint32_t val = valid ? vals_in[idx] : 0u;
    const uint32_t d = valid ? ((key >> shift) & (kRadixBuckets - 1)) : (uint32_t)kRadixBuckets;
#pragma unroll
    for (int w = 0; w < kWarps; w++) s_wc[w][tid] = 0;
    __syncthreads();
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt_mask);
    if (valid && rank == 0) s_wc[wid][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kWarps; w++) {
        const uint32_t c = s_wc[w][tid];
        s_wc[w][tid] = run;
        run += c;
      }
      s_round[tid] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = s_base[d] + s_wc[wid][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
    __syncthreads();
    s_base[tid] += s_round[tid];
    __syncthreads();
  }
}

// Per-tile [start, end) of the sorted list.
__global__ void __launch_bounds__(256)
k_ranges(const uint32_t* __restrict__ keys, const WsHeader* __restrict__ hdr,
         int2* __restrict__ ranges) {
  const int E = hdr->n_entries;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < E; i += gridDim.x * blockDim.x) {
    const uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = i;
    if (i == E - 1 || keys[i + 1] != t) ranges[t].y = i + 1;
  }
}

// ---------------------------------------------------------------------------
cudaError_t launch_project(const gs2d_plan& p, void* ws, const float* params, cudaStream_t s) {
  const int work = p.n > p.num_tiles ? p.n : p.num_tiles;
  const int blocks = (work + 255) / 256;
  k_project<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(
      p.n, p.width, p.height, p.tiles_x, p.num_tiles, p.cfg.sigma_cut, p.cfg.alpha_min,
      p.cfg.det_eps, params, ws_ptr<float4>(ws, p, kOffRec), ws_ptr<int4>(ws, p, kOffRect),
      ws_ptr<int>(ws, p, kOffCount), ws_ptr<int2>(ws, p, kOffRanges));
  return cudaGetLastError();
}

cudaError_t launch_bin_sort(const gs2d_plan& p, void* ws, cudaStream_t s) {
  WsHeader* hdr = ws_ptr<WsHeader>(ws, p, kOffHeader);
  int* count = ws_ptr<int>(ws, p, kOffCount);
  long long* bsum = ws_ptr<long long>(ws, p, kOffBlockSum);
  const int nblocks = (p.n + kScanChunk - 1) / kScanChunk;
  if (nblocks > 0) k_scan_reduce<<<nblocks, kScanThreads, 0, s>>>(p.n, count, bsum);
  k_scan_top<<<1, 32, 0, s>>>(nblocks, p.n, p.max_entries, bsum, count, hdr);
  if (nblocks > 0) k_scan_down<<<nblocks, kScanThreads, 0, s>>>(p.n, count, bsum);
  uint32_t* ka = ws_ptr<uint32_t>(ws, p, kOffKeysA);
  uint32_t* kb = ws_ptr<uint32_t>(ws, p, kOffKeysB);
  uint32_t* va = ws_ptr<uint32_t>(ws, p, kOffValsA);
  uint32_t* vb = ws_ptr<uint32_t>(ws, p, kOffValsB);
  if (p.n > 0)
    k_emit<<<(p.n + 255) / 256, 256, 0, s>>>(p.n, p.tiles_x, ws_ptr<int4>(ws, p, kOffRect), count,
                                             hdr, ka, va);
  uint32_t* hist = ws_ptr<uint32_t>(ws, p, kOffHist);
  const int nb = p.sort_blocks;
  for (int pass = 0; pass < p.sort_passes; pass++) {
    const int shift = pass * kRadixBits;
    const uint32_t* kin = (pass & 1) ? kb : ka;
    const uint32_t* vin = (pass & 1) ? vb : va;
    uint32_t* kout = (pass & 1) ? ka : kb;
    uint32_t* vout = (pass & 1) ? va : vb;
    k_radix_upsweep<<<nb, kSortThreads, 0, s>>>(kin, hdr, nb, shift, hist);
    k_radix_scan<<<1, kScanThreads, 0, s>>>(kRadixBuckets * nb, hist);
    k_radix_downsweep<<<nb, kSortThreads, 0, s>>>(kin, vin, kout, vout, hdr, nb, shift, hist);
  }
  const uint32_t* sorted = (p.sort_passes & 1) ? kb : ka;
  k_ranges<<<4 * 152, 256, 0, s>>>(sorted, hdr, ws_ptr<int2>(ws, p, kOffRanges));
  return cudaGetLastError();
}

}  // namespace gs2d
