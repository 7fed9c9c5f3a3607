// Tile binning and depth sort ("tile-based", "depth-sorted" rasterization, Sec.
// "Preliminary" of the paper).
//
// Result: for every global tile, the visible records whose footprint ellipse (where
// alpha can reach the 1/255 floor, with a 0.2% margin) meets the tile's box of pixel
// centres, ordered by (FP32 depth bits, record index), concatenated tile after tile.
// Candidate tiles are those under the footprint's bounding box (gs_project's rect);
// the exact ellipse-box test (tile_hit) removes the rest.
//
// Instead of one wide radix sort on (tile << 32 | depth) keys over all duplicates,
// the order is built in two stable stages that give the same permutation:
//   1. the visible records (one entry each) are compacted in record order and
//      sorted by their 32-bit depth key (stable LSD radix sort, 4 x 8-bit passes);
//   2. every record, taken in depth order, emits one entry per tile its footprint
//      meets, and the entries are stably sorted by tile id alone. The first LSD
//      digit of that sort (the low FB bits of the tile id) is fused into the
//      emission: a counting pass histograms each warp batch's hits by that digit,
//      a scan turns the (digit, batch) counts into cursors, and the emitting pass
//      writes every entry straight to its digit-partitioned position. The remaining
//      high bits take ceil((bits - FB) / 8) ordinary passes (none when the tile id
//      has at most 8 bits).
// A stable sort by tile of a depth-ordered sequence is ordered by (tile, depth,
// record). Stage 2 moves 8 bytes per duplicate per pass instead of 12 bytes per
// pass for 5-6 passes.
//
// Every count is read from device memory (no host round trip), so the whole
// sequence can be captured into a CUDA graph. All grids are fixed-size and every
// block derives its share of the work from the device-side count.
#include "gs_common.cuh"
#include "scan.cuh"

namespace gs {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;  // 2048 keys per tile
constexpr int kRsBins = 256;

// ------------------------------------------------------------------ LSD radix sort pass
// Digit histograms per block (digit-major: hist[d * G + b]).
__global__ void __launch_bounds__(kRsThreads) rs_upsweep_kernel(const uint32_t *__restrict__ keys,
                                                                const uint32_t *d_n, const uint32_t *d_skip,
                                                                int shift, uint32_t mask, uint32_t *hist) {
  __shared__ uint32_t h[kRsWarps][kRsBins];
  const int G = gridDim.x;
  const uint64_t n = (d_skip && *d_skip) ? 0 : *d_n;
  uint64_t begin, end;
  chunk_of(n, G, kRsTile, begin, end);
  const int warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRsWarps * kRsBins; d += kRsThreads) (&h[0][0])[d] = 0;
  __syncthreads();
  uint64_t i = begin + 4 * threadIdx.x;
  for (; i + 3 < end; i += 4 * kRsThreads) {
    const uint4 k = *reinterpret_cast<const uint4 *>(keys + i);
    atomicAdd(&h[warp][(k.x >> shift) & mask], 1u);
    atomicAdd(&h[warp][(k.y >> shift) & mask], 1u);
    atomicAdd(&h[warp][(k.z >> shift) & mask], 1u);
    atomicAdd(&h[warp][(k.w >> shift) & mask], 1u);
  }
  for (; i < end; ++i) atomicAdd(&h[warp][(keys[i] >> shift) & mask], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kRsBins; d += kRsThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) s += h[w][d];
    hist[(uint64_t)d * G + blockIdx.x] = s;
  }
}

// Per-digit exclusive scan of the digit-major histogram hist[256][G] over blocks,
// in place: one warp per digit (grid of 256 warps), so every row is read and
// written coalesced and all rows proceed in parallel; the digit total goes to
// totals[d]. The digit bases (exclusive scan of totals) are added by the downsweep.
__global__ void __launch_bounds__(32) rs_scan_kernel(uint32_t *hist, int G, uint32_t *totals,
                                                      const uint32_t *d_skip) {
  if (d_skip && *d_skip) return;
  const int lane = threadIdx.x, d = blockIdx.x;
  uint32_t *row = hist + (size_t)d * G;
  uint32_t carry = 0;
  for (int b0 = 0; b0 < G; b0 += 32) {
    const int b = b0 + lane;
    const uint32_t x = b < G ? row[b] : 0u;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (b < G) row[b] = carry + incl - x;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) totals[d] = carry;
}

// Stable scatter. Each warp ranks a contiguous slice of the tile, 32 keys per
// step in order; slices are then offset by the warps before them, staged in shared
// memory in digit order and written out coalesced. Ranking within a step: for
// digits of NB <= 6 bits (BITS = NB), the peers of a key are the AND of NB
// ballots (one per digit bit) and lane l keeps the running counts of digits l and
// l + 32 in registers; wider digits (BITS = 0) use __match_any_sync and a per-warp
// shared-memory count.
template <int BITS>
__global__ void __launch_bounds__(kRsThreads, 4) rs_downsweep_kernel(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, uint32_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, const uint32_t *d_n, const uint32_t *d_skip, int shift, uint32_t mask,
    const uint32_t *__restrict__ hist, const uint32_t *__restrict__ totals) {
  static_assert(BITS >= 0 && BITS <= 6, "ballot ranking covers digits of at most 6 bits");
  constexpr int kSlots = BITS == 0 ? 0 : ((1 << BITS) + 31) / 32;
  __shared__ uint32_t s_keys[kRsTile];
  __shared__ uint32_t s_vals[kRsTile];
  __shared__ uint32_t s_whist[kRsWarps][kRsBins + 1];
  __shared__ uint32_t s_goff[kRsBins];
  __shared__ uint32_t s_tstart[kRsBins + 1];
  const int G = gridDim.x;
  const uint64_t n = (d_skip && *d_skip) ? 0 : *d_n;
  uint64_t begin, end;
  chunk_of(n, G, kRsTile, begin, end);
  if (begin >= end) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    // digit bases: exclusive scan of the digit totals, then this block's column
    uint32_t all;
    const uint32_t dbase = block_exclusive_scan<uint32_t>(totals[threadIdx.x], &all);
    s_goff[threadIdx.x] = dbase + hist[(uint64_t)threadIdx.x * G + blockIdx.x];
  }
  if (BITS > 0) {   // digits >= 2^BITS never occur: zero once
    for (int d = lane; d < kRsBins + 1; d += 32) s_whist[warp][d] = 0;
  }
  const uint32_t lt_mask = lanemask_lt();
  for (uint64_t tb = begin; tb < end; tb += kRsTile) {
    const uint32_t tile_n = (uint32_t)min((uint64_t)kRsTile, end - tb);
    if (BITS == 0) {
      for (int d = lane; d < kRsBins + 1; d += 32) s_whist[warp][d] = 0;
      __syncwarp();
    }
    uint32_t k[kRsItems], v[kRsItems], dig[kRsItems], rank[kRsItems];
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
      const uint32_t li = warp * (32 * kRsItems) + j * 32 + lane;   // warp slice of 32 * kRsItems keys
      const bool valid = li < tile_n;
      k[j] = valid ? keys_in[tb + li] : 0u;
      v[j] = valid ? vals_in[tb + li] : 0u;
      dig[j] = valid ? ((k[j] >> shift) & mask) : (uint32_t)kRsBins;
    }
    if (BITS == 0) {
#pragma unroll
      for (int j = 0; j < kRsItems; ++j) {
        const uint32_t peers = __match_any_sync(0xffffffffu, dig[j]);
        const uint32_t before = __popc(peers & lt_mask);
        const uint32_t base = s_whist[warp][dig[j]];
        __syncwarp();
        rank[j] = base + before;
        if (before == 0) s_whist[warp][dig[j]] = base + __popc(peers);
        __syncwarp();
      }
    } else {
      uint32_t cnt[kSlots > 0 ? kSlots : 1];
#pragma unroll
      for (int q = 0; q < kSlots; ++q) cnt[q] = 0;
#pragma unroll
      for (int j = 0; j < kRsItems; ++j) {
        const uint32_t d = dig[j];
        const uint32_t vm = __ballot_sync(0xffffffffu, d < (uint32_t)kRsBins);
        uint32_t mb[BITS > 0 ? BITS : 1];
        uint32_t peers = vm;
#pragma unroll
        for (int b = 0; b < BITS; ++b) {
          mb[b] = __ballot_sync(0xffffffffu, (d >> b) & 1u);
          peers &= ((d >> b) & 1u) ? mb[b] : ~mb[b];
        }
        uint32_t base = __shfl_sync(0xffffffffu, cnt[0], d & 31u);
        if (kSlots > 1) {
          const uint32_t hi = __shfl_sync(0xffffffffu, cnt[kSlots > 1 ? 1 : 0], d & 31u);
          base = ((d >> 5) & 1u) ? hi : base;
        }
        rank[j] = base + __popc(peers & lt_mask);
#pragma unroll
        for (int q = 0; q < kSlots; ++q) {
          const uint32_t own = lane + 32u * q;   // digit whose count this lane keeps
          uint32_t m = vm;
#pragma unroll
          for (int b = 0; b < BITS; ++b) m &= ((own >> b) & 1u) ? mb[b] : ~mb[b];
          if (own < (1u << BITS)) cnt[q] += __popc(m);
        }
      }
#pragma unroll
      for (int q = 0; q < kSlots; ++q)
        if (lane + 32 * q < (1 << BITS)) s_whist[warp][lane + 32 * q] = cnt[q];
    }
    __syncthreads();
    uint32_t tot = 0;
    for (int d = threadIdx.x; d < kRsBins + 1; d += kRsThreads) {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kRsWarps; ++w) {
        const uint32_t c = s_whist[w][d];
        s_whist[w][d] = run;
        run += c;
      }
      if (d < kRsBins) tot = run;
    }
    uint32_t all;
    const uint32_t start = block_exclusive_scan<uint32_t>(tot, &all);
    s_tstart[threadIdx.x] = start;
    if (threadIdx.x == 0) s_tstart[kRsBins] = all;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
      if (BITS > 0 && dig[j] >= (uint32_t)kRsBins) continue;   // not counted: past the tile's end
      const uint32_t pos = s_tstart[dig[j]] + s_whist[warp][dig[j]] + rank[j];
      s_keys[pos] = k[j];
      s_vals[pos] = v[j];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tile_n; i += kRsThreads) {
      const uint32_t key = s_keys[i];
      const uint32_t d = (key >> shift) & mask;
      const uint32_t gpos = s_goff[d] + (i - s_tstart[d]);
      if (keys_out) keys_out[gpos] = key;
      vals_out[gpos] = s_vals[i];
    }
    __syncthreads();
    s_goff[threadIdx.x] += tot;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ bin/sort functors
struct VisibleCompact {
  const int32_t *radius;
  const float *depth;
  uint64_t n;
  uint32_t *keys, *vals, *n_vis;
  __device__ uint64_t count() const { return n; }
  __device__ uint32_t value(uint64_t i) const { return radius[i] > 0 ? 1u : 0u; }
  __device__ void emit(uint64_t i, uint64_t pre, uint32_t v) const {
    if (v) {
      keys[pre] = __float_as_uint(depth[i]);
      vals[pre] = (uint32_t)i;
    }
  }
  __device__ void total(uint64_t t) const { *n_vis = (uint32_t)t; }
};

// Exclusive scan, in place, of the (digit, batch) hit counts stored digit-major
// (hist[d * NB + b], NB = number of 32-record batches): the result is each batch's
// first output position for each digit. The total is M; above the duplicate
// capacity the frame overflows.
struct HistScan {
  uint32_t *hist;
  const uint32_t *n_vis;
  int fbits;
  uint64_t capacity;
  uint32_t *m_total;          // M (0 on overflow)
  uint32_t *overflow;
  int64_t *d_count;
  int32_t *d_error;
  __device__ uint64_t count() const { return ((uint64_t)(*n_vis) + 31u) / 32u << fbits; }
  __device__ uint32_t value(uint64_t i) const { return hist[i]; }
  __device__ void emit(uint64_t i, uint64_t pre, uint32_t) const {
    if (pre <= 0xffffffffull) hist[i] = (uint32_t)pre;
  }
  __device__ void total(uint64_t t) const {
    *d_count = (int64_t)t;
    const bool over = t > capacity;
    *overflow = over ? 1u : 0u;
    *m_total = over ? 0u : (uint32_t)t;
    if (over && d_error) atomicOr(d_error, (int32_t)GS_ERR_CAPACITY);
  }
};

struct RecordTiles {
  uint32_t x0, y0, w, n;     // candidate rectangle (origin, width, count)
  float u, v, A, beta, gamma, qb, ab, inv_den;
  int W, H, toff, gx;
};

__device__ __forceinline__ RecordTiles record_tiles(const gs_proj_t &P, const gs_camera_t *cams, int n_views,
                                                   int64_t n_per_view, uint32_t r) {
  RecordTiles t;
  const uint2 q = reinterpret_cast<const uint2 *>(P.rect)[r];
  t.x0 = q.x & 0xffffu;
  t.y0 = q.x >> 16;
  const uint32_t x1 = q.y & 0xffffu, y1 = q.y >> 16;
  t.w = x1 > t.x0 ? x1 - t.x0 : 0u;
  t.n = (x1 > t.x0 && y1 > t.y0) ? t.w * (y1 - t.y0) : 0u;
  const float2 m = reinterpret_cast<const float2 *>(P.mean2d)[r];
  const float4 co = reinterpret_cast<const float4 *>(P.conic_opacity)[r];
  t.u = m.x; t.v = m.y; t.A = co.x; t.beta = co.y; t.gamma = co.z;
  t.qb = __fmul_rn(reinterpret_cast<const float4 *>(P.rgb)[r].w, kBinMargin);
  tile_hit_consts(t.A, t.beta, t.gamma, t.ab, t.inv_den);
  const int view = n_views == 1 ? 0 : (int)((int64_t)r / n_per_view);
  t.W = cams[view].width; t.H = cams[view].height; t.toff = cams[view].tile_offset; t.gx = cams[view].grid_x;
  return t;
}

// Candidate c of the record's rectangle: global tile id and whether the footprint
// ellipse meets the tile's box of pixel centres.
__device__ __forceinline__ bool candidate(const RecordTiles &t, uint32_t c, int tw, int th, uint32_t &tile) {
  const uint32_t tx = t.x0 + c % t.w, ty = t.y0 + c / t.w;
  tile = (uint32_t)t.toff + ty * (uint32_t)t.gx + tx;
  const float X0 = (float)(tx * tw) + 0.5f, X1 = (float)min((int)(tx + 1) * tw, t.W) - 0.5f;
  const float Y0 = (float)(ty * th) + 0.5f, Y1 = (float)min((int)(ty + 1) * th, t.H) - 0.5f;
  return tile_hit(t.u, t.v, t.A, t.beta, t.gamma, t.ab, t.inv_den, t.qb, X0, X1, Y0, Y1);
}

// Warp-cooperative pass over the candidate tiles of 32 depth-ordered records at a
// time (one batch): lane l loads record k0 + l (one round of independent loads),
// the 32 candidate lists are concatenated by a warp scan, and each lane then takes
// one candidate per step, finding its record by a binary search over the scan and
// reading that record's fields with shuffles. Hits are kept in candidate order per
// digit d = tile & (2^fbits - 1): the count pass (EMIT = false) writes the batch's
// hits per digit to hist[d * NB + batch]; the emitting pass starts each digit's
// cursor at the scanned hist entry and writes (tile id, record) at the cursor.
constexpr int kMaxFusedBits = 8;

template <bool EMIT>
__global__ void __launch_bounds__(256) candidates_kernel(gs_proj_t P, const uint32_t *__restrict__ order,
                                                         const uint32_t *n_vis, const uint32_t *overflow,
                                                         const gs_camera_t *__restrict__ cams, int n_views,
                                                         int64_t n_per_view, int tw, int th, int fbits,
                                                         uint32_t *__restrict__ hist, uint32_t *__restrict__ dkeys,
                                                         uint32_t *__restrict__ dvals) {
  __shared__ uint32_t s_cur[8][1 << kMaxFusedBits];   // per warp: hits (count) / next position (emit) per digit
  if (EMIT && *overflow) return;
  const uint32_t nv = *n_vis;
  const uint32_t NB = (nv + 31u) / 32u;
  const uint32_t nd = 1u << fbits, dmask = nd - 1u;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t k0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; k0 < nv; k0 += nw * 32) {
    const uint32_t batch = k0 / 32u;
    for (uint32_t d = lane; d < nd; d += 32) s_cur[wib][d] = EMIT ? hist[(uint64_t)d * NB + batch] : 0u;
    const uint32_t k = k0 + lane;
    RecordTiles t{};
    uint32_t r = 0;
    if (k < nv) {
      r = order[k];
      t = record_tiles(P, cams, n_views, n_per_view, r);
    }
    uint32_t incl = t.n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t excl = incl - t.n;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    for (uint32_t c0 = 0; c0 < total; c0 += 32) {
      const uint32_t g = c0 + lane;
      // owner: the last record j whose candidates start at or before g
      int j = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t e = __shfl_sync(0xffffffffu, excl, j + step);
        if (j + step < 32 && e <= g) j += step;
      }
      RecordTiles o;
      o.x0 = __shfl_sync(0xffffffffu, t.x0, j);
      o.y0 = __shfl_sync(0xffffffffu, t.y0, j);
      o.w = __shfl_sync(0xffffffffu, t.w, j);
      o.n = __shfl_sync(0xffffffffu, t.n, j);
      o.u = __shfl_sync(0xffffffffu, t.u, j);
      o.v = __shfl_sync(0xffffffffu, t.v, j);
      o.A = __shfl_sync(0xffffffffu, t.A, j);
      o.beta = __shfl_sync(0xffffffffu, t.beta, j);
      o.gamma = __shfl_sync(0xffffffffu, t.gamma, j);
      o.qb = __shfl_sync(0xffffffffu, t.qb, j);
      o.ab = __shfl_sync(0xffffffffu, t.ab, j);
      o.inv_den = __shfl_sync(0xffffffffu, t.inv_den, j);
      o.W = __shfl_sync(0xffffffffu, t.W, j);
      o.H = __shfl_sync(0xffffffffu, t.H, j);
      o.toff = __shfl_sync(0xffffffffu, t.toff, j);
      o.gx = __shfl_sync(0xffffffffu, t.gx, j);
      const uint32_t c = g - __shfl_sync(0xffffffffu, excl, j);
      uint32_t tile = 0;
      const bool hit = g < total && candidate(o, c, tw, th, tile);
      const uint32_t dig = tile & dmask;
      // hits of this step with the same digit, in lane (= candidate) order
      const uint32_t peers = __match_any_sync(0xffffffffu, hit ? dig : 0xffffffffu);
      const uint32_t r_j = EMIT ? __shfl_sync(0xffffffffu, r, j) : 0u;
      uint32_t cur = 0;
      if (hit) cur = s_cur[wib][dig];
      __syncwarp();
      if (hit) {
        if (EMIT) {
          const uint32_t pos = cur + __popc(peers & lt);
          dkeys[pos] = tile;
          dvals[pos] = r_j;
        }
        if ((peers & lt) == 0) s_cur[wib][dig] = cur + __popc(peers);
      }
      __syncwarp();
    }
    if (!EMIT)
      for (uint32_t d = lane; d < nd; d += 32) hist[(uint64_t)d * NB + batch] = s_cur[wib][d];
    __syncwarp();
  }
}

// ranges[t] = [first index with key >= t, first index with key > t) over the sorted keys.
__global__ void ranges_kernel(const uint32_t *__restrict__ keys, const uint32_t *m_total, const uint32_t *overflow,
                              int n_tiles, uint2 *__restrict__ ranges) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (*overflow) {
    for (int64_t t = tid; t < n_tiles; t += stride) ranges[t] = make_uint2(0u, 0u);
    return;
  }
  const uint32_t M = *m_total;
  for (int64_t i = tid; i <= (int64_t)M; i += stride) {
    const int64_t prev = i > 0 ? (int64_t)keys[i - 1] : -1;
    const int64_t cur = i < (int64_t)M ? (int64_t)keys[i] : (int64_t)n_tiles;
    for (int64_t t = prev + 1; t <= cur && t < n_tiles; ++t) ranges[t].x = (uint32_t)i;
    for (int64_t t = prev < 0 ? 0 : prev; t < cur && t < n_tiles; ++t) ranges[t].y = (uint32_t)i;
  }
}

__global__ void keys64_kernel(const uint32_t *__restrict__ tiles, const uint32_t *__restrict__ vals,
                              const float *__restrict__ depth, const uint32_t *m_total, const uint32_t *overflow,
                              uint64_t *__restrict__ keys) {
  if (*overflow) return;
  const uint32_t M = *m_total;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x)
    keys[i] = ((uint64_t)tiles[i] << 32) | __float_as_uint(depth[vals[i]]);
}

// ------------------------------------------------------------------ host side
struct BinWs {
  uint32_t *vk0, *vv0, *vk1, *vv1;   // visible records: depth keys / record ids (double buffered)
  uint32_t *dhist;                   // (digit, batch) hit counts -> emission cursors
  uint32_t *dk0, *dk1, *dv1;         // duplicate tile keys (double buffered) + second value buffer
  uint64_t *block_sums;
  uint32_t *hist;
  uint32_t *counters;                // [0] n_vis, [1] M, [2] overflow
  size_t bytes;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static BinWs bin_ws_layout(void *base, int64_t R, int64_t cap, int fbits) {
  BinWs w{};
  char *p = static_cast<char *>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) -> void * {
    void *q = p ? p + off : nullptr;
    off += align256(bytes);
    return q;
  };
  w.vk0 = (uint32_t *)take(4 * (size_t)R + 16);
  w.vv0 = (uint32_t *)take(4 * (size_t)R + 16);
  w.vk1 = (uint32_t *)take(4 * (size_t)R + 16);
  w.vv1 = (uint32_t *)take(4 * (size_t)R + 16);
  w.dhist = (uint32_t *)take(4 * ((((size_t)R + 31) / 32) << fbits) + 16);
  w.dk0 = (uint32_t *)take(4 * (size_t)cap + 16);
  w.dk1 = (uint32_t *)take(4 * (size_t)cap + 16);
  w.dv1 = (uint32_t *)take(4 * (size_t)cap + 16);
  w.block_sums = (uint64_t *)take(8 * kMaxBlocks);
  w.hist = (uint32_t *)take(4 * (size_t)kRsBins * (kMaxBlocks + 1));   // + digit totals
  w.counters = (uint32_t *)take(64);
  w.bytes = off;
  return w;
}


// Blocks of the radix passes: four per SM (the downsweep holds 8 keys per thread).
static int radix_blocks() {
  const int g = 4 * num_sms();
  return g > kMaxBlocks ? kMaxBlocks : g;
}

// Stable LSD radix sort of (key, val) pairs on bits [first_bit, n_bits), ping-ponging between
// buffer 0 and 1; returns in *in_b0 whether the result is in buffer 0.
static gs_status_t radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, const uint32_t *d_n,
                              const uint32_t *d_skip, int first_bit, int n_bits, bool keep_keys, uint32_t *hist,
                              cudaStream_t s, bool *in_b0) {
  const int G = radix_blocks();
  const int span = n_bits - first_bit;
  const int passes = span > 0 ? (span + 7) / 8 : 0;
  const int bits = passes > 0 ? (span + passes - 1) / passes : 0;
  bool cur0 = true;
  for (int p = 0; p < passes; ++p) {
    const int shift = first_bit + p * bits;
    const int nb = (shift + bits > n_bits) ? n_bits - shift : bits;
    const uint32_t mask = (1u << nb) - 1u;
    uint32_t *ki = cur0 ? k0 : k1, *vi = cur0 ? v0 : v1, *ko = cur0 ? k1 : k0, *vo = cur0 ? v1 : v0;
    rs_upsweep_kernel<<<G, kRsThreads, 0, s>>>(ki, d_n, d_skip, shift, mask, hist);
    GS_LAUNCH_CHECK();
    rs_scan_kernel<<<kRsBins, 32, 0, s>>>(hist, G, hist + (size_t)kRsBins * kMaxBlocks, d_skip);
    GS_LAUNCH_CHECK();
    const bool last = p == passes - 1;
    uint32_t *kout = (last && !keep_keys) ? nullptr : ko;
    const uint32_t *tot = hist + (size_t)kRsBins * kMaxBlocks;
    switch (nb) {
#define GS_RS_DOWN(B)                                                                                          \
  case B:                                                                                                      \
    rs_downsweep_kernel<B><<<G, kRsThreads, 0, s>>>(ki, vi, kout, vo, d_n, d_skip, shift, mask, hist, tot); \
    break;
      GS_RS_DOWN(1) GS_RS_DOWN(2) GS_RS_DOWN(3) GS_RS_DOWN(4) GS_RS_DOWN(5) GS_RS_DOWN(6)
#undef GS_RS_DOWN
      default:
        rs_downsweep_kernel<0><<<G, kRsThreads, 0, s>>>(ki, vi, kout, vo, d_n, d_skip, shift, mask, hist, tot);
    }
    GS_LAUNCH_CHECK();
    cur0 = !cur0;
  }
  *in_b0 = cur0;
  return GS_OK;
}

static int bits_for(uint32_t max_value) {
  int b = 1;
  while (b < 32 && (max_value >> b) != 0) ++b;
  return b;
}

// Tile-id bits and the low digit fused into the emission: every bit above it is
// covered by ceil((bits - fbits) / 8) radix passes, with fbits as small as that
// pass count allows (a smaller digit means a smaller (digit, batch) histogram).
static void tile_sort_plan(int n_tiles, int &tile_bits, int &fbits) {
  tile_bits = bits_for((uint32_t)(n_tiles > 0 ? n_tiles - 1 : 0));
  if (tile_bits <= kMaxFusedBits) {
    fbits = tile_bits;
    return;
  }
  const int passes = (tile_bits - kMaxFusedBits + 7) / 8;
  fbits = tile_bits - 8 * passes;
  if (fbits < 1) fbits = 1;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_bin_sort_workspace_size(int64_t n_records, int64_t dup_capacity, const gs_frame_t *frame) {
  if (n_records < 0 || dup_capacity < 0) return 0;
  int tile_bits = 32, fbits = kMaxFusedBits;
  if (frame) tile_sort_plan(frame->n_tiles, tile_bits, fbits);
  return bin_ws_layout(nullptr, n_records, dup_capacity, fbits).bytes;
}

extern "C" gs_status_t gs_bin_sort(const gs_proj_t *proj, const gs_frame_t *frame, gs_bins_t *bins, void *ws,
                                   size_t ws_bytes, int32_t *d_error, gs_stream_t stream) {
  if (!proj || !frame || !bins || !ws || !frame->cams_dev || frame->n_views <= 0 || frame->n_tiles <= 0)
    return GS_ERR_INVALID_ARG;
  if (!bins->vals || !bins->ranges || !bins->d_count || bins->capacity < 0 || bins->capacity >= (1ll << 31))
    return GS_ERR_INVALID_ARG;
  const int64_t R = proj->n_records;
  if (R < 0 || R >= (1ll << 31) || R % frame->n_views != 0) return GS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return GS_ERR_INVALID_ARG;
  int tile_bits, fbits;
  tile_sort_plan(frame->n_tiles, tile_bits, fbits);
  const BinWs w = bin_ws_layout(ws, R, bins->capacity, fbits);
  if (ws_bytes < w.bytes) return GS_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  const int G = scan_blocks();
  uint32_t *n_vis = w.counters + 0, *m_total = w.counters + 1, *overflow = w.counters + 2;
  GS_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 64, s));

  // 1. compact visible records (record order) with their FP32 depth bits as keys
  VisibleCompact vc{proj->radius, proj->depth, (uint64_t)R, w.vk0, w.vv0, n_vis};
  if (gs_status_t st = run_scan(vc, w.block_sums, G, s)) return st;
  // 2. stable sort by depth
  bool in0 = true;
  if (gs_status_t st = radix_sort(w.vk0, w.vv0, w.vk1, w.vv1, n_vis, nullptr, 0, 32, false, w.hist, s, &in0))
    return st;
  const uint32_t *order = in0 ? w.vv0 : w.vv1;
  // 3. hits per (low tile digit, batch of 32 depth-ordered records), scanned into
  //    emission cursors; M and the capacity check
  const int64_t n_per_view = R / frame->n_views;
  const int eg = num_sms() * 8;
  candidates_kernel<false><<<eg, 256, 0, s>>>(*proj, order, n_vis, nullptr, frame->cams_dev, frame->n_views,
                                              n_per_view, frame->tile_w, frame->tile_h, fbits, w.dhist, nullptr,
                                              nullptr);
  GS_LAUNCH_CHECK();
  HistScan hs{w.dhist, n_vis, fbits, (uint64_t)bins->capacity, m_total, overflow, bins->d_count, d_error};
  if (gs_status_t st = run_scan(hs, w.block_sums, G, s)) return st;
  // 4. emit (tile, record) partitioned by the low digit, in depth order within it,
  //    into the buffer the remaining passes end in
  const int passes = (tile_bits - fbits + 7) / 8;
  uint32_t *A_k = w.dk0, *A_v = bins->vals, *B_k = w.dk1, *B_v = w.dv1;
  const bool emit_to_A = (passes % 2) == 0;
  candidates_kernel<true><<<eg, 256, 0, s>>>(*proj, order, n_vis, overflow, frame->cams_dev, frame->n_views,
                                             n_per_view, frame->tile_w, frame->tile_h, fbits, w.dhist,
                                             emit_to_A ? A_k : B_k, emit_to_A ? A_v : B_v);
  GS_LAUNCH_CHECK();
  // 5. stable sort by the remaining tile-id bits
  bool res0 = true;
  if (emit_to_A) {
    if (gs_status_t st = radix_sort(A_k, A_v, B_k, B_v, m_total, overflow, fbits, tile_bits, true, w.hist, s, &res0))
      return st;
  } else {
    if (gs_status_t st = radix_sort(B_k, B_v, A_k, A_v, m_total, overflow, fbits, tile_bits, true, w.hist, s, &res0))
      return st;
    res0 = !res0;
  }
  // 6. per-tile ranges (and optional 64-bit keys)
  ranges_kernel<<<eg, 256, 0, s>>>(A_k, m_total, overflow, frame->n_tiles, reinterpret_cast<uint2 *>(bins->ranges));
  GS_LAUNCH_CHECK();
  if (bins->keys) {
    keys64_kernel<<<eg, 256, 0, s>>>(A_k, A_v, proj->depth, m_total, overflow, bins->keys);
    GS_LAUNCH_CHECK();
  }
  return GS_OK;
}
