// Tile binning and depth sort ("tile-based", "depth-sorted" rasterization, Sec.
// "Preliminary" of the paper).
//
// Result: for every global tile, the visible records whose footprint ellipse (where
// alpha can reach the 1/255 floor, with a 0.2% margin) meets the tile's box of pixel
// centres, ordered by (FP32 depth bits, record index), concatenated tile after tile.
// Candidate tiles are those under the footprint's bounding box (gs_project's rect);
// per tile row, the ellipse's x-extent over the row's pixel centres keeps a
// contiguous run of columns (the exact ellipse-box test, band_span_rn).
//
// Instead of one wide radix sort on (tile << 32 | depth) keys over all duplicates,
// the order is built in two stable stages that give the same permutation:
//   1. the visible records (one entry each) are stably sorted by their FP32 depth
//      bits (LSD radix sort, 8-bit digits over the bits the visible depth range
//      spans; the first pass reads the records and drops the invisible ones);
//   2. every record, taken in depth order, emits one entry per tile its footprint
//      meets, and the entries are stably sorted by tile id alone. The first LSD
//      digit of that sort (the low FB bits of the tile id) is fused into the
//      emission: a counting pass histograms each warp batch's hits by that digit,
//      a scan turns the (digit, batch) counts into cursors, and the emitting pass
//      writes every entry straight to its digit-partitioned position (as one packed
//      8-byte (tile, record) pair when a single pass follows). The remaining high
//      bits take ceil((bits - FB) / 8) ordinary passes (none when the tile id has at
//      most 8 bits).
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

#ifdef GS_DEBUG
GS_DEBUG_TAKE(debug_take_bin_sort)
#endif

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;  // 2048 keys per tile
constexpr int kRsBins = 256;      // digits of a tile-id pass
constexpr int kDepthBins = 256;   // digits of a depth pass (8 bits; 9-bit passes measured slower)

// ------------------------------------------------------------------ LSD radix sort pass
// One pass sorts stably by the digit (key >> shift) & (2^nb - 1), nb <= log2(BINS):
// per-block digit histograms (upsweep), their per-digit scan over blocks, and a
// stable scatter (downsweep). The depth sort's first pass reads the records
// themselves (FROM_RECORDS): it keeps the visible ones (radius > 0) in record order,
// keyed by their FP32 depth bits minus the smallest visible depth's bits, and so
// compacts and sorts in one go; its later passes run only while the key range
// needs more digits, and the pass that ends the sort writes its record ids to a
// fixed output buffer.
struct RsSrc {
  const uint32_t *keys;      // keys and values of the pass (unless FROM_RECORDS)
  const uint32_t *vals;
  const int32_t *radius;     // FROM_RECORDS: visibility and depth of record i
  const float *depth;
  uint64_t n;                // FROM_RECORDS: the record count (else *d_n elements)
  const uint32_t *d_n;
  const uint32_t *d_skip;    // non-zero: the pass does nothing
  const uint32_t *range;     // depth sort: [0] ~min, [1] max of the visible depth bits (else null)
  int shift, nb;
};

// Bits of the depth sort's keys (0 without visible records).
__device__ __forceinline__ int depth_key_bits(const uint32_t *range) {
  const uint32_t mn = ~range[0], mx = range[1];
  return mx >= mn && mx != mn ? 32 - __clz(mx - mn) : 0;
}

__device__ __forceinline__ bool rs_active(const RsSrc &s) {
  if (s.d_skip && *s.d_skip) return false;
  return !s.range || s.shift == 0 || depth_key_bits(s.range) > s.shift;
}

__device__ __forceinline__ uint64_t rs_count(const RsSrc &s, bool from_records) {
  return from_records ? s.n : (uint64_t)*s.d_n;
}

// Visible-record count and the range of their FP32 depth bits (atomics on zeroed
// words: range[0] collects the largest ~bits, i.e. the smallest bits).
__global__ void __launch_bounds__(256) depth_range_kernel(const int32_t *__restrict__ radius,
                                                          const float *__restrict__ depth, int64_t n,
                                                          uint32_t *n_vis, uint32_t *range) {
  uint32_t cnt = 0, mx = 0, nmn = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t rad = radius[i];
    const uint32_t b = __float_as_uint(depth[i]);   // both loads in flight at once
    if (rad > 0) {
      ++cnt;
      mx = max(mx, b);
      nmn = max(nmn, ~b);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nmn = max(nmn, __shfl_xor_sync(0xffffffffu, nmn, o));
  }
  __shared__ uint32_t s_red[3][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    s_red[0][warp] = cnt;
    s_red[1][warp] = mx;
    s_red[2][warp] = nmn;
  }
  __syncthreads();
  if (warp == 0) {
    cnt = lane < nw ? s_red[0][lane] : 0u;
    mx = lane < nw ? s_red[1][lane] : 0u;
    nmn = lane < nw ? s_red[2][lane] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      nmn = max(nmn, __shfl_xor_sync(0xffffffffu, nmn, o));
    }
    if (lane == 0 && cnt) {
      atomicAdd(n_vis, cnt);
      atomicMax(&range[1], mx);
      atomicMax(&range[0], nmn);
    }
  }
}

// Digit histograms per block (digit-major: hist[d * G + b]).
// Element sources of a pass: plain keys, depth-sort keys (the pass may be inactive
// or end the sort), or the records themselves (the depth sort's first pass).
// kSrcPacked: (key, value) pairs stored as one uint2 each (the emission's output when a
// single tile-id pass follows).
constexpr int kSrcKeys = 0, kSrcDepthKeys = 1, kSrcRecords = 2, kSrcPacked = 3;

template <int BINS, int SRC>
__global__ void __launch_bounds__(kRsThreads) rs_upsweep_kernel(RsSrc src, uint32_t *hist) {
  constexpr bool FROM_RECORDS = SRC == kSrcRecords;
  __shared__ uint32_t h[kRsWarps][BINS];
  if (!rs_active(src)) return;
  const int G = gridDim.x;
  const uint64_t n = rs_count(src, FROM_RECORDS);
  uint64_t begin, end;
  chunk_of(n, G, kRsTile, begin, end);
  const int warp = threadIdx.x >> 5;
  const int shift = src.shift;
  const uint32_t mask = (1u << src.nb) - 1u;
  for (int d = threadIdx.x; d < kRsWarps * BINS; d += kRsThreads) (&h[0][0])[d] = 0;
  __syncthreads();
  if (FROM_RECORDS) {
    const uint32_t mn = ~src.range[0];
    for (uint64_t i = begin + threadIdx.x; i < end; i += kRsThreads) {
      const int32_t rad = src.radius[i];
      const uint32_t b = __float_as_uint(src.depth[i]);
      if (rad > 0) atomicAdd(&h[warp][((b - mn) >> shift) & mask], 1u);
    }
  } else if (SRC == kSrcPacked) {
    // two pairs per 16-byte load (chunks start at even indices)
    const uint2 *pk = reinterpret_cast<const uint2 *>(src.keys);
    uint64_t i = begin + 2 * threadIdx.x;
    for (; i + 1 < end; i += 2 * kRsThreads) {
      const uint4 k = *reinterpret_cast<const uint4 *>(pk + i);
      atomicAdd(&h[warp][(k.x >> shift) & mask], 1u);
      atomicAdd(&h[warp][(k.z >> shift) & mask], 1u);
    }
    for (; i < end; ++i) atomicAdd(&h[warp][(pk[i].x >> shift) & mask], 1u);
  } else {
    const uint32_t *keys = src.keys;
    uint64_t i = begin + 4 * threadIdx.x;
    for (; i + 3 < end; i += 4 * kRsThreads) {
      const uint4 k = *reinterpret_cast<const uint4 *>(keys + i);
      atomicAdd(&h[warp][(k.x >> shift) & mask], 1u);
      atomicAdd(&h[warp][(k.y >> shift) & mask], 1u);
      atomicAdd(&h[warp][(k.z >> shift) & mask], 1u);
      atomicAdd(&h[warp][(k.w >> shift) & mask], 1u);
    }
    for (; i < end; ++i) atomicAdd(&h[warp][(keys[i] >> shift) & mask], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < BINS; d += kRsThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) s += h[w][d];
    hist[(uint64_t)d * G + blockIdx.x] = s;
  }
}

// Per-digit exclusive scan of the digit-major histogram hist[BINS][G] over blocks,
// in place: one block of kRsThreads per digit (G <= 4 * kRsThreads), each thread
// taking up to four consecutive entries of the row; the digit total goes to
// totals[d]. The digit bases (exclusive scan of totals) are added by the downsweep.
__global__ void __launch_bounds__(kRsThreads) rs_scan_kernel(RsSrc src, uint32_t *hist, int G, uint32_t *totals) {
  if (!rs_active(src)) return;
  uint32_t *row = hist + (size_t)blockIdx.x * G;
  const int per = (G + kRsThreads - 1) / kRsThreads;
  const int b0 = threadIdx.x * per;
  uint32_t x[4] = {0u, 0u, 0u, 0u}, sum = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (i < per && b0 + i < G) {
      x[i] = row[b0 + i];
      sum += x[i];
    }
  uint32_t all;
  uint32_t run = block_exclusive_scan<uint32_t>(sum, &all);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (i < per && b0 + i < G) {
      row[b0 + i] = run;
      run += x[i];
    }
  if (threadIdx.x == 0) totals[blockIdx.x] = all;
}

// Stable scatter. Each warp ranks a contiguous slice of the tile, 32 keys per
// step in order: the lanes sharing a digit come from one ballot per digit bit
// (faster here than __match_any_sync), their base from a per-warp shared-memory
// digit count;
// slices are then offset by the warps before them, staged in shared memory in
// digit order and written out coalesced. Elements that are not kept (invisible
// records, the ragged end) take the sentinel digit BINS and are staged last.
// keys_out null: the pass writes no keys. A depth-sort pass that ends the sort
// writes only the record ids, to vals_last.
template <int BINS, int SRC, int NBC>
__global__ void __launch_bounds__(kRsThreads, 4) rs_downsweep_kernel(RsSrc src, uint32_t *__restrict__ keys_out,
                                                                     uint32_t *__restrict__ vals_out,
                                                                     uint32_t *__restrict__ vals_last,
                                                                     const uint32_t *__restrict__ hist,
                                                                     const uint32_t *__restrict__ totals) {
  constexpr bool FROM_RECORDS = SRC == kSrcRecords;
  constexpr int DPT = BINS / kRsThreads;   // digits per thread
  static_assert(DPT * kRsThreads == BINS, "BINS is a multiple of the block size");
  __shared__ uint32_t s_keys[kRsTile];
  __shared__ uint32_t s_vals[kRsTile];
  __shared__ uint32_t s_whist[kRsWarps][BINS + 1];
  __shared__ uint32_t s_goff[BINS];
  __shared__ uint32_t s_tstart[BINS + 1];
  if (!rs_active(src)) return;
  const int G = gridDim.x;
  const uint64_t n = rs_count(src, FROM_RECORDS);
  uint64_t begin, end;
  chunk_of(n, G, kRsTile, begin, end);
  if (begin >= end) return;
  const bool last = (SRC == kSrcRecords || SRC == kSrcDepthKeys) && depth_key_bits(src.range) <= src.shift + src.nb;
  uint32_t *ko = last ? nullptr : keys_out;
  uint32_t *vo = last ? vals_last : vals_out;
  const int shift = src.shift;
  const uint32_t mask = (1u << src.nb) - 1u;
  const uint32_t mn = FROM_RECORDS ? ~src.range[0] : 0u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int d0 = threadIdx.x * DPT;
  {
    // digit bases: exclusive scan of the digit totals, then this block's column
    uint32_t tv[DPT], sum = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      tv[q] = totals[d0 + q];
      sum += tv[q];
    }
    uint32_t all;
    uint32_t base = block_exclusive_scan<uint32_t>(sum, &all);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      s_goff[d0 + q] = base + hist[(uint64_t)(d0 + q) * G + blockIdx.x];
      base += tv[q];
    }
  }
  const uint32_t lt_mask = lanemask_lt();
  for (uint64_t tb = begin; tb < end; tb += kRsTile) {
    const uint32_t tile_n = (uint32_t)min((uint64_t)kRsTile, end - tb);
    for (int d = lane; d < BINS + 1; d += 32) s_whist[warp][d] = 0;
    __syncwarp();
    uint32_t k[kRsItems], v[kRsItems], dig[kRsItems], rank[kRsItems];
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
      const uint32_t li = warp * (32 * kRsItems) + j * 32 + lane;   // warp slice of 32 * kRsItems keys
      bool valid = li < tile_n;
      if (FROM_RECORDS) {
        const int32_t rad = valid ? src.radius[tb + li] : 0;
        const uint32_t b = valid ? __float_as_uint(src.depth[tb + li]) : 0u;
        valid = rad > 0;
        k[j] = valid ? b - mn : 0u;
        v[j] = (uint32_t)(tb + li);
      } else if (SRC == kSrcPacked) {
        const uint2 kv = valid ? reinterpret_cast<const uint2 *>(src.keys)[tb + li] : make_uint2(0u, 0u);
        k[j] = kv.x;
        v[j] = kv.y;
      } else {
        k[j] = valid ? src.keys[tb + li] : 0u;
        v[j] = valid ? src.vals[tb + li] : 0u;
      }
      dig[j] = valid ? ((k[j] >> shift) & mask) : (uint32_t)BINS;
    }
    // peers: the lanes holding the same digit, from one ballot per digit bit (a
    // lane with bit value v keeps ballot ^ (v - 1): the ballot, or its complement),
    // unrolled when the digit width is known at compile time; the sentinel bit takes
    // one more, needed only where sentinels can occur (the ragged end of the keys,
    // and the invisible records of the depth sort's first pass)
    const bool sentinels = FROM_RECORDS || tile_n < (uint32_t)kRsTile;
    uint32_t pm[kRsItems];
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
      uint32_t p = 0xffffffffu;
      if (NBC > 0) {
#pragma unroll
        for (int b = 0; b < NBC; ++b) {
          const uint32_t bit = (dig[j] >> b) & 1u;
          p &= __ballot_sync(0xffffffffu, bit) ^ (bit - 1u);
        }
      } else {
        for (int b = 0; b < src.nb; ++b) {
          const uint32_t bit = (dig[j] >> b) & 1u;
          p &= __ballot_sync(0xffffffffu, bit) ^ (bit - 1u);
        }
      }
      if (sentinels) {
        const uint32_t sb = dig[j] == (uint32_t)BINS ? 1u : 0u;
        p &= __ballot_sync(0xffffffffu, sb) ^ (sb - 1u);
      }
      pm[j] = p;
    }
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
      const uint32_t peers = pm[j];
      const uint32_t before = __popc(peers & lt_mask);
      const uint32_t base = s_whist[warp][dig[j]];
      __syncwarp();
      rank[j] = base + before;
      if (before == 0) s_whist[warp][dig[j]] = base + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per digit: the warps' exclusive offsets and the tile's count (the last thread
    // also takes the sentinel digit, which stays out of the counts)
    uint32_t tot[DPT], local = 0;
#pragma unroll
    for (int q = 0; q < DPT + 1; ++q) {
      const int d = q < DPT ? d0 + q : BINS;
      if (q == DPT && threadIdx.x != kRsThreads - 1) break;
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kRsWarps; ++w) {
        const uint32_t c = s_whist[w][d];
        s_whist[w][d] = run;
        run += c;
      }
      if (q < DPT) {
        tot[q] = run;
        local += run;
      }
    }
    uint32_t all;
    uint32_t start = block_exclusive_scan<uint32_t>(local, &all);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      s_tstart[d0 + q] = start;
      start += tot[q];
    }
    if (threadIdx.x == 0) s_tstart[BINS] = all;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
      const uint32_t pos = s_tstart[dig[j]] + s_whist[warp][dig[j]] + rank[j];
      s_keys[pos] = k[j];
      s_vals[pos] = v[j];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < all; i += kRsThreads) {
      const uint32_t key = s_keys[i];
      const uint32_t d = (key >> shift) & mask;
      const uint32_t gpos = s_goff[d] + (i - s_tstart[d]);
      if (ko) ko[gpos] = key;
      vo[gpos] = s_vals[i];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < DPT; ++q) s_goff[d0 + q] += tot[q];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ bin/sort functors
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
  const unsigned long long *units;   // length of the binning's unit list, held in the list buffers
  int64_t *d_count;
  int32_t *d_error;
  __device__ uint64_t count() const { return ((uint64_t)(*n_vis) + 31u) / 32u << fbits; }
  __device__ uint32_t value(uint64_t i) const { return hist[i]; }
  __device__ void emit(uint64_t i, uint64_t pre, uint32_t) const {
    if (pre <= 0xffffffffull) hist[i] = (uint32_t)pre;
  }
  __device__ void total(uint64_t t) const {
    const uint64_t nu = *units;
    const bool over = t > capacity || nu > capacity;
    // on overflow: a capacity that holds both the entries and the unit list
    *d_count = (int64_t)(over && nu > t ? nu : t);
    *overflow = over ? 1u : 0u;
    *m_total = over ? 0u : (uint32_t)t;
    if (over && d_error) atomicOr(d_error, (int32_t)GS_ERR_CAPACITY);
  }
};

// Per record of a batch (one warp's 32 depth-ordered records), in shared memory:
// the ellipse constants and the candidate rectangle with its view's layout.
struct BinRec {
  float u, v, inv_A, beta, gamma, qb, dyr;
  uint32_t rec;
  uint32_t x0, x1, y0;       // candidate tile rectangle (columns [x0, x1), first row y0)
  int W, H, toff, gx;
  uint32_t nrow;             // tile rows of the rectangle (0: nothing to bin)
};
static_assert(sizeof(BinRec) == 64, "BinRec is four 16-byte words");

// Columns of one tile row that the band's x-extent [xl, xr] covers: the first tx in
// [x0, x1) whose pixel-centre box ends at or after xl and the last one that starts
// at or before xr (exact float compares against the box edges; the scaled
// coordinate, with inv_tw ~ 1 / tw, only seeds the search). Returns the count (0 if
// none) and the first column in lo.
__device__ __forceinline__ uint32_t band_columns(float xl, float xr, int x0, int x1, int tw, float inv_tw, int W,
                                                 int &lo) {
  auto X0 = [&](int tx) { return (float)(tx * tw) + 0.5f; };
  auto X1 = [&](int tx) { return (float)min((tx + 1) * tw, W) - 0.5f; };
  int a = (int)fminf(fmaxf(ceilf((xl + 0.5f) * inv_tw) - 1.f, (float)x0), (float)x1);
  while (a < x1 && X1(a) < xl) ++a;
  while (a > x0 && X1(a - 1) >= xl) --a;
  int b = (int)fminf(fmaxf(floorf((xr - 0.5f) * inv_tw), (float)(x0 - 1)), (float)(x1 - 1));
  while (b >= x0 && X0(b) > xr) --b;
  while (b + 1 < x1 && X0(b + 1) <= xr) ++b;
  lo = a;
  return b >= a ? (uint32_t)(b - a + 1) : 0u;
}

// Binning of 32 depth-ordered records per warp (one batch), one tile row of a
// record's candidate rectangle (a "unit") at a time: the ellipse's x-extent over the
// row's band of pixel centres (band_span_rn) selects a contiguous run of tile
// columns. Two passes over the batches:
// bin_count_kernel spreads the batch's units over the lanes (the rows concatenated
// by a warp scan, each lane finding its record by a binary search), adds every run's
// tiles to the batch's histogram of the low tile digit d = tile & (2^fbits - 1),
// written to hist[d * NB + batch], and stores each unit's run (first tile id; record
// slot << 24 | length) in a unit list, in (record, row) order, at a range the batch
// reserves from a counter (ubatch[batch] = (first unit, units)).
// bin_emit_kernel reads the batch's units back, concatenates their hits (a scan over
// the run lengths) and spreads them over the lanes; each hit goes to its digit's
// cursor, which starts at the scanned hist entry and advances in (record, row,
// column) order, so each digit's entries stay in depth order.
constexpr int kMaxFusedBits = 8;
constexpr int kCountUnits = 64;    // units per round of the counting pass (two per lane)
constexpr int kUnits = 128;        // units per round of the emitting pass (four per lane)
constexpr int kWinCap = 256;   // 32-hit windows per round located by bit masks (else a binary search)
constexpr uint32_t kRunBits = 24;

__global__ void __launch_bounds__(256) bin_count_kernel(gs_proj_t P, const uint32_t *__restrict__ order,
                                                        const uint32_t *n_vis, const gs_camera_t *__restrict__ cams,
                                                        int n_views, int64_t n_per_view, int tw, int th,
                                                        float inv_tw, int fbits, uint32_t *__restrict__ hist,
                                                        uint2 *__restrict__ ubatch, uint32_t *__restrict__ ut0,
                                                        uint32_t *__restrict__ uinf,
                                                        unsigned long long *units_total, uint64_t unit_cap,
                                                        uint32_t *work) {
  __shared__ BinRec s_rec[8][32];
  __shared__ uint32_t s_cur[8][1 << kMaxFusedBits];
  const uint32_t nv = *n_vis;
  const uint32_t NB = (nv + 31u) / 32u;
  const uint32_t nd = 1u << fbits, dmask = nd - 1u;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // batches are claimed one at a time from a counter (zeroed before the launch):
  // their hit counts vary widely, so a fixed assignment leaves SMs idle at the end
  for (;;) {
    uint32_t batch = 0;
    if (lane == 0) batch = atomicAdd(work, 1u);
    batch = __shfl_sync(0xffffffffu, batch, 0);
    if (batch >= NB) break;
    const uint32_t k0 = batch * 32u;
    for (uint32_t d = lane; d < nd; d += 32) s_cur[wib][d] = 0u;
    // this lane's record: constants to shared memory, its row count to the scan
    uint32_t nrow = 0;
    {
      const uint32_t k = k0 + lane;
      BinRec br{};
      if (k < nv) {
        const uint32_t r = order[k];
        const uint2 q = reinterpret_cast<const uint2 *>(P.rect)[r];
        const uint32_t x0 = q.x & 0xffffu, y0 = q.x >> 16, x1 = q.y & 0xffffu, y1 = q.y >> 16;
        const float2 m = reinterpret_cast<const float2 *>(P.mean2d)[r];
        const float4 co = reinterpret_cast<const float4 *>(P.conic_opacity)[r];
        const int view = n_views == 1 ? 0 : (int)((int64_t)r / n_per_view);
        br.u = m.x; br.v = m.y; br.beta = co.y; br.gamma = co.z;
        br.qb = __fmul_rn(reinterpret_cast<const float4 *>(P.rgb)[r].w, kBinMargin);
        band_consts_rn(co.x, br.beta, br.gamma, br.qb, br.dyr, br.inv_A);
        br.rec = r;
        br.x0 = x0; br.x1 = x1; br.y0 = y0;
        br.W = cams[view].width; br.H = cams[view].height; br.toff = cams[view].tile_offset; br.gx = cams[view].grid_x;
        nrow = (x1 > x0 && y1 > y0) ? y1 - y0 : 0u;
        br.nrow = nrow;
      }
      s_rec[wib][lane] = br;
    }
    uint32_t incl = nrow;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t rexcl = incl - nrow;
    const uint32_t n_units = __shfl_sync(0xffffffffu, incl, 31);
    // the batch's range of the unit list; past the list's capacity nothing is stored
    // (the frame then overflows and the emitting pass does not run)
    unsigned long long ub = 0;
    if (lane == 0) ub = atomicAdd(units_total, (unsigned long long)n_units);
    ub = __shfl_sync(0xffffffffu, ub, 0);
    const bool keep = ub + n_units <= unit_cap;
    if (lane == 0) ubatch[batch] = make_uint2(keep ? (uint32_t)ub : 0u, keep ? n_units : 0u);
    __syncwarp();
    for (uint32_t u0 = 0; u0 < n_units; u0 += kCountUnits) {
#pragma unroll
      for (int i = 0; i < kCountUnits / 32; ++i) {
        const uint32_t u = u0 + lane + 32 * i;
        // owner: the last record j whose rows start at or before u
        int j = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t e = __shfl_sync(0xffffffffu, rexcl, j + step);
          if (j + step < 32 && e <= u) j += step;
        }
        const uint32_t row_j = u - __shfl_sync(0xffffffffu, rexcl, j);
        if (u < n_units) {
          const BinRec &b = s_rec[wib][j];
          const int ty = (int)(b.y0 + row_j);
          const float Y0 = (float)(ty * th) + 0.5f, Y1 = (float)min((ty + 1) * th, b.H) - 0.5f;
          float xl, xr;
          int lo = 0;
          uint32_t run = 0;
          if (band_span_rn(b.u, b.v, b.beta, b.gamma, b.qb, b.dyr, b.inv_A, Y0, Y1, xl, xr))
            run = band_columns(xl, xr, (int)b.x0, (int)b.x1, tw, inv_tw, b.W, lo);
          const uint32_t t0 = (uint32_t)(b.toff + ty * b.gx + lo);
          if (keep && GS_CHECK(ub + u < unit_cap, 4, ub + u)) {
            ut0[ub + u] = t0;
            uinf[ub + u] = ((uint32_t)j << kRunBits) | run;
          }
          if (run > 0) {
            // tiles t0 .. t0 + run - 1: digit (t0 + i) & dmask gets ceil((run - i) / nd)
            const uint32_t nrep = run < nd ? run : nd;
            for (uint32_t q = 0; q < nrep; ++q)
              atomicAdd(&s_cur[wib][(t0 + q) & dmask], (run - q + nd - 1) >> fbits);
          }
        }
      }
    }
    __syncwarp();
    for (uint32_t d = lane; d < nd; d += 32) hist[(uint64_t)d * NB + batch] = s_cur[wib][d];
    __syncwarp();
  }
}

// PACKED: each hit is written as one 8-byte (tile, record) pair at dkeys (as uint2)
// instead of two 4-byte words in two arrays: the scattered stores are what the
// emission's time goes to, and one store per hit halves their sectors.
template <bool PACKED>
__global__ void __launch_bounds__(256) bin_emit_kernel(const uint32_t *__restrict__ order, const uint32_t *n_vis,
                                                       const uint32_t *overflow, int fbits,
                                                       const uint32_t *__restrict__ hist,
                                                       const uint2 *__restrict__ ubatch,
                                                       const uint32_t *__restrict__ ut0,
                                                       const uint32_t *__restrict__ uinf,
                                                       uint32_t *__restrict__ dkeys, uint32_t *__restrict__ dvals,
                                                       uint32_t *work, uint64_t cap) {
  __shared__ uint32_t s_recid[8][32];
  __shared__ uint2 s_unit[8][kUnits];            // (record slot << 24 | run length, tile id of the run's first column)
  __shared__ uint32_t s_hpre[8][kUnits + 1];     // exclusive scan of the run lengths
  __shared__ uint32_t s_mask[8][kWinCap];        // per 32-hit window: bits at the hits that start a unit
  __shared__ uint8_t s_uid[8][kUnits];           // k-th non-empty unit of the round
  __shared__ uint32_t s_cur[8][1 << kMaxFusedBits];
  if (*overflow) return;
  const uint32_t nv = *n_vis;
  const uint32_t NB = (nv + 31u) / 32u;
  const uint32_t nd = 1u << fbits, dmask = nd - 1u;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  const uint32_t le = lt | (1u << lane);
  for (;;) {
    uint32_t batch = 0;
    if (lane == 0) batch = atomicAdd(work, 1u);
    batch = __shfl_sync(0xffffffffu, batch, 0);
    if (batch >= NB) break;
    const uint32_t k0 = batch * 32u;
    for (uint32_t d = lane; d < nd; d += 32) s_cur[wib][d] = hist[(uint64_t)d * NB + batch];
    s_recid[wib][lane] = k0 + lane < nv ? order[k0 + lane] : 0u;
    const uint2 ubn = ubatch[batch];
    const uint32_t ub = ubn.x, n_units = ubn.y;
    __syncwarp();
    for (uint32_t u0 = 0; u0 < n_units; u0 += kUnits) {
      uint32_t run[kUnits / 32];
#pragma unroll
      for (int i = 0; i < kUnits / 32; ++i) {
        const uint32_t u = u0 + lane + 32 * i;
        run[i] = 0;
        if (u < n_units) {
          const uint32_t inf = uinf[ub + u];
          run[i] = inf & ((1u << kRunBits) - 1u);
          s_unit[wib][u - u0] = make_uint2(inf, ut0[ub + u]);
        }
      }
      // concatenate the round's runs and spread the hits over the lanes
      uint32_t total = 0;
#pragma unroll
      for (int i = 0; i < kUnits / 32; ++i) {
        uint32_t c = run[i];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, c, o);
          if (lane >= o) c += y;
        }
        s_hpre[wib][32 * i + lane] = total + c - run[i];
        total += __shfl_sync(0xffffffffu, c, 31);
      }
      if (lane == 0) s_hpre[wib][kUnits] = total;
      __syncwarp();
      const uint32_t nu = min((uint32_t)kUnits, n_units - u0);
      // the unit of hit h is the last non-empty one starting at or before h: mark the
      // starts in per-window bit masks and number the non-empty units, so that a lane
      // finds its unit by a popcount instead of a binary search over s_hpre
      const uint32_t nwin = (total + 31) >> 5;
      const bool masks = nwin <= (uint32_t)kWinCap;
      if (masks) {
        for (uint32_t w = lane; w < nwin; w += 32) s_mask[wib][w] = 0u;
        __syncwarp();
        uint32_t kbase = 0;
#pragma unroll
        for (int i = 0; i < kUnits / 32; ++i) {
          const bool ne = run[i] > 0;
          const uint32_t bal = __ballot_sync(0xffffffffu, ne);
          if (ne) {
            const uint32_t pos = s_hpre[wib][32 * i + lane];
            atomicOr(&s_mask[wib][pos >> 5], 1u << (pos & 31));
            s_uid[wib][kbase + __popc(bal & lt)] = (uint8_t)(32 * i + lane);
          }
          kbase += __popc(bal);
        }
        __syncwarp();
      }
      uint32_t starts = 0;   // non-empty units starting before the window
      for (uint32_t h0 = 0; h0 < total; h0 += 32) {
        const uint32_t h = h0 + lane;
        const bool hit = h < total;
        uint32_t tile = 0, r = 0, u = 0;
        if (masks) {
          const uint32_t m = s_mask[wib][h0 >> 5];
          u = s_uid[wib][starts + __popc(m & le) - 1u];
          starts += __popc(m);
        } else if (hit) {
          uint32_t lo = 0, hi = nu;   // invariant: s_hpre[lo] <= h < s_hpre[hi]
          while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_hpre[wib][mid] <= h) lo = mid; else hi = mid;
          }
          u = lo;
        }
        if (hit) {
          const uint2 un = s_unit[wib][u];
          tile = un.y + (h - s_hpre[wib][u]);
          r = s_recid[wib][un.x >> kRunBits];
        }
        const uint32_t dig = tile & dmask;
        const uint32_t peers = __match_any_sync(0xffffffffu, hit ? dig : 0xffffffffu);
        uint32_t cur = 0;
        if (hit) cur = s_cur[wib][dig];
        __syncwarp();
        if (hit) {
          const uint32_t pos = cur + __popc(peers & lt);
          if (GS_CHECK(pos < cap, 4, pos)) {
            if (PACKED) {
              reinterpret_cast<uint2 *>(dkeys)[pos] = make_uint2(tile, r);
            } else {
              dkeys[pos] = tile;
              dvals[pos] = r;
            }
          }
          if ((peers & lt) == 0) s_cur[wib][dig] = cur + __popc(peers);
        }
        __syncwarp();
      }
      __syncwarp();
    }
    __syncwarp();
  }
}

// ranges[t] = [first index with key >= t, first index with key > t) over the sorted
// keys. Each thread takes four consecutive boundaries i = 4g .. 4g+3 (one 16-byte
// load) and writes the tiles whose range starts or ends there; i = M closes the rest.
__device__ __forceinline__ void range_boundary(int64_t i, int64_t prev, int64_t cur, int n_tiles,
                                               uint2 *__restrict__ ranges) {
  for (int64_t t = prev + 1; t <= cur && t < n_tiles; ++t) ranges[t].x = (uint32_t)i;
  for (int64_t t = prev < 0 ? 0 : prev; t < cur && t < n_tiles; ++t) ranges[t].y = (uint32_t)i;
}

__global__ void ranges_kernel(const uint32_t *__restrict__ keys, const uint32_t *m_total, const uint32_t *overflow,
                              int n_tiles, uint2 *__restrict__ ranges) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (*overflow) {
    for (int64_t t = tid; t < n_tiles; t += stride) ranges[t] = make_uint2(0u, 0u);
    return;
  }
  const int64_t M = *m_total;
  for (int64_t g = tid; 4 * g <= M; g += stride) {
    const int64_t i0 = 4 * g;
    int64_t prev = i0 > 0 ? (int64_t)keys[i0 - 1] : -1;
    if (i0 + 3 < M) {
      const uint4 k = *reinterpret_cast<const uint4 *>(keys + i0);
      const int64_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (kk[j] != prev) range_boundary(i0 + j, prev, kk[j], n_tiles, ranges);
        prev = kk[j];
      }
    } else {
      for (int64_t i = i0; i <= M && i < i0 + 4; ++i) {
        const int64_t cur = i < M ? (int64_t)keys[i] : (int64_t)n_tiles;
        if (cur != prev) range_boundary(i, prev, cur, n_tiles, ranges);
        prev = cur;
      }
    }
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
  uint32_t *order;                   // visible record ids in depth order
  uint32_t *dhist;                   // (digit, batch) hit counts -> emission cursors
  uint2 *ubatch;                     // per batch of 32 depth-ordered records: (first unit, units)
  uint32_t *dk0, *dk1, *dv1;         // duplicate tile keys (double buffered) + second value buffer
  uint64_t *block_sums;
  uint32_t *hist;
  uint32_t *counters;                // [0] n_vis, [1] M, [2] overflow, [3] [4] batch counters of the
                                     // counting and the emitting pass, [6..7] units (64-bit),
                                     // [8] [9] range of the visible depth bits (~min, max)
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
  w.ubatch = (uint2 *)take(8 * (((size_t)R + 31) / 32) + 16);
  w.dk0 = (uint32_t *)take(4 * (size_t)cap + 16);
  // dk1 and dv1 are adjacent: together they hold cap packed 8-byte (tile, record) pairs
  w.dk1 = (uint32_t *)take(4 * (size_t)cap + 16);
  w.dv1 = (uint32_t *)take(4 * (size_t)cap + 16);
  w.block_sums = (uint64_t *)take(8 * kMaxBlocks);
  w.order = (uint32_t *)take(4 * (size_t)R + 16);
  w.hist = (uint32_t *)take(4 * (size_t)kDepthBins * (kMaxBlocks + 1));   // + digit totals
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
// packed: the first pass reads buffer 0 as (key, value) uint2 pairs at k0.
static gs_status_t radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, const uint32_t *d_n,
                              const uint32_t *d_skip, int first_bit, int n_bits, bool keep_keys, uint32_t *hist,
                              cudaStream_t s, bool *in_b0, bool packed = false) {
  const int G = radix_blocks();
  const int span = n_bits - first_bit;
  const int passes = span > 0 ? (span + 7) / 8 : 0;
  const int bits = passes > 0 ? (span + passes - 1) / passes : 0;
  uint32_t *totals = hist + (size_t)kDepthBins * kMaxBlocks;
  bool cur0 = true;
  for (int p = 0; p < passes; ++p) {
    const int shift = first_bit + p * bits;
    const int nb = (shift + bits > n_bits) ? n_bits - shift : bits;
    uint32_t *ki = cur0 ? k0 : k1, *vi = cur0 ? v0 : v1, *ko = cur0 ? k1 : k0, *vo = cur0 ? v1 : v0;
    const RsSrc src{ki, vi, nullptr, nullptr, 0, d_n, d_skip, nullptr, shift, nb};
    const bool pk = packed && p == 0;
    if (pk)
      rs_upsweep_kernel<kRsBins, kSrcPacked><<<G, kRsThreads, 0, s>>>(src, hist);
    else
      rs_upsweep_kernel<kRsBins, kSrcKeys><<<G, kRsThreads, 0, s>>>(src, hist);
    GS_LAUNCH_CHECK();
    rs_scan_kernel<<<kRsBins, kRsThreads, 0, s>>>(src, hist, G, totals);
    GS_LAUNCH_CHECK();
    const bool last = p == passes - 1;
    uint32_t *kw = (last && !keep_keys) ? nullptr : ko;
    if (pk && nb == 8)
      rs_downsweep_kernel<kRsBins, kSrcPacked, 8><<<G, kRsThreads, 0, s>>>(src, kw, vo, nullptr, hist, totals);
    else if (pk)
      rs_downsweep_kernel<kRsBins, kSrcPacked, 0><<<G, kRsThreads, 0, s>>>(src, kw, vo, nullptr, hist, totals);
    else if (nb == 8)
      rs_downsweep_kernel<kRsBins, kSrcKeys, 8><<<G, kRsThreads, 0, s>>>(src, kw, vo, nullptr, hist, totals);
    else
      rs_downsweep_kernel<kRsBins, kSrcKeys, 0><<<G, kRsThreads, 0, s>>>(src, kw, vo, nullptr, hist, totals);
    GS_LAUNCH_CHECK();
    cur0 = !cur0;
  }
  *in_b0 = cur0;
  return GS_OK;
}

// Stable sort of the visible records by FP32 depth bits (ties: record order) into
// w.order[0, n_vis): the visible count and depth range first, then 8-bit passes
// over the keys (depth bits minus the smallest visible depth's bits), the later ones
// only while the range needs them (three when the visible depths span less than an
// octave: 24 bits). The first pass compacts the visible records as it sorts.
static gs_status_t depth_sort(const gs_proj_t *proj, int64_t R, const BinWs &w, uint32_t *n_vis,
                              uint32_t *range, cudaStream_t s) {
  const int G = radix_blocks();
  depth_range_kernel<<<num_sms() * 4, 256, 0, s>>>(proj->radius, proj->depth, R, n_vis, range);
  GS_LAUNCH_CHECK();
  static const int kPass[4][2] = {{0, 8}, {8, 8}, {16, 8}, {24, 8}};   // (shift, bits)
  uint32_t *totals = w.hist + (size_t)kDepthBins * kMaxBlocks;
  for (int p = 0; p < 4; ++p) {
    // pass p reads buffer (p + 1) % 2 and writes buffer p % 2 (pass 0: the records)
    uint32_t *ki = (p % 2) ? w.vk0 : w.vk1, *vi = (p % 2) ? w.vv0 : w.vv1;
    uint32_t *ko = (p % 2) ? w.vk1 : w.vk0, *vo = (p % 2) ? w.vv1 : w.vv0;
    const RsSrc src{ki, vi, proj->radius, proj->depth, (uint64_t)R, n_vis, nullptr, range, kPass[p][0],
                    kPass[p][1]};
    if (p == 0) {
      rs_upsweep_kernel<kDepthBins, kSrcRecords><<<G, kRsThreads, 0, s>>>(src, w.hist);
    } else {
      rs_upsweep_kernel<kDepthBins, kSrcDepthKeys><<<G, kRsThreads, 0, s>>>(src, w.hist);
    }
    GS_LAUNCH_CHECK();
    rs_scan_kernel<<<kDepthBins, kRsThreads, 0, s>>>(src, w.hist, G, totals);
    GS_LAUNCH_CHECK();
    if (p == 0) {
      rs_downsweep_kernel<kDepthBins, kSrcRecords, 8><<<G, kRsThreads, 0, s>>>(src, ko, vo, w.order, w.hist, totals);
    } else {
      rs_downsweep_kernel<kDepthBins, kSrcDepthKeys, 8><<<G, kRsThreads, 0, s>>>(src, ko, vo, w.order, w.hist,
                                                                              totals);
    }
    GS_LAUNCH_CHECK();
  }
  return GS_OK;
}

static int bits_for(uint32_t max_value) {
  int b = 1;
  while (b < 32 && (max_value >> b) != 0) ++b;
  return b;
}

// Tile-id bits and the low digit fused into the emission: every bit above it is
// covered by ceil((bits - 8) / 8) radix passes and fbits takes what they leave.
// Fewer digits are cheaper to emit: the emission ranks each step's hits by digit
// and scatters them over 2^fbits output runs (16 digits and one 8-bit pass beat
// 64 digits and one 6-bit pass on a 4056-tile frame).
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

// The frame's plan: tile_sort_plan, or the frame's sort_fused_bits when set.
// Returns false for an override outside 1..min(8, tile bits).
static bool frame_sort_plan(const gs_frame_t *frame, int &tile_bits, int &fbits) {
  tile_sort_plan(frame->n_tiles, tile_bits, fbits);
  const int f = frame->sort_fused_bits;
  if (f == 0) return true;
  if (f < 1 || f > kMaxFusedBits || f > tile_bits) return false;
  fbits = f;
  return true;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_bin_sort_workspace_size(int64_t n_records, int64_t dup_capacity, const gs_frame_t *frame) {
  if (n_records < 0 || dup_capacity < 0) return 0;
  int tile_bits = 32, fbits = kMaxFusedBits;
  if (frame && !frame_sort_plan(frame, tile_bits, fbits)) return 0;
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
  if (!frame_sort_plan(frame, tile_bits, fbits)) return GS_ERR_INVALID_ARG;
  const BinWs w = bin_ws_layout(ws, R, bins->capacity, fbits);
  if (ws_bytes < w.bytes) return GS_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  const int G = scan_blocks();
  uint32_t *n_vis = w.counters + 0, *m_total = w.counters + 1, *overflow = w.counters + 2;
  GS_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 64, s));

  // 1-2. the visible records, compacted in record order and stably sorted by depth
  if (gs_status_t st = depth_sort(proj, R, w, n_vis, w.counters + 8, s)) return st;
  const uint32_t *order = w.order;
  // 3. hits per (low tile digit, batch of 32 depth-ordered records), scanned into
  //    emission cursors; M and the capacity check
  const int64_t n_per_view = R / frame->n_views;
  const int eg = num_sms() * 8;
  const int passes = (tile_bits - fbits + 7) / 8;
  uint32_t *A_k = w.dk0, *A_v = bins->vals, *B_k = w.dk1, *B_v = w.dv1;
  const bool emit_to_A = (passes % 2) == 0;
  // the unit list lives in the list buffer pair the emission does not write
  uint32_t *ut0 = emit_to_A ? B_k : A_k, *uinf = emit_to_A ? B_v : A_v;
  unsigned long long *units = reinterpret_cast<unsigned long long *>(w.counters + 6);
  const float inv_tw = 1.f / (float)frame->tile_w;
  bin_count_kernel<<<eg, 256, 0, s>>>(*proj, order, n_vis, frame->cams_dev, frame->n_views, n_per_view,
                                      frame->tile_w, frame->tile_h, inv_tw, fbits, w.dhist, w.ubatch, ut0, uinf,
                                      units, (uint64_t)bins->capacity, w.counters + 3);
  GS_LAUNCH_CHECK();
  HistScan hs{w.dhist, n_vis, fbits, (uint64_t)bins->capacity, m_total, overflow, units, bins->d_count, d_error};
  if (gs_status_t st = run_scan(hs, w.block_sums, G, s)) return st;
  // 4. emit (tile, record) partitioned by the low digit, in depth order within it,
  //    into the buffer the remaining passes end in
  //    With exactly one pass to follow (9-16 tile-id bits), the hits go out as packed
  //    (tile, record) pairs over the contiguous workspace words dk1 | dv1, which
  //    hold 8 * capacity bytes, and that pass reads them.
  const bool packed = passes == 1;
  if (packed && reinterpret_cast<const char *>(w.dv1) - reinterpret_cast<const char *>(w.dk1) <
                    (ptrdiff_t)(4 * (size_t)bins->capacity))
    return GS_ERR_INVALID_ARG;   // the layout keeps dk1 | dv1 adjacent; never taken
  if (packed)
    bin_emit_kernel<true><<<eg, 256, 0, s>>>(order, n_vis, overflow, fbits, w.dhist, w.ubatch, ut0, uinf, B_k,
                                             nullptr, w.counters + 4, (uint64_t)bins->capacity);
  else
    bin_emit_kernel<false><<<eg, 256, 0, s>>>(order, n_vis, overflow, fbits, w.dhist, w.ubatch, ut0, uinf,
                                              emit_to_A ? A_k : B_k, emit_to_A ? A_v : B_v, w.counters + 4,
                                              (uint64_t)bins->capacity);
  GS_LAUNCH_CHECK();
  // 5. stable sort by the remaining tile-id bits
  bool res0 = true;
  if (emit_to_A) {
    if (gs_status_t st = radix_sort(A_k, A_v, B_k, B_v, m_total, overflow, fbits, tile_bits, true, w.hist, s, &res0))
      return st;
  } else {
    if (gs_status_t st = radix_sort(B_k, B_v, A_k, A_v, m_total, overflow, fbits, tile_bits, true, w.hist, s, &res0,
                                    packed))
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
