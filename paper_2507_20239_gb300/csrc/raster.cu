// Front-to-back alpha compositing (the paper's Eq. 2) and its gradient.
//
// Forward: one CTA per tile, two horizontally adjacent pixels per thread; each warp
// owns an 8x8 block of the tile and walks the tile's depth-ordered list on its own,
// 32 entries at a time, keeping only the entries whose footprint ellipse (where
// alpha can reach the 1/255 floor) meets its block. A pixel stops before the entry
// that would drive its transmittance below 1e-4; a warp leaves once its 64 pixels
// have stopped. Optionally it stores each pixel's stop index and, for the per-splat
// backward, a checkpoint (T, composited colour) every 64 list entries.
//
// Both backward kernels re-walk the lists front to back with exactly the forward's
// FP32 decisions and need, per pixel, only <dL/dout, out>:
//   dL/dsigma_i = T_i <c_i, g> - (<out, g> - sum_{j<=i} <c_j, g> sigma_j T_j) / (1 - sigma_i).
// Per (pixel, Gaussian) they accumulate six moments of the falloff gradient and
// three colour terms, turned into the record gradients once per (tile, record).
// raster_bwd_kernel is parallel over pixels: the terms are summed over a thread's
// two pixels in registers, across the warp with a transposing shuffle reduction and
// across the CTA's warps in shared memory, then added with vector reductions.
// raster_bwd_splat_kernel is parallel over list entries (one lane per entry, the
// pixels flowing through the warp from the forward's checkpoints), so each lane
// sums its own entry's terms and no reduction is needed.
#include "gs_common.cuh"

namespace gs {

#ifdef GS_DEBUG
GS_DEBUG_TAKE(debug_take_raster)
#endif

struct TileCoord {
  int view, tx, ty, W, H;
  int64_t pix_off;
};

__device__ __forceinline__ TileCoord tile_coord(const gs_camera_t *cams, int n_views, int tile) {
  TileCoord c;
  c.view = view_of_tile(cams, n_views, tile);
  const gs_camera_t &cam = cams[c.view];
  const int lt = tile - cam.tile_offset;
  c.tx = lt % cam.grid_x;
  c.ty = lt / cam.grid_x;
  c.W = cam.width;
  c.H = cam.height;
  c.pix_off = cam.pixel_offset;
  return c;
}

// Checkpoint buckets of the per-splat backward: list positions [32 b, 32 b + 32) of
// tile t (whose list starts at s_t in the sorted order) own bucket floor(s_t / 32) +
// t + b. Consecutive tiles' buckets never overlap (floor(s_t / 32) + ceil(len_t / 32)
// <= floor(s_{t+1} / 32) + 1), so no per-tile scan is needed and, for M listed
// entries, every bucket is below ceil(M / 32) + n_tiles.
__device__ __forceinline__ uint64_t ckpt_bucket(uint32_t list_start, uint32_t tile) {
  return (uint64_t)(list_start >> 5) + tile;
}

// Checkpoint buffer: only the (bucket, 8 x 8 pixel block) pairs a forward warp
// actually walks hold data. Layout (caller-owned, sized by gs_raster_ckpt_size):
//   pools [kCkptPools] u32       slots claimed from each pool by the last forward
//   table [buckets x blocks] u32 slot of (bucket, block), kCkptNone past a pool's end
//   slots [n_slots][64] float4   (T, R, G, B) of the block's 64 pixels, row-major
// A warp claims a slot from pool (tile * blocks + block) mod n_pools, which spreads
// the claims over n_pools counters (a power of two up to kCkptPools, about 32 of the
// frame's blocks each, so that pools fill evenly); pool p owns slots [p P, (p + 1) P),
// P = floor(n_slots / n_pools). A buffer with a slot for every table entry maps
// the entry to its own slot instead (nothing can overflow; the pools still count).
// The table needs no clearing: the backward only looks up (bucket, block) pairs
// holding a live pixel, which the forward walked in the same frame.
constexpr int kCkptPools = 256;
constexpr uint32_t kCkptNone = 0xffffffffu;

struct CkptLayout {
  uint32_t *pools, *table;
  float4 *slots;
  uint64_t n_slots, pool_size, table_entries;
  uint32_t n_pools;
  size_t bytes;
};

// Pools of a frame with `blocks` 8 x 8 blocks in all: the largest power of two up to
// kCkptPools with at least 32 blocks per pool.
__host__ __device__ inline uint32_t ckpt_pools(uint64_t blocks) {
  uint32_t p = 1;
  while (p < (uint32_t)kCkptPools && (uint64_t)p * 2 * 32 <= blocks) p *= 2;
  return p;
}

__host__ __device__ inline size_t ckpt_a256(size_t x) { return (x + 255) & ~(size_t)255; }

__host__ __device__ inline CkptLayout ckpt_layout(void *base, uint64_t table_entries, uint64_t n_slots,
                                                   uint32_t n_pools = kCkptPools) {
  CkptLayout L;
  char *p = static_cast<char *>(base);
  size_t off = 0;
  L.pools = reinterpret_cast<uint32_t *>(p + off);
  off += ckpt_a256(4 * (size_t)kCkptPools);
  L.table = reinterpret_cast<uint32_t *>(p + off);
  off += ckpt_a256(4 * (size_t)table_entries);
  L.slots = reinterpret_cast<float4 *>(p + off);
  off += (size_t)n_slots * 64 * sizeof(float4);
  L.n_slots = n_slots;
  L.n_pools = n_pools;
  L.pool_size = n_slots / n_pools;
  L.table_entries = table_entries;
  L.bytes = off;
  return L;
}

// Pixel mapping: warp w owns the 8x8 block (w % (TW/8), w / (TW/8)) of the tile;
// lane l owns pixels (2 (l % 4), l / 4) and (2 (l % 4) + 1, l / 4) of that block.
template <int TW>
__device__ __forceinline__ void pixel_of(int t, int &lx, int &ly) {
  const int w = t >> 5, l = t & 31;
  lx = (w % (TW / 8)) * 8 + 2 * (l & 3);
  ly = (w / (TW / 8)) * 8 + (l >> 2);
}

// Stage list entry r: position, pre-scaled conic (k A, beta, k gamma, o) with
// k = -1/2 log2 e, colour; colour.w holds the mask of the tile's BW x BH blocks
// (one per warp) whose pixel centres the footprint ellipse (q <= q_max with the
// binning's margin) meets, so a warp can skip records that miss its block. co_raw
// returns the unscaled (A, beta, gamma, o).
template <int TW, int TH, int BW, int BH>
__device__ __forceinline__ void stage(const float2 *__restrict__ mean2d, const float4 *__restrict__ conic_o,
                                      const float4 *__restrict__ rgb, uint32_t r, int x0, int y0, int W, int H,
                                      float2 &xy, float4 &co, float4 &c, float4 &co_raw) {
  constexpr int NB = (TW / BW) * (TH / BH);
  xy = mean2d[r];
  co_raw = conic_o[r];
  c = rgb[r];
  uint32_t m = 1u;
  if (NB > 1) {
    const EllipseRows e = ellipse_rows(xy.x, xy.y, co_raw.x, co_raw.y, co_raw.z, c.w * kBinMargin);
    m = 0u;
#pragma unroll
    for (int by = 0; by < TH / BH; ++by) {
      const int yb = y0 + by * BH;
      float xl, xr;
      if (yb >= H || !row_span(e, (float)yb + 0.5f, (float)min(yb + BH, H) - 0.5f, xl, xr)) continue;
#pragma unroll
      for (int bx = 0; bx < TW / BW; ++bx) {
        const int xb = x0 + bx * BW;
        if (xb < W && (float)min(xb + BW, W) - 0.5f >= xl && (float)xb + 0.5f <= xr) m |= 1u << (by * (TW / BW) + bx);
      }
    }
  }
  co = make_float4(__fmul_rn(co_raw.x, kNegHalfLog2e), co_raw.y, __fmul_rn(co_raw.z, kNegHalfLog2e), co_raw.w);
  c.w = __uint_as_float(m);
}

// The staged positions j < cnt whose block mask has this warp's bit, in order, into
// list[] (one ballot per 32 entries); returns their number. The walk then visits
// only those, without a per-entry mask test.
__device__ __forceinline__ int warp_select(const float4 *s_rgb, int cnt, int warp, int lane, uint8_t *list) {
  const uint32_t lt = (1u << lane) - 1u;
  int nsel = 0;
  for (int j0 = 0; j0 < cnt; j0 += 32) {
    const int j = j0 + lane;
    const bool sel = j < cnt && ((__float_as_uint(s_rgb[j].w) >> warp) & 1u);
    const uint32_t b = __ballot_sync(0xffffffffu, sel);
    if (sel) list[nsel + __popc(b & lt)] = (uint8_t)j;
    nsel += __popc(b);
  }
  __syncwarp();
  return nsel;
}

// Forward without CTA-wide steps: each warp walks its tile's list on its own, 32
// entries at a time. Lane l gathers entry base + l, tests it against the warp's
// 8x8 block (the ellipse's x-extent over the block's rows against its columns) and
// stages it in the warp's shared slots if it passes; the warp then composites the
// passing entries in list order. A warp leaves as soon as its 64 pixels have
// stopped, so neither barriers nor finished neighbours hold it (one-warp CTAs,
// which also free a finished warp's slot, measured no faster).
struct FwdArgs {
  const float2 *__restrict__ mean2d;
  const float4 *__restrict__ conic_o;
  const float4 *__restrict__ rgb;
  const uint32_t *__restrict__ vals;
  const uint2 *__restrict__ ranges;
  const gs_camera_t *__restrict__ cams;
  int n_views;
  float bg0, bg1, bg2;
  float *__restrict__ image;
  float *__restrict__ T_final;
  uint32_t *__restrict__ stop_out;
  CkptLayout ckpt;
  uint64_t n_records, list_cap;   // bounds of the record ids and list positions (debug checks)
};

// One warp's 8 x 8 block `warp` of `tile`, with the warp's staging slots.
template <int TW, int TH, bool CKPT>
__device__ __forceinline__ void fwd_warp_block(const FwdArgs &a, int tile, int warp, int lane, float2 *sxy,
                                               float4 *sco, float4 *srgb) {
  constexpr int NW = TW * TH / 64;
  const float2 *__restrict__ mean2d = a.mean2d;
  const float4 *__restrict__ conic_o = a.conic_o;
  const float4 *__restrict__ rgb = a.rgb;
  const uint32_t *__restrict__ vals = a.vals;
  const CkptLayout &ckpt = a.ckpt;
  const TileCoord tc = tile_coord(a.cams, a.n_views, tile);
  int lx, ly;
  pixel_of<TW>(warp * 32 + lane, lx, ly);
  const int py = tc.ty * TH + ly;
  const int px = tc.tx * TW + lx;
  const bool in0 = py < tc.H && px < tc.W, in1 = py < tc.H && px + 1 < tc.W;
  const float fy = (float)py + 0.5f;
  const float2 fx = f2((float)px + 0.5f, (float)px + 1.5f), ONE = f2(1.f);
  // the warp's block of pixel centres
  const int bx = tc.tx * TW + (warp % (TW / 8)) * 8, by = tc.ty * TH + (warp / (TW / 8)) * 8;
  const float X0 = (float)bx + 0.5f, X1 = (float)min(bx + 8, tc.W) - 0.5f;
  const float Y0 = (float)by + 0.5f, Y1 = (float)min(by + 8, tc.H) - 0.5f;
  float2 T = f2(1.f), cr = f2(0.f), cg = f2(0.f), cb = f2(0.f);   // (pixel 0, pixel 1)
  uint32_t st0 = 0, st1 = 0;
  bool done0 = !in0, done1 = !in1;
  uint2 rg = a.ranges[tile];
  if (!GS_CHECK(rg.x <= rg.y && (uint64_t)rg.y <= a.list_cap, 2, tile)) rg = make_uint2(0u, 0u);
  const int n = (int)(rg.y - rg.x);
  // software pipeline: the record id two steps ahead, the record one step ahead
  uint32_t r_next = lane < n ? vals[rg.x + lane] : 0u;
  uint32_t r_next2 = 32 + lane < n ? vals[rg.x + 32 + lane] : 0u;
  float2 xy_n = make_float2(0.f, 0.f);
  float4 co_n = make_float4(0.f, 0.f, 0.f, 0.f), c_n = co_n;
  if (lane < n && GS_CHECK(r_next < a.n_records, 1, r_next)) {
    xy_n = mean2d[r_next];
    co_n = conic_o[r_next];
    c_n = rgb[r_next];
  }
  // checkpoint slot claims (lane 0): the pool of this (tile, block), and the claim for
  // the first step
  const uint32_t pool = CKPT ? (((uint32_t)tile * NW + warp) & (ckpt.n_pools - 1)) : 0u;
  uint32_t claim = 0;
  if (CKPT && lane == 0 && n > 0) claim = atomicAdd(ckpt.pools + pool, 1u);
  for (int base = 0; base < n; base += 32) {
    if (__all_sync(0xffffffffu, done0 && done1)) break;
    if (CKPT && (base & 63) == 0) {
      // state before list position base: (T, accumulated colour) for the per-splat
      // backward (whose buckets are 64 entries long), in the slot claimed for (32-entry
      // step, this warp's 8 x 8 block); the claim for the next checkpoint is issued now
      // and its result used two steps later, so the atomic's round trip overlaps the
      // compositing
      uint32_t slot = kCkptNone;
      if (lane == 0) {
        const uint64_t idx = (ckpt_bucket(rg.x, tile) + (uint64_t)(base >> 5)) * NW + warp;
        if (ckpt.n_slots >= ckpt.table_entries) slot = (uint32_t)idx;      // room for every pair
        else if (claim < ckpt.pool_size) slot = (uint32_t)(pool * ckpt.pool_size + claim);
        if (GS_CHECK(idx < ckpt.table_entries, 3, idx)) ckpt.table[idx] = slot;
        if (base + 64 < n) claim = atomicAdd(ckpt.pools + pool, 1u);
      }
      slot = __shfl_sync(0xffffffffu, slot, 0);
      if (slot != kCkptNone && GS_CHECK(slot < ckpt.n_slots, 3, slot)) {
        float4 *ck = ckpt.slots + (uint64_t)slot * 64 + (lane >> 2) * 8 + 2 * (lane & 3);
        if (!done0) ck[0] = make_float4(T.x, cr.x, cg.x, cb.x);
        if (!done1) ck[1] = make_float4(T.y, cr.y, cg.y, cb.y);
      }
    }
    const int j = base + lane;
    const float2 xy = xy_n;
    const float4 co = co_n, c = c_n;
    // issue the next step's gathers and the id after it before compositing this one
    r_next = r_next2;
    if (j + 32 < n && GS_CHECK(r_next < a.n_records, 1, r_next)) {
      xy_n = mean2d[r_next];
      co_n = conic_o[r_next];
      c_n = rgb[r_next];
    }
    r_next2 = j + 64 < n ? vals[rg.x + j + 64] : 0u;
    bool sel = false;
    if (j < n) {
      const EllipseRows e = ellipse_rows(xy.x, xy.y, co.x, co.y, co.z, c.w * kBinMargin);
      float xl, xr;
      sel = row_span(e, Y0, Y1, xl, xr) && X1 >= xl && X0 <= xr;
      if (sel) {
        sxy[lane] = xy;
        sco[lane] = make_float4(__fmul_rn(co.x, kNegHalfLog2e), co.y, __fmul_rn(co.z, kNegHalfLog2e), co.w);
        srgb[lane] = c;
      }
    }
    uint32_t b = __ballot_sync(0xffffffffu, sel);
    __syncwarp();
    // both pixels in packed pairs, without branches: an entry a pixel skips (done,
    // below the floor, or the one that would cross the cut-off) gets weight 0 and
    // leaves T, the colour and the stop index as they are
    while (b) {
      const int i = __ffs(b) - 1;
      b &= b - 1u;
      const float2 xy = sxy[i];
      const float4 co = sco[i];
      float2 al;
      if (CKPT) {
        // the falloff in scalar form (its operands are the entry's, broadcast to both
        // pixels, so packing them costs register moves); the two pixels share dy and
        // gamma dy^2: lane for lane the operations and roundings of falloff(). Measured
        // faster with checkpoints (0.319 -> 0.305 ms on the benchmark view) and slower
        // without (0.270 -> 0.300 ms), so each form keeps the faster one
        const float dx0 = __fsub_rn(xy.x, fx.x), dx1 = __fsub_rn(xy.x, fx.y), dy = __fsub_rn(xy.y, fy);
        const float gdd = __fmul_rn(co.z, __fmul_rn(dy, dy));
        const float t0 = __fmaf_rn(co.y, dy, dx0), t1 = __fmaf_rn(co.y, dy, dx1);
        const float e0 = __fmaf_rn(__fmul_rn(co.x, t0), t0, gdd), e1 = __fmaf_rn(__fmul_rn(co.x, t1), t1, gdd);
        al = f2(fminf(kAlphaMax, __fmul_rn(co.w, ex2_approx(e0))), fminf(kAlphaMax, __fmul_rn(co.w, ex2_approx(e1))));
      } else {
        al = falloff2(xy.x, xy.y, co.x, co.y, co.z, co.w, fx, fy).alpha;
      }
      const bool a0 = !done0 && al.x >= kAlphaMin, a1 = !done1 && al.y >= kAlphaMin;
      // transmittance and weight: genuinely per-pixel pairs, packed
      const float2 Tn = f2_mul(T, f2_sub(ONE, al));
      const bool c0 = a0 && !(Tn.x < kTMin), c1 = a1 && !(Tn.y < kTMin);
      done0 = done0 || (a0 && !c0);
      done1 = done1 || (a1 && !c1);
      const float2 w = f2_mul(f2(c0 ? al.x : 0.f, c1 ? al.y : 0.f), T);
      const float4 c = srgb[i];
      if (CKPT) {
        cr = f2(fmaf(c.x, w.x, cr.x), fmaf(c.x, w.y, cr.y));
        cg = f2(fmaf(c.y, w.x, cg.x), fmaf(c.y, w.y, cg.y));
        cb = f2(fmaf(c.z, w.x, cb.x), fmaf(c.z, w.y, cb.y));
      } else {
        cr = f2_fma(f2(c.x), w, cr);
        cg = f2_fma(f2(c.y), w, cg);
        cb = f2_fma(f2(c.z), w, cb);
      }
      T = f2(c0 ? Tn.x : T.x, c1 ? Tn.y : T.y);
      st0 = c0 ? base + i + 1 : st0;
      st1 = c1 ? base + i + 1 : st1;
    }
    __syncwarp();
  }
  const float T0 = T.x, T1 = T.y;
  const float r0 = cr.x, g0 = cg.x, b0 = cb.x, r1 = cr.y, g1 = cg.y, b1 = cb.y;
  const int64_t p0 = (int64_t)py * tc.W + px;
  const int64_t plane = (int64_t)tc.W * tc.H;
  float *img = a.image + 3 * tc.pix_off;
  if (in0) {
    img[p0] = fmaf(T0, a.bg0, r0);
    img[plane + p0] = fmaf(T0, a.bg1, g0);
    img[2 * plane + p0] = fmaf(T0, a.bg2, b0);
    a.T_final[tc.pix_off + p0] = T0;
    if (a.stop_out) a.stop_out[tc.pix_off + p0] = st0;
  }
  if (in1) {
    img[p0 + 1] = fmaf(T1, a.bg0, r1);
    img[plane + p0 + 1] = fmaf(T1, a.bg1, g1);
    img[2 * plane + p0 + 1] = fmaf(T1, a.bg2, b1);
    a.T_final[tc.pix_off + p0 + 1] = T1;
    if (a.stop_out) a.stop_out[tc.pix_off + p0 + 1] = st1;
  }
}

// One CTA per tile, warp w on the tile's block w.
template <int TW, int TH, bool CKPT>
__global__ void __launch_bounds__(TW *TH / 2) raster_fwd_warp_kernel(const FwdArgs a) {
  constexpr int NW = TW * TH / 64;
  __shared__ float2 s_xy[NW][32];
  __shared__ float4 s_co[NW][32];
  __shared__ float4 s_rgb[NW][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  fwd_warp_block<TW, TH, CKPT>(a, blockIdx.x, warp, lane, s_xy[warp], s_co[warp], s_rgb[warp]);
}

// Persistent form: a resident grid whose warps claim (tile, block) units from a
// counter (zeroed before the launch) in tile order, so that a warp whose block
// stopped early takes the next unit instead of idling until its CTA's slowest warp
// is done. Units are independent; no warp ever waits on another.
constexpr int kQueueWarps = 4;

template <int TW, int TH, bool CKPT>
__global__ void __launch_bounds__(32 * kQueueWarps) raster_fwd_queue_kernel(const FwdArgs a, int n_tiles,
                                                                           uint32_t *queue) {
  constexpr int NW = TW * TH / 64;
  __shared__ float2 s_xy[kQueueWarps][32];
  __shared__ float4 s_co[kQueueWarps][32];
  __shared__ float4 s_rgb[kQueueWarps][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t units = (uint32_t)n_tiles * NW;
  for (;;) {
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(queue, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= units) break;
    fwd_warp_block<TW, TH, CKPT>(a, (int)(u / NW), (int)(u % NW), lane, s_xy[w], s_co[w], s_rgb[w]);
    __syncwarp();
  }
}

template <int TW, int TH, bool COUNT>
__global__ void __launch_bounds__(TW *TH / 2) raster_fwd_kernel(
    const float2 *__restrict__ mean2d, const float4 *__restrict__ conic_o, const float4 *__restrict__ rgb,
    const uint32_t *__restrict__ vals, const uint2 *__restrict__ ranges, const gs_camera_t *__restrict__ cams,
    int n_views, float bg0, float bg1, float bg2, float *__restrict__ image, float *__restrict__ T_final,
    uint32_t *__restrict__ stop_out, uint32_t *__restrict__ counts, uint64_t n_records, uint64_t list_cap) {
  constexpr int NT = TW * TH / 2;
  static_assert(NT <= 256, "list positions are bytes");
  __shared__ float2 s_xy[NT];
  __shared__ float4 s_co[NT];
  __shared__ float4 s_rgb[NT];
  __shared__ uint8_t s_list[NT / 32][NT];
  const TileCoord tc = tile_coord(cams, n_views, blockIdx.x);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  int lx, ly;
  pixel_of<TW>(t, lx, ly);
  const int py = tc.ty * TH + ly;
  const int px = tc.tx * TW + lx;
  const bool in0 = py < tc.H && px < tc.W, in1 = py < tc.H && px + 1 < tc.W;
  const float fy = (float)py + 0.5f, fx0 = (float)px + 0.5f, fx1 = (float)px + 1.5f;
  float T0 = 1.f, T1 = 1.f;
  float r0 = 0.f, g0 = 0.f, b0 = 0.f, r1 = 0.f, g1 = 0.f, b1 = 0.f;
  uint32_t st0 = 0, st1 = 0;
  uint32_t ex0 = 0, ex1 = 0, nc0 = 0, nc1 = 0;
  bool done0 = !in0, done1 = !in1;
  uint2 rg = ranges[blockIdx.x];
  if (!GS_CHECK(rg.x <= rg.y && (uint64_t)rg.y <= list_cap, 2, blockIdx.x)) rg = make_uint2(0u, 0u);
  const int n = (int)(rg.y - rg.x);
  for (int base = 0; base < n; base += NT) {
    if (__syncthreads_count(!(done0 && done1)) == 0) break;
    if (base + t < n) {
      float4 co_raw;
      const uint32_t r = vals[rg.x + base + t];
      if (GS_CHECK(r < n_records, 1, r))
        stage<TW, TH, 8, 8>(mean2d, conic_o, rgb, r, tc.tx * TW, tc.ty * TH, tc.W, tc.H, s_xy[t], s_co[t],
                            s_rgb[t], co_raw);
    }
    __syncthreads();
    if (__all_sync(0xffffffffu, done0 && done1)) continue;
    const int cnt = min(NT, n - base);
    const int nsel = COUNT ? cnt : warp_select(s_rgb, cnt, warp, lane, s_list[warp]);
#pragma unroll 2
    for (int i = 0; i < nsel; ++i) {
      const int j = COUNT ? i : s_list[warp][i];
      const float2 xy = s_xy[j];
      const float4 co = s_co[j];
      if (!done0) {
        if (COUNT) ++ex0;
        const Falloff f = falloff(xy.x, xy.y, co.x, co.y, co.z, co.w, fx0, fy);
        if (f.alpha >= kAlphaMin) {
          const float Tn = __fmul_rn(T0, __fsub_rn(1.f, f.alpha));
          if (Tn < kTMin) {
            done0 = true;
          } else {
            if (COUNT) ++nc0;
            const float4 c = s_rgb[j];
            const float w = f.alpha * T0;
            r0 = fmaf(c.x, w, r0); g0 = fmaf(c.y, w, g0); b0 = fmaf(c.z, w, b0);
            T0 = Tn;
            st0 = base + j + 1;
          }
        }
      }
      if (!done1) {
        if (COUNT) ++ex1;
        const Falloff f = falloff(xy.x, xy.y, co.x, co.y, co.z, co.w, fx1, fy);
        if (f.alpha >= kAlphaMin) {
          const float Tn = __fmul_rn(T1, __fsub_rn(1.f, f.alpha));
          if (Tn < kTMin) {
            done1 = true;
          } else {
            if (COUNT) ++nc1;
            const float4 c = s_rgb[j];
            const float w = f.alpha * T1;
            r1 = fmaf(c.x, w, r1); g1 = fmaf(c.y, w, g1); b1 = fmaf(c.z, w, b1);
            T1 = Tn;
            st1 = base + j + 1;
          }
        }
      }
    }
  }
  const int64_t p0 = (int64_t)py * tc.W + px;
  if (COUNT) {
    if (in0) reinterpret_cast<uint2 *>(counts)[tc.pix_off + p0] = make_uint2(ex0, nc0);
    if (in1) reinterpret_cast<uint2 *>(counts)[tc.pix_off + p0 + 1] = make_uint2(ex1, nc1);
    return;
  }
  const int64_t plane = (int64_t)tc.W * tc.H;
  float *img = image + 3 * tc.pix_off;
  if (in0) {
    img[p0] = fmaf(T0, bg0, r0);
    img[plane + p0] = fmaf(T0, bg1, g0);
    img[2 * plane + p0] = fmaf(T0, bg2, b0);
    T_final[tc.pix_off + p0] = T0;
    if (stop_out) stop_out[tc.pix_off + p0] = st0;
  }
  if (in1) {
    img[p0 + 1] = fmaf(T1, bg0, r1);
    img[plane + p0 + 1] = fmaf(T1, bg1, g1);
    img[2 * plane + p0 + 1] = fmaf(T1, bg2, b1);
    T_final[tc.pix_off + p0 + 1] = T1;
    if (stop_out) stop_out[tc.pix_off + p0 + 1] = st1;
  }
}

// Sum 9 per-lane values over the warp and add the totals to acc[0..8] in shared
// memory. Values 0..7 are reduced by a transposing butterfly (each step exchanges
// half of the remaining values), value 8 by a plain butterfly: 14 shuffles.
__device__ __forceinline__ void warp_reduce9_add(const float v[9], float *acc, int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float a[4], b[2];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float send = b4 ? v[k] : v[k + 4];
    const float keep = b4 ? v[k + 4] : v[k];
    a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = b3 ? a[k] : a[k + 2];
    const float keep = b3 ? a[k + 2] : a[k];
    b[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float c;
  {
    const float send = b2 ? b[0] : b[1];
    const float keep = b2 ? b[1] : b[0];
    c = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  float e = v[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((lane & 3) == 0) atomicAdd(&acc[lane >> 2], c);   // value index 4*b4 + 2*b3 + b2
  if (lane == 0) atomicAdd(&acc[8], e);
}

// R = <out, g> - sum_{j<=i} <c_j, g> sigma_j T_j, the numerator of the second term
// of dL/dsigma_i, kept as a running remainder.
struct PixBwd {
  float fx, T, R, d0, d1, d2;
  bool done;
  uint32_t stop;   // STOP: one past the pixel's last composited list position
};

// One pixel's contribution of the current Gaussian. With m = dL/dalpha * G on
// pixels where alpha is not clamped at 0.99, v[9] accumulates the moments
// (sum m t, sum m dy, sum m t^2, sum m t dy, sum m dy^2, sum m) and the colour
// gradient (sum d alpha T); the per-record epilogue turns the moments into the
// gradients w.r.t. (u, v, A, beta, gamma, o) of the quadratic form
// A (dx + beta dy)^2 + gamma dy^2 with dG/dq = -G/2. co = (k A, beta, k gamma, o).
// STOP: the forward's stop index bounds the walk (list position jg); before it the
// transmittance cut-off cannot trigger, so it is not tested.
template <bool STOP>
__device__ __forceinline__ bool pix_bwd(PixBwd &p, uint32_t jg, float fy, const float2 xy, const float4 co,
                                        const float4 c, float *v) {
  if (STOP ? jg >= p.stop : p.done) return false;
  const Falloff f = falloff(xy.x, xy.y, co.x, co.y, co.z, co.w, p.fx, fy);
  if (!(f.alpha >= kAlphaMin)) return false;
  const float one_m = __fsub_rn(1.f, f.alpha);
  const float Tn = __fmul_rn(p.T, one_m);
  if (!STOP && Tn < kTMin) {
    p.done = true;
    return false;
  }
  const float w = f.alpha * p.T;
  const float cd = c.x * p.d0 + c.y * p.d1 + c.z * p.d2;
  p.R = fmaf(-cd, w, p.R);
  const float dLda = p.T * cd - __fdividef(p.R, one_m);
  p.T = Tn;
  v[6] = fmaf(p.d0, w, v[6]);
  v[7] = fmaf(p.d1, w, v[7]);
  v[8] = fmaf(p.d2, w, v[8]);
  const float m = f.raw <= kAlphaMax ? dLda * f.G : 0.f;
  const float mt = m * f.t, mdy = m * f.dy;
  v[0] += mt;
  v[1] += mdy;
  v[2] = fmaf(mt, f.t, v[2]);
  v[3] = fmaf(mt, f.dy, v[3]);
  v[4] = fmaf(mdy, f.dy, v[4]);
  v[5] += m;
  return true;
}

// PX pixels per thread: lane l of warp w owns the 2 x (PX/2) block at column
// 2 (l % 4), row (PX/2) (l / 4) of the warp's 8 x 4PX block, so the per-entry
// overhead and the warp reduction are shared by PX pixels.
// STOP: stop_in holds the forward's per-pixel stop indices; each warp walks up to
// its pixels' largest, the CTA up to its largest. HALF: each CTA step stages half
// as many list entries as the CTA has threads (a finer step, more barriers).
template <int TW, int TH, int PX, bool STOP, bool HALF>
__global__ void __launch_bounds__(TW *TH / PX) raster_bwd_kernel(
    const float2 *__restrict__ mean2d, const float4 *__restrict__ conic_o, const float4 *__restrict__ rgb,
    const uint32_t *__restrict__ vals, const uint2 *__restrict__ ranges, const gs_camera_t *__restrict__ cams,
    int n_views, const float *__restrict__ image, const float *__restrict__ d_image,
    const uint32_t *__restrict__ stop_in, float *__restrict__ g_mean2d, float *__restrict__ g_co,
    float *__restrict__ g_rgb, uint64_t n_records, uint64_t list_cap) {
  constexpr int NT = TW * TH / PX, CH = HALF ? NT / 2 : NT, BW = 8, BH = 4 * PX;
  __shared__ float2 s_xy[CH];
  __shared__ float4 s_co[CH];
  __shared__ float4 s_rgb[CH];
  __shared__ uint32_t s_rec[CH];
  __shared__ float4 s_cu[CH];
  __shared__ float s_acc[CH * 9];
  __shared__ uint8_t s_list[NT / 32][CH];
  static_assert(NT <= 256, "list positions are bytes");
  const TileCoord tc = tile_coord(cams, n_views, blockIdx.x);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int lx = (warp % (TW / BW)) * BW + 2 * (lane & 3);
  const int ly = (warp / (TW / BW)) * BH + (PX / 2) * (lane >> 2);
  const int64_t plane = (int64_t)tc.W * tc.H;
  const float *img = image + 3 * tc.pix_off;
  const float *dim = d_image + 3 * tc.pix_off;
  PixBwd q[PX];
  float fy[PX / 2];
#pragma unroll
  for (int k = 0; k < PX; ++k) {
    const int px = tc.tx * TW + lx + (k & 1), py = tc.ty * TH + ly + (k >> 1);
    const bool in = py < tc.H && px < tc.W;
    q[k] = PixBwd{(float)px + 0.5f, 1.f, 0.f, 0.f, 0.f, 0.f, !in, 0u};
    if ((k & 1) == 0) fy[k >> 1] = (float)py + 0.5f;
    if (in) {
      const int64_t p = (int64_t)py * tc.W + px;
      if (STOP) q[k].stop = stop_in[tc.pix_off + p];
      q[k].d0 = dim[p]; q[k].d1 = dim[plane + p]; q[k].d2 = dim[2 * plane + p];
      q[k].R = q[k].d0 * img[p] + q[k].d1 * img[plane + p] + q[k].d2 * img[2 * plane + p];
    }
  }
  auto all_done = [&]() {
    bool d = true;
#pragma unroll
    for (int k = 0; k < PX; ++k) d = d && q[k].done;
    return d;
  };
  uint2 rg = ranges[blockIdx.x];
  if (!GS_CHECK(rg.x <= rg.y && (uint64_t)rg.y <= list_cap, 2, blockIdx.x)) rg = make_uint2(0u, 0u);
  int n = (int)(rg.y - rg.x);
  uint32_t wstop = 0;
  if (STOP) {
    __shared__ uint32_t s_cstop;
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < PX; ++k) m = max(m, q[k].stop);
    wstop = __reduce_max_sync(0xffffffffu, m);
    if (t == 0) s_cstop = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&s_cstop, wstop);
    __syncthreads();
    n = min(n, (int)s_cstop);
  }
  for (int base = 0; base < n; base += CH) {
    if (STOP) {
      __syncthreads();
    } else if (__syncthreads_count(!all_done()) == 0) {
      break;
    }
    const int cnt = min(CH, n - base);
    if (t < cnt) {
      uint32_t r = vals[rg.x + base + t];
      if (!GS_CHECK(r < n_records, 1, r)) r = 0;
      s_rec[t] = r;
      stage<TW, TH, BW, BH>(mean2d, conic_o, rgb, r, tc.tx * TW, tc.ty * TH, tc.W, tc.H, s_xy[t], s_co[t], s_rgb[t],
                            s_cu[t]);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k)
      if (k * NT + t < 9 * CH) s_acc[k * NT + t] = 0.f;
    __syncthreads();
    const int jend = STOP ? min(cnt, (int)wstop - base) : cnt;
    if (STOP ? jend > 0 : !__all_sync(0xffffffffu, all_done())) {
      float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const int nsel = warp_select(s_rgb, jend, warp, lane, s_list[warp]);
      for (int i = 0; i < nsel; ++i) {
        const int j = s_list[warp][i];
        const float4 c = s_rgb[j];
        const float2 xy = s_xy[j];
        const float4 co = s_co[j];
        bool any = false;
#pragma unroll
        for (int k = 0; k < PX; ++k) any |= pix_bwd<STOP>(q[k], (uint32_t)(base + j), fy[k >> 1], xy, co, c, v);
        if (__any_sync(0xffffffffu, any)) {
          warp_reduce9_add(v, s_acc + j * 9, lane);
#pragma unroll
          for (int k = 0; k < 9; ++k) v[k] = 0.f;   // lanes without a contribution kept zeros
        }
      }
    }
    __syncthreads();
    if (t < cnt) {
      const float *a = s_acc + t * 9;
      const float mt = a[0], mdy = a[1], mtt = a[2], mtdy = a[3], mdydy = a[4], m = a[5];
      const float k0 = a[6], k1 = a[7], k2 = a[8];
      if (mt != 0.f || mdy != 0.f || mtt != 0.f || mtdy != 0.f || mdydy != 0.f || m != 0.f || k0 != 0.f ||
          k1 != 0.f || k2 != 0.f) {
        const uint32_t r = s_rec[t];
        const float4 cu = s_cu[t];   // (A, beta, gamma, o)
        const float oA = cu.w * cu.x, ho = -0.5f * cu.w;
        red_add_v2(g_mean2d + 2 * (size_t)r, -oA * mt, -(oA * cu.y * mt + cu.w * cu.z * mdy));
        red_add_v4(g_co + 4 * (size_t)r, ho * mtt, -oA * mtdy, ho * mdydy, m);
        red_add_v4(g_rgb + 4 * (size_t)r, k0, k1, k2, 0.f);
      }
    }
  }
}

// Per-splat backward (the per-splat parallel back-propagation of the Taming-3DGS
// lineage that the paper's base trainer uses): the same gradient as
// raster_bwd_kernel, parallel over list entries instead of pixels. The warps of a
// tile's CTAs claim its 64-entry buckets (up to the tile's largest stop index) one
// at a time, two consecutive entries per lane. A bucket's live pixels (stop index
// beyond its first position) start from the forward's checkpoint (T and the colour
// composited before the bucket) and flow through the warp diagonally: at step s lane
// l works on live pixel s - l, taking its (T, R) from lane l - 1, which handled that
// pixel one step earlier, and passes it through its two entries in list order. The
// two entries' falloff and their moment sums are independent, so they run as packed
// FP32 pairs (add/sub/mul/fma.rn.f32x2); only the transmittance chain through the two
// entries stays scalar. A tile's buckets are shared by kSplatSplit CTAs, so a tile with
// a long list does not hold the end of the launch. Each lane sums its entries' moments
// over the tile's pixels in registers and adds them to the record gradients once,
// with no cross-lane reduction. Since the lanes only ever read 32 consecutive live
// pixels, a warp keeps them in a 64-slot ring refilled every 32 steps (the next 32
// pixels' checkpoints are loaded meanwhile). A pixel's falloff, floor and stop
// decisions are the forward's own (same operations, same roundings). Needs the stop
// indices and the checkpoints written by the forward (gs_raster_fwd_ckpt).
constexpr int kSplatThreads = 128;
constexpr int kSplatSplit = 2;     // CTAs per tile (bucket b goes to CTA b % kSplatSplit)
constexpr int kSplatRing = 64;
constexpr int kSplatBlocks = 6;    // resident CTAs per SM the register budget targets (80 registers)

// rcp.approx.ftz.f32: the reciprocal __fdividef uses.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int TW, int TH>
__global__ void __launch_bounds__(kSplatThreads, kSplatBlocks) raster_bwd_splat_kernel(
    const float2 *__restrict__ mean2d, const float4 *__restrict__ conic_o, const float4 *__restrict__ rgb,
    const uint32_t *__restrict__ vals, const uint2 *__restrict__ ranges, const gs_camera_t *__restrict__ cams,
    int n_views, const float *__restrict__ image, const float *__restrict__ d_image,
    const uint32_t *__restrict__ stop_in, const CkptLayout ckpt, float *__restrict__ g_mean2d,
    float *__restrict__ g_co, float *__restrict__ g_rgb, uint64_t n_records, uint64_t list_cap) {
  constexpr int NP = TW * TH, NW = kSplatThreads / 32, NB = TW * TH / 64;
  static_assert(NP % 32 == 0 && NP <= 65536, "whole warps of pixels, 16-bit indices");
  __shared__ float4 s_g[NP];                       // (dL/dout, <out, dL/dout>)
  __shared__ uint32_t s_stop[NP];
  __shared__ uint16_t s_live[NW][NP];
  // ring of live pixels at index i % 64: ra = (dL/dout, stop bits), rb = (x, y, T, R)
  // at the bucket start; one base address, immediate offsets
  __shared__ float4 s_ring[NW][2][kSplatRing];
  __shared__ uint32_t s_max, s_next;
  const int tile = blockIdx.x / kSplatSplit, part = blockIdx.x % kSplatSplit;
  const TileCoord tc = tile_coord(cams, n_views, tile);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  if (t == 0) {
    s_max = 0;
    s_next = NW;
  }
  __syncthreads();
  {
    const int64_t plane = (int64_t)tc.W * tc.H;
    const float *img = image + 3 * tc.pix_off;
    const float *dim = d_image + 3 * tc.pix_off;
    uint32_t mx = 0;
    for (int p = t; p < NP; p += kSplatThreads) {
      const int px = tc.tx * TW + p % TW, py = tc.ty * TH + p / TW;
      uint32_t st = 0;
      float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
      if (px < tc.W && py < tc.H) {
        const int64_t q = (int64_t)py * tc.W + px;
        st = stop_in[tc.pix_off + q];
        g.x = dim[q]; g.y = dim[plane + q]; g.z = dim[2 * plane + q];
        g.w = g.x * img[q] + g.y * img[plane + q] + g.z * img[2 * plane + q];
      }
      s_g[p] = g;
      s_stop[p] = st;
      mx = max(mx, st);
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) atomicMax(&s_max, mx);
  }
  __syncthreads();
  uint2 rg = ranges[tile];
  if (!GS_CHECK(rg.x <= rg.y && (uint64_t)rg.y <= list_cap, 2, tile)) rg = make_uint2(0u, 0u);
  const int n = min((int)(rg.y - rg.x), (int)s_max);
  const int nb = (n + 63) >> 6;                     // buckets of 64 list entries
  const uint64_t bk0 = ckpt_bucket(rg.x, tile);
  uint16_t *live = s_live[warp];
  float4 *ra = s_ring[warp][0], *rb = s_ring[warp][1];
  const float4 *rw = s_ring[warp][0];
  for (int b = part + kSplatSplit * warp; b < nb;) {
    // this lane's two consecutive list entries (a, b) = (64 b + 2 lane, 64 b + 2 lane + 1)
    const int ja = 64 * b + 2 * lane, jb = ja + 1;
    float2 xya = make_float2(0.f, 0.f), xyb = xya;
    float4 cua = make_float4(0.f, 0.f, 0.f, 0.f), cub = cua, ca = cua, cb = cua;
    if (ja < n) {
      const uint32_t r = vals[rg.x + ja];
      if (GS_CHECK(r < n_records, 1, r)) {
        xya = mean2d[r];
        cua = conic_o[r];
        ca = rgb[r];
      }
    }
    if (jb < n) {
      const uint32_t r = vals[rg.x + jb];
      if (GS_CHECK(r < n_records, 1, r)) {
        xyb = mean2d[r];
        cub = conic_o[r];
        cb = rgb[r];
      }
    }
    int nl = 0;
    for (int p0 = 0; p0 < NP; p0 += 32) {
      const int p = p0 + lane;
      const bool on = s_stop[p] > (uint32_t)(64 * b);
      const uint32_t bal = __ballot_sync(0xffffffffu, on);
      if (on) live[nl + __popc(bal & lt)] = (uint16_t)p;
      nl += __popc(bal);
    }
    __syncwarp();
    // the checkpoint slot of each 8 x 8 block at the bucket's first position (the
    // forward's 32-entry step 2 b; lane k holds block k's); a block holding a live pixel
    // was walked by its forward warp, so its entry is current
    uint32_t bslot = kCkptNone;
    if (lane < NB) {
      const uint64_t ti = (bk0 + 2 * (uint64_t)b) * NB + lane;
      if (GS_CHECK(ti < ckpt.table_entries, 3, ti)) bslot = ckpt.table[ti];
    }
    // live pixel `slot` for this lane: its index (-1 past the list) and checkpoint
    int pn = -1;
    float4 kn = make_float4(1.f, 0.f, 0.f, 0.f);
    auto fetch = [&](int slot) {
      pn = slot < nl ? (int)live[slot] : -1;
      const int px = pn & (TW - 1), py = pn / TW;
      const uint32_t sl = __shfl_sync(0xffffffffu, bslot, (py >> 3) * (TW / 8) + (px >> 3));
      kn = make_float4(1.f, 0.f, 0.f, 0.f);
      if (pn >= 0 && sl != kCkptNone && GS_CHECK(sl < ckpt.n_slots, 3, sl))
        kn = ckpt.slots[(uint64_t)sl * 64 + (py & 7) * 8 + (px & 7)];
    };
    fetch(lane);
    // ring slots 32..63 read as stopped until the second chunk replaces them
    ra[32 + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    rb[32 + lane] = make_float4(0.f, 0.f, 1.f, 0.f);
    // moments accumulated negated (see nd below), colour terms as they are; .x the
    // sums of entry a, .y of entry b
    float2 v0 = f2(0.f), v1 = f2(0.f), v2 = f2(0.f), v3 = f2(0.f), v4 = f2(0.f), v5 = f2(0.f);
    float2 v6 = f2(0.f), v7 = f2(0.f), v8 = f2(0.f);
    float T = 1.f, Rr = 0.f;
    const uint32_t jja = (uint32_t)ja, jjb = (uint32_t)jb;
    const float2 U = f2(xya.x, xyb.x), V = f2(xya.y, xyb.y);
    const float2 A2 = f2(__fmul_rn(cua.x, kNegHalfLog2e), __fmul_rn(cub.x, kNegHalfLog2e));
    const float2 BE = f2(cua.y, cub.y);
    const float2 G2 = f2(__fmul_rn(cua.z, kNegHalfLog2e), __fmul_rn(cub.z, kNegHalfLog2e));
    const float2 O = f2(cua.w, cub.w);
    const float2 NCX = f2(-ca.x, -cb.x), NCY = f2(-ca.y, -cb.y), NCZ = f2(-ca.z, -cb.z);
    for (int s0 = 0; s0 < nl + 31; s0 += 32) {
      {
        // ring slots s0 .. s0 + 31; past the list a slot reads as stopped (stop 0)
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = make_float4(0.f, 0.f, 1.f, 0.f);
        if (pn >= 0) {
          const float4 g = s_g[pn];
          A = make_float4(g.x, g.y, g.z, __uint_as_float(s_stop[pn]));
          B = make_float4((float)(tc.tx * TW + pn % TW) + 0.5f, (float)(tc.ty * TH + pn / TW) + 0.5f, kn.x,
                          g.w - (kn.y * g.x + kn.z * g.y + kn.w * g.z));
        }
        ra[(s0 + lane) & (kSplatRing - 1)] = A;
        rb[(s0 + lane) & (kSplatRing - 1)] = B;
        fetch(s0 + 32 + lane);
        __syncwarp();
      }
      const int s1 = min(s0 + 32, nl + 31);
#pragma unroll 8
      for (int s = s0; s < s1; ++s) {
        const float4 *q = rw + ((s - lane) & (kSplatRing - 1));
        const float Tin = __shfl_up_sync(0xffffffffu, T, 1);
        const float Rin = __shfl_up_sync(0xffffffffu, Rr, 1);
        const float4 g = q[0], p = q[kSplatRing];
        T = lane == 0 ? p.z : Tin;
        Rr = lane == 0 ? p.w : Rin;
        // falloff of both entries at this pixel: the forward's operations and roundings
        // (the pixel's coordinates are a broadcast operand: two scalar subtractions
        // cost less than a packed one and the moves that would build its pair)
        const float2 dx = f2(__fsub_rn(U.x, p.x), __fsub_rn(U.y, p.x));
        const float2 dy = f2(__fsub_rn(V.x, p.y), __fsub_rn(V.y, p.y));
        const float2 tt = f2_fma(BE, dy, dx);
        const float2 e = f2_fma(f2_mul(A2, tt), tt, f2_mul(G2, f2_mul(dy, dy)));
        const float2 G = f2(ex2_approx(e.x), ex2_approx(e.y));
        const float2 raw = f2_mul(O, G);
        const float2 al = f2(fminf(kAlphaMax, raw.x), fminf(kAlphaMax, raw.y));
        // a position before the pixel's stop (false on stopped pixels and for lanes
        // without an entry) where sigma reaches the floor; elsewhere sigma 0 leaves T,
        // R and every sum as they are
        const uint32_t stop = __float_as_uint(g.w);
        const bool oka = jja < stop && al.x >= kAlphaMin, okb = jjb < stop && al.y >= kAlphaMin;
        const float2 ncd = f2_fma(NCZ, f2(g.z), f2_fma(NCY, f2(g.y), f2_mul(NCX, f2(g.x))));   // -<c, g>
        // entry a, then entry b, in list order: -dL/dsigma = -T <c, g> + R / (1 - sigma)
        const float sa = oka ? al.x : 0.f;
        const float oma = __fsub_rn(1.f, sa);
        const float wa = sa * T;
        Rr = fmaf(ncd.x, wa, Rr);
        const float nda = fmaf(T, ncd.x, Rr * rcp_approx(oma));
        T = __fmul_rn(T, oma);
        const float sb = okb ? al.y : 0.f;
        const float omb = __fsub_rn(1.f, sb);
        const float wb = sb * T;
        Rr = fmaf(ncd.y, wb, Rr);
        const float ndb = fmaf(T, ncd.y, Rr * rcp_approx(omb));
        T = __fmul_rn(T, omb);
        const float2 w = f2(wa, wb);
        v6 = f2_fma(f2(g.x), w, v6);
        v7 = f2_fma(f2(g.y), w, v7);
        v8 = f2_fma(f2(g.z), w, v8);
        const float2 m = f2(oka && raw.x <= kAlphaMax ? nda * G.x : 0.f, okb && raw.y <= kAlphaMax ? ndb * G.y : 0.f);
        const float2 mt = f2_mul(m, tt), mdy = f2_mul(m, dy);
        v0 = f2_add(v0, mt);
        v1 = f2_add(v1, mdy);
        v2 = f2_fma(mt, tt, v2);
        v3 = f2_fma(mt, dy, v3);
        v4 = f2_fma(mdy, dy, v4);
        v5 = f2_add(v5, m);
      }
      __syncwarp();   // this chunk's reads before the next chunk's ring writes
    }
    // each entry's sums once into its record's gradients (record and conic read again)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int jh = h == 0 ? ja : jb;
      const float v[9] = {-(h == 0 ? v0.x : v0.y), -(h == 0 ? v1.x : v1.y), -(h == 0 ? v2.x : v2.y),
                          -(h == 0 ? v3.x : v3.y), -(h == 0 ? v4.x : v4.y), -(h == 0 ? v5.x : v5.y),
                          h == 0 ? v6.x : v6.y, h == 0 ? v7.x : v7.y, h == 0 ? v8.x : v8.y};
      if (jh < n && (v[0] != 0.f || v[1] != 0.f || v[2] != 0.f || v[3] != 0.f || v[4] != 0.f ||
                     v[5] != 0.f || v[6] != 0.f || v[7] != 0.f || v[8] != 0.f)) {
        const uint32_t r = vals[rg.x + jh];
        if (!GS_CHECK(r < n_records, 1, r)) continue;
        const float4 cu = conic_o[r];
        const float oA = cu.w * cu.x, ho = -0.5f * cu.w;
        red_add_v2(g_mean2d + 2 * (size_t)r, -oA * v[0], -(oA * cu.y * v[0] + cu.w * cu.z * v[1]));
        red_add_v4(g_co + 4 * (size_t)r, ho * v[2], -oA * v[3], ho * v[4], v[5]);
        red_add_v4(g_rgb + 4 * (size_t)r, v[6], v[7], v[8], 0.f);
      }
    }
    __syncwarp();   // the next bucket rewrites this warp's live list
    uint32_t nxt = 0;
    if (lane == 0) nxt = atomicAdd(&s_next, 1u);
    b = part + kSplatSplit * (int)__shfl_sync(0xffffffffu, nxt, 0);
  }
}

__device__ __forceinline__ float l1_term(float a, float t, float inv, float &g) {
  const float d = a - t;
  g = d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
  return fabsf(d);
}

// VEC (image, target and d_image on 16-byte boundaries): the view's elements as a
// scalar head up to the first 16-byte boundary, float4s, and a scalar tail, so that
// each thread keeps 32 bytes of loads in flight instead of 8.
template <bool VEC>
__global__ void __launch_bounds__(256) l1_loss_grad_kernel(const gs_camera_t *__restrict__ cams,
                                                           const float *__restrict__ image,
                                                           const float *__restrict__ target,
                                                           float *__restrict__ d_image, float *loss) {
  const int v = blockIdx.y;
  const gs_camera_t &cam = cams[v];
  const int64_t n = 3ll * cam.width * cam.height;
  const int64_t off = 3 * cam.pixel_offset;
  const float inv = 1.f / (float)n;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  float acc = 0.f;
  int64_t head = n, nv4 = 0;
  if (VEC) {
    head = min(n, (int64_t)((4 - (off & 3)) & 3));
    nv4 = (n - head) >> 2;
    const float4 *im4 = reinterpret_cast<const float4 *>(image + off + head);
    const float4 *tg4 = reinterpret_cast<const float4 *>(target + off + head);
    float4 *dg4 = reinterpret_cast<float4 *>(d_image + off + head);
    for (int64_t i = tid; i < nv4; i += stride) {
      const float4 a = im4[i], t = tg4[i];
      float4 g;
      acc += l1_term(a.x, t.x, inv, g.x);
      acc += l1_term(a.y, t.y, inv, g.y);
      acc += l1_term(a.z, t.z, inv, g.z);
      acc += l1_term(a.w, t.w, inv, g.w);
      dg4[i] = g;
    }
  }
  // the scalar elements: [0, head) and [head + 4 nv4, n) (all of them without VEC)
  const int64_t tail0 = head + 4 * nv4;
  const int64_t n_scalar = head + (n - tail0);
  for (int64_t k = tid; k < n_scalar; k += stride) {
    const int64_t i = k < head ? k : tail0 + (k - head);
    float g;
    acc += l1_term(image[off + i], target[off + i], inv, g);
    d_image[off + i] = g;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += ws[i];
    atomicAdd(loss + v, s * inv);
  }
}

template <int TW, int TH, bool COUNT = false>
static gs_status_t launch_fwd(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                              const gs_raster_cfg_t *cfg, float *image, float *T_final, uint32_t *stop,
                              cudaStream_t s, uint32_t *counts = nullptr, const CkptLayout *ckpt = nullptr) {
  if (!COUNT) {
    FwdArgs a;
    a.mean2d = reinterpret_cast<const float2 *>(proj->mean2d);
    a.conic_o = reinterpret_cast<const float4 *>(proj->conic_opacity);
    a.rgb = reinterpret_cast<const float4 *>(proj->rgb);
    a.vals = bins->vals;
    a.ranges = reinterpret_cast<const uint2 *>(bins->ranges);
    a.cams = frame->cams_dev;
    a.n_views = frame->n_views;
    a.bg0 = cfg->bg[0];
    a.bg1 = cfg->bg[1];
    a.bg2 = cfg->bg[2];
    a.image = image;
    a.T_final = T_final;
    a.stop_out = cfg->store_stop ? stop : nullptr;
    a.ckpt = ckpt ? *ckpt : CkptLayout{};
    a.n_records = (uint64_t)proj->n_records;
    a.list_cap = (uint64_t)bins->capacity;
    if (cfg->d_queue) {
      // persistent grid: every CTA the SMs hold at once
      GS_CUDA_TRY(cudaMemsetAsync(cfg->d_queue, 0, sizeof(uint32_t), s));
      auto kern = ckpt ? raster_fwd_queue_kernel<TW, TH, true> : raster_fwd_queue_kernel<TW, TH, false>;
      int per_sm = 0;
      GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kQueueWarps, 0));
      if (per_sm < 1) per_sm = 1;
      kern<<<num_sms() * per_sm, 32 * kQueueWarps, 0, s>>>(a, frame->n_tiles, cfg->d_queue);
    } else {
      auto kern = ckpt ? raster_fwd_warp_kernel<TW, TH, true> : raster_fwd_warp_kernel<TW, TH, false>;
      kern<<<frame->n_tiles, TW * TH / 2, 0, s>>>(a);
    }
    GS_LAUNCH_CHECK();
    return GS_OK;
  }
  raster_fwd_kernel<TW, TH, COUNT><<<frame->n_tiles, TW * TH / 2, 0, s>>>(
      reinterpret_cast<const float2 *>(proj->mean2d), reinterpret_cast<const float4 *>(proj->conic_opacity),
      reinterpret_cast<const float4 *>(proj->rgb), bins->vals, reinterpret_cast<const uint2 *>(bins->ranges),
      frame->cams_dev, frame->n_views, cfg->bg[0], cfg->bg[1], cfg->bg[2], image, T_final,
      cfg->store_stop ? stop : nullptr, counts, (uint64_t)proj->n_records, (uint64_t)bins->capacity);
  GS_LAUNCH_CHECK();
  return GS_OK;
}

template <int TW, int TH>
static gs_status_t launch_bwd(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                              const float *image, const float *d_image, const uint32_t *stop, bool half,
                              gs_rec_grads_t *g, cudaStream_t s) {
  const size_t R = (size_t)proj->n_records;
  GS_CUDA_TRY(cudaMemsetAsync(g->d_mean2d, 0, R * 2 * sizeof(float), s));
  GS_CUDA_TRY(cudaMemsetAsync(g->d_conic_opacity, 0, R * 4 * sizeof(float), s));
  GS_CUDA_TRY(cudaMemsetAsync(g->d_rgb, 0, R * 4 * sizeof(float), s));
  // 2 pixels per thread: 8 x 8 warp blocks skip more records than 8 x 16 ones
  // (4 pixels per thread) save in shared per-entry work.
  constexpr int PX = 2;
  const auto *m2 = reinterpret_cast<const float2 *>(proj->mean2d);
  const auto *co = reinterpret_cast<const float4 *>(proj->conic_opacity);
  const auto *c = reinterpret_cast<const float4 *>(proj->rgb);
  const auto *rg = reinterpret_cast<const uint2 *>(bins->ranges);
#define GS_BWD(STOPV, HALFV)                                                                               \
  raster_bwd_kernel<TW, TH, PX, STOPV, HALFV><<<frame->n_tiles, TW * TH / PX, 0, s>>>(                       \
      m2, co, c, bins->vals, rg, frame->cams_dev, frame->n_views, image, d_image, stop, g->d_mean2d,          \
      g->d_conic_opacity, g->d_rgb, (uint64_t)proj->n_records, (uint64_t)bins->capacity)
  if (stop)
    half ? GS_BWD(true, true) : GS_BWD(true, false);
  else
    half ? GS_BWD(false, true) : GS_BWD(false, false);
#undef GS_BWD
  GS_LAUNCH_CHECK();
  return GS_OK;
}

template <int TW, int TH>
static gs_status_t launch_bwd_splat(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                                    const float *image, const float *d_image, const uint32_t *stop,
                                    const CkptLayout &ckpt, gs_rec_grads_t *g, cudaStream_t s) {
  const size_t R = (size_t)proj->n_records;
  GS_CUDA_TRY(cudaMemsetAsync(g->d_mean2d, 0, R * 2 * sizeof(float), s));
  GS_CUDA_TRY(cudaMemsetAsync(g->d_conic_opacity, 0, R * 4 * sizeof(float), s));
  GS_CUDA_TRY(cudaMemsetAsync(g->d_rgb, 0, R * 4 * sizeof(float), s));
  raster_bwd_splat_kernel<TW, TH><<<frame->n_tiles * kSplatSplit, kSplatThreads, 0, s>>>(
      reinterpret_cast<const float2 *>(proj->mean2d), reinterpret_cast<const float4 *>(proj->conic_opacity),
      reinterpret_cast<const float4 *>(proj->rgb), bins->vals, reinterpret_cast<const uint2 *>(bins->ranges),
      frame->cams_dev, frame->n_views, image, d_image, stop, ckpt, g->d_mean2d, g->d_conic_opacity, g->d_rgb,
      (uint64_t)proj->n_records, (uint64_t)bins->capacity);
  GS_LAUNCH_CHECK();
  return GS_OK;
}

static bool a16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace gs

using namespace gs;

extern "C" int32_t gs_tile_supported(int32_t tw, int32_t th) {
  return (tw == 16 && th == 16) || (tw == 8 && th == 8) || (tw == 16 && th == 32) || (tw == 32 && th == 16);
}

extern "C" gs_status_t gs_raster_fwd(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                                     const gs_raster_cfg_t *cfg, float *image, float *T_final, uint32_t *stop,
                                     gs_stream_t stream) {
  if (!proj || !bins || !frame || !cfg || !image || !T_final || !frame->cams_dev || frame->n_tiles <= 0)
    return GS_ERR_INVALID_ARG;
  if (!bins->vals || !bins->ranges || !proj->mean2d || !a16(proj->conic_opacity) || !a16(proj->rgb))
    return GS_ERR_INVALID_ARG;
  if (cfg->store_stop && !stop) return GS_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  if (frame->tile_w == 16 && frame->tile_h == 16) return launch_fwd<16, 16>(proj, bins, frame, cfg, image, T_final, stop, s);
  if (frame->tile_w == 8 && frame->tile_h == 8) return launch_fwd<8, 8>(proj, bins, frame, cfg, image, T_final, stop, s);
  if (frame->tile_w == 16 && frame->tile_h == 32) return launch_fwd<16, 32>(proj, bins, frame, cfg, image, T_final, stop, s);
  if (frame->tile_w == 32 && frame->tile_h == 16) return launch_fwd<32, 16>(proj, bins, frame, cfg, image, T_final, stop, s);
  return GS_ERR_UNSUPPORTED;
}

extern "C" gs_status_t gs_raster_bwd(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                                     const gs_raster_cfg_t *cfg, const float *image, const float *d_image,
                                     const uint32_t *stop, gs_rec_grads_t *grads, gs_stream_t stream) {
  if (!proj || !bins || !frame || !cfg || !image || !d_image || !grads || !frame->cams_dev || frame->n_tiles <= 0)
    return GS_ERR_INVALID_ARG;
  if (!grads->d_mean2d || !a16(grads->d_conic_opacity) || !a16(grads->d_rgb) || !grads->d_conic_opacity ||
      !grads->d_rgb || ((reinterpret_cast<uintptr_t>(grads->d_mean2d) & 7u) != 0))
    return GS_ERR_INVALID_ARG;
  if (cfg->stage_depth != 0 && cfg->stage_depth != 1) return GS_ERR_INVALID_ARG;
  const bool half = cfg->stage_depth == 1;
  cudaStream_t s = as_stream(stream);
  if (frame->tile_w == 16 && frame->tile_h == 16) return launch_bwd<16, 16>(proj, bins, frame, image, d_image, stop, half, grads, s);
  if (frame->tile_w == 8 && frame->tile_h == 8) return launch_bwd<8, 8>(proj, bins, frame, image, d_image, stop, half, grads, s);
  if (frame->tile_w == 16 && frame->tile_h == 32) return launch_bwd<16, 32>(proj, bins, frame, image, d_image, stop, half, grads, s);
  if (frame->tile_w == 32 && frame->tile_h == 16) return launch_bwd<32, 16>(proj, bins, frame, image, d_image, stop, half, grads, s);
  return GS_ERR_UNSUPPORTED;
}

// Table entries of a frame whose lists hold at most `capacity` entries: one per
// (bucket, 8 x 8 block); 0 for an unsupported frame.
static uint64_t ckpt_table_entries(const gs_frame_t *frame, int64_t capacity) {
  if (!frame || capacity < 0 || frame->n_tiles <= 0 || !gs_tile_supported(frame->tile_w, frame->tile_h)) return 0;
  const uint64_t buckets = ((uint64_t)capacity + 31u) / 32u + (uint64_t)frame->n_tiles;
  return buckets * (uint64_t)(frame->tile_w * frame->tile_h / 64);
}

// The largest slot count a buffer of `bytes` holds for this frame and capacity.
static bool ckpt_from_bytes(const gs_frame_t *frame, int64_t capacity, void *base, size_t bytes, CkptLayout &L) {
  const uint64_t te = ckpt_table_entries(frame, capacity);
  if (te == 0) return false;
  const size_t head = ckpt_layout(nullptr, te, 0).bytes;
  if (bytes < head) return false;
  const uint32_t pools = ckpt_pools((uint64_t)frame->n_tiles * (frame->tile_w * frame->tile_h / 64));
  L = ckpt_layout(base, te, (bytes - head) / (64 * sizeof(float4)), pools);
  return true;
}

extern "C" size_t gs_raster_ckpt_size(const gs_frame_t *frame, int64_t capacity, int64_t n_slots) {
  const uint64_t te = ckpt_table_entries(frame, capacity);
  if (te == 0) return 0;
  // a slot for every (bucket, block) pair the lists can have: enough whatever the
  // stop indices
  const uint64_t slots = n_slots < 0 ? te : (uint64_t)n_slots;
  return ckpt_layout(nullptr, te, slots).bytes;
}

__global__ void ckpt_usage_kernel(const uint32_t *__restrict__ pools, uint32_t n_pools, uint64_t pool_size,
                                  bool direct, int64_t *out) {
  // one warp: the slots the last forward needed (n_pools x the fullest pool, the
  // size at which no pool overflows) and whether any pool overflowed
  uint32_t mx = 0;
  for (uint32_t i = threadIdx.x; i < n_pools; i += 32) mx = max(mx, pools[i]);
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (threadIdx.x == 0) {
    out[0] = (int64_t)mx * n_pools;
    out[1] = (!direct && (uint64_t)mx > pool_size) ? 1 : 0;
  }
}

extern "C" gs_status_t gs_raster_ckpt_usage(const gs_frame_t *frame, int64_t capacity, const void *ckpt,
                                            size_t ckpt_bytes, int64_t *d_usage, gs_stream_t stream) {
  if (!frame || !ckpt || !d_usage || !a16(ckpt) || (reinterpret_cast<uintptr_t>(d_usage) & 7u) != 0)
    return GS_ERR_INVALID_ARG;
  CkptLayout L;
  if (!ckpt_from_bytes(frame, capacity, const_cast<void *>(ckpt), ckpt_bytes, L)) return GS_ERR_INVALID_ARG;
  ckpt_usage_kernel<<<1, 32, 0, as_stream(stream)>>>(L.pools, L.n_pools, L.pool_size,
                                                     L.n_slots >= L.table_entries, d_usage);
  GS_LAUNCH_CHECK();
  return GS_OK;
}

extern "C" gs_status_t gs_raster_fwd_ckpt(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                                          const gs_raster_cfg_t *cfg, float *image, float *T_final, uint32_t *stop,
                                          void *ckpt, size_t ckpt_bytes, gs_stream_t stream) {
  if (!proj || !bins || !frame || !cfg || !image || !T_final || !stop || !ckpt || !frame->cams_dev ||
      frame->n_tiles <= 0)
    return GS_ERR_INVALID_ARG;
  if (!bins->vals || !bins->ranges || !proj->mean2d || !a16(proj->conic_opacity) || !a16(proj->rgb) || !a16(ckpt))
    return GS_ERR_INVALID_ARG;
  if (!gs_tile_supported(frame->tile_w, frame->tile_h)) return GS_ERR_UNSUPPORTED;
  CkptLayout L;
  if (!ckpt_from_bytes(frame, bins->capacity, ckpt, ckpt_bytes, L)) return GS_ERR_INVALID_ARG;
  gs_raster_cfg_t c = *cfg;
  c.store_stop = 1;
  cudaStream_t s = as_stream(stream);
  GS_CUDA_TRY(cudaMemsetAsync(L.pools, 0, 4 * kCkptPools, s));
  if (frame->tile_w == 16 && frame->tile_h == 16) return launch_fwd<16, 16>(proj, bins, frame, &c, image, T_final, stop, s, nullptr, &L);
  if (frame->tile_w == 8 && frame->tile_h == 8) return launch_fwd<8, 8>(proj, bins, frame, &c, image, T_final, stop, s, nullptr, &L);
  if (frame->tile_w == 16 && frame->tile_h == 32) return launch_fwd<16, 32>(proj, bins, frame, &c, image, T_final, stop, s, nullptr, &L);
  if (frame->tile_w == 32 && frame->tile_h == 16) return launch_fwd<32, 16>(proj, bins, frame, &c, image, T_final, stop, s, nullptr, &L);
  return GS_ERR_UNSUPPORTED;
}

extern "C" gs_status_t gs_raster_bwd_splat(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                                           const float *image, const float *d_image, const uint32_t *stop,
                                           const void *ckpt, size_t ckpt_bytes, gs_rec_grads_t *grads,
                                           gs_stream_t stream) {
  if (!proj || !bins || !frame || !image || !d_image || !stop || !ckpt || !grads || !frame->cams_dev ||
      frame->n_tiles <= 0)
    return GS_ERR_INVALID_ARG;
  if (!bins->vals || !bins->ranges || !a16(proj->conic_opacity) || !a16(proj->rgb) || !a16(ckpt))
    return GS_ERR_INVALID_ARG;
  if (!grads->d_mean2d || !a16(grads->d_conic_opacity) || !a16(grads->d_rgb) || !grads->d_conic_opacity ||
      !grads->d_rgb || ((reinterpret_cast<uintptr_t>(grads->d_mean2d) & 7u) != 0))
    return GS_ERR_INVALID_ARG;
  if (!gs_tile_supported(frame->tile_w, frame->tile_h)) return GS_ERR_UNSUPPORTED;
  CkptLayout L;
  if (!ckpt_from_bytes(frame, bins->capacity, const_cast<void *>(ckpt), ckpt_bytes, L)) return GS_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  if (frame->tile_w == 16 && frame->tile_h == 16) return launch_bwd_splat<16, 16>(proj, bins, frame, image, d_image, stop, L, grads, s);
  if (frame->tile_w == 8 && frame->tile_h == 8) return launch_bwd_splat<8, 8>(proj, bins, frame, image, d_image, stop, L, grads, s);
  if (frame->tile_w == 16 && frame->tile_h == 32) return launch_bwd_splat<16, 32>(proj, bins, frame, image, d_image, stop, L, grads, s);
  if (frame->tile_w == 32 && frame->tile_h == 16) return launch_bwd_splat<32, 16>(proj, bins, frame, image, d_image, stop, L, grads, s);
  return GS_ERR_UNSUPPORTED;
}

extern "C" gs_status_t gs_raster_count(const gs_proj_t *proj, const gs_bins_t *bins, const gs_frame_t *frame,
                                       uint32_t *counts, gs_stream_t stream) {
  if (!proj || !bins || !frame || !counts || !frame->cams_dev || frame->n_tiles <= 0 || !bins->vals ||
      !bins->ranges || !a16(proj->conic_opacity) || !a16(proj->rgb) ||
      (reinterpret_cast<uintptr_t>(counts) & 7u) != 0)
    return GS_ERR_INVALID_ARG;
  gs_raster_cfg_t cfg{};
  cudaStream_t s = as_stream(stream);
  if (frame->tile_w == 16 && frame->tile_h == 16) return launch_fwd<16, 16, true>(proj, bins, frame, &cfg, nullptr, nullptr, nullptr, s, counts);
  if (frame->tile_w == 8 && frame->tile_h == 8) return launch_fwd<8, 8, true>(proj, bins, frame, &cfg, nullptr, nullptr, nullptr, s, counts);
  if (frame->tile_w == 16 && frame->tile_h == 32) return launch_fwd<16, 32, true>(proj, bins, frame, &cfg, nullptr, nullptr, nullptr, s, counts);
  if (frame->tile_w == 32 && frame->tile_h == 16) return launch_fwd<32, 16, true>(proj, bins, frame, &cfg, nullptr, nullptr, nullptr, s, counts);
  return GS_ERR_UNSUPPORTED;
}

extern "C" gs_status_t gs_l1_loss_grad(const gs_frame_t *frame, const float *image, const float *target,
                                       float *d_image, float *loss_dev, gs_stream_t stream) {
  if (!frame || !frame->cams_dev || frame->n_views <= 0 || !image || !target || !d_image || !loss_dev)
    return GS_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  GS_CUDA_TRY(cudaMemsetAsync(loss_dev, 0, sizeof(float) * frame->n_views, s));
  const bool vec = ((reinterpret_cast<uintptr_t>(image) | reinterpret_cast<uintptr_t>(target) |
                     reinterpret_cast<uintptr_t>(d_image)) & 15u) == 0;
  const int64_t per_view = 3ll * frame->max_width * frame->max_height;
  int bx = (int)((per_view / (vec ? 4 : 1) + 255) / 256);
  const int cap = num_sms() * 8;   // a full SM of 256-thread blocks, shared by the views
  const int cap_view = (cap + frame->n_views - 1) / frame->n_views;
  if (bx > cap_view) bx = cap_view;
  if (bx < 1) bx = 1;
  if (vec)
    l1_loss_grad_kernel<true><<<dim3(bx, frame->n_views), 256, 0, s>>>(frame->cams_dev, image, target, d_image,
                                                                       loss_dev);
  else
    l1_loss_grad_kernel<false><<<dim3(bx, frame->n_views), 256, 0, s>>>(frame->cams_dev, image, target, d_image,
                                                                        loss_dev);
  GS_LAUNCH_CHECK();
  return GS_OK;
}
