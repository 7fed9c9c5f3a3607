// Reduce-then-scan over a device-side element count, shared by binning and
// densification. Fixed grids; each block derives its chunk from the count, so no
// host round trip is needed and no block ever waits on another.
#pragma once

#include "gs_common.cuh"

namespace gs {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kMaxBlocks = 1024;

// Blocks of the fixed-size scan / sort grids: two per SM.
inline int scan_blocks() {
  const int g = 2 * num_sms();
  return g > kMaxBlocks ? kMaxBlocks : g;
}


__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Exclusive scan over the block (kScanThreads threads); returns the block total in *total.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T *total) {
  __shared__ T warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    T w = lane < nw ? warp_sums[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < nw) warp_sums[lane] = wi - w;
    if (lane == nw - 1) warp_sums[31] = wi;
  }
  __syncthreads();
  const T res = warp_sums[warp] + incl - x;
  *total = warp_sums[31];
  __syncthreads();
  return res;
}

__device__ __forceinline__ void chunk_of(uint64_t n, int G, int align, uint64_t &begin, uint64_t &end) {
  uint64_t chunk = (n + G - 1) / G;
  chunk = (chunk + align - 1) / align * align;
  begin = (uint64_t)blockIdx.x * chunk;
  end = begin + chunk;
  if (begin > n) begin = n;
  if (end > n) end = n;
}

// ------------------------------------------------------------------ reduce-then-scan
// Functor interface: uint64_t count() (device-side element count), uint32_t value(i),
// void emit(i, exclusive_prefix, value). A skip flag makes every kernel a no-op.

template <typename F>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(F f, uint64_t *block_sums) {
  const uint64_t n = f.count();
  uint64_t begin, end;
  chunk_of(n, gridDim.x, kScanTile, begin, end);
  uint64_t s = 0;
  for (uint64_t i = begin + threadIdx.x; i < end; i += kScanThreads) s += f.value(i);
  uint64_t tot;
  block_exclusive_scan<uint64_t>(s, &tot);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

template <typename F>
__global__ void __launch_bounds__(1024) scan_top_kernel(F f, uint64_t *block_sums, int G) {
  // one block of 1024 threads, G <= 1024: Hillis-Steele scan of the block sums
  __shared__ uint64_t s[1024];
  const int t = threadIdx.x;
  const uint64_t own = t < G ? block_sums[t] : 0;
  s[t] = own;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint64_t y = t >= o ? s[t - o] : 0;
    __syncthreads();
    s[t] += y;
    __syncthreads();
  }
  if (t < G) block_sums[t] = s[t] - own;
  if (t == 1023) f.total(s[1023]);
}

template <typename F>
__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(F f, const uint64_t *block_offsets) {
  const uint64_t n = f.count();
  uint64_t begin, end;
  chunk_of(n, gridDim.x, kScanTile, begin, end);
  uint64_t run = block_offsets[blockIdx.x];
  for (uint64_t base = begin; base < end; base += kScanTile) {
    uint32_t v[kScanItems];
    uint64_t local = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      const uint64_t i = base + (uint64_t)threadIdx.x * kScanItems + j;
      v[j] = i < end ? f.value(i) : 0u;
      local += v[j];
    }
    uint64_t tot;
    uint64_t pre = block_exclusive_scan<uint64_t>(local, &tot) + run;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      const uint64_t i = base + (uint64_t)threadIdx.x * kScanItems + j;
      if (i < end) f.emit(i, pre, v[j]);
      pre += v[j];
    }
    run += tot;
  }
}


template <typename F>
inline gs_status_t run_scan(const F &f, uint64_t *block_sums, int G, cudaStream_t s) {
  scan_reduce_kernel<F><<<G, kScanThreads, 0, s>>>(f, block_sums);
  GS_LAUNCH_CHECK();
  scan_top_kernel<F><<<1, 1024, 0, s>>>(f, block_sums, G);
  GS_LAUNCH_CHECK();
  scan_down_kernel<F><<<G, kScanThreads, 0, s>>>(f, block_sums);
  GS_LAUNCH_CHECK();
  return GS_OK;
}


}  // namespace gs
