// Densification bookkeeping of the paper's training loop.
//
//  * split/clone selection on the view-space gradient statistic (Sec.
//    "Preliminary": norm of the average position gradient above a threshold; split
//    when the largest scale exceeds a scale threshold, clone otherwise), with the
//    global-to-local gating of Sec. "Global-to-local framework" (clone disabled in
//    the first, global phase) and the single-operation variants;
//  * the pruning threshold: fixed, or the adaptive tau = min(alpha_sorted[floor(N p)],
//    tau_u) of Sec. "Adaptive Opacity Pruning", taken in logit space over the
//    post-densification multiset by an exact weighted radix select;
//  * compaction: survivors, clones and split children written in a fixed order.
// Every predicate is evaluated in FP32 with one rounding per operation.
#include <math.h>

#include <mutex>

#include "gs_common.cuh"
#include "scan.cuh"

namespace gs {

constexpr int kSelThreads = 256;

// Monotone map of an FP32 value to an unsigned key (unsigned order == float order).
__device__ __forceinline__ uint32_t ordered_bits(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_ordered_bits(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

struct SelectState {      // scratch of the selection (lives in the caller's workspace)
  unsigned long long n_post;   // post-densification count (before pruning)
  unsigned long long n_keep;   // count after pruning
  uint32_t prefix;             // radix-select prefix of the k-th key
  uint32_t k_rem;              // rank still to find inside the current bucket
  uint32_t pad[2];
  uint32_t hist[256];
};

__device__ __forceinline__ void block_add_u64(unsigned long long x, unsigned long long *dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __shared__ unsigned long long ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += ws[i];
    if (s) atomicAdd(dst, s);
  }
}

__global__ void __launch_bounds__(kSelThreads) select_kernel(gs_densify_cfg_t cfg, const float *__restrict__ log_scales,
                                                             const float *__restrict__ accum,
                                                             const int32_t *__restrict__ count, int64_t n,
                                                             uint8_t *__restrict__ split, uint8_t *__restrict__ clone,
                                                             SelectState *st) {
  unsigned long long post = 0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = count[g];
    const float avg = c > 0 ? __fdiv_rn(accum[g], (float)c) : 0.f;
    const bool ok = avg > cfg.grad_threshold;
    const float m = fmaxf(fmaxf(log_scales[3 * g + 0], log_scales[3 * g + 1]), log_scales[3 * g + 2]);
    const bool big = m > cfg.log_scale_threshold;
    bool sp = false, cl = false;
    switch (cfg.mode) {
      case GS_DENSIFY_ADAPTIVE: sp = ok && big; cl = ok && !big; break;
      case GS_DENSIFY_SPLIT_ONLY: sp = ok && big; break;
      case GS_DENSIFY_ALL_SPLIT: sp = ok; break;
      default: cl = ok; break;
    }
    split[g] = sp;
    clone[g] = cl;
    post += (sp || cl) ? 2 : 1;
  }
  block_add_u64(post, &st->n_post);
}

// Radix select, most significant byte first: histogram of the current byte over
// the keys that match the prefix found so far, weighted by multiplicity.
__global__ void __launch_bounds__(kSelThreads) kth_hist_kernel(const float *__restrict__ logits,
                                                               const uint8_t *__restrict__ split,
                                                               const uint8_t *__restrict__ clone, int64_t n,
                                                               int shift, SelectState *st) {
  __shared__ uint32_t h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t prefix = st->prefix;
  const uint32_t hi_mask = shift >= 24 ? 0u : (0xffffffffu << (shift + 8));
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t key = ordered_bits(logits[g]);
    if ((key & hi_mask) != (prefix & hi_mask)) continue;
    atomicAdd(&h[(key >> shift) & 0xffu], (split[g] | clone[g]) ? 2u : 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&st->hist[i], h[i]);
}

__global__ void kth_find_kernel(int shift, double ratio, SelectState *st) {
  // single thread: walk the 256 buckets to the one holding rank k_rem
  if (threadIdx.x != 0) return;
  if (shift == 24) {
    const unsigned long long N = st->n_post;
    unsigned long long k = (unsigned long long)floor((double)N * ratio);
    if (k > N - 1) k = N - 1;
    st->k_rem = (uint32_t)k;
    st->prefix = 0;
  }
  uint32_t k = st->k_rem, b = 0;
  for (; b < 255; ++b) {
    const uint32_t c = st->hist[b];
    if (k < c) break;
    k -= c;
  }
  st->k_rem = k;
  st->prefix |= b << shift;
  for (int i = 0; i < 256; ++i) st->hist[i] = 0;
}

__global__ void tau_kernel(gs_densify_cfg_t cfg, SelectState *st, float *tau) {
  if (threadIdx.x != 0) return;
  float t = cfg.prune_logit;
  if (cfg.prune_adaptive) t = fminf(from_ordered_bits(st->prefix), cfg.prune_upper_logit);
  *tau = t;
}

__global__ void __launch_bounds__(kSelThreads) count_keep_kernel(const float *__restrict__ logits,
                                                                 const uint8_t *__restrict__ split,
                                                                 const uint8_t *__restrict__ clone, int64_t n,
                                                                 const float *__restrict__ tau, SelectState *st,
                                                                 int64_t *d_new_n) {
  const float t = *tau;
  unsigned long long c = 0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    if (logits[g] < t) continue;
    c += split[g] ? 2 : (clone[g] ? 2 : 1);
  }
  block_add_u64(c, &st->n_keep);
}

__global__ void publish_kernel(SelectState *st, int64_t *d_new_n) {
  if (threadIdx.x == 0) *d_new_n = (int64_t)st->n_keep;
}

// ------------------------------------------------------------------ compaction
struct SectionFlag {
  const float *logits;
  const uint8_t *split, *clone;
  const float *tau;
  int64_t n;
  int kind;                // 0: survivor (kept, not split), 1: clone, 2: split parent
  uint32_t *pos;
  uint32_t *total_out;
  __device__ uint64_t count() const { return (uint64_t)n; }
  __device__ uint32_t value(uint64_t g) const {
    if (logits[g] < *tau) return 0u;
    if (kind == 0) return split[g] ? 0u : 1u;
    if (kind == 1) return clone[g] ? 1u : 0u;
    return split[g] ? 1u : 0u;
  }
  __device__ void emit(uint64_t g, uint64_t pre, uint32_t) const { pos[g] = (uint32_t)pre; }
  __device__ void total(uint64_t t) const { *total_out = (uint32_t)t; }
};

constexpr int kMaxExtra = 16;
struct ExtraList {
  gs_extra_array_t a[kMaxExtra];
  int n;
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Rows [g0, g0 + cnt) of a w-wide array, copied by one warp: the batch's rows are
// one contiguous block of the source, read coalesced; each element goes to its
// row's survivor and clone destinations (< 0: none) and, with `children`, to both
// rows of a split child pair. zero_new: clones and children get zeros instead (the
// rows new Gaussians start from, e.g. optimiser moments).
template <typename T>
__device__ __forceinline__ void warp_copy_rows(const T *__restrict__ src, T *__restrict__ dst, int w, int64_t g0,
                                               int cnt, const int64_t *ds, const int64_t *dc, const int64_t *dp,
                                               bool children, bool zero_new, int lane) {
  const int tot = cnt * w;
  // element e = lane + 32 k sits at row e / w, column e % w; both advance by
  // (32 / w, 32 % w) per step, wrapping the column at most once
  const int q = 32 / w, rem = 32 - q * w;
  int r = lane / w, c = lane - (lane / w) * w;
  const T *s = src + g0 * w;
  constexpr int U = 4;   // loads issued before their stores: the copy is latency-bound
  for (int e0 = lane; e0 < tot; e0 += 32 * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = e0 + 32 * u < tot ? s[e0 + 32 * u] : T(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (e0 + 32 * u < tot) {
        const T nv = zero_new ? T(0) : v[u];
        const int64_t a = ds[r], b = dc[r];
        if (a >= 0) dst[a * w + c] = v[u];
        if (b >= 0) dst[b * w + c] = nv;
        if (children) {
          const int64_t d = dp[r];
          if (d >= 0) {
            dst[d * w + c] = nv;
            dst[(d + 1) * w + c] = nv;
          }
        }
      }
      r += q;
      c += rem;
      if (c >= w) {
        c -= w;
        ++r;
      }
    }
  }
}

// The same copy in 16-byte vectors, for rows of w = 4 w4 floats whose arrays start on
// 16-byte boundaries (quaternions, SH rows, their optimiser moments: most of the
// bytes): four times the bytes in flight per load, which is what this latency-bound
// copy is short of.
__device__ __forceinline__ void warp_copy_rows4(const float4 *__restrict__ src, float4 *__restrict__ dst, int w4,
                                                int64_t g0, int cnt, const int64_t *ds, const int64_t *dc,
                                                const int64_t *dp, bool children, bool zero_new, int lane) {
  const int tot = cnt * w4;
  const int q = 32 / w4, rem = 32 - q * w4;
  int r = lane / w4, c = lane - (lane / w4) * w4;
  const float4 *s = src + g0 * w4;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  constexpr int U = 4;
  for (int e0 = lane; e0 < tot; e0 += 32 * U) {
    float4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = e0 + 32 * u < tot ? s[e0 + 32 * u] : z;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (e0 + 32 * u < tot) {
        const float4 nv = zero_new ? z : v[u];
        const int64_t a = ds[r], b = dc[r];
        if (a >= 0) dst[a * w4 + c] = v[u];
        if (b >= 0) dst[b * w4 + c] = nv;
        if (children) {
          const int64_t d = dp[r];
          if (d >= 0) {
            dst[d * w4 + c] = nv;
            dst[(d + 1) * w4 + c] = nv;
          }
        }
      }
      r += q;
      c += rem;
      if (c >= w4) {
        c -= w4;
        ++r;
      }
    }
  }
}

// Row copy of a float array: in 16-byte vectors where the width and alignment allow.
__device__ __forceinline__ void copy_rows(const float *src, float *dst, int w, int64_t g0, int cnt,
                                          const int64_t *ds, const int64_t *dc, const int64_t *dp, bool children,
                                          bool zero_new, int lane) {
  if ((w & 3) == 0 && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0)
    warp_copy_rows4(reinterpret_cast<const float4 *>(src), reinterpret_cast<float4 *>(dst), w >> 2, g0, cnt, ds, dc,
                    dp, children, zero_new, lane);
  else
    warp_copy_rows(src, dst, w, g0, cnt, ds, dc, dp, children, zero_new, lane);
}

constexpr int kScatThreads = 256;

// Compaction, one warp per batch of 32 consecutive Gaussians: each lane finds its
// Gaussian's destinations (survivor row, clone row, first child row), then every
// array is copied by the warp with coalesced reads (warp_copy_rows); split children's
// means (Philox4x32-10 draw, Box-Muller, R(q) exp(s) z) and log-scales are computed
// per lane.
__global__ void __launch_bounds__(kScatThreads) scatter_kernel(
    gs_densify_cfg_t cfg, gs_params_t in, const uint8_t *__restrict__ split, const uint8_t *__restrict__ clone,
    const float *__restrict__ tau, gs_params_out_t out, ExtraList extra, gs_provenance_t prov,
    const uint32_t *__restrict__ pos_s, const uint32_t *__restrict__ pos_c, const uint32_t *__restrict__ pos_p,
    const uint32_t *totals, int64_t capacity, int64_t *d_new_n, int32_t *d_error) {
  __shared__ int64_t s_d[kScatThreads / 32][3][32];
  const uint32_t n_s = totals[0], n_c = totals[1], n_p = totals[2];
  const int64_t new_n = (int64_t)n_s + n_c + 2ll * n_p;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *d_new_n = new_n;
    if (new_n > capacity && d_error) atomicOr(d_error, (int32_t)GS_ERR_CAPACITY);
  }
  if (new_n > capacity) return;
  const float t = *tau;
  const int shw = in.sh_stride * 3;
  const float ls_div = 0.47000362924573558f;   // FP32 of log(1.6)
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int64_t *ds = s_d[wib][0], *dc = s_d[wib][1], *dp = s_d[wib][2];
  const int64_t n_batches = (in.n + 31) / 32;
  for (int64_t bt = blockIdx.x * (int64_t)(kScatThreads / 32) + wib; bt < n_batches;
       bt += (int64_t)gridDim.x * (kScatThreads / 32)) {
    const int64_t g0 = bt * 32, g = g0 + lane;
    const int cnt = (int)min((int64_t)32, in.n - g0);
    bool keep = false, sp = false, cl = false;
    if (g < in.n) {
      keep = !(in.opacity_logits[g] < t);
      sp = keep && split[g];
      cl = keep && clone[g];
    }
    ds[lane] = (keep && !sp) ? (int64_t)pos_s[g] : -1;
    dc[lane] = cl ? (int64_t)n_s + pos_c[g] : -1;
    dp[lane] = sp ? (int64_t)n_s + n_c + 2ll * pos_p[g] : -1;
    __syncwarp();
    warp_copy_rows(in.means, out.means, 3, g0, cnt, ds, dc, dp, false, false, lane);
    warp_copy_rows(in.log_scales, out.log_scales, 3, g0, cnt, ds, dc, dp, false, false, lane);
    copy_rows(in.quats, out.quats, 4, g0, cnt, ds, dc, dp, true, false, lane);
    warp_copy_rows(in.opacity_logits, out.opacity_logits, 1, g0, cnt, ds, dc, dp, true, false, lane);
    copy_rows(in.sh, out.sh, shw, g0, cnt, ds, dc, dp, true, false, lane);
    for (int e = 0; e < extra.n; ++e)
      copy_rows(extra.a[e].src, extra.a[e].dst, extra.a[e].width, g0, cnt, ds, dc, dp, true, true, lane);
    if (prov.origin_in != nullptr && g < in.n && keep) {
      const int32_t po = prov.origin_in[g], ps = prov.splits_in[g], pc = prov.clones_in[g];
      if (ds[lane] >= 0) {
        prov.origin_out[ds[lane]] = po;
        prov.splits_out[ds[lane]] = ps;
        prov.clones_out[ds[lane]] = pc;
      }
      if (cl) {
        prov.origin_out[dc[lane]] = po;
        prov.splits_out[dc[lane]] = ps;
        prov.clones_out[dc[lane]] = pc + 1;
      }
      if (sp)
        for (int c = 0; c < 2; ++c) {
          prov.origin_out[dp[lane] + c] = po;
          prov.splits_out[dp[lane] + c] = ps + 1;
          prov.clones_out[dp[lane] + c] = pc;
        }
    }
    if (sp) {
      const float4 q = reinterpret_cast<const float4 *>(in.quats)[g];
      const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
      const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
      const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                          2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                          2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
      const float s3[3] = {expf(in.log_scales[3 * g + 0]), expf(in.log_scales[3 * g + 1]),
                           expf(in.log_scales[3 * g + 2])};
      for (int c = 0; c < 2; ++c) {
        const int64_t o = dp[lane] + c;
        const uint4 bits = philox4x32_10(
            make_uint4((uint32_t)g, (uint32_t)((uint64_t)g >> 32), cfg.event, (uint32_t)c),
            make_uint2((uint32_t)cfg.seed, (uint32_t)(cfg.seed >> 32)));
        const float u0 = ((float)(bits.x >> 8) + 0.5f) * 5.9604644775390625e-08f;   // 2^-24
        const float u1 = ((float)(bits.y >> 8) + 0.5f) * 5.9604644775390625e-08f;
        const float u2 = ((float)(bits.z >> 8) + 0.5f) * 5.9604644775390625e-08f;
        const float u3 = ((float)(bits.w >> 8) + 0.5f) * 5.9604644775390625e-08f;
        const float r0 = sqrtf(-2.f * logf(u0)), r1 = sqrtf(-2.f * logf(u2));
        float sn0, cs0, sn1, cs1;
        sincospif(2.f * u1, &sn0, &cs0);
        sincospif(2.f * u3, &sn1, &cs1);
        const float zl[3] = {r0 * cs0 * s3[0], r0 * sn0 * s3[1], r1 * cs1 * s3[2]};
#pragma unroll
        for (int i = 0; i < 3; ++i)
          out.means[3 * o + i] = in.means[3 * g + i] + R[3 * i + 0] * zl[0] + R[3 * i + 1] * zl[1] + R[3 * i + 2] * zl[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) out.log_scales[3 * o + i] = __fsub_rn(in.log_scales[3 * g + i], ls_div);
      }
    }
    __syncwarp();   // the next batch rewrites this warp's destinations
  }
}

struct DensWs {
  SelectState *st;
  uint32_t *pos_s, *pos_c, *pos_p, *totals;
  uint64_t *block_sums;
  size_t bytes;
};

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

static DensWs dens_layout(void *base, int64_t n) {
  DensWs w{};
  char *p = static_cast<char *>(base);
  size_t off = 0;
  auto take = [&](size_t b) -> void * {
    void *q = p ? p + off : nullptr;
    off += a256(b);
    return q;
  };
  w.st = (SelectState *)take(sizeof(SelectState));
  w.pos_s = (uint32_t *)take(4 * (size_t)n + 16);
  w.pos_c = (uint32_t *)take(4 * (size_t)n + 16);
  w.pos_p = (uint32_t *)take(4 * (size_t)n + 16);
  w.totals = (uint32_t *)take(16);
  w.block_sums = (uint64_t *)take(8 * kMaxBlocks);
  w.bytes = off;
  return w;
}

static int dgrid(int64_t n) {
  int64_t g = (n + kSelThreads - 1) / kSelThreads;
  const int64_t cap = (int64_t)num_sms() * 8;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_densify_workspace_size(int64_t n) {
  if (n < 0) return 0;
  return dens_layout(nullptr, n).bytes;
}

extern "C" gs_status_t gs_densify_select(const gs_densify_cfg_t *cfg, const float *log_scales,
                                         const float *opacity_logits, const float *accum, const int32_t *count,
                                         int64_t n, uint8_t *split, uint8_t *clone, float *d_tau_logit,
                                         int64_t *d_new_n, void *ws, size_t ws_bytes, gs_stream_t stream) {
  if (!cfg || !log_scales || !opacity_logits || !accum || !count || n <= 0 || n >= (1ll << 31) || !split ||
      !clone || !d_tau_logit || !d_new_n || !ws)
    return GS_ERR_INVALID_ARG;
  if (cfg->mode < 0 || cfg->mode > 3) return GS_ERR_INVALID_ARG;
  if (cfg->prune_adaptive && !(cfg->prune_ratio > 0.0 && cfg->prune_ratio < 1.0)) return GS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return GS_ERR_INVALID_ARG;
  const DensWs w = dens_layout(ws, n);
  if (ws_bytes < w.bytes) return GS_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  GS_CUDA_TRY(cudaMemsetAsync(w.st, 0, sizeof(SelectState), s));
  const int G = dgrid(n);
  select_kernel<<<G, kSelThreads, 0, s>>>(*cfg, log_scales, accum, count, n, split, clone, w.st);
  GS_LAUNCH_CHECK();
  if (cfg->prune_adaptive) {
    for (int shift = 24; shift >= 0; shift -= 8) {
      kth_hist_kernel<<<G, kSelThreads, 0, s>>>(opacity_logits, split, clone, n, shift, w.st);
      GS_LAUNCH_CHECK();
      kth_find_kernel<<<1, 32, 0, s>>>(shift, cfg->prune_ratio, w.st);
      GS_LAUNCH_CHECK();
    }
  }
  tau_kernel<<<1, 32, 0, s>>>(*cfg, w.st, d_tau_logit);
  GS_LAUNCH_CHECK();
  count_keep_kernel<<<G, kSelThreads, 0, s>>>(opacity_logits, split, clone, n, d_tau_logit, w.st, d_new_n);
  GS_LAUNCH_CHECK();
  publish_kernel<<<1, 32, 0, s>>>(w.st, d_new_n);
  GS_LAUNCH_CHECK();
  return GS_OK;
}

extern "C" gs_status_t gs_densify_apply(const gs_densify_cfg_t *cfg, const gs_params_t *in, const uint8_t *split,
                                        const uint8_t *clone, const float *d_tau_logit, gs_params_out_t *out,
                                        const gs_extra_array_t *extra, int32_t n_extra, const gs_provenance_t *prov,
                                        int64_t out_capacity, int64_t *d_new_n, int32_t *d_error, void *ws,
                                        size_t ws_bytes, gs_stream_t stream) {
  if (!cfg || !in || !split || !clone || !d_tau_logit || !out || !d_new_n || !ws || in->n <= 0 ||
      in->n >= (1ll << 31) || out_capacity < 0)
    return GS_ERR_INVALID_ARG;
  if (!in->means || !in->log_scales || !in->quats || !in->opacity_logits || !in->sh || in->sh_stride <= 0)
    return GS_ERR_INVALID_ARG;
  if (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->sh) return GS_ERR_INVALID_ARG;
  if (n_extra < 0 || n_extra > kMaxExtra || (n_extra > 0 && !extra)) return GS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || (reinterpret_cast<uintptr_t>(in->quats) & 15u) != 0)
    return GS_ERR_INVALID_ARG;
  const DensWs w = dens_layout(ws, in->n);
  if (ws_bytes < w.bytes) return GS_ERR_INVALID_ARG;
  gs_provenance_t pv{};
  if (prov) {
    if (!prov->origin_in || !prov->splits_in || !prov->clones_in || !prov->origin_out || !prov->splits_out ||
        !prov->clones_out)
      return GS_ERR_INVALID_ARG;
    pv = *prov;
  }
  ExtraList el{};
  el.n = n_extra;
  for (int i = 0; i < n_extra; ++i) {
    if (!extra[i].src || !extra[i].dst || extra[i].width <= 0) return GS_ERR_INVALID_ARG;
    el.a[i] = extra[i];
  }
  cudaStream_t s = as_stream(stream);
  const int G = scan_blocks();
  for (int kind = 0; kind < 3; ++kind) {
    uint32_t *pos = kind == 0 ? w.pos_s : (kind == 1 ? w.pos_c : w.pos_p);
    SectionFlag f{in->opacity_logits, split, clone, d_tau_logit, in->n, kind, pos, w.totals + kind};
    if (gs_status_t st = run_scan(f, w.block_sums, G, s)) return st;
  }
  int sg = (int)((in->n + 32 * (kScatThreads / 32) - 1) / (32 * (kScatThreads / 32)));
  // at most the blocks the device keeps resident: with more, a second partial wave
  // of the grid-stride loop runs on a part of the GPU
  static int resident = 0;
  if (resident == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scatter_kernel, kScatThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 4;
    resident = per_sm * num_sms();
  }
  if (sg > resident) sg = resident;
  scatter_kernel<<<sg, kScatThreads, 0, s>>>(*cfg, *in, split, clone, d_tau_logit, *out, el, pv, w.pos_s,
                                                      w.pos_c, w.pos_p, w.totals, out_capacity, d_new_n, d_error);
  GS_LAUNCH_CHECK();
  return GS_OK;
}

// ------------------------------------------------------------------ allocation-free variant
// Some callers cannot allocate device memory for a workspace: custom operators and
// plugins that run inside another runtime's execution callbacks, where allocating
// is forbidden or would bypass the host runtime's memory accounting, and
// fixed-budget deployments that must not grow their device footprint at run time.
// gs_densify_select_static serves them with its scratch (the selection state: two
// counters, the radix-select prefix and a 256-bin histogram) in this file-scope
// device array instead of a caller workspace. Every GPU that loads the library holds
// it until the process exits.
static __device__ __align__(256) SelectState g_select_scratch;

namespace {
constexpr int kMaxScratchDevices = 64;
std::mutex g_scratch_mutex;
SelectState *g_scratch_addr[kMaxScratchDevices] = {};
}  // namespace

// Device address of g_select_scratch on the current device. The array's name is
// only a host-side stand-in for it, so the address is looked up once per device
// (with that device current) and cached; the cache does not survive a
// cudaDeviceReset of that device.
static gs_status_t static_select_scratch(SelectState **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxScratchDevices) return GS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_select_scratch);
    if (e != cudaSuccess || p == nullptr) return GS_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<SelectState *>(p);
  }
  *out = g_scratch_addr[dev];
  return GS_OK;
}

extern "C" gs_status_t gs_densify_select_static(const gs_densify_cfg_t *cfg, const float *log_scales,
                                                const float *opacity_logits, const float *accum,
                                                const int32_t *count, int64_t n, uint8_t *split, uint8_t *clone,
                                                float *d_tau_logit, int64_t *d_new_n, gs_stream_t stream) {
  if (!cfg || !log_scales || !opacity_logits || !accum || !count || n <= 0 || !split || !clone || !d_tau_logit ||
      !d_new_n)
    return GS_ERR_INVALID_ARG;
  if (n > GS_DENSIFY_SELECT_STATIC_MAX_N) return GS_ERR_INVALID_ARG;   // beyond the scratch's counters
  if (cfg->mode < 0 || cfg->mode > 3) return GS_ERR_INVALID_ARG;
  if (cfg->prune_adaptive && !(cfg->prune_ratio > 0.0 && cfg->prune_ratio < 1.0)) return GS_ERR_INVALID_ARG;
  SelectState *st = nullptr;
  if (gs_status_t e = static_select_scratch(&st)) return e;
  cudaStream_t s = as_stream(stream);
  // the previous call's contents are still there: clear the counters and histogram
  GS_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(SelectState), s));
  const int G = dgrid(n);
  select_kernel<<<G, kSelThreads, 0, s>>>(*cfg, log_scales, accum, count, n, split, clone, st);
  GS_LAUNCH_CHECK();
  if (cfg->prune_adaptive) {
    for (int shift = 24; shift >= 0; shift -= 8) {
      kth_hist_kernel<<<G, kSelThreads, 0, s>>>(opacity_logits, split, clone, n, shift, st);
      GS_LAUNCH_CHECK();
      kth_find_kernel<<<1, 32, 0, s>>>(shift, cfg->prune_ratio, st);
      GS_LAUNCH_CHECK();
    }
  }
  tau_kernel<<<1, 32, 0, s>>>(*cfg, st, d_tau_logit);
  GS_LAUNCH_CHECK();
  count_keep_kernel<<<G, kSelThreads, 0, s>>>(opacity_logits, split, clone, n, d_tau_logit, st, d_new_n);
  GS_LAUNCH_CHECK();
  publish_kernel<<<1, 32, 0, s>>>(st, d_new_n);
  GS_LAUNCH_CHECK();
  return GS_OK;
}
