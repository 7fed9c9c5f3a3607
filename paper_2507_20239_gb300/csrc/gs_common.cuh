// Shared device helpers of libgs (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

#define GS_CUDA_TRY(expr)                                        \
  do {                                                           \
    cudaError_t _e = (expr);                                     \
    if (_e != cudaSuccess) { return GS_ERR_CUDA; }               \
  } while (0)

namespace gs {
// Number of kernels this library has enqueued since it was loaded (host side).
void count_launch();
}  // namespace gs

#define GS_LAUNCH_CHECK()   \
  do {                      \
    gs::count_launch();     \
    GS_CUDA_TRY(cudaGetLastError()); \
  } while (0)

namespace gs {

// Debug builds (-DGS_DEBUG, libgs_debug.so): the hot path's index accesses (record
// ids read from the tile lists, the lists' ranges, checkpoint table entries and
// slots, the emitted list positions) are checked before they are made. A failed check
// records (code << 48 | index) in the translation unit's debug word, the first failure
// winning, and the access is skipped, so the launch completes and gs_debug_status
// reports what went wrong. Release builds compile every check to `true`.
// Codes: 1 record id >= records, 2 tile range outside the list, 3 checkpoint table
// index or slot out of range, 4 list position >= capacity.
#ifdef GS_DEBUG
static __device__ unsigned long long g_gs_debug_word;
__device__ __forceinline__ bool debug_check(bool ok, uint32_t code, uint64_t index) {
  if (!ok) atomicCAS(&g_gs_debug_word, 0ull, ((unsigned long long)code << 48) | (index & 0xffffffffffffull));
  return ok;
}
#define GS_CHECK(cond, code, index) ::gs::debug_check((cond), (code), (uint64_t)(index))
// Host side of a translation unit's word: read and clear it (synchronising).
#define GS_DEBUG_TAKE(fn)                                                          \
  uint64_t fn() {                                                                \
    unsigned long long v = 0, z = 0;                                             \
    if (cudaMemcpyFromSymbol(&v, g_gs_debug_word, sizeof(v)) != cudaSuccess) return ~0ull; \
    if (cudaMemcpyToSymbol(g_gs_debug_word, &z, sizeof(z)) != cudaSuccess) return ~0ull;   \
    return v;                                                                    \
  }
uint64_t debug_take_raster();
uint64_t debug_take_bin_sort();
#else
#define GS_CHECK(cond, code, index) true
#endif

constexpr float kNear = 0.2f;            // default near plane (the camera carries its own)
constexpr float kDilation = 0.3f;        // low-pass dilation added to the 2D covariance (px^2)
constexpr float kFovClamp = 1.3f;        // J is evaluated with t_x/t_z clamped to +-1.3 (W/2)/f
constexpr float kAlphaMax = 0.99f;       // sigma = min(0.99, o G)
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;           // transmittance cut-off
constexpr float kLog2e = 1.4426950408889634f;

inline cudaStream_t as_stream(gs_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

inline int num_sms() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
      cached = n;
    else
      cached = 148;
  }
  return cached;
}

// 2^x on the MUFU unit (PTX ex2.approx.ftz.f32).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float kBinMargin = 1.002f;    // tile test keeps q_min <= q_max * 1.002

// Gaussian falloff term of Eq. 2 at one pixel. The conic is carried factored as
// (A, beta, gamma): d^T Sigma''^-1 d = A (dx + beta dy)^2 + gamma dy^2, a sum of two
// non-negative terms that does not cancel for thin, elongated splats. Every
// rounding is explicit so that the forward and backward kernels take identical
// skip / stop decisions.
struct Falloff {
  float dx, dy, t, G, raw, alpha;
};

// The quadratic form is non-negative by construction (A, gamma > 0), so no entry
// needs the "exponent > 0" rejection. The kernels stage the conic pre-scaled,
// a2 = k A and g2 = k gamma with k = -1/2 log2 e, so that G = 2^(a2 t^2 + g2 dy^2)
// with t = dx + beta dy; d = mean - pixel centre.
constexpr float kNegHalfLog2e = -0.72134752044448170f;

__device__ __forceinline__ Falloff falloff(float u, float v, float a2, float beta, float g2, float o,
                                           float px, float py) {
  Falloff f;
  f.dx = __fsub_rn(u, px);
  f.dy = __fsub_rn(v, py);
  f.t = __fmaf_rn(beta, f.dy, f.dx);
  const float e = __fmaf_rn(__fmul_rn(a2, f.t), f.t, __fmul_rn(g2, __fmul_rn(f.dy, f.dy)));
  f.G = ex2_approx(e);
  f.raw = __fmul_rn(o, f.G);
  f.alpha = fminf(kAlphaMax, f.raw);
  return f;
}

// Packed FP32 pairs (sm_100 family: add/sub/mul/fma.rn.f32x2). Each lane of the
// pair is one IEEE round-to-nearest operation, identical to the scalar __fadd_rn /
// __fsub_rn / __fmul_rn / __fmaf_rn, so a packed evaluation takes exactly the
// decisions of the scalar one; it halves the issue slots of paired FP32 work.
__device__ __forceinline__ uint64_t f2_pack(float2 a) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(uint64_t r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(d);
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(d);
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(d);
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)), "l"(f2_pack(c)));
  return f2_unpack(d);
}
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// falloff() at two pixel centres of one row, (px.x, py) and (px.y, py), with packed
// pairs: lane for lane the same operations and roundings as two falloff() calls.
struct Falloff2 {
  float2 t, G, raw, alpha;
  float dy;
};

__device__ __forceinline__ Falloff2 falloff2(float u, float v, float a2, float beta, float g2, float o, float2 px,
                                             float py) {
  Falloff2 f;
  const float2 dx = f2_sub(f2(u), px);
  f.dy = __fsub_rn(v, py);
  f.t = f2_fma(f2(beta), f2(f.dy), dx);
  const float gdd = __fmul_rn(g2, __fmul_rn(f.dy, f.dy));
  const float2 e = f2_fma(f2_mul(f2(a2), f.t), f.t, f2(gdd));
  f.G = make_float2(ex2_approx(e.x), ex2_approx(e.y));
  f.raw = f2_mul(f2(o), f.G);
  f.alpha = make_float2(fminf(kAlphaMax, f.raw.x), fminf(kAlphaMax, f.raw.y));
  return f;
}

// The binning's ellipse-box test, in two steps with one IEEE FP32 rounding per
// operation (no contraction), so that the decision is reproducible op for op:
// band_consts_rn once per record, band_span_rn once per row of tiles (the x-extent of
// the ellipse A (dx + beta dy)^2 + gamma dy^2 <= qb, d = mean - p, over the band of
// pixel-centre rows [Y0, Y1]; derivation beside EllipseRows below), and a box
// [X0, X1] x [Y0, Y1] meets the ellipse iff ok && xl <= xr && X1 >= xl && X0 <= xr.
__device__ __forceinline__ void band_consts_rn(float A, float beta, float gamma, float qb, float &dyr,
                                               float &inv_A) {
  const float ab = __fmul_rn(A, beta);
  const float den = __fadd_rn(__fmul_rn(ab, beta), gamma);
  dyr = __fmul_rn(beta, __fsqrt_rn(__fdiv_rn(__fmul_rn(qb, A), __fmul_rn(gamma, den))));
  inv_A = __fdiv_rn(1.f, A);
}

__device__ __forceinline__ bool band_span_rn(float u, float v, float beta, float gamma, float qb, float dyr,
                                             float inv_A, float Y0, float Y1, float &xl, float &xr) {
  const float dyl = __fsub_rn(v, Y1), dyh = __fsub_rn(v, Y0);
  const float dr = fminf(fmaxf(dyr, dyl), dyh), dl = fminf(fmaxf(-dyr, dyl), dyh);
  const float wr = __fsub_rn(qb, __fmul_rn(gamma, __fmul_rn(dr, dr)));
  const float wl = __fsub_rn(qb, __fmul_rn(gamma, __fmul_rn(dl, dl)));
  xr = __fadd_rn(__fadd_rn(u, __fmul_rn(beta, dr)), __fsqrt_rn(__fmul_rn(fmaxf(wr, 0.f), inv_A)));
  xl = __fsub_rn(__fadd_rn(u, __fmul_rn(beta, dl)), __fsqrt_rn(__fmul_rn(fmaxf(wl, 0.f), inv_A)));
  return (wr >= 0.f || wl >= 0.f) && xl <= xr;
}

// x-extent of the ellipse A (dx + beta dy)^2 + gamma dy^2 <= qb (d = mean - p) over
// a band of pixel-centre rows Y0 <= y <= Y1. At fixed dy the ellipse spans
// x = u + beta dy +- sqrt((qb - gamma dy^2) / A); the right end is concave in dy and
// peaks at the rightmost point of the ellipse, dy_r = beta sqrt(qb A / (gamma (A beta^2
// + gamma))), the left end bottoms out at -dy_r, so over the band each end is taken
// at the clamped extreme. A box [X0, X1] x [Y0, Y1] meets the ellipse iff the band is
// not empty and [X0, X1] meets [xl, xr]. Approximate (MUFU) square root and
// reciprocal: callers use it as a conservative skip test with a margin in qb far
// above their few-ulp error.
struct EllipseRows {
  float u, v, beta, gamma, inv_A, qb, dyr;
};

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ EllipseRows ellipse_rows(float u, float v, float A, float beta, float gamma, float qb) {
  EllipseRows e;
  e.u = u; e.v = v; e.beta = beta; e.gamma = gamma; e.qb = qb;
  e.inv_A = __fdividef(1.f, A);
  const float den = fmaf(A * beta, beta, gamma);
  e.dyr = beta * sqrt_approx(__fdividef(qb * A, gamma * den));
  return e;
}

__device__ __forceinline__ bool row_span(const EllipseRows &e, float Y0, float Y1, float &xl, float &xr) {
  const float dyl = e.v - Y1, dyh = e.v - Y0;
  const float dr = fminf(fmaxf(e.dyr, dyl), dyh), dl = fminf(fmaxf(-e.dyr, dyl), dyh);
  const float wr = e.qb - e.gamma * dr * dr, wl = e.qb - e.gamma * dl * dl;
  if (wr < 0.f && wl < 0.f) return false;
  xr = fmaf(e.beta, dr, e.u) + sqrt_approx(fmaxf(wr, 0.f) * e.inv_A);
  xl = fmaf(e.beta, dl, e.u) - sqrt_approx(fmaxf(wl, 0.f) * e.inv_A);
  return true;
}

// Find the view owning global tile t (views are few; a linear scan of the cameras).
__device__ __forceinline__ int view_of_tile(const gs_camera_t *cams, int n_views, int t) {
  int v = 0;
  for (int i = 1; i < n_views; ++i)
    if (cams[i].tile_offset <= t) v = i;
  return v;
}

// Vector reductions to global memory (sm_90+), fire-and-forget.
__device__ __forceinline__ void red_add_v2(float *addr, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

}  // namespace gs
