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

// Per-Gaussian form of the conic used by the rasterizer. With (A, B, C) the conic,
// dx = u - p_x, dy = v - p_y:
//   A dx^2 + 2 B dx dy + C dy^2 = A (dx + beta dy)^2 + gamma dy^2,
//   beta = B / A, gamma = (A C - B^2) / A,
// a sum of two non-negative terms: unlike the expanded form it does not cancel for
// thin, elongated splats. A C - B^2 is computed with Kahan's FMA-compensated 2x2
// determinant. Returns (A, beta, gamma, opacity).
__device__ __forceinline__ float4 stage_conic(float4 co) {
  const float A = co.x, B = co.y, C = co.z;
  const float w = __fmul_rn(B, B);
  const float e = __fmaf_rn(-B, B, w);   // w - B^2, exact
  const float f = __fmaf_rn(A, C, -w);
  const float det = __fadd_rn(f, e);
  return make_float4(A, __fdiv_rn(B, A), __fdiv_rn(det, A), co.w);
}

// Gaussian falloff term of Eq. 2 at one pixel, from the staged (A, beta, gamma, o).
// Every rounding is explicit so that the forward and backward kernels take
// identical skip / stop decisions.
struct Falloff {
  float dx, dy, t, power, G, raw, alpha;
};

__device__ __forceinline__ Falloff falloff(float u, float v, float A, float beta, float gamma, float o,
                                           float px, float py) {
  Falloff f;
  f.dx = __fsub_rn(u, px);
  f.dy = __fsub_rn(v, py);
  f.t = __fmaf_rn(beta, f.dy, f.dx);
  const float q = __fmaf_rn(__fmul_rn(A, f.t), f.t, __fmul_rn(gamma, __fmul_rn(f.dy, f.dy)));
  f.power = __fmul_rn(-0.5f, q);
  f.G = ex2_approx(__fmul_rn(f.power, kLog2e));
  f.raw = __fmul_rn(o, f.G);
  f.alpha = fminf(kAlphaMax, f.raw);
  return f;
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
