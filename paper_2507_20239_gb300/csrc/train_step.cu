// The rest of a training step around the rasterizer: the photometric loss of
// Eq. 3 with its gradient, (1 - lambda) L1 + lambda D-SSIM, and the optimiser
// update (Adam; sparse Adam skips Gaussians no view of the step saw), with the
// opacity reset of the densification schedule.
//
// SSIM: per channel, an 11 x 11 Gaussian window (sigma 1.5, normalised) applied
// separably with zero padding; mu_x, mu_y and the windowed second moments Sxx, Syy,
// Sxy give map = (2 mu_x mu_y + C1)(2 (Sxy - mu_x mu_y) + C2) /
// ((mu_x^2 + mu_y^2 + C1)(Sxx - mu_x^2 + Syy - mu_y^2 + C2)). Its gradient w.r.t. the
// rendered image x is the window's adjoint (the same symmetric window, zero
// padded) applied to d map / d mu_x, d map / d Sxx and d map / d Sxy, combined as
// W*(d/dmu) + 2 x W*(d/dSxx) + y W*(d/dSxy). Four separable passes per view, every
// view of the frame in one launch each; the sums for the loss are FP64.
#include <cmath>

#include "gs_common.cuh"

namespace gs {

constexpr int kWin = 11, kHalf = 5;
constexpr float kSsimC1 = 0.01f * 0.01f, kSsimC2 = 0.03f * 0.03f;
constexpr int kPlanes = 8;   // scratch planes per pixel value

struct float5_t {
  float v[5];
};

__device__ __forceinline__ void window(float *w) {
  if (threadIdx.x < kWin && threadIdx.y == 0) {
    const float d = (float)((int)threadIdx.x - kHalf);
    w[threadIdx.x] = expf(-d * d / (2.f * 1.5f * 1.5f));
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    float s = 0.f;
    for (int i = 0; i < kWin; ++i) s += w[i];
    w[kWin] = 1.f / s;
  }
  __syncthreads();
}

struct ViewPlane {
  int W, H;
  int64_t base;   // offset of this (view, channel) plane in the planar batch layout
  bool ok;
};

__device__ __forceinline__ ViewPlane view_plane(const gs_camera_t *cams) {
  ViewPlane p;
  const int v = blockIdx.z / 3, c = blockIdx.z - 3 * v;
  const gs_camera_t &cam = cams[v];
  p.W = cam.width;
  p.H = cam.height;
  p.base = 3 * cam.pixel_offset + (int64_t)c * p.W * p.H;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  p.ok = x < p.W && y < p.H;
  return p;
}

// pass 1: horizontal window sums of x, y, x^2, y^2, x y (planes 0..4); L1 sum.
__global__ void ssim_h1_kernel(const gs_camera_t *__restrict__ cams, const float *__restrict__ img,
                               const float *__restrict__ tgt, float *__restrict__ ws, int64_t stride,
                               double *__restrict__ l1) {
  __shared__ float w[kWin + 1];
  __shared__ float s_red[8];
  window(w);
  const ViewPlane p = view_plane(cams);
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  float ad = 0.f;
  if (p.ok) {
    float a[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int64_t row = p.base + (int64_t)y * p.W;
    for (int k = -kHalf; k <= kHalf; ++k) {
      const int xx = x + k;
      if (xx < 0 || xx >= p.W) continue;
      const float wk = w[k + kHalf], xi = img[row + xx], yi = tgt[row + xx];
      a[0] = fmaf(wk, xi, a[0]);
      a[1] = fmaf(wk, yi, a[1]);
      a[2] = fmaf(wk, xi * xi, a[2]);
      a[3] = fmaf(wk, yi * yi, a[3]);
      a[4] = fmaf(wk, xi * yi, a[4]);
    }
    const float n = w[kWin];
    for (int q = 0; q < 5; ++q) ws[q * stride + row + x] = a[q] * n;
    ad = fabsf(img[row + x] - tgt[row + x]);
  }
  // block sum of |x - y| (16 x 16 threads)
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ad += __shfl_xor_sync(0xffffffffu, ad, o);
  if ((t & 31) == 0) s_red[t >> 5] = ad;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x * blockDim.y) / 32; ++i) s += s_red[i];
    atomicAdd(l1 + blockIdx.z / 3, s);
  }
}

// pass 2: vertical window sums -> SSIM map (summed) and its partial derivatives
// w.r.t. mu_x, Sxx, Sxy (planes 5..7).
__global__ void ssim_v1_kernel(const gs_camera_t *__restrict__ cams, float *__restrict__ ws, int64_t stride,
                               double *__restrict__ ssim_sum) {
  __shared__ float w[kWin + 1];
  __shared__ double s_dred[8];
  window(w);
  const ViewPlane p = view_plane(cams);
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  float mapv = 0.f;
  if (p.ok) {
    float a[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = -kHalf; k <= kHalf; ++k) {
      const int yy = y + k;
      if (yy < 0 || yy >= p.H) continue;
      const float wk = w[k + kHalf];
      const int64_t i = p.base + (int64_t)yy * p.W + x;
      for (int q = 0; q < 5; ++q) a[q] = fmaf(wk, ws[q * stride + i], a[q]);
    }
    const float n = w[kWin];
    const float mx = a[0] * n, my = a[1] * n, sxx = a[2] * n, syy = a[3] * n, sxy = a[4] * n;
    const float A1 = 2.f * mx * my + kSsimC1, A2 = 2.f * (sxy - mx * my) + kSsimC2;
    const float B1 = mx * mx + my * my + kSsimC1, B2 = (sxx - mx * mx) + (syy - my * my) + kSsimC2;
    const float inv = 1.f / (B1 * B2);
    mapv = A1 * A2 * inv;
    const int64_t i = p.base + (int64_t)y * p.W + x;
    ws[5 * stride + i] = (2.f * my * (A2 - A1)) * inv - mapv * (2.f * mx * (B2 - B1)) * inv;   // d map / d mu_x
    ws[6 * stride + i] = -mapv / B2;                                                         // d map / d Sxx
    ws[7 * stride + i] = 2.f * A1 * inv;                                                     // d map / d Sxy
  }
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  double m = mapv;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  if ((t & 31) == 0) s_dred[t >> 5] = m;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x * blockDim.y) / 32; ++i) s += s_dred[i];
    atomicAdd(ssim_sum + blockIdx.z / 3, s);
  }
}

// pass 3: horizontal adjoint window over planes 5..7 -> planes 0..2.
__global__ void ssim_h2_kernel(const gs_camera_t *__restrict__ cams, float *__restrict__ ws, int64_t stride) {
  __shared__ float w[kWin + 1];
  window(w);
  const ViewPlane p = view_plane(cams);
  if (!p.ok) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  const int64_t row = p.base + (int64_t)y * p.W;
  float a[3] = {0.f, 0.f, 0.f};
  for (int k = -kHalf; k <= kHalf; ++k) {
    const int xx = x + k;
    if (xx < 0 || xx >= p.W) continue;
    const float wk = w[k + kHalf];
    for (int q = 0; q < 3; ++q) a[q] = fmaf(wk, ws[(5 + q) * stride + row + xx], a[q]);
  }
  for (int q = 0; q < 3; ++q) ws[q * stride + row + x] = a[q] * w[kWin];
}

// pass 4: vertical adjoint window -> d loss / d image.
__global__ void ssim_v2_kernel(const gs_camera_t *__restrict__ cams, const float *__restrict__ img,
                               const float *__restrict__ tgt, const float *__restrict__ ws, int64_t stride,
                               float lambda, float *__restrict__ d_image) {
  __shared__ float w[kWin + 1];
  window(w);
  const ViewPlane p = view_plane(cams);
  if (!p.ok) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  float a[3] = {0.f, 0.f, 0.f};
  for (int k = -kHalf; k <= kHalf; ++k) {
    const int yy = y + k;
    if (yy < 0 || yy >= p.H) continue;
    const float wk = w[k + kHalf];
    const int64_t i = p.base + (int64_t)yy * p.W + x;
    for (int q = 0; q < 3; ++q) a[q] = fmaf(wk, ws[q * stride + i], a[q]);
  }
  const float n = w[kWin];
  const int64_t i = p.base + (int64_t)y * p.W + x;
  const float xi = img[i], yi = tgt[i], d = xi - yi;
  const float inv_n = 1.f / (3.f * (float)p.W * (float)p.H);
  const float g_ssim = (a[0] * n + 2.f * xi * (a[1] * n) + yi * (a[2] * n)) * inv_n;
  const float g_l1 = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
  d_image[i] = (1.f - lambda) * g_l1 - lambda * g_ssim;
}

__global__ void photometric_finalize_kernel(const gs_camera_t *__restrict__ cams, int n_views, float lambda,
                                            const double *__restrict__ l1, const double *__restrict__ ssim,
                                            float *__restrict__ loss) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_views) return;
  const double n = 3.0 * cams[v].width * (double)cams[v].height;
  loss[v] = (float)((1.0 - lambda) * l1[v] / n + lambda * (1.0 - ssim[v] / n));
}

// ------------------------------------------------------------------ optimiser
__global__ void adam_kernel(gs_params_out_t P, gs_param_grads_t G, gs_adam_state_t S, int64_t n, int32_t sh_width,
                            float5_t step_size, float beta1, float beta2, float eps, float sqrt_bc2,
                            const int32_t *__restrict__ radius, int32_t n_views) {
  const int grp = blockIdx.y;
  float *p;
  const float *g;
  int width;
  switch (grp) {
    case 0: p = P.means; g = G.d_means; width = 3; break;
    case 1: p = P.log_scales; g = G.d_log_scales; width = 3; break;
    case 2: p = P.quats; g = G.d_quats; width = 4; break;
    case 3: p = P.opacity_logits; g = G.d_opacity_logits; width = 1; break;
    default: p = P.sh; g = G.d_sh; width = sh_width; break;
  }
  float *m = S.m[grp], *v = S.v[grp];
  const float ss = step_size.v[grp];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  auto visible = [&](int64_t row) {
    bool seen = false;
    for (int k = 0; k < n_views; ++k) seen |= radius[(int64_t)k * n + row] > 0;
    return seen;
  };
  auto update = [&](float &pi, float &mi, float &vi, float gi) {
    mi = beta1 * mi + (1.f - beta1) * gi;
    vi = beta2 * vi + (1.f - beta2) * gi * gi;
    pi -= ss * mi / (sqrtf(vi) / sqrt_bc2 + eps);
  };
  const bool vec = (width & 3) == 0 && ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(g) |
                                         reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) & 15u) == 0;
  if (vec) {
    // rows of a multiple of four floats on 16-byte boundaries (quaternions, SH rows):
    // four elements of one row per thread and 16-byte accesses, one visibility test
    // per vector; the same per-element update
    const int w4 = width >> 2;
    const int64_t total4 = n * w4;
    float4 *p4 = reinterpret_cast<float4 *>(p), *m4 = reinterpret_cast<float4 *>(m), *v4 = reinterpret_cast<float4 *>(v);
    const float4 *g4 = reinterpret_cast<const float4 *>(g);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total4; i += stride) {
      if (radius && !visible(i / w4)) continue;
      const float4 gi = g4[i];
      float4 pi = p4[i], mi = m4[i], vi = v4[i];
      update(pi.x, mi.x, vi.x, gi.x);
      update(pi.y, mi.y, vi.y, gi.y);
      update(pi.z, mi.z, vi.z, gi.z);
      update(pi.w, mi.w, vi.w, gi.w);
      m4[i] = mi;
      v4[i] = vi;
      p4[i] = pi;
    }
    return;
  }
  const int64_t total = n * width;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += stride) {
    if (radius && !visible(i / width)) continue;
    float pi = p[i], mi = m[i], vi = v[i];
    update(pi, mi, vi, g[i]);
    m[i] = mi;
    v[i] = vi;
    p[i] = pi;
  }
}

__global__ void opacity_reset_kernel(float *__restrict__ logits, float *__restrict__ m, float *__restrict__ v,
                                     int64_t n, float cap) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    logits[i] = fminf(logits[i], cap);
    if (m) m[i] = 0.f;
    if (v) v[i] = 0.f;
  }
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_photometric_workspace_size(const gs_frame_t *frame) {
  if (!frame || frame->n_views <= 0 || frame->n_pixels <= 0) return 0;
  return sizeof(float) * kPlanes * 3 * (size_t)frame->n_pixels + 2 * sizeof(double) * (size_t)frame->n_views + 256;
}

extern "C" gs_status_t gs_photometric_loss_grad(const gs_frame_t *frame, const float *image, const float *target,
                                                float lambda, float *d_image, float *loss_dev, void *ws,
                                                size_t ws_bytes, gs_stream_t stream) {
  if (!frame || !frame->cams_dev || frame->n_views <= 0 || !image || !target || !d_image || !loss_dev || !ws)
    return GS_ERR_INVALID_ARG;
  if (!(lambda >= 0.f && lambda <= 1.f) || ws_bytes < gs_photometric_workspace_size(frame) ||
      (reinterpret_cast<uintptr_t>(ws) & 15u) != 0)
    return GS_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  const int64_t stride = 3 * frame->n_pixels;
  float *planes = static_cast<float *>(ws);
  double *l1 = reinterpret_cast<double *>(planes + kPlanes * stride);
  double *ssim = l1 + frame->n_views;
  GS_CUDA_TRY(cudaMemsetAsync(l1, 0, 2 * sizeof(double) * frame->n_views, s));
  const dim3 block(16, 16);
  const dim3 grid((frame->max_width + 15) / 16, (frame->max_height + 15) / 16, 3 * frame->n_views);
  ssim_h1_kernel<<<grid, block, 0, s>>>(frame->cams_dev, image, target, planes, stride, l1);
  GS_LAUNCH_CHECK();
  ssim_v1_kernel<<<grid, block, 0, s>>>(frame->cams_dev, planes, stride, ssim);
  GS_LAUNCH_CHECK();
  ssim_h2_kernel<<<grid, block, 0, s>>>(frame->cams_dev, planes, stride);
  GS_LAUNCH_CHECK();
  ssim_v2_kernel<<<grid, block, 0, s>>>(frame->cams_dev, image, target, planes, stride, lambda, d_image);
  GS_LAUNCH_CHECK();
  photometric_finalize_kernel<<<(frame->n_views + 127) / 128, 128, 0, s>>>(frame->cams_dev, frame->n_views, lambda,
                                                                           l1, ssim, loss_dev);
  GS_LAUNCH_CHECK();
  return GS_OK;
}

extern "C" gs_status_t gs_adam_step(const gs_adam_cfg_t *cfg, gs_params_out_t *params, int64_t n, int32_t sh_stride,
                                    const gs_param_grads_t *grads, gs_adam_state_t *state, const int32_t *radius,
                                    int32_t n_views, gs_stream_t stream) {
  if (!cfg || !params || !grads || !state || n < 0 || sh_stride < 1 || cfg->step < 1) return GS_ERR_INVALID_ARG;
  if (radius && n_views < 1) return GS_ERR_INVALID_ARG;
  if (!params->means || !params->log_scales || !params->quats || !params->opacity_logits || !params->sh ||
      !grads->d_means || !grads->d_log_scales || !grads->d_quats || !grads->d_opacity_logits || !grads->d_sh)
    return GS_ERR_INVALID_ARG;
  for (int k = 0; k < 5; ++k)
    if (!state->m[k] || !state->v[k]) return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  const double bc1 = 1.0 - std::pow(cfg->beta1, (double)cfg->step);
  const double bc2 = 1.0 - std::pow(cfg->beta2, (double)cfg->step);
  float5_t ss;
  for (int k = 0; k < 5; ++k) ss.v[k] = (float)(cfg->lr[k] / bc1);
  const int64_t widest = n * 3 * (int64_t)sh_stride;
  const int gx = (int)std::min<int64_t>((widest + 255) / 256, (int64_t)num_sms() * 8);
  adam_kernel<<<dim3(gx, 5), 256, 0, as_stream(stream)>>>(*params, *grads, *state, n, 3 * sh_stride, ss,
                                                          (float)cfg->beta1, (float)cfg->beta2, cfg->eps,
                                                          (float)std::sqrt(bc2), radius, n_views);
  GS_LAUNCH_CHECK();
  return GS_OK;
}

extern "C" gs_status_t gs_opacity_reset(float *opacity_logits, float *m, float *v, int64_t n, float max_opacity,
                                        gs_stream_t stream) {
  if (!opacity_logits || n < 0 || !(max_opacity > 0.f && max_opacity < 1.f)) return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  const float cap = (float)std::log((double)max_opacity / (1.0 - (double)max_opacity));
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
  opacity_reset_kernel<<<grid, 256, 0, as_stream(stream)>>>(opacity_logits, m, v, n, cap);
  GS_LAUNCH_CHECK();
  return GS_OK;
}
