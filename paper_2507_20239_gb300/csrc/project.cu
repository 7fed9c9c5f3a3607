// EWA projection + SH colour (forward) and its vector-Jacobian product.
//
// Forward per (view, Gaussian) record: Eq. 1's covariance Sigma = R S S^T R^T,
// the affine projection Sigma' = J W Sigma W^T J^T (Sec. "Preliminary"), the conic
// (Sigma' + 0.3 I)^-1, the footprint where alpha can reach the 1/255 floor (the
// ellipse d^T Sigma''^-1 d <= 2 ln(255 o); its bounding box, with the binning
// margin, gives the extent), the pixel mean, the tile rectangle and the
// SH-evaluated colour c_i of Eq. 2.  Backward per Gaussian: the chain rule through
// all of the above, summed over views, with the optional densification statistic.
#include <math.h>

#include "gs_common.cuh"

namespace gs {

// Real SH with the Condon-Shortley phase, index k = l^2 + l + m. Each constant is
// K_lm (times sqrt 2 for m != 0) of the polynomial written beside it.
constexpr float kC0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kC1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float kC2a = 1.0925484305920792f;   // sqrt(15/pi)/2        xy, yz, xz
constexpr float kC2b = 0.31539156525252005f;  // sqrt(5/pi)/4         3z^2 - 1
constexpr float kC2c = 0.5462742152960396f;   // sqrt(15/pi)/4        x^2 - y^2
constexpr float kC3a = 0.5900435899266435f;   // sqrt(35/(2 pi))/4    y(3x^2-y^2), x(x^2-3y^2)
constexpr float kC3b = 2.890611442640554f;    // sqrt(105/pi)/2       xyz
constexpr float kC3c = 0.4570457994644658f;   // sqrt(21/(2 pi))/4    y(5z^2-1), x(5z^2-1)
constexpr float kC3d = 0.3731763325901154f;   // sqrt(7/pi)/4         z(5z^2-3)
constexpr float kC3e = 1.445305721320277f;    // sqrt(105/pi)/4       z(x^2-y^2)

// Visit every basis function k < (DEG+1)^2 with its value and its gradient w.r.t.
// the (unnormalised) direction components, without materialising arrays:
// f(k, Y, dY/dx, dY/dy, dY/dz).
template <int DEG, typename F>
__device__ __forceinline__ void sh_visit(float x, float y, float z, F &&f) {
  f(0, kC0, 0.f, 0.f, 0.f);
  if (DEG >= 1) {
    f(1, -kC1 * y, 0.f, -kC1, 0.f);
    f(2, kC1 * z, 0.f, 0.f, kC1);
    f(3, -kC1 * x, -kC1, 0.f, 0.f);
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    f(4, kC2a * x * y, kC2a * y, kC2a * x, 0.f);
    f(5, -kC2a * y * z, 0.f, -kC2a * z, -kC2a * y);
    f(6, kC2b * (3.f * zz - 1.f), 0.f, 0.f, 6.f * kC2b * z);
    f(7, -kC2a * x * z, -kC2a * z, 0.f, -kC2a * x);
    f(8, kC2c * (xx - yy), 2.f * kC2c * x, -2.f * kC2c * y, 0.f);
    if (DEG >= 3) {
      f(9, -kC3a * y * (3.f * xx - yy), -6.f * kC3a * x * y, -3.f * kC3a * (xx - yy), 0.f);
      f(10, kC3b * x * y * z, kC3b * y * z, kC3b * x * z, kC3b * x * y);
      f(11, -kC3c * y * (5.f * zz - 1.f), 0.f, -kC3c * (5.f * zz - 1.f), -10.f * kC3c * y * z);
      f(12, kC3d * z * (5.f * zz - 3.f), 0.f, 0.f, kC3d * (15.f * zz - 3.f));
      f(13, -kC3c * x * (5.f * zz - 1.f), -kC3c * (5.f * zz - 1.f), 0.f, -10.f * kC3c * x * z);
      f(14, kC3e * z * (xx - yy), 2.f * kC3e * x * z, -2.f * kC3e * y * z, kC3e * (xx - yy));
      f(15, -kC3a * x * (xx - 3.f * yy), -3.f * kC3a * (xx - yy), 6.f * kC3a * x * y, 0.f);
    }
  }
}

struct Rot {
  float m[9];
};

// Rotation of the normalised quaternion (w, x, y, z).
__device__ __forceinline__ Rot quat_rot(float w, float x, float y, float z) {
  Rot R;
  R.m[0] = 1.f - 2.f * (y * y + z * z); R.m[1] = 2.f * (x * y - w * z);       R.m[2] = 2.f * (x * z + w * y);
  R.m[3] = 2.f * (x * y + w * z);       R.m[4] = 1.f - 2.f * (x * x + z * z); R.m[5] = 2.f * (y * z - w * x);
  R.m[6] = 2.f * (x * z - w * y);       R.m[7] = 2.f * (y * z + w * x);       R.m[8] = 1.f - 2.f * (x * x + y * y);
  return R;
}

// Everything the forward computes for one record up to the conic, reused by the VJP.
struct ProjGeom {
  float tx, ty, tz;
  float rx, ry;         // clamped t_x/t_z, t_y/t_z
  bool clx, cly;        // clamp active
  float T0[3], T1[3];   // rows of J W
  float K0[3], K1[3];   // rows of K = (J W) (R S), so that Sigma' = K K^T
  float a, b, c, det;   // Sigma' + 0.3 I and its determinant
};

__device__ __forceinline__ void camera_space(const gs_camera_t &cam, float mx, float my, float mz,
                                             float &tx, float &ty, float &tz) {
  tx = fmaf(cam.R[0], mx, fmaf(cam.R[1], my, fmaf(cam.R[2], mz, cam.t[0])));
  ty = fmaf(cam.R[3], mx, fmaf(cam.R[4], my, fmaf(cam.R[5], mz, cam.t[1])));
  tz = fmaf(cam.R[6], mx, fmaf(cam.R[7], my, fmaf(cam.R[8], mz, cam.t[2])));
}

// Sigma' = J W Sigma W^T J^T with Sigma = M M^T, M = R S, formed as K K^T with
// K = (J W) M so that Sigma is never built (building it squares the condition number
// of thin Gaussians). det(Sigma' + 0.3 I) uses the Lagrange identity
// |K0|^2 |K1|^2 - (K0.K1)^2 = |K0 x K1|^2, which has no cancellation.
__device__ __forceinline__ void project_cov(const gs_camera_t &cam, const float *M, ProjGeom &P) {
  const float itz = 1.f / P.tz;
  const float limx = kFovClamp * 0.5f * (float)cam.width / cam.fx;
  const float limy = kFovClamp * 0.5f * (float)cam.height / cam.fy;
  const float rx0 = P.tx * itz, ry0 = P.ty * itz;
  P.rx = fminf(fmaxf(rx0, -limx), limx);
  P.ry = fminf(fmaxf(ry0, -limy), limy);
  P.clx = (rx0 < -limx) || (rx0 > limx);
  P.cly = (ry0 < -limy) || (ry0 > limy);
  const float J00 = cam.fx * itz, J02 = -cam.fx * P.rx * itz;
  const float J11 = cam.fy * itz, J12 = -cam.fy * P.ry * itz;
  const float *W = cam.R;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    P.T0[k] = J00 * W[k] + J02 * W[6 + k];
    P.T1[k] = J11 * W[3 + k] + J12 * W[6 + k];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    P.K0[j] = P.T0[0] * M[j] + P.T0[1] * M[3 + j] + P.T0[2] * M[6 + j];
    P.K1[j] = P.T1[0] * M[j] + P.T1[1] * M[3 + j] + P.T1[2] * M[6 + j];
  }
  const float n0 = P.K0[0] * P.K0[0] + P.K0[1] * P.K0[1] + P.K0[2] * P.K0[2];
  const float n1 = P.K1[0] * P.K1[0] + P.K1[1] * P.K1[1] + P.K1[2] * P.K1[2];
  const float x0 = P.K0[1] * P.K1[2] - P.K0[2] * P.K1[1];
  const float x1 = P.K0[2] * P.K1[0] - P.K0[0] * P.K1[2];
  const float x2 = P.K0[0] * P.K1[1] - P.K0[1] * P.K1[0];
  P.a = n0 + kDilation;
  P.b = P.K0[0] * P.K1[0] + P.K0[1] * P.K1[1] + P.K0[2] * P.K1[2];
  P.c = n1 + kDilation;
  P.det = (x0 * x0 + x1 * x1 + x2 * x2) + kDilation * (n0 + n1) + kDilation * kDilation;
}

// M = R diag(s).
__device__ __forceinline__ void scale_rot(const Rot &R, float s0, float s1, float s2, float *M) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    M[3 * i + 0] = R.m[3 * i + 0] * s0;
    M[3 * i + 1] = R.m[3 * i + 1] * s1;
    M[3 * i + 2] = R.m[3 * i + 2] * s2;
  }
}

__device__ __forceinline__ void camera_centre(const gs_camera_t &cam, float &cx, float &cy, float &cz) {
  const float *W = cam.R;
  cx = -(W[0] * cam.t[0] + W[3] * cam.t[1] + W[6] * cam.t[2]);
  cy = -(W[1] * cam.t[0] + W[4] * cam.t[1] + W[7] * cam.t[2]);
  cz = -(W[2] * cam.t[0] + W[5] * cam.t[1] + W[8] * cam.t[2]);
}

// VEC: the SH rows start on 16-byte boundaries (sh_stride a multiple of 4), so a
// thread reads its row as float4s: 4 coefficients x 3 channels per three loads.
template <int DEG, bool VEC>
__global__ void __launch_bounds__(256) project_fwd_kernel(gs_params_t P, const gs_camera_t *__restrict__ cams,
                                                          int n_views, int tile_w, int tile_h, gs_proj_t out) {
  const int64_t R = (int64_t)n_views * P.n;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int v = (int)(r / P.n);
    const int64_t g = r - (int64_t)v * P.n;
    const gs_camera_t &cam = cams[v];
    // every geometric input is requested at once (the few records behind the near
    // plane read 32 bytes they do not use), so a record waits for one round trip
    // before its SH row instead of two
    const float mx = P.means[3 * g + 0], my = P.means[3 * g + 1], mz = P.means[3 * g + 2];
    const float4 q = reinterpret_cast<const float4 *>(P.quats)[g];
    const float ls0 = P.log_scales[3 * g + 0], ls1 = P.log_scales[3 * g + 1], ls2 = P.log_scales[3 * g + 2];
    const float logit = P.opacity_logits[g];
    ProjGeom G;
    camera_space(cam, mx, my, mz, G.tx, G.ty, G.tz);
    bool ok = G.tz > cam.near_plane;
    int radius = 0, x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    float u = 0.f, vv = 0.f, A = 0.f, B = 0.f, C = 0.f, qmax = 0.f;   // (A, B, C) = (A, beta, gamma)
    float o_ = 0.f;
    if (ok) {
      const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
      const Rot Rq = quat_rot(q.x * inv, q.y * inv, q.z * inv, q.w * inv);
      const float s0 = expf(ls0);
      const float s1 = expf(ls1);
      const float s2 = expf(ls2);
      float M[9];
      scale_rot(Rq, s0, s1, s2, M);
      project_cov(cam, M, G);
      o_ = 1.f / (1.f + expf(-logit));
      ok = G.det > 0.f && o_ >= kAlphaMin;
      if (ok) {
        // factored conic: A = c/det, beta = -b/c, gamma = 1/c
        A = G.c / G.det;
        B = -G.b / G.c;
        C = 1.f / G.c;
        // alpha = min(0.99, o G) reaches 1/255 only where d^T Sigma''^-1 d <= q_max
        qmax = 2.f * logf(255.f * o_);
        const float qb = __fmul_rn(qmax, kBinMargin);
        const float hx = sqrtf(qb * G.a), hy = sqrtf(qb * G.c);
        radius = (int)fminf(ceilf(fmaxf(hx, hy)), 1.0e9f);
        const float itz = 1.f / G.tz;
        u = cam.fx * G.tx * itz + cam.cx;
        vv = cam.fy * G.ty * itz + cam.cy;
        // tiles under the footprint's bounding box: one rounded FP32 add/sub and one
        // division per bound
        const float ftw = (float)tile_w, fth = (float)tile_h;
        x0 = (int)fminf(fmaxf(floorf(__fdiv_rn(__fsub_rn(u, hx), ftw)), 0.f), (float)cam.grid_x);
        y0 = (int)fminf(fmaxf(floorf(__fdiv_rn(__fsub_rn(vv, hy), fth)), 0.f), (float)cam.grid_y);
        x1 = (int)fminf(fmaxf(floorf(__fdiv_rn(__fadd_rn(u, hx), ftw)) + 1.f, 0.f), (float)cam.grid_x);
        y1 = (int)fminf(fmaxf(floorf(__fdiv_rn(__fadd_rn(vv, hy), fth)) + 1.f, 0.f), (float)cam.grid_y);
        ok = (x1 > x0) && (y1 > y0);
      }
    }
    if (!ok) {
      reinterpret_cast<float2 *>(out.mean2d)[r] = make_float2(0.f, 0.f);
      reinterpret_cast<float4 *>(out.conic_opacity)[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      reinterpret_cast<float4 *>(out.rgb)[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      out.depth[r] = 0.f;
      out.radius[r] = 0;
      reinterpret_cast<uint2 *>(out.rect)[r] = make_uint2(0u, 0u);
      out.clamped[r] = 0;
      continue;
    }
    // SH colour, direction from the camera centre to the mean
    float ccx, ccy, ccz;
    camera_centre(cam, ccx, ccy, ccz);
    float dx = mx - ccx, dy = my - ccy, dz = mz - ccz;
    const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= il; dy *= il; dz *= il;
    const float *sh = P.sh + (int64_t)g * P.sh_stride * 3;
    float cr = 0.5f, cg = 0.5f, cb = 0.5f;
    if (VEC) {
      constexpr int K = (DEG + 1) * (DEG + 1);
      float Y[K];
      sh_visit<DEG>(dx, dy, dz, [&](int k, float y, float, float, float) { Y[k] = y; });
      const float4 *sh4 = reinterpret_cast<const float4 *>(sh);
#pragma unroll
      for (int q = 0; q < (K + 3) / 4; ++q) {
        const float4 a = sh4[3 * q], b = sh4[3 * q + 1], c = sh4[3 * q + 2];
        const float f[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (4 * q + i >= K) break;
          cr = fmaf(Y[4 * q + i], f[3 * i + 0], cr);
          cg = fmaf(Y[4 * q + i], f[3 * i + 1], cg);
          cb = fmaf(Y[4 * q + i], f[3 * i + 2], cb);
        }
      }
    } else {
      sh_visit<DEG>(dx, dy, dz, [&](int k, float Y, float, float, float) {
        cr = fmaf(Y, sh[3 * k + 0], cr);
        cg = fmaf(Y, sh[3 * k + 1], cg);
        cb = fmaf(Y, sh[3 * k + 2], cb);
      });
    }
    const uint8_t cl = (cr < 0.f ? 1 : 0) | (cg < 0.f ? 2 : 0) | (cb < 0.f ? 4 : 0);
    reinterpret_cast<float2 *>(out.mean2d)[r] = make_float2(u, vv);
    reinterpret_cast<float4 *>(out.conic_opacity)[r] = make_float4(A, B, C, o_);
    reinterpret_cast<float4 *>(out.rgb)[r] = make_float4(fmaxf(cr, 0.f), fmaxf(cg, 0.f), fmaxf(cb, 0.f), qmax);
    out.depth[r] = G.tz;
    out.radius[r] = radius;
    const uint32_t lo = (uint32_t)x0 | ((uint32_t)y0 << 16), hi = (uint32_t)x1 | ((uint32_t)y1 << 16);
    reinterpret_cast<uint2 *>(out.rect)[r] = make_uint2(lo, hi);
    out.clamped[r] = cl;
  }
}

// Projection VJP, geometric part: conic, pixel mean and opacity gradients of every
// view -> means (through t = W mu + t_w and J), log-scales, quaternion, opacity
// logit; the densification statistic is fused. The colour part is project_bwd_sh.
// Every input is requested at entry, before the visibility test (with several views
// the per-view records follow it): the parameters of a Gaussian no view sees are read
// and not used, but a thread waits for one round trip instead of two.
template <bool ONE_VIEW>
__global__ void __launch_bounds__(128, 5) project_bwd_geom_kernel(gs_params_t P, const gs_camera_t *__restrict__ cams,
                                                               int n_views, gs_proj_t proj, gs_rec_grads_t rg,
                                                               gs_param_grads_t out, float *accum, int32_t *count) {
  const int64_t n = P.n;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    {
    const float mx = P.means[3 * g + 0], my = P.means[3 * g + 1], mz = P.means[3 * g + 2];
    const float4 q = reinterpret_cast<const float4 *>(P.quats)[g];
    const float ls0 = P.log_scales[3 * g + 0], ls1 = P.log_scales[3 * g + 1], ls2 = P.log_scales[3 * g + 2];
    const float logit = P.opacity_logits[g];
    int rad1 = 0;
    float2 gm1 = make_float2(0.f, 0.f);
    float4 gco1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ONE_VIEW) {
      rad1 = proj.radius[g];
      gm1 = reinterpret_cast<const float2 *>(rg.d_mean2d)[g];
      gco1 = reinterpret_cast<const float4 *>(rg.d_conic_opacity)[g];
    }
    float d_mean[3] = {0.f, 0.f, 0.f};
    float dM[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // dL/dM, M = R S
    float d_logit = 0.f;
    float acc = accum ? accum[g] : 0.f;
    int cnt = count ? count[g] : 0;
    bool any = false;
    // view-independent pieces, computed on first use
    float qinv = 0.f, s0 = 0.f, s1 = 0.f, s2 = 0.f, M[9];
    Rot Rq;
    for (int v = 0; v < (ONE_VIEW ? 1 : n_views); ++v) {
      const int64_t r = (int64_t)v * n + g;
      if ((ONE_VIEW ? rad1 : proj.radius[r]) <= 0) continue;
      const gs_camera_t &cam = cams[v];
      if (!any) {
        any = true;
        qinv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        Rq = quat_rot(q.x * qinv, q.y * qinv, q.z * qinv, q.w * qinv);
        s0 = expf(ls0);
        s1 = expf(ls1);
        s2 = expf(ls2);
        scale_rot(Rq, s0, s1, s2, M);
      }
      ProjGeom G;
      camera_space(cam, mx, my, mz, G.tx, G.ty, G.tz);
      project_cov(cam, M, G);
      const float2 gm = ONE_VIEW ? gm1 : reinterpret_cast<const float2 *>(rg.d_mean2d)[r];
      const float4 gco = ONE_VIEW ? gco1 : reinterpret_cast<const float4 *>(rg.d_conic_opacity)[r];
      if (accum) {
        const float gx = __fmul_rn(gm.x, 0.5f * (float)cam.width);
        const float gy = __fmul_rn(gm.y, 0.5f * (float)cam.height);
        acc = __fadd_rn(acc, __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy))));
        cnt += 1;
      }
      // factored conic (A, beta, gamma) = (c/det, -b/c, 1/c)  ->  (a, b, c)
      const float b = G.b, c = G.c;
      const float id2 = 1.f / (G.det * G.det), ic = 1.f / c, ic2 = ic * ic;
      const float da = -c * c * id2 * gco.x;
      const float db = 2.f * b * c * id2 * gco.x - ic * gco.y;
      const float dc = -b * b * id2 * gco.x + b * ic2 * gco.y - ic2 * gco.z;
      // a = |K0|^2 + 0.3, b = K0.K1, c = |K1|^2 + 0.3 with K = T M
      float dK0[3], dK1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        dK0[k] = 2.f * da * G.K0[k] + db * G.K1[k];
        dK1[k] = db * G.K0[k] + 2.f * dc * G.K1[k];
      }
      // K = T M: dT = dK M^T, dM += T^T dK
      float dT0[3], dT1[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        dT0[i] = dK0[0] * M[3 * i + 0] + dK0[1] * M[3 * i + 1] + dK0[2] * M[3 * i + 2];
        dT1[i] = dK1[0] * M[3 * i + 0] + dK1[1] * M[3 * i + 1] + dK1[2] * M[3 * i + 2];
#pragma unroll
        for (int j = 0; j < 3; ++j) dM[3 * i + j] += G.T0[i] * dK0[j] + G.T1[i] * dK1[j];
      }
      // T = J W  ->  dJ = dT W^T (only the non-zero entries of J matter)
      const float *W = cam.R;
      const float dJ00 = dT0[0] * W[0] + dT0[1] * W[1] + dT0[2] * W[2];
      const float dJ02 = dT0[0] * W[6] + dT0[1] * W[7] + dT0[2] * W[8];
      const float dJ11 = dT1[0] * W[3] + dT1[1] * W[4] + dT1[2] * W[5];
      const float dJ12 = dT1[0] * W[6] + dT1[1] * W[7] + dT1[2] * W[8];
      const float itz = 1.f / G.tz, itz2 = itz * itz;
      float dtx = 0.f, dty = 0.f, dtz = 0.f;
      dtz += -dJ00 * cam.fx * itz2 - dJ11 * cam.fy * itz2;
      if (G.clx) {
        dtz += dJ02 * cam.fx * G.rx * itz2;
      } else {
        dtx += -dJ02 * cam.fx * itz2;
        dtz += 2.f * dJ02 * cam.fx * G.tx * itz2 * itz;
      }
      if (G.cly) {
        dtz += dJ12 * cam.fy * G.ry * itz2;
      } else {
        dty += -dJ12 * cam.fy * itz2;
        dtz += 2.f * dJ12 * cam.fy * G.ty * itz2 * itz;
      }
      // pixel mean u = fx tx / tz + cx, v = fy ty / tz + cy
      dtx += gm.x * cam.fx * itz;
      dty += gm.y * cam.fy * itz;
      dtz += -(gm.x * cam.fx * G.tx + gm.y * cam.fy * G.ty) * itz2;
      // t = W mu + t_w
      d_mean[0] += W[0] * dtx + W[3] * dty + W[6] * dtz;
      d_mean[1] += W[1] * dtx + W[4] * dty + W[7] * dtz;
      d_mean[2] += W[2] * dtx + W[5] * dty + W[8] * dtz;
      // opacity = sigmoid(logit)
      const float o = 1.f / (1.f + expf(-logit));
      d_logit += gco.w * o * (1.f - o);
    }
    float d_ls[3] = {0.f, 0.f, 0.f};
    float d_q[4] = {0.f, 0.f, 0.f, 0.f};
    if (any) {
      // M = R diag(s)
      const float sc[3] = {s0, s1, s2};
      float dR[9];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        float ds = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          ds += dM[3 * i + j] * Rq.m[3 * i + j];
          dR[3 * i + j] = dM[3 * i + j] * sc[j];
        }
        d_ls[j] = ds * sc[j];
      }
      // R(q_hat) -> q_hat -> q (through the normalisation)
      const float w = q.x * qinv, x = q.y * qinv, y = q.z * qinv, z = q.w * qinv;
      const float dw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
      const float dx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] +
                              w * dR[7] - 2.f * x * dR[8]);
      const float dy = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                              z * dR[7] - 2.f * y * dR[8]);
      const float dz = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] +
                              y * dR[5] + x * dR[6] + y * dR[7]);
      const float proj_ = w * dw + x * dx + y * dy + z * dz;
      d_q[0] = (dw - w * proj_) * qinv;
      d_q[1] = (dx - x * proj_) * qinv;
      d_q[2] = (dy - y * proj_) * qinv;
      d_q[3] = (dz - z * proj_) * qinv;
    }
    out.d_means[3 * g + 0] = d_mean[0];
    out.d_means[3 * g + 1] = d_mean[1];
    out.d_means[3 * g + 2] = d_mean[2];
    out.d_log_scales[3 * g + 0] = d_ls[0];
    out.d_log_scales[3 * g + 1] = d_ls[1];
    out.d_log_scales[3 * g + 2] = d_ls[2];
    reinterpret_cast<float4 *>(out.d_quats)[g] = make_float4(d_q[0], d_q[1], d_q[2], d_q[3]);
    out.d_opacity_logits[g] = d_logit;
    if (accum) {
      accum[g] = acc;
      count[g] = cnt;
    }
    }
  }
}

// Projection VJP, colour part: SH coefficient gradients (zero through a clamped
// channel) and the colour's dependence on the viewing direction, added to the
// mean gradients that project_bwd_geom_kernel wrote. STAGED (sh_stride ==
// (DEG+1)^2): each warp moves the SH rows of its 32 Gaussians and their gradients
// between global and shared memory with coalesced accesses (rows padded by one float).
// ONE_VIEW: with a single view each coefficient's gradient is written once, right
// after the coefficient has been read, so it overwrites the staged row in place and
// one shared buffer suffices (twice the resident blocks).
template <int DEG, bool STAGED, bool ONE_VIEW>
__global__ void __launch_bounds__(128, ONE_VIEW ? 8 : 4) project_bwd_sh_kernel(
    gs_params_t P, const gs_camera_t *__restrict__ cams, int n_views, gs_proj_t proj, gs_rec_grads_t rg,
    gs_param_grads_t out, bool vec) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int RW = 3 * K, RP = RW + 1;
  constexpr bool IN_PLACE = STAGED && ONE_VIEW;
  __shared__ float s_sh[STAGED ? 4 * 32 * RP : 1];
  __shared__ float s_dsh[IN_PLACE ? 1 : 4 * 32 * RP];
  const int64_t n = P.n;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float *wsh = s_sh + (STAGED ? wib * 32 * RP : 0);
  float *dsh_row = IN_PLACE ? wsh + lane * RP : s_dsh + (wib * 32 + lane) * RP;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = base + threadIdx.x;
    const int64_t g0 = base + wib * 32;
    const int rows = (int)(n - g0 < 0 ? 0 : (n - g0 > 32 ? 32 : n - g0));
    // with one view, the record's inputs are requested before the row staging, so
    // they arrive while it runs
    int rad1 = 0;
    float mx1 = 0.f, my1 = 0.f, mz1 = 0.f;
    float4 grgb1 = make_float4(0.f, 0.f, 0.f, 0.f);
    uint8_t cl1 = 0;
    if (ONE_VIEW && g < n) {
      rad1 = proj.radius[g];
      mx1 = P.means[3 * g + 0]; my1 = P.means[3 * g + 1]; mz1 = P.means[3 * g + 2];
      grgb1 = reinterpret_cast<const float4 *>(rg.d_rgb)[g];
      cl1 = proj.clamped[g];
    }
    if (STAGED) {
      // rows of Gaussians culled in every view are not read: their coefficients are
      // never used and their gradient rows are zero
      bool seen = false;
      if (ONE_VIEW)
        seen = rad1 > 0;
      else if (g < n)
        for (int v = 0; v < n_views && !seen; ++v) seen = proj.radius[(int64_t)v * n + g] > 0;
      const uint32_t vmask = __ballot_sync(0xffffffffu, seen);
      const float *src = P.sh + g0 * RW;
      if (RW % 4 == 0 && vec) {   // rows of 3K floats, K = 4 or 16: whole float4s, none across rows
        for (int f4 = lane; f4 < rows * RW / 4; f4 += 32) {
          const int row = (4 * f4) / RW;
          if (!((vmask >> row) & 1u)) continue;
          const float4 x = reinterpret_cast<const float4 *>(src)[f4];
          float *d = wsh + row * RP + (4 * f4) % RW;
          d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
        }
      } else {
        for (int f = lane; f < rows * RW; f += 32)
          if ((vmask >> (f / RW)) & 1u) wsh[(f / RW) * RP + (f % RW)] = src[f];
      }
      __syncwarp();
    }
    if (g < n) {
      const float *sh = STAGED ? wsh + lane * RP : P.sh + (int64_t)g * P.sh_stride * 3;
      if (!IN_PLACE) {
#pragma unroll
        for (int k = 0; k < RW; ++k) dsh_row[k] = 0.f;
      }
      const float mx = ONE_VIEW ? mx1 : P.means[3 * g + 0], my = ONE_VIEW ? my1 : P.means[3 * g + 1],
                  mz = ONE_VIEW ? mz1 : P.means[3 * g + 2];
      float dm0 = 0.f, dm1 = 0.f, dm2 = 0.f;
      bool any = false;
      for (int v = 0; v < (ONE_VIEW ? 1 : n_views); ++v) {
        const int64_t r = (int64_t)v * n + g;
        if ((ONE_VIEW ? rad1 : proj.radius[r]) <= 0) continue;
        any = true;
        const gs_camera_t &cam = cams[v];
        const float4 grgb = ONE_VIEW ? grgb1 : reinterpret_cast<const float4 *>(rg.d_rgb)[r];
        const uint8_t cl = ONE_VIEW ? cl1 : proj.clamped[r];
        const float g0c = (cl & 1) ? 0.f : grgb.x, g1c = (cl & 2) ? 0.f : grgb.y, g2c = (cl & 4) ? 0.f : grgb.z;
        float ccx, ccy, ccz;
        camera_centre(cam, ccx, ccy, ccz);
        const float ex = mx - ccx, ey = my - ccy, ez = mz - ccz;
        const float il = rsqrtf(ex * ex + ey * ey + ez * ez);
        const float dxn = ex * il, dyn = ey * il, dzn = ez * il;
        float gdx = 0.f, gdy = 0.f, gdz = 0.f;
        sh_visit<DEG>(dxn, dyn, dzn, [&](int k, float Y, float yx, float yy, float yz) {
          const float wk = g0c * sh[3 * k + 0] + g1c * sh[3 * k + 1] + g2c * sh[3 * k + 2];
          if (IN_PLACE) {
            dsh_row[3 * k + 0] = g0c * Y;
            dsh_row[3 * k + 1] = g1c * Y;
            dsh_row[3 * k + 2] = g2c * Y;
          } else {
            dsh_row[3 * k + 0] += g0c * Y;
            dsh_row[3 * k + 1] += g1c * Y;
            dsh_row[3 * k + 2] += g2c * Y;
          }
          gdx = fmaf(wk, yx, gdx);
          gdy = fmaf(wk, yy, gdy);
          gdz = fmaf(wk, yz, gdz);
        });
        // dir = (mu - centre) / |mu - centre|
        const float dd = gdx * dxn + gdy * dyn + gdz * dzn;
        dm0 += (gdx - dd * dxn) * il;
        dm1 += (gdy - dd * dyn) * il;
        dm2 += (gdz - dd * dzn) * il;
      }
      if (any) {
        out.d_means[3 * g + 0] += dm0;
        out.d_means[3 * g + 1] += dm1;
        out.d_means[3 * g + 2] += dm2;
      } else if (IN_PLACE) {
#pragma unroll
        for (int k = 0; k < RW; ++k) dsh_row[k] = 0.f;   // culled: zero gradient
      }
      if (!STAGED) {
        float *dsh = out.d_sh + (int64_t)g * P.sh_stride * 3;
#pragma unroll
        for (int k = 0; k < RW; ++k) dsh[k] = dsh_row[k];
        for (int k = K; k < P.sh_stride; ++k) dsh[3 * k + 0] = dsh[3 * k + 1] = dsh[3 * k + 2] = 0.f;
      }
    }
    if (STAGED) {
      __syncwarp();
      float *dst = out.d_sh + g0 * RW;
      const float *srow = IN_PLACE ? wsh : s_dsh + wib * 32 * RP;
      if (RW % 4 == 0 && vec) {
        for (int f4 = lane; f4 < rows * RW / 4; f4 += 32) {
          const float *q = srow + ((4 * f4) / RW) * RP + (4 * f4) % RW;
          reinterpret_cast<float4 *>(dst)[f4] = make_float4(q[0], q[1], q[2], q[3]);
        }
      } else {
        for (int f = lane; f < rows * RW; f += 32) dst[f] = srow[(f / RW) * RP + (f % RW)];
      }
      __syncwarp();
    }
  }
}

__global__ void densify_accum_kernel(const float *__restrict__ d_mean2d, const int32_t *__restrict__ radius,
                                     const gs_camera_t *__restrict__ cams, int n_views, int64_t n,
                                     float *accum, int32_t *count) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    float acc = accum[g];
    int cnt = count[g];
    for (int v = 0; v < n_views; ++v) {
      const int64_t r = (int64_t)v * n + g;
      if (radius[r] <= 0) continue;
      const float2 gm = reinterpret_cast<const float2 *>(d_mean2d)[r];
      const float gx = __fmul_rn(gm.x, 0.5f * (float)cams[v].width);
      const float gy = __fmul_rn(gm.y, 0.5f * (float)cams[v].height);
      acc = __fadd_rn(acc, __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy))));
      cnt += 1;
    }
    accum[g] = acc;
    count[g] = cnt;
  }
}

template <int DEG, bool STAGED>
static void launch_bwd_k(int grid, cudaStream_t s, const gs_params_t &P, const gs_frame_t *frame, const gs_proj_t &proj,
                         const gs_rec_grads_t &rg, const gs_param_grads_t &out, float *acc, int32_t *cnt) {
  if (frame->n_views == 1)
    project_bwd_geom_kernel<true><<<grid, 128, 0, s>>>(P, frame->cams_dev, 1, proj, rg, out, acc, cnt);
  else
    project_bwd_geom_kernel<false><<<grid, 128, 0, s>>>(P, frame->cams_dev, frame->n_views, proj, rg, out, acc, cnt);
  count_launch();
  // float4 staging needs both SH arrays on 16-byte boundaries (rows of 3K floats, K = 4 or 16)
  const bool vec = (reinterpret_cast<uintptr_t>(P.sh) & 15u) == 0 && (reinterpret_cast<uintptr_t>(out.d_sh) & 15u) == 0;
  if (frame->n_views == 1)
    project_bwd_sh_kernel<DEG, STAGED, true><<<grid, 128, 0, s>>>(P, frame->cams_dev, 1, proj, rg, out, vec);
  else
    project_bwd_sh_kernel<DEG, STAGED, false><<<grid, 128, 0, s>>>(P, frame->cams_dev, frame->n_views, proj, rg, out,
                                                                   vec);
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static bool params_ok(const gs_params_t *p) {
  return p && p->n >= 0 && p->means && p->log_scales && p->quats && p->opacity_logits && p->sh &&
         p->sh_degree >= 0 && p->sh_degree <= 3 && p->sh_stride >= (p->sh_degree + 1) * (p->sh_degree + 1) &&
         aligned16(p->quats);
}

static int grid_for(int64_t n, int threads) {
  const int64_t want = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * 32;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_project(const gs_params_t *params, const gs_frame_t *frame, gs_proj_t *out,
                                  gs_stream_t stream) {
  if (!params_ok(params) || !frame || !out || !frame->cams_dev || frame->n_views <= 0) return GS_ERR_INVALID_ARG;
  if (!out->mean2d || !out->conic_opacity || !out->rgb || !out->depth || !out->radius || !out->rect ||
      !out->clamped || !aligned16(out->conic_opacity) || !aligned16(out->rgb))
    return GS_ERR_INVALID_ARG;
  const int64_t R = (int64_t)frame->n_views * params->n;
  if (out->n_records < R) return GS_ERR_INVALID_ARG;
  if (R == 0) return GS_OK;
  const int grid = grid_for(R, 256);
  cudaStream_t s = as_stream(stream);
  const bool vec = params->sh_stride % 4 == 0 && aligned16(params->sh);
#define GS_PROJ_FWD(D)                                                                                        \
  (vec ? project_fwd_kernel<D, true><<<grid, 256, 0, s>>>(*params, frame->cams_dev, frame->n_views,           \
                                                          frame->tile_w, frame->tile_h, *out)                \
       : project_fwd_kernel<D, false><<<grid, 256, 0, s>>>(*params, frame->cams_dev, frame->n_views,          \
                                                           frame->tile_w, frame->tile_h, *out))
  switch (params->sh_degree) {
    case 0: GS_PROJ_FWD(0); break;
    case 1: GS_PROJ_FWD(1); break;
    case 2: GS_PROJ_FWD(2); break;
    default: GS_PROJ_FWD(3); break;
  }
#undef GS_PROJ_FWD
  GS_LAUNCH_CHECK();
  return GS_OK;
}

extern "C" gs_status_t gs_project_bwd(const gs_params_t *params, const gs_frame_t *frame, const gs_proj_t *proj,
                                      const gs_rec_grads_t *rg, gs_param_grads_t *out, float *densify_accum,
                                      int32_t *densify_count, gs_stream_t stream) {
  if (!params_ok(params) || !frame || !proj || !rg || !out || !frame->cams_dev || frame->n_views <= 0)
    return GS_ERR_INVALID_ARG;
  if (!rg->d_mean2d || !rg->d_conic_opacity || !rg->d_rgb || !out->d_means || !out->d_log_scales ||
      !out->d_quats || !out->d_opacity_logits || !out->d_sh || !aligned16(out->d_quats))
    return GS_ERR_INVALID_ARG;
  if ((densify_accum == nullptr) != (densify_count == nullptr)) return GS_ERR_INVALID_ARG;
  if (proj->n_records < (int64_t)frame->n_views * params->n) return GS_ERR_INVALID_ARG;
  if (params->n == 0) return GS_OK;
  const int grid = grid_for(params->n, 128);
  cudaStream_t s = as_stream(stream);
  const int K = (params->sh_degree + 1) * (params->sh_degree + 1);
  const bool staged = params->sh_stride == K;
  switch (params->sh_degree) {
    case 0: staged ? launch_bwd_k<0, true>(grid, s, *params, frame, *proj, *rg, *out, densify_accum, densify_count)
                  : launch_bwd_k<0, false>(grid, s, *params, frame, *proj, *rg, *out, densify_accum, densify_count); break;
    case 1: staged ? launch_bwd_k<1, true>(grid, s, *params, frame, *proj, *rg, *out, densify_accum, densify_count)
                  : launch_bwd_k<1, false>(grid, s, *params, frame, *proj, *rg, *out, densify_accum, densify_count); break;
    case 2: staged ? launch_bwd_k<2, true>(grid, s, *params, frame, *proj, *rg, *out, densify_accum, densify_count)
                  : launch_bwd_k<2, false>(grid, s, *params, frame, *proj, *rg, *out, densify_accum, densify_count); break;
    default: staged ? launch_bwd_k<3, true>(grid, s, *params, frame, *proj, *rg, *out, densify_accum, densify_count)
                  : launch_bwd_k<3, false>(grid, s, *params, frame, *proj, *rg, *out, densify_accum, densify_count); break;
  }
  GS_LAUNCH_CHECK();
  return GS_OK;
}

extern "C" gs_status_t gs_densify_accum(const float *d_mean2d, const int32_t *radius, const gs_frame_t *frame,
                                        int64_t n, float *accum, int32_t *count, gs_stream_t stream) {
  if (!d_mean2d || !radius || !frame || !frame->cams_dev || frame->n_views <= 0 || n < 0 || !accum || !count)
    return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  densify_accum_kernel<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(d_mean2d, radius, frame->cams_dev,
                                                                         frame->n_views, n, accum, count);
  GS_LAUNCH_CHECK();
  return GS_OK;
}
