// Energy of training images across resolutions, for the coarse-to-fine schedule
// (Sec. "Energy-aware multi-resolution"): the anti-aliased bilinear downscale
// D_r and the L1 norm of the 2D Fourier magnitude, ||E(I)||_1.
//
// D_r: separable triangle filter whose support widens with the scale s = W / W_r
// (W_r = floor(W/r + 1/2)); output column j samples the input at c = (j + 1/2) s - 1/2
// with weights max(0, 1 - |k - c| / s) over the input columns k inside the image,
// normalised to sum 1; rows likewise.
//
// ||E(I)||_1: a 2D DFT of each channel as two 1D DFT passes -- rows (real input,
// every row in one block, twiddles from a shared table indexed by n k mod W, the
// index advanced incrementally) and columns (complex input, the magnitude of each
// coefficient summed in FP64 per block and added once per block). Images are a
// few megapixels and the schedule is computed once per scene, so direct O(N^2) DFTs
// per row and column suffice; no FFT library is used.
#include <algorithm>

#include "gs_common.cuh"

namespace gs {

constexpr int kEnergyMaxDim = 4096;
constexpr int kEnergyThreads = 256;

__device__ __forceinline__ void aa_taps(int j, int n_in, int n_out, float &c, float &s, int &k0, int &k1,
                                        float &norm) {
  s = (float)n_in / (float)n_out;
  c = ((float)j + 0.5f) * s - 0.5f;
  k0 = max(0, (int)ceilf(c - s));
  k1 = min(n_in - 1, (int)floorf(c + s));
  float sum = 0.f;
  for (int k = k0; k <= k1; ++k) sum += fmaxf(0.f, 1.f - fabsf((float)k - c) / s);
  norm = 1.f / sum;
}

__global__ void downscale_kernel(const float *__restrict__ img, int C, int H, int W, float *__restrict__ out,
                                 int Hr, int Wr) {
  const int64_t total = (int64_t)Hr * Wr;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(p / Wr), x = (int)(p - (int64_t)y * Wr);
    float cx, sx, nx, cy, sy, ny;
    int x0, x1, y0, y1;
    aa_taps(x, W, Wr, cx, sx, x0, x1, nx);
    aa_taps(y, H, Hr, cy, sy, y0, y1, ny);
    for (int ch = 0; ch < C; ++ch) {
      const float *src = img + (int64_t)ch * H * W;
      float acc = 0.f;
      for (int ky = y0; ky <= y1; ++ky) {
        const float wy = fmaxf(0.f, 1.f - fabsf((float)ky - cy) / sy);
        float row = 0.f;
        for (int kx = x0; kx <= x1; ++kx) row = fmaf(fmaxf(0.f, 1.f - fabsf((float)kx - cx) / sx), src[(int64_t)ky * W + kx], row);
        acc = fmaf(wy, row, acc);
      }
      out[(int64_t)ch * Hr * Wr + p] = acc * nx * ny;
    }
  }
}

// tw[q] = exp(-2 pi i q / N), q in [0, N)
__device__ __forceinline__ void fill_twiddles(float2 *tw, int N) {
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)q / (double)N, &sn, &cs);
    tw[q] = make_float2((float)cs, (float)-sn);
  }
}

// One block per (channel, row): X[ch][h][k] = sum_n I[ch][h][n] exp(-2 pi i n k / W).
__global__ void __launch_bounds__(kEnergyThreads) dft_rows_kernel(const float *__restrict__ img, int W,
                                                                  float2 *__restrict__ X) {
  extern __shared__ float4 s_raw[];
  float2 *tw = reinterpret_cast<float2 *>(s_raw);
  float *row = reinterpret_cast<float *>(tw + W);
  const int64_t base = (int64_t)blockIdx.x * W;
  fill_twiddles(tw, W);
  for (int n = threadIdx.x; n < W; n += blockDim.x) row[n] = img[base + n];
  __syncthreads();
  for (int k = threadIdx.x; k < W; k += blockDim.x) {
    float re = 0.f, im = 0.f;
    int q = 0;
    for (int n = 0; n < W; ++n) {
      const float2 t = tw[q];
      re = fmaf(row[n], t.x, re);
      im = fmaf(row[n], t.y, im);
      q += k;
      if (q >= W) q -= W;
    }
    X[base + k] = make_float2(re, im);
  }
}

// One block per (channel, column k): Y[m] = sum_h X[h][k] exp(-2 pi i h m / H);
// the block adds sum_m |Y[m]| to *sum.
__global__ void __launch_bounds__(kEnergyThreads) dft_cols_l1_kernel(const float2 *__restrict__ X, int H, int W,
                                                                     double *sum) {
  extern __shared__ float4 s_raw[];
  float2 *tw = reinterpret_cast<float2 *>(s_raw);
  float2 *col = tw + H;
  __shared__ double s_part[kEnergyThreads / 32];
  const int ch = blockIdx.x / W, k = blockIdx.x - ch * W;
  const float2 *src = X + (int64_t)ch * H * W + k;
  fill_twiddles(tw, H);
  for (int h = threadIdx.x; h < H; h += blockDim.x) col[h] = src[(int64_t)h * W];
  __syncthreads();
  double part = 0.0;
  for (int m = threadIdx.x; m < H; m += blockDim.x) {
    float re = 0.f, im = 0.f;
    int q = 0;
    for (int h = 0; h < H; ++h) {
      const float2 t = tw[q], x = col[h];
      re = fmaf(x.x, t.x, fmaf(-x.y, t.y, re));
      im = fmaf(x.x, t.y, fmaf(x.y, t.x, im));
      q += m;
      if (q >= H) q -= H;
    }
    part += sqrt((double)re * re + (double)im * im);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kEnergyThreads / 32; ++w) b += s_part[w];
    atomicAdd(sum, b);
  }
}

static bool dims_ok(int C, int H, int W) {
  return C > 0 && H > 0 && W > 0 && H <= kEnergyMaxDim && W <= kEnergyMaxDim;
}

}  // namespace gs

using namespace gs;

extern "C" int32_t gs_downscaled_size(int32_t n, int32_t r) {
  if (n <= 0 || r < 1) return 0;
  const int64_t m = (2 * (int64_t)n + r) / (2 * (int64_t)r);   // floor(n / r + 1/2)
  return (int32_t)(m > 0 ? m : 1);
}

extern "C" gs_status_t gs_downscale(const float *image, int32_t C, int32_t H, int32_t W, int32_t r, float *out,
                                    gs_stream_t stream) {
  if (!image || !out || C <= 0 || H <= 0 || W <= 0 || r < 1) return GS_ERR_INVALID_ARG;
  const int Hr = gs_downscaled_size(H, r), Wr = gs_downscaled_size(W, r);
  const int64_t total = (int64_t)Hr * Wr;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16);
  downscale_kernel<<<grid, 256, 0, as_stream(stream)>>>(image, C, H, W, out, Hr, Wr);
  GS_LAUNCH_CHECK();
  return GS_OK;
}

extern "C" size_t gs_spectrum_workspace_size(int32_t C, int32_t H, int32_t W) {
  if (!dims_ok(C, H, W)) return 0;
  return sizeof(float2) * (size_t)C * H * W;
}

extern "C" gs_status_t gs_spectrum_l1(const float *image, int32_t C, int32_t H, int32_t W, double *d_sum, void *ws,
                                      size_t ws_bytes, gs_stream_t stream) {
  if (!image || !d_sum || !ws || !dims_ok(C, H, W)) return GS_ERR_INVALID_ARG;
  if (ws_bytes < gs_spectrum_workspace_size(C, H, W) || (reinterpret_cast<uintptr_t>(ws) & 15u) != 0)
    return GS_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  float2 *X = static_cast<float2 *>(ws);
  const size_t smem_rows = (size_t)W * (sizeof(float2) + sizeof(float));
  const size_t smem_cols = (size_t)H * 2 * sizeof(float2);
  GS_CUDA_TRY(cudaFuncSetAttribute(dft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows));
  GS_CUDA_TRY(cudaFuncSetAttribute(dft_cols_l1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols));
  GS_CUDA_TRY(cudaMemsetAsync(d_sum, 0, sizeof(double), s));
  dft_rows_kernel<<<C * H, kEnergyThreads, smem_rows, s>>>(image, W, X);
  GS_LAUNCH_CHECK();
  dft_cols_l1_kernel<<<C * W, kEnergyThreads, smem_cols, s>>>(X, H, W, d_sum);
  GS_LAUNCH_CHECK();
  return GS_OK;
}
