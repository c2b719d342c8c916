// k_autofocus.cu -- the parts of the learned autofocus that are not FFT passes:
// the Tamura coefficient from per-frame amplitude sums, and the network input
// (log-magnitude spectrum, 2 x 2 binned, standardised, bfloat16).
//
// The plain z-sweep the network replaces: for every distance z_j, the angular
// spectrum propagation of the mean-removed hologram (Sec. III-B.1's ASP with the
// DC bin of the transfer function set to zero) and the Tamura coefficient
// sqrt(sigma / mu) of the amplitude |U| over the frame.
#include <cuda_bf16.h>

#include "hv_internal.h"

namespace hv {

namespace {

// metric[i] = sqrt(sigma / mu) of frame-and-distance i from (sum |u|, sum |u|^2)
// over P pixels; 0 when mu = 0.
__global__ void k_tamura_finish(const double* acc, uint32_t count, double P, float* metric) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const double mu = acc[2 * i] / P;
    const double var = acc[2 * i + 1] / P - mu * mu;
    const double sigma = var > 0.0 ? sqrt(var) : 0.0;
    metric[i] = mu > 0.0 ? float(sqrt(sigma / mu)) : 0.f;
  }
}

constexpr int FT_NT = 512;

// Binned log-magnitude of cell (r, c): the centred spectrum's 2 x 2 block
// rows 2r, 2r+1 and columns 2c, 2c+1; centred row y is unshifted row
// (y + H/2) mod H. The DC bin counts as zero (the mean is removed).
__device__ __forceinline__ float cell_value(const float2* F, uint32_t W, uint32_t H, uint32_t r, uint32_t c) {
  float m = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const uint32_t y = (2 * r + a + H / 2) & (H - 1);
      const uint32_t x = (2 * c + b + W / 2) & (W - 1);
      const float2 v = F[size_t(y) * W + x];
      if (x | y) m += sqrtf(fmaf(v.x, v.x, v.y * v.y));
    }
  return log1pf(0.25f * m);
}

// One CTA per frame: mean and deviation of the cells in float64, then the
// standardised cells rounded to bfloat16 (nearest, ties to even).
__global__ void __launch_bounds__(FT_NT) k_af_features(const float2* spec, uint32_t W, uint32_t H,
                                                       __nv_bfloat16* out) {
  const uint32_t f = blockIdx.x;
  const float2* F = spec + size_t(f) * W * H;
  const uint32_t cw = W / 2, ncell = (W / 2) * (H / 2);
  // a thread's few cells summed in float32 (values below ~20), the block in float64
  float f1 = 0.f, f2 = 0.f;
  for (uint32_t e = threadIdx.x; e < ncell; e += FT_NT) {
    const float v = cell_value(F, W, H, e / cw, e % cw);
    f1 += v;
    f2 = fmaf(v, v, f2);
  }
  double s1 = f1, s2 = f2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  __shared__ double red[2][FT_NT / 32];
  __shared__ float stat[2];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s1;
    red[1][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < FT_NT / 32; ++w) {
      t1 += red[0][w];
      t2 += red[1][w];
    }
    const double mean = t1 / ncell;
    const double var = t2 / ncell - mean * mean;
    stat[0] = float(mean);
    stat[1] = var > 0.0 ? float(1.0 / sqrt(var)) : 0.f;
  }
  __syncthreads();
  const float mean = stat[0], inv = stat[1];
  __nv_bfloat16* o = out + size_t(f) * ncell;
  for (uint32_t e = threadIdx.x; e < ncell; e += FT_NT)
    o[e] = __float2bfloat16_rn((cell_value(F, W, H, e / cw, e % cw) - mean) * inv);
}

// The network input from precomputed cells, one CTA per frame: the frame's mean
// and deviation from its float64 sums (once), then (v - mean) / deviation rounded
// to bfloat16 (as k_af_features).
__global__ void __launch_bounds__(FT_NT) k_af_standardize(const float* cells, const double* sums, uint32_t stride,
                                                         uint32_t ncell, __nv_bfloat16* out) {
  const uint32_t f = blockIdx.x;
  __shared__ float stat[2];
  if (threadIdx.x == 0) {
    const double mean = sums[size_t(f) * stride] / ncell;
    const double var = sums[size_t(f) * stride + 1] / ncell - mean * mean;
    stat[0] = float(mean);
    stat[1] = var > 0.0 ? float(1.0 / sqrt(var)) : 0.f;
  }
  __syncthreads();
  const float m = stat[0], inv = stat[1];
  const float* c = cells + size_t(f) * ncell;
  __nv_bfloat16* o = out + size_t(f) * ncell;
  for (uint32_t e = threadIdx.x; e < ncell; e += FT_NT) o[e] = __float2bfloat16_rn((c[e] - m) * inv);
}

}  // namespace

cudaError_t launch_af_standardize(const float* cells, const double* sums, uint32_t sum_stride, uint32_t n,
                                  uint32_t ncell, void* out_bf16, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_af_standardize<<<n, FT_NT, 0, s>>>(cells, sums, sum_stride, ncell, static_cast<__nv_bfloat16*>(out_bf16));
  return cudaGetLastError();
}

cudaError_t launch_tamura_finish(const double* acc, uint32_t count, uint32_t pixels, float* metric, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const uint32_t blocks = (count + 255) / 256;
  k_tamura_finish<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(acc, count, double(pixels), metric);
  return cudaGetLastError();
}

cudaError_t launch_af_features(const float2* spec, uint32_t n, uint32_t W, uint32_t H, void* out_bf16,
                               cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_af_features<<<n, FT_NT, 0, s>>>(spec, W, H, static_cast<__nv_bfloat16*>(out_bf16));
  return cudaGetLastError();
}

}  // namespace hv
