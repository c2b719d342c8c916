// k_post.cu -- post-processing of rendered images (Sec. III-B, "post processing and
// image accumulation"): periodic K x K convolution, re-normalisation by the mean,
// moving average over the last A images of each output.
//
// Rendered images of one call are [window][image][H][W]. Each image, after the
// convolution, goes to slot (count + window) mod R of a ring that keeps the last
// R images of every output (R >= A - 1 + windows per call), with its float64 sum
// beside it (kPostSub partial sums, added by the CTAs that write the slot); the
// moving average then reads the slots it needs, so every window of the call is
// averaged in parallel. Without a convolution the STFT epilogue writes the slots
// and their sums itself, and only the average runs here.
#include "hv_internal.h"

namespace hv {

namespace {

constexpr int PT = 16;  // output tile side of the convolution

// ring[slot][m][y][x] = sum_{a,b} k[a][b] img[(y + a - c) mod H][(x + b - c) mod W]
// for image m of window w (slot = (count + w) mod R); K = 0 copies. Re-normalising,
// the tile's sum goes into one of the slot image's partial sums.
__global__ void __launch_bounds__(PT* PT) k_post_conv(const float* __restrict__ img, PostArgs a) {
  extern __shared__ float sm[];
  const int K = a.K, c = K / 2, S = PT + (K > 0 ? K - 1 : 0);
  float* tile = sm;          // S x S
  float* kw = sm + S * S;    // K x K
  const uint32_t tiles_x = a.W / PT;
  const int ty0 = int(blockIdx.x / tiles_x) * PT, tx0 = int(blockIdx.x % tiles_x) * PT;
  const uint32_t im = blockIdx.y;  // w * nout + m
  const uint32_t w = im / a.nout, m = im % a.nout;
  const size_t hw = size_t(a.W) * a.H;
  const float* src = img + size_t(im) * hw;
  for (int e = threadIdx.x; e < K * K; e += PT * PT) kw[e] = a.kern[e];
  const int off = K > 0 ? c : 0;
  for (int e = threadIdx.x; e < S * S; e += PT * PT) {
    const int y = (ty0 + e / S - off) & int(a.H - 1), x = (tx0 + e % S - off) & int(a.W - 1);
    tile[e] = src[size_t(y) * a.W + x];
  }
  __syncthreads();
  const int ly = threadIdx.x / PT, lx = threadIdx.x % PT;
  float v;
  if (K > 0) {
    v = 0.f;
    for (int p = 0; p < K; ++p)
      for (int q = 0; q < K; ++q) v = fmaf(kw[p * K + q], tile[(ly + p) * S + lx + q], v);
  } else {
    v = tile[ly * S + lx];
  }
  const uint32_t slot = uint32_t((a.count + w) % a.R);
  a.ring[(size_t(slot) * a.nout + m) * hw + size_t(ty0 + ly) * a.W + tx0 + lx] = v;
  if (a.renorm) {
    double t = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    __shared__ double red[PT * PT / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double u = 0.0;
      for (int i = 0; i < PT * PT / 32; ++i) u += red[i];
      atomicAdd(&a.sums[(size_t(slot) * a.nout + m) * kPostSub + blockIdx.x % kPostSub], u);
    }
  }
}

// out[w][m][p] = mean over the last min(A, count + w + 1) slots of image m,
// each divided by its mean when re-normalising.
__global__ void __launch_bounds__(256) k_post_avg(float* __restrict__ out, PostArgs a) {
  __shared__ double scale[64];  // hw / sum of each slot read (A <= 64)
  const uint32_t im = blockIdx.y, w = im / a.nout, m = im % a.nout;
  const size_t hw = size_t(a.W) * a.H;
  const uint64_t newest = a.count + w;
  const uint32_t n = uint32_t(newest + 1 < a.A ? newest + 1 : a.A);
  if (a.renorm) {
    for (uint32_t j = threadIdx.x >> 5; j < n; j += blockDim.x >> 5) {
      const uint32_t slot = uint32_t((newest - j) % a.R);
      double t = a.sums[(size_t(slot) * a.nout + m) * kPostSub + (threadIdx.x & 31)];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if ((threadIdx.x & 31) == 0) scale[j] = t != 0.0 ? double(hw) / t : 0.0;
    }
    __syncthreads();
  }
  for (size_t p = blockIdx.x * size_t(blockDim.x) + threadIdx.x; p < hw; p += size_t(gridDim.x) * blockDim.x) {
    float acc = 0.f;
    for (uint32_t j = 0; j < n; ++j) {
      const uint32_t slot = uint32_t((newest - j) % a.R);
      float v = a.ring[(size_t(slot) * a.nout + m) * hw + p];
      if (a.renorm) v = float(double(v) * scale[j]);
      acc += v;
    }
    out[size_t(im) * hw + p] = acc / float(n);
  }
}

}  // namespace

cudaError_t launch_post_zero(const PostArgs& a, uint32_t nwin, cudaStream_t s) {
  if (!a.renorm || nwin == 0) return cudaSuccess;
  // the slots (count + w) mod R of the call, w < nwin <= R: one run, or two across the wrap
  const size_t per_slot = size_t(a.nout) * kPostSub * sizeof(double);
  const uint32_t first = uint32_t(a.count % a.R);
  const uint32_t run = nwin < a.R - first ? nwin : a.R - first;
  cudaError_t e = cudaMemsetAsync(a.sums + size_t(first) * a.nout * kPostSub, 0, run * per_slot, s);
  if (e == cudaSuccess && run < nwin) e = cudaMemsetAsync(a.sums, 0, (nwin - run) * per_slot, s);
  return e;
}

cudaError_t launch_post(float* images, uint32_t nwin, const PostArgs& a, cudaStream_t s, int* launches) {
  if (nwin == 0) return cudaSuccess;
  if (nwin > a.R || a.A > 64) return cudaErrorInvalidValue;
  const uint32_t nimg = nwin * a.nout;
  cudaError_t e;
  if (!a.fused) {
    e = launch_post_zero(a, nwin, s);
    if (e != cudaSuccess) return e;
    const int S = PT + (a.K > 0 ? a.K - 1 : 0);
    const size_t smem = (size_t(S) * S + size_t(a.K) * a.K) * sizeof(float);
    k_post_conv<<<dim3((a.W / PT) * (a.H / PT), nimg), PT * PT, smem, s>>>(images, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *launches += 1;
  }
  const size_t hw = size_t(a.W) * a.H;
  const unsigned gx = unsigned((hw + 255) / 256 < 64 ? (hw + 255) / 256 : 64);
  k_post_avg<<<dim3(gx, nimg), 256, 0, s>>>(images, a);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace hv
