// k_spatial.cu -- spatial demodulation of raw interferograms (Sec. III-B.1).
//
// Angular-spectrum propagation  U = IFFT2( FFT2(u) . H ),
//   H(kx, ky) = exp(i z sqrt(k^2 - kx^2 - ky^2)) (0 where evanescent),
// and the single-FFT Fresnel transform  U = FFT2( u . exp(i pi (x^2+y^2)/(lam z)) ),
// with fftshift folded into the input as the exact modulation (-1)^(x+y).
//
// A 2-D FFT is two batches of 1-D FFTs. Every pass below is one batched 1-D FFT
// along the frame's non-contiguous axis with the contiguous axis as the batch,
// so that loads and stores of 16 adjacent lines are coalesced; the transpose
// that a 2-D transform needs is done in shared memory on the way out.
//
//  P1  column FFT of the raw frame (conversion to complex and the Fresnel chirp
//      fused into the load), stored transposed  -> S1[x][ky]
//  P2a (ASP) row FFT of S1, multiply by H (1/(W H) folded in), row IFFT,
//      stored transposed back -> S2[ky][x]
//  P3a (ASP) column IFFT of S2 -> time queue [y][x]
//  P2f (Fresnel) row FFT of S1, stored transposed -> time queue [ky][kx]
#include "fft_dev.cuh"
#include "hv_internal.h"
#include "../../include/hv.h"

namespace hv {

constexpr int SP_BT = 16;  // lines per CTA in every spatial pass

template <int L>
struct SpCfg {
  static constexpr int BT = SP_BT;
  static constexpr int NT = FftThreads<L, BT>::value;
  static constexpr int LD = BT + 1;  // padded: transposed smem reads are conflict-free
  static constexpr size_t SMEM = size_t(L) * LD * sizeof(float2);
};

// P1: raw [H][W] -> column FFT (length L = H) -> S1[x][ky]
template <int L>
__global__ void __launch_bounds__(SpCfg<L>::NT) k_p1(SpatialArgs a) {
  using C = SpCfg<L>;
  extern __shared__ float2 smem[];
  const int tid = threadIdx.x;
  const uint32_t W = a.W;
  const uint32_t b0 = blockIdx.x * C::BT;
  const uint32_t i = blockIdx.y;
  const size_t rslot = (a.raw.slot0 + i) % a.raw.cap;
  const bool chirp = a.spatial == HV_SPATIAL_FRESNEL;
  for (int idx = tid; idx < L * C::BT; idx += C::NT) {
    const int b = idx % C::BT, y = idx / C::BT;
    const size_t off = rslot * size_t(W) * L + size_t(y) * W + b0 + b;
    float v = a.in_kind == IN_U8 ? float(static_cast<const uint8_t*>(a.raw.base)[off])
                                 : float(static_cast<const uint16_t*>(a.raw.base)[off]);
    float2 c = make_float2(v, 0.f);
    if (chirp) c = cscale(cmul(__ldg(&a.chirp_y[y]), __ldg(&a.chirp_x[b0 + b])), v);
    smem[y * C::LD + b] = c;
  }
  __syncthreads();
  StoreSmem<C::LD> epi{smem};
  fft_lines<L, -1, C::BT, C::NT, C::LD>(smem, a.tw_h, epi);
  __syncthreads();
  float2* s1 = a.scratch1 + size_t(i) * W * L;
  for (int idx = tid; idx < L * C::BT; idx += C::NT) {
    const int k = idx % L, b = idx / L;
    s1[size_t(b0 + b) * L + k] = smem[k * C::LD + b];
  }
}

// Multiply bin kx of line b by the transposed transfer function, then store.
template <int LD>
struct AspMulEpi {
  float2* buf;
  const float2* ht;  // [kx][ky]
  uint32_t H, b0;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const {
    buf[k * LD + b] = cmul(v, __ldg(&ht[size_t(k) * H + b0 + b]));
  }
};

// P2a: S1[x][ky] -> row FFT (L = W) -> x H -> row IFFT -> S2[ky][x]
template <int L>
__global__ void __launch_bounds__(SpCfg<L>::NT) k_p2_asp(SpatialArgs a) {
  using C = SpCfg<L>;
  extern __shared__ float2 smem[];
  const int tid = threadIdx.x;
  const uint32_t H = a.H;
  const uint32_t b0 = blockIdx.x * C::BT;
  const uint32_t i = blockIdx.y;
  const float2* s1 = a.scratch1 + size_t(i) * H * L;
  for (int idx = tid; idx < L * C::BT; idx += C::NT) {
    const int b = idx % C::BT, x = idx / C::BT;
    smem[x * C::LD + b] = s1[size_t(x) * H + b0 + b];
  }
  __syncthreads();
  AspMulEpi<C::LD> mul{smem, a.asp_ht, H, b0};
  fft_lines<L, -1, C::BT, C::NT, C::LD>(smem, a.tw_w, mul);
  __syncthreads();
  StoreSmem<C::LD> st{smem};
  fft_lines<L, +1, C::BT, C::NT, C::LD>(smem, a.tw_w, st);
  __syncthreads();
  float2* s2 = a.scratch2 + size_t(i) * H * L;
  for (int idx = tid; idx < L * C::BT; idx += C::NT) {
    const int x = idx % L, b = idx / L;
    s2[size_t(b0 + b) * L + x] = smem[x * C::LD + b];
  }
}

struct StoreGlobal {
  float2* out;
  uint32_t ld, b0;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const {
    out[size_t(k) * ld + b0 + b] = v;
  }
};

// P3a: S2[ky][x] -> column IFFT (L = H) -> time queue [y][x]
template <int L>
__global__ void __launch_bounds__(SpCfg<L>::NT) k_p3_asp(SpatialArgs a) {
  using C = SpCfg<L>;
  extern __shared__ float2 smem[];
  const int tid = threadIdx.x;
  const uint32_t W = a.W;
  const uint32_t b0 = blockIdx.x * C::BT;
  const uint32_t i = blockIdx.y;
  const float2* s2 = a.scratch2 + size_t(i) * W * L;
  for (int idx = tid; idx < L * C::BT; idx += C::NT) {
    const int b = idx % C::BT, y = idx / C::BT;
    smem[y * C::LD + b] = s2[size_t(y) * W + b0 + b];
  }
  __syncthreads();
  const size_t tslot = (a.tq.slot0 + i) % a.tq.cap;
  StoreGlobal st{static_cast<float2*>(a.tq.base) + tslot * size_t(W) * L, W, b0};
  fft_lines<L, +1, C::BT, C::NT, C::LD>(smem, a.tw_h, st);
}

// P2f: S1[x][ky] -> row FFT (L = W) -> time queue [ky][kx]
template <int L>
__global__ void __launch_bounds__(SpCfg<L>::NT) k_p2_fresnel(SpatialArgs a) {
  using C = SpCfg<L>;
  extern __shared__ float2 smem[];
  const int tid = threadIdx.x;
  const uint32_t H = a.H;
  const uint32_t b0 = blockIdx.x * C::BT;
  const uint32_t i = blockIdx.y;
  const float2* s1 = a.scratch1 + size_t(i) * H * L;
  for (int idx = tid; idx < L * C::BT; idx += C::NT) {
    const int b = idx % C::BT, x = idx / C::BT;
    smem[x * C::LD + b] = s1[size_t(x) * H + b0 + b];
  }
  __syncthreads();
  StoreSmem<C::LD> st{smem};
  fft_lines<L, -1, C::BT, C::NT, C::LD>(smem, a.tw_w, st);
  __syncthreads();
  const size_t tslot = (a.tq.slot0 + i) % a.tq.cap;
  float2* out = static_cast<float2*>(a.tq.base) + tslot * size_t(H) * L;
  for (int idx = tid; idx < L * C::BT; idx += C::NT) {
    const int k = idx % L, b = idx / L;
    out[size_t(b0 + b) * L + k] = smem[k * C::LD + b];
  }
}

// No spatial transform: conversion only.
__global__ void k_convert(SpatialArgs a) {
  const size_t hw = size_t(a.W) * a.H;
  const size_t total = hw * a.n;
  for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < total;
       e += size_t(gridDim.x) * blockDim.x) {
    const uint32_t i = uint32_t(e / hw);
    const size_t p = e % hw;
    const size_t roff = ((a.raw.slot0 + i) % a.raw.cap) * hw + p;
    const float v = a.in_kind == IN_U8 ? float(static_cast<const uint8_t*>(a.raw.base)[roff])
                                       : float(static_cast<const uint16_t*>(a.raw.base)[roff]);
    static_cast<float2*>(a.tq.base)[((a.tq.slot0 + i) % a.tq.cap) * hw + p] = make_float2(v, 0.f);
  }
}

template <class K>
static cudaError_t launch_pass(K kern, size_t smem, dim3 grid, int nt, const SpatialArgs& a,
                               cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  kern<<<grid, nt, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LH, int LW>
static cudaError_t spatial_fixed(const SpatialArgs& a, cudaStream_t s, int* launches) {
  cudaError_t e;
  const dim3 g1(a.W / SP_BT, a.n), g2(a.H / SP_BT, a.n);
  e = launch_pass(k_p1<LH>, SpCfg<LH>::SMEM, g1, SpCfg<LH>::NT, a, s);
  if (e != cudaSuccess) return e;
  ++*launches;
  if (a.spatial == HV_SPATIAL_ASP) {
    e = launch_pass(k_p2_asp<LW>, SpCfg<LW>::SMEM, g2, SpCfg<LW>::NT, a, s);
    if (e != cudaSuccess) return e;
    e = launch_pass(k_p3_asp<LH>, SpCfg<LH>::SMEM, g1, SpCfg<LH>::NT, a, s);
    *launches += 2;
  } else {
    e = launch_pass(k_p2_fresnel<LW>, SpCfg<LW>::SMEM, g2, SpCfg<LW>::NT, a, s);
    *launches += 1;
  }
  return e;
}

template <int LH>
static cudaError_t spatial_w(const SpatialArgs& a, cudaStream_t s, int* launches) {
  switch (a.W) {
    case 16: return spatial_fixed<LH, 16>(a, s, launches);
    case 32: return spatial_fixed<LH, 32>(a, s, launches);
    case 64: return spatial_fixed<LH, 64>(a, s, launches);
    case 128: return spatial_fixed<LH, 128>(a, s, launches);
    case 256: return spatial_fixed<LH, 256>(a, s, launches);
    case 512: return spatial_fixed<LH, 512>(a, s, launches);
    case 1024: return spatial_fixed<LH, 1024>(a, s, launches);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_spatial(const SpatialArgs& a, cudaStream_t s, int* launches) {
  if (a.n == 0) return cudaSuccess;
  if (a.spatial == HV_SPATIAL_NONE) {
    const size_t total = size_t(a.W) * a.H * a.n;
    const int nb = int((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
    k_convert<<<nb, 256, 0, s>>>(a);
    ++*launches;
    return cudaGetLastError();
  }
  if (a.use_fused && spatial_fused_supported(a)) return launch_spatial_fused(a, s, launches);
  if (a.use_cluster && spatial_cluster_supported(a)) return launch_spatial_cluster(a, s, launches);
  if (a.use_pp && spatial_pp_supported(a)) return launch_spatial_pp(a, s, launches);
  switch (a.H) {
    case 16: return spatial_w<16>(a, s, launches);
    case 32: return spatial_w<32>(a, s, launches);
    case 64: return spatial_w<64>(a, s, launches);
    case 128: return spatial_w<128>(a, s, launches);
    case 256: return spatial_w<256>(a, s, launches);
    case 512: return spatial_w<512>(a, s, launches);
    case 1024: return spatial_w<1024>(a, s, launches);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hv
