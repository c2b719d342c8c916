// k_cnn.cu -- the autofocus network's training and inference kernels.
//
// Network (input 1 x 128 x 128, the binned log-spectrum of a hologram):
//   four 3 x 3 convolutions, stride 2, zero padding 1, channels 1 -> 16 -> 32 ->
//   64 -> 64, each followed by ReLU (outputs 64^2, 32^2, 16^2, 8^2); global average
//   pool; dense 64 -> 32 with ReLU; dense 32 -> 1. The output predicts the
//   normalised distance (z - 0.35) / 0.25; the loss is the batch mean of the
//   squared error.
// Arithmetic: activations and convolution weights in bfloat16, every product
// accumulated in float32 (the forward of layers 2-4 on the tensor cores, in
// k_conv_tc.cu; layer 1 and the backward pass here on the CUDA cores); the dense layers, gradients and the Adam state in
// float32. Layouts: activations [n][c][h][w]; the flat float32 parameter vector
// holds w1 [16][1][3][3], b1, w2 [32][16][3][3], b2, w3, b3, w4, b4, f1w [32][64],
// f1b, f2w [1][32], f2b; a bfloat16 mirror of it feeds the convolutions.
#include <cuda_bf16.h>

#include "cnn_internal.h"

namespace hv {
namespace cnn {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// ------------------------------------------------------------------ forward
//
// y[n][o][i][j] = relu(b[o] + sum_{c,di,dj} w[o][c][di][dj] x[n][c][2i+di-1][2j+dj-1]).
// A CTA covers image n, NR output rows and all CO channels; a thread owns 4
// channels (4 cg .. 4 cg + 3) x 4 neighbouring pixels of one row. Input rows
// and weights are staged in shared memory CK channels at a time.
template <int CI, int CO, int HI>
__global__ void __launch_bounds__(NT) k_conv_fwd(const __nv_bfloat16* __restrict__ x,
                                                 const __nv_bfloat16* __restrict__ w,
                                                 const float* __restrict__ bias, __nv_bfloat16* __restrict__ y) {
  constexpr int WI = HI, HO = HI / 2, WO = HO;
  constexpr int CG = CO / 4, PG = NT / CG, TPX = 4 * PG;
  constexpr int NR = TPX / WO;
  static_assert(TPX % WO == 0 && NR <= HO && HO % NR == 0, "tile");
  constexpr int CK = CI < 8 ? CI : 8;
  constexpr int SR = 2 * NR + 1, SC = WI + 2;
  __shared__ float xs[CK][SR][SC];
  __shared__ __align__(16) float ws[CK][9][CO];
  constexpr int TILES = HO / NR;
  const int n = blockIdx.x / TILES, r0 = (blockIdx.x % TILES) * NR;
  const int tid = threadIdx.x, cg = tid % CG, pg = tid / CG;
  const int p0 = pg * 4, il = p0 / WO, j0 = p0 % WO;
  float acc[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[k][q] = 0.f;
  for (int c0 = 0; c0 < CI; c0 += CK) {
    __syncthreads();
    for (int e = tid; e < CK * SR * SC; e += NT) {
      const int c = e / (SR * SC), rr = (e / SC) % SR, cc = e % SC;
      const int yy = 2 * r0 - 1 + rr, xx = cc - 1;
      float v = 0.f;
      if (yy >= 0 && yy < HI && xx >= 0 && xx < WI) v = bf(x[((size_t(n) * CI + c0 + c) * HI + yy) * WI + xx]);
      xs[c][rr][cc] = v;
    }
    for (int e = tid; e < CK * 9 * CO; e += NT) {
      const int o = e % CO, t = (e / CO) % 9, c = e / (9 * CO);
      ws[c][t][o] = bf(w[(size_t(o) * CI + c0 + c) * 9 + t]);
    }
    __syncthreads();
#pragma unroll 2
    for (int c = 0; c < CK; ++c)
#pragma unroll
      for (int di = 0; di < 3; ++di)
#pragma unroll
        for (int dj = 0; dj < 3; ++dj) {
          const float4 wv = *reinterpret_cast<const float4*>(&ws[c][di * 3 + dj][4 * cg]);
          float xv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) xv[q] = xs[c][2 * il + di][2 * (j0 + q) + dj];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            acc[0][q] = fmaf(wv.x, xv[q], acc[0][q]);
            acc[1][q] = fmaf(wv.y, xv[q], acc[1][q]);
            acc[2][q] = fmaf(wv.z, xv[q], acc[2][q]);
            acc[3][q] = fmaf(wv.w, xv[q], acc[3][q]);
          }
        }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int o = 4 * cg + k;
    const float b = bias[o];
    __align__(8) __nv_bfloat16 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = __float2bfloat16_rn(fmaxf(acc[k][q] + b, 0.f));
    *reinterpret_cast<uint2*>(y + ((size_t(n) * CO + o) * HO + r0 + il) * WO + j0) = *reinterpret_cast<uint2*>(v);
  }
}

// ------------------------------------------------------------ input gradient
//
// dX[n][c][y][x] = sum_{o,di,dj: y = 2i+di-1, x = 2j+dj-1} w[o][c][di][dj] dZ[n][o][i][j],
// times the ReLU mask of the layer input (its stored activation > 0): the
// result is the previous layer's dZ. For even y only di = 1 (i = y/2) reaches
// y; for odd y, di = 0 (i = (y+1)/2) and di = 2 (i = (y-1)/2); columns alike.
// A CTA covers image n, NRI = 4 input rows, all CI channels; a thread owns 4
// channels x 4 pixels x = 2(b0+q) + px of one row, and the pixels of a warp
// share (y mod 2, x mod 2), so the taps a warp visits are uniform.
template <int CI, int CO, int HI>
__global__ void __launch_bounds__(NT) k_conv_dx(const float* __restrict__ dz, const __nv_bfloat16* __restrict__ w,
                                                const __nv_bfloat16* __restrict__ aprev, float* __restrict__ dprev) {
  constexpr int WI = HI, HO = HI / 2, WO = HO;
  constexpr int NRI = 4, CG = CI / 4;
  static_assert(CG * NRI * (WI / 4) == NT, "one thread per 4 channels x 4 pixels");
  static_assert((CI * WI) % 512 == 0, "warp-uniform parity classes");
  constexpr int CK = 8;
  constexpr int SRZ = NRI / 2 + 2, SCZ = WO + 1;
  __shared__ float zs[CK][SRZ][SCZ];
  __shared__ __align__(16) float ws[CK][9][CI];
  constexpr int TILES = HI / NRI;
  const int n = blockIdx.x / TILES, y0 = (blockIdx.x % TILES) * NRI;
  const int tid = threadIdx.x, cg = tid % CG, g = tid / CG;
  constexpr int GPC = (NRI / 2) * (WI / 8);  // pixel groups per parity class
  const int cls = g / GPC, rem = g % GPC;
  const int py = cls >> 1, px = cls & 1;
  const int r = rem / (WI / 8), b0 = 4 * (rem % (WI / 8));
  const int yy = y0 + py + 2 * r;
  const int ibase = y0 / 2 - 1;  // staged dZ row 0
  float acc[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[k][q] = 0.f;
  for (int o0 = 0; o0 < CO; o0 += CK) {
    __syncthreads();
    for (int e = tid; e < CK * SRZ * SCZ; e += NT) {
      const int o = e / (SRZ * SCZ), rr = (e / SCZ) % SRZ, cc = e % SCZ;
      const int i = ibase + rr;
      float v = 0.f;
      if (i >= 0 && i < HO && cc < WO) v = dz[((size_t(n) * CO + o0 + o) * HO + i) * WO + cc];
      zs[o][rr][cc] = v;
    }
    for (int e = tid; e < CK * 9 * CI; e += NT) {
      const int c = e % CI, t = (e / CI) % 9, o = e / (9 * CI);
      ws[o][t][c] = bf(w[(size_t(o0 + o) * CI + c) * 9 + t]);
    }
    __syncthreads();
    // taps of this class: (di, staged dZ row) and (dj, column offset from b)
    const int ndi = py ? 2 : 1, ndj = px ? 2 : 1;
#pragma unroll 2
    for (int o = 0; o < CK; ++o)
      for (int a = 0; a < ndi; ++a) {
        const int di = py ? 2 * a : 1;              // odd y: di = 0 or 2
        const int zr = py ? (a == 0 ? r + 2 : r + 1) : r + 1;
        for (int bq = 0; bq < ndj; ++bq) {
          const int dj = px ? 2 * bq : 1;
          const int jo = px ? (bq == 0 ? 1 : 0) : 0;  // j = b + jo
          const float4 wv = *reinterpret_cast<const float4*>(&ws[o][di * 3 + dj][4 * cg]);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float d = zs[o][zr][b0 + q + jo];
            acc[0][q] = fmaf(wv.x, d, acc[0][q]);
            acc[1][q] = fmaf(wv.y, d, acc[1][q]);
            acc[2][q] = fmaf(wv.z, d, acc[2][q]);
            acc[3][q] = fmaf(wv.w, d, acc[3][q]);
          }
        }
      }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const size_t row = ((size_t(n) * CI + 4 * cg + k) * HI + yy) * WI;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int xx = 2 * (b0 + q) + px;
      dprev[row + xx] = bf(aprev[row + xx]) > 0.f ? acc[k][q] : 0.f;
    }
  }
}

// ----------------------------------------------------------- weight gradient
//
// dW[o][c][t] = sum over pixels (n, i, j) of dZ[n][o][i][j] x[n][c][2i+di-1][2j+dj-1]
// (t = 3 di + dj, k = 9 c + t), db[o] = sum dZ. A CTA covers all CO channels,
// KT groups of 4 k and one chunk of the pixels; a thread owns 4 o x 4 k.
// Partial sums go to part[chunk][o][k] and partb[chunk][o] (reduced later in a
// fixed order, so the result does not depend on scheduling).
template <int CI, int CO, int HI>
struct DwCfg {
  static constexpr int K = 9 * CI, KG = (K + 3) / 4, CG = CO / 4;
  static constexpr int KT = KG < NT / CG ? KG : NT / CG;
  static constexpr int KTILES = (KG + KT - 1) / KT;
  static constexpr int THREADS = CG * KT;
  static constexpr int TP = 32;
};

template <int CI, int CO, int HI>
__global__ void __launch_bounds__(DwCfg<CI, CO, HI>::THREADS) k_conv_dw(const float* __restrict__ dz,
                                                                         const __nv_bfloat16* __restrict__ x,
                                                                         uint32_t npix, uint32_t chunk,
                                                                         float* __restrict__ part,
                                                                         float* __restrict__ partb) {
  using D = DwCfg<CI, CO, HI>;
  constexpr int WI = HI, HO = HI / 2, WO = HO, K = D::K, KT = D::KT, CG = D::CG, TP = D::TP;
  __shared__ __align__(16) float zs[TP][CO];
  __shared__ __align__(16) float xs[TP][4 * KT];
  const int tid = threadIdx.x, cg = tid % CG, kg = tid / CG;
  const int k0 = blockIdx.x * KT * 4;  // first k of this CTA
  const uint32_t pbeg = blockIdx.y * chunk;
  const uint32_t pend = pbeg + chunk < npix ? pbeg + chunk : npix;
  float acc[4][4], accb[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    accb[a] = 0.f;
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  }
  for (uint32_t p0 = pbeg; p0 < pend; p0 += TP) {
    __syncthreads();
    for (int e = tid; e < TP * CO; e += D::THREADS) {
      const int pl = e / CO, o = e % CO;
      const uint32_t p = p0 + pl;
      float v = 0.f;
      if (p < pend) {
        const uint32_t n = p / (HO * WO), ij = p % (HO * WO);
        v = dz[(size_t(n) * CO + o) * HO * WO + ij];
      }
      zs[pl][o] = v;
    }
    for (int e = tid; e < TP * 4 * KT; e += D::THREADS) {
      const int pl = e / (4 * KT), kl = e % (4 * KT);
      const int k = k0 + kl;
      const uint32_t p = p0 + pl;
      float v = 0.f;
      if (p < pend && k < K) {
        const uint32_t n = p / (HO * WO), ij = p % (HO * WO);
        const int i = ij / WO, j = ij % WO, c = k / 9, t = k % 9;
        const int yy = 2 * i + t / 3 - 1, xx = 2 * j + t % 3 - 1;
        if (yy >= 0 && yy < HI && xx >= 0 && xx < WI) v = bf(x[((size_t(n) * CI + c) * HI + yy) * WI + xx]);
      }
      xs[pl][kl] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int pl = 0; pl < TP; ++pl) {
      const float4 zv = *reinterpret_cast<const float4*>(&zs[pl][4 * cg]);
      const float4 xv = *reinterpret_cast<const float4*>(&xs[pl][4 * kg]);
      const float zz[4] = {zv.x, zv.y, zv.z, zv.w}, xx[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        accb[a] += zz[a];
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(zz[a], xx[b], acc[a][b]);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int o = 4 * cg + a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int k = k0 + 4 * kg + b;
      if (k < K) part[(size_t(blockIdx.y) * CO + o) * K + k] = acc[a][b];
    }
    if (blockIdx.x == 0 && kg == 0) partb[size_t(blockIdx.y) * CO + o] = accb[a];
  }
}

// grad[off + e] = sum over chunks of part[chunk][e] (e < count), in chunk order.
__global__ void k_sum_chunks(const float* __restrict__ part, uint32_t count, uint32_t nchunks, float* __restrict__ out) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (uint32_t c = 0; c < nchunks; ++c) s += part[size_t(c) * count + e];
    out[e] = s;
  }
}

// --------------------------------------------------------------------- head
//
// One CTA of 64 threads per image: pool, dense layers, output. With training,
// also the loss term, the gradient of the pooled features and dZ4 (times the
// ReLU mask of a4). Scratch per image: g[64], h[32], dh[32], dy, err.
constexpr int HS = 64 + 32 + 32 + 2;

__global__ void __launch_bounds__(64) k_head(const __nv_bfloat16* __restrict__ a4, const float* __restrict__ prm,
                                            const float* __restrict__ ztarget, uint32_t n, float* __restrict__ zout,
                                            float* __restrict__ scratch, float* __restrict__ dz4) {
  const int t = blockIdx.x, c = threadIdx.x;
  __shared__ float g[64], h[32], dh[32], s_dy;
  const __nv_bfloat16* src = a4 + (size_t(t) * 64 + c) * 64;
  float s = 0.f;
  for (int e = 0; e < 64; ++e) s += bf(src[e]);
  g[c] = s * (1.f / 64.f);
  __syncthreads();
  const float* f1w = prm + OFF_F1W;
  const float* f1b = prm + OFF_F1B;
  const float* f2w = prm + OFF_F2W;
  if (c < 32) {
    float v = f1b[c];
    for (int k = 0; k < 64; ++k) v = fmaf(f1w[c * 64 + k], g[k], v);
    h[c] = fmaxf(v, 0.f);
  }
  __syncthreads();
  if (c == 0) {
    float v = prm[OFF_F2B];
    for (int k = 0; k < 32; ++k) v = fmaf(f2w[k], h[k], v);
    if (zout) zout[t] = 0.35f + 0.25f * v;
    if (ztarget) {
      const float err = v - (ztarget[t] - 0.35f) * 4.0f;  // (z - 0.35) / 0.25
      s_dy = 2.f * err / float(n);
      scratch[size_t(t) * HS + 128] = s_dy;
      scratch[size_t(t) * HS + 129] = err;
    }
  }
  if (!ztarget) return;
  __syncthreads();
  if (c < 32) dh[c] = h[c] > 0.f ? s_dy * f2w[c] : 0.f;
  __syncthreads();
  float dg = 0.f;
  for (int k = 0; k < 32; ++k) dg = fmaf(dh[k], f1w[k * 64 + c], dg);
  dg *= 1.f / 64.f;
  float* d = dz4 + (size_t(t) * 64 + c) * 64;
  for (int e = 0; e < 64; ++e) d[e] = bf(src[e]) > 0.f ? dg : 0.f;
  float* sc = scratch + size_t(t) * HS;
  sc[c] = g[c];
  if (c < 32) {
    sc[64 + c] = h[c];
    sc[96 + c] = dh[c];
  }
}

// Dense-layer gradients summed over the batch in image order, and the loss.
__global__ void k_head_grads(const float* __restrict__ scratch, uint32_t n, float* __restrict__ grad,
                             float* __restrict__ loss) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  float s = 0.f;
  if (e < 2048) {  // f1w[k][c] = sum dh[k] g[c]
    const int k = e / 64, c = e % 64;
    for (uint32_t t = 0; t < n; ++t) s = fmaf(scratch[t * HS + 96 + k], scratch[t * HS + c], s);
    grad[OFF_F1W + e] = s;
  } else if (e < 2080) {  // f1b[k] = sum dh[k]
    for (uint32_t t = 0; t < n; ++t) s += scratch[t * HS + 96 + (e - 2048)];
    grad[OFF_F1B + e - 2048] = s;
  } else if (e < 2112) {  // f2w[k] = sum dy h[k]
    for (uint32_t t = 0; t < n; ++t) s = fmaf(scratch[t * HS + 128], scratch[t * HS + 64 + (e - 2080)], s);
    grad[OFF_F2W + e - 2080] = s;
  } else if (e == 2112) {  // f2b = sum dy
    for (uint32_t t = 0; t < n; ++t) s += scratch[t * HS + 128];
    grad[OFF_F2B] = s;
  } else if (e == 2113 && loss) {
    for (uint32_t t = 0; t < n; ++t) s = fmaf(scratch[t * HS + 129], scratch[t * HS + 129], s);
    *loss = s / float(n);
  }
}

// ---------------------------------------------------------------------- Adam

__global__ void k_adam(float* __restrict__ prm, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ prm_bf, uint32_t count, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * g);
    const float vi = fmaf(b2, v[i], (1.f - b2) * g * g);
    m[i] = mi;
    v[i] = vi;
    const float p = prm[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    prm[i] = p;
    prm_bf[i] = __float2bfloat16_rn(p);
  }
}

__global__ void k_to_bf16(const float* __restrict__ prm, __nv_bfloat16* __restrict__ out, uint32_t count) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(prm[i]);
}

// ------------------------------------------------------------------ launchers

template <int CI, int CO, int HI>
cudaError_t conv_fwd(const Net& t, const __nv_bfloat16* x, int off_w, int off_b, __nv_bfloat16* y, uint32_t n,
                     cudaStream_t s) {
  constexpr int WO = HI / 2, CG = CO / 4, TPX = 4 * (NT / CG), NR = TPX / WO;
  k_conv_fwd<CI, CO, HI><<<n * (HI / 2 / NR), NT, 0, s>>>(x, t.prm_bf + off_w, t.prm + off_b, y);
  return cudaGetLastError();
}

template <int CI, int CO, int HI>
cudaError_t conv_bwd(const Net& t, const float* dz, const __nv_bfloat16* x, int off_w, int off_b, float* dprev,
                     uint32_t n, cudaStream_t s) {
  using D = DwCfg<CI, CO, HI>;
  const uint32_t npix = n * (HI / 2) * (HI / 2);
  uint32_t nchunks = t.dw_chunks;
  uint32_t chunk = (npix + nchunks - 1) / nchunks;
  chunk = (chunk + D::TP - 1) / D::TP * D::TP;
  nchunks = (npix + chunk - 1) / chunk;
  k_conv_dw<CI, CO, HI><<<dim3(D::KTILES, nchunks), D::THREADS, 0, s>>>(dz, x, npix, chunk, t.part, t.partb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint32_t cw = CO * D::K;
  k_sum_chunks<<<(cw + 255) / 256, 256, 0, s>>>(t.part, cw, nchunks, t.grad + off_w);
  k_sum_chunks<<<1, CO, 0, s>>>(t.partb, CO, nchunks, t.grad + off_b);
  if (dprev) {
    if constexpr (CI >= 16) {
      k_conv_dx<CI, CO, HI><<<n * (HI / 4), NT, 0, s>>>(dz, t.prm_bf + off_w, x, dprev);
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t net_forward(const Net& t, const void* x, uint32_t n, const float* ztarget, float* zout, cudaStream_t s) {
  const auto* xi = static_cast<const __nv_bfloat16*>(x);
  cudaError_t e = conv_fwd<1, 16, 128>(t, xi, OFF_W1, OFF_B1, t.a1, n, s);
  // layers 2-4 (K = 144, 288, 576): implicit GEMMs on the tensor cores
  if (e == cudaSuccess) e = conv_tc<16, 32, 64>(t.a1, t.prm_bf + OFF_W2, t.prm + OFF_B2, t.a2, n, t.err, s);
  if (e == cudaSuccess) e = conv_tc<32, 64, 32>(t.a2, t.prm_bf + OFF_W3, t.prm + OFF_B3, t.a3, n, t.err, s);
  if (e == cudaSuccess) e = conv_tc<64, 64, 16>(t.a3, t.prm_bf + OFF_W4, t.prm + OFF_B4, t.a4, n, t.err, s);
  if (e != cudaSuccess) return e;
  k_head<<<n, 64, 0, s>>>(t.a4, t.prm, ztarget, n, zout, t.head, t.dbuf0);
  return cudaGetLastError();
}

cudaError_t net_backward(const Net& t, const void* x, uint32_t n, float* loss, cudaStream_t s) {
  // dZ4 is in dbuf0 (from the head); dZ3 -> dbuf1, dZ2 -> dbuf0, dZ1 -> dbuf1
  k_head_grads<<<(2114 + 255) / 256, 256, 0, s>>>(t.head, n, t.grad, loss);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = conv_bwd<64, 64, 16>(t, t.dbuf0, t.a3, OFF_W4, OFF_B4, t.dbuf1, n, s);
  if (e == cudaSuccess) e = conv_bwd<32, 64, 32>(t, t.dbuf1, t.a2, OFF_W3, OFF_B3, t.dbuf0, n, s);
  if (e == cudaSuccess) e = conv_bwd<16, 32, 64>(t, t.dbuf0, t.a1, OFF_W2, OFF_B2, t.dbuf1, n, s);
  if (e == cudaSuccess)
    e = conv_bwd<1, 16, 128>(t, t.dbuf1, static_cast<const __nv_bfloat16*>(x), OFF_W1, OFF_B1, nullptr, n, s);
  return e;
}

cudaError_t net_adam(const Net& t, float lr, float b1, float b2, float eps, float c1, float c2, cudaStream_t s) {
  k_adam<<<(NPARAMS + 255) / 256, 256, 0, s>>>(t.prm, t.grad, t.m, t.v, t.prm_bf, NPARAMS, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t net_sync_bf16(const Net& t, cudaStream_t s) {
  k_to_bf16<<<(NPARAMS + 255) / 256, 256, 0, s>>>(t.prm, t.prm_bf, NPARAMS);
  return cudaGetLastError();
}

size_t dw_part_floats(uint32_t nchunks) { return size_t(nchunks) * 64 * 9 * 64; }

}  // namespace cnn
}  // namespace hv
