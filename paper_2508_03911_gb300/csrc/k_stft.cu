// k_stft.cu -- short-time FFT along the frame axis and band moments (Sec. III-B.1).
//
// For every pixel p and window w (frames wS .. wS+T-1 of the time queue):
//   S_k(p) = sum_t U_{wS+t}(p) exp(-2 pi i k t / T),   P_k = |S_k|^2,
//   M0 = sum_{k=klo..khi} P_k,  M1 = sum f_k P_k,  M2 = sum f_k^2 P_k  (f_k in kHz),
//   M1N = M1 / M0 and M2N = sqrt(M2 / M0) in float64 (0 where M0 = 0).
//
// One CTA owns BT adjacent pixels and walks all windows of the launch. Their
// samples sit in a shared-memory ring of T slots (frame o of the launch in slot
// o mod T), so overlapping windows (S < T) load each propagated frame from HBM
// once per launch: a window only brings in its S newest frames. The ring holds
// the window circularly rotated; a rotation multiplies S_k by a unit phase and
// leaves P_k, hence every moment, unchanged, so the FFT reads the ring as is.
// The frame-to-time-axis transpose is this load: pixel-contiguous rows of the
// time queue land batch-fastest in shared memory.
#include "fft_dev.cuh"
#include "hv_internal.h"
#include "../../include/hv.h"

namespace hv {

template <int T>
struct StftCfg {
  static constexpr int BT = T <= 8 ? 32 : (T <= 256 ? 16 : 8);
  static constexpr int NT = FftThreads<T, BT>::value;
  static constexpr size_t SMEM = 2 * size_t(T) * BT * sizeof(float2) + 3 * NT * sizeof(float);
};

template <int T>
struct MomentEpi {
  uint32_t klo, khi;
  float fscale;
  float m0 = 0.f, m1 = 0.f, m2 = 0.f;
  __device__ __forceinline__ void operator()(int, int k, float2 v) {
    if (uint32_t(k) >= klo && uint32_t(k) <= khi) {
      const float P = fmaf(v.x, v.x, v.y * v.y);
      const float f = float(k < T / 2 ? k : k - T) * fscale;
      m0 += P;
      m1 = fmaf(f, P, m1);
      m2 = fmaf(f, f * P, m2);
    }
  }
};

template <int T>
__global__ void __launch_bounds__(StftCfg<T>::NT) k_stft(StftArgs a) {
  using C = StftCfg<T>;
  constexpr int BT = C::BT, NT = C::NT;
  extern __shared__ float2 smem[];
  float2* ring = smem;
  float2* work = smem + T * BT;
  float* red = reinterpret_cast<float*>(work + T * BT);
  const int tid = threadIdx.x;
  const size_t HW = size_t(a.W) * a.H;
  const uint32_t p0 = blockIdx.x * BT;
  const float2* tq = static_cast<const float2*>(a.tq.base);

  for (uint32_t w = 0; w < a.nwin; ++w) {
    const uint32_t lo = w * a.S;
    const uint32_t new_lo = (w == 0 || a.S >= uint32_t(T)) ? lo : lo + T - a.S;
    const uint32_t nnew = lo + T - new_lo;
    for (uint32_t idx = tid; idx < nnew * BT; idx += NT) {
      const uint32_t b = idx % BT, o = new_lo + idx / BT;
      const size_t slot = (size_t(a.tq.slot0) + o) % a.tq.cap;
      ring[(o & (T - 1)) * BT + b] = tq[slot * HW + p0 + b];
    }
    __syncthreads();
    MomentEpi<T> epi{a.klo, a.khi, a.fscale};
    fft_stages<T, 1, -1, BT, NT, BT>(ring, BT, work, a.tw_t, epi);
    red[tid] = epi.m0;
    red[NT + tid] = epi.m1;
    red[2 * NT + tid] = epi.m2;
    __syncthreads();
    if (tid < BT) {
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      for (int t = tid; t < NT; t += BT) {
        s0 += red[t];
        s1 += red[NT + t];
        s2 += red[2 * NT + t];
      }
      float* o = a.out + size_t(w) * a.nout * HW + p0 + tid;
      int q = 0;
      if (a.mask & HV_MOM_M0) o[HW * q++] = s0;
      if (a.mask & HV_MOM_M1) o[HW * q++] = s1;
      if (a.mask & HV_MOM_M2) o[HW * q++] = s2;
      const double d0 = s0;
      if (a.mask & HV_MOM_M1N) o[HW * q++] = d0 > 0.0 ? float(double(s1) / d0) : 0.f;
      if (a.mask & HV_MOM_M2N) {
        const double r = d0 > 0.0 ? double(s2) / d0 : 0.0;
        o[HW * q++] = float(sqrt(r > 0.0 ? r : 0.0));
      }
    }
    __syncthreads();
  }
}

template <int T>
static cudaError_t launch_t(const StftArgs& a, cudaStream_t s) {
  using C = StftCfg<T>;
  const size_t hw = size_t(a.W) * a.H;
  if (hw % C::BT) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_stft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(C::SMEM));
  if (e != cudaSuccess) return e;
  k_stft<T><<<unsigned(hw / C::BT), C::NT, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_stft(const StftArgs& a, cudaStream_t s, int* launches) {
  if (a.nwin == 0) return cudaSuccess;
  ++*launches;
  switch (a.T) {
    case 8: return launch_t<8>(a, s);
    case 16: return launch_t<16>(a, s);
    case 32: return launch_t<32>(a, s);
    case 64: return launch_t<64>(a, s);
    case 128: return launch_t<128>(a, s);
    case 256: return launch_t<256>(a, s);
    case 512: return launch_t<512>(a, s);
    case 1024: return launch_t<1024>(a, s);
  }
  return cudaErrorInvalidValue;
}

__global__ void k_copy_frames(RingRef tq, uint32_t n, size_t hw, float2* out) {
  const size_t total = hw * n;
  for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < total;
       e += size_t(gridDim.x) * blockDim.x) {
    const size_t i = e / hw, p = e % hw;
    out[e] = static_cast<const float2*>(tq.base)[((tq.slot0 + i) % tq.cap) * hw + p];
  }
}

cudaError_t launch_copy_frames(const RingRef& tq, uint32_t n, uint32_t hw, float* out,
                               cudaStream_t s, int* launches) {
  if (n == 0) return cudaSuccess;
  const size_t total = size_t(hw) * n;
  const int nb = int((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
  k_copy_frames<<<nb, 256, 0, s>>>(tq, n, hw, reinterpret_cast<float2*>(out));
  ++*launches;
  return cudaGetLastError();
}

}  // namespace hv
