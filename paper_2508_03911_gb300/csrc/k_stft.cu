// k_stft.cu -- short-time FFT along the frame axis and band moments (Sec. III-B.1).
//
// For every pixel p and window w (frames wS .. wS+T-1 of the time queue):
//   S_k(p) = sum_t U_{wS+t}(p) exp(-2 pi i k t / T),   P_k = |S_k|^2,
//   M0 = sum_{k=klo..khi} P_k,  M1 = sum f_k P_k,  M2 = sum f_k^2 P_k  (f_k in kHz),
//   M1N = M1 / M0 and M2N = sqrt(M2 / M0) in float64 (0 where M0 = 0).
//
// One CTA owns BT adjacent pixels and walks all windows of the launch, so
// overlapping windows (S < T) load each propagated frame from HBM once per
// launch: a window only brings in its S newest frames. The frame-to-time-axis
// transpose is that load: pixel-contiguous rows of the time queue land in a
// per-pixel ring in shared memory.
#include "fft_dev.cuh"
#include "hv_internal.h"
#include "../../include/hv.h"

namespace hv {

// ------------------------------------------------------------------------
// Kernel layout: 8 warps per CTA; each pixel's FFT is carried by LP lanes of one
// warp (LP = 32 for T >= 256, fewer for short windows, a warp then holding
// 32 / LP pixels). A pixel's samples sit in a shared ring of RS = T + min(S, T)
// slots, so the S frames that the next window adds are fetched with cp.async
// while the current window is transformed (S < T: frame o of the launch in slot
// o mod RS; S >= T: windows alternate between the two halves). The FFT is a
// Stockham pass sequence private to the warp (only __syncwarp between stages)
// through a padded work row, index i at i + i/16, which keeps the stage
// accesses of a pixel at two wavefronts. When the band lies below T/2 the last
// stage only forms the lower half of its outputs.

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ int wpad(int i) { return i + (i >> 4); }

struct MomAcc {
  uint32_t klo, khi;
  float fscale;
  float m0, m1, m2;
  template <int T>
  __device__ __forceinline__ void add(int k, float2 v) {
    if (uint32_t(k) - klo <= khi - klo) {
      const float P = fmaf(v.x, v.x, v.y * v.y);
      const float f = float(k < T / 2 ? k : k - T) * fscale;
      m0 += P;
      m1 = fmaf(f, P, m1);
      m2 = fmaf(f, f * P, m2);
    }
  }
};

// Lower half X_0 .. X_{R/2-1} of an R-point forward DFT.
template <int R>
__device__ __forceinline__ void dft_lower(float2* v) {
  if constexpr (R == 32) {
    float2 e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    dft<16, -1>(e);
    dft<16, -1>(o);
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = cadd(e[k], tw32<-1>(o[k], k));
  } else if constexpr (R == 16) {
    dft<16, -1>(v);
  } else if constexpr (R == 2) {
    v[0] = cadd(v[0], v[1]);
  } else if constexpr (R == 4) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = mul_i<-1>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[1] = cadd(t1, t3);
  } else {
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft<4, -1>(e);
    dft<4, -1>(o);
    const float c = 0.70710678118654752440f;
    v[0] = cadd(e[0], o[0]);
    v[1] = cadd(e[1], make_float2(c * (o[1].x + o[1].y), c * (o[1].y - o[1].x)));
    v[2] = cadd(e[2], mul_i<-1>(o[2]));
    v[3] = cadd(e[3], make_float2(c * (-o[3].x + o[3].y), c * (-o[3].y - o[3].x)));
  }
}

// Radix plan of the time FFT: two register-heavy stages where the length allows
// it (one exchange through shared memory), else radix 8, 4, 2.
template <int T>
struct WarpPlan {
  static constexpr int R1 = T == 1024 ? 32 : (T >= 128 ? 16 : RadixOf<T>::value);
  static constexpr int R2 = T == 128 ? 8 : (T == 256 ? 16 : (T >= 512 ? 32 : 0));
  static constexpr int RMAX = R1 > R2 ? R1 : R2;
  template <int NS>
  __host__ __device__ static constexpr int radix() {
    if constexpr (R2 != 0) return NS == 1 ? R1 : R2;
    else return RadixOf<T / NS>::value;
  }
};

// Lanes per pixel: every stage's butterflies spread evenly over LP lanes (at
// most 32); a warp then holds 32 / LP pixels.
template <int T>
struct WarpLayout {
  static constexpr int NBMIN = T / WarpPlan<T>::RMAX;
  static constexpr int LP = NBMIN < 32 ? NBMIN : 32;
  static constexpr int PW = 32 / LP;                                  // pixels per warp
  static constexpr int NW = PW >= 8 ? 1 : 8 / PW;                     // warps per CTA
  static constexpr int NT = 32 * NW;
  static constexpr int BT = NW * PW;                                  // pixels per CTA (>= 8)
  static constexpr int WLD = T + T / 16;                              // work row stride
};

// Stockham stages of one pixel's length-T forward FFT, carried by the LP lanes
// of its group (jl = lane within the group): stage 1 reads the ring, later
// stages the pixel's work row; the last stage feeds the moment accumulator.
template <int T, int NS, int LP>
__device__ __forceinline__ void warp_fft(const float2* ring, int rbase, int RS, float2* work,
                                         const float2* tw, int jl, MomAcc& acc, bool lower) {
  constexpr int R = WarpPlan<T>::template radix<NS>();
  constexpr int NB = T / R;
  static_assert(NB % LP == 0, "lanes per pixel must divide the butterflies");
  constexpr int IT = NB / LP;
  float2 v[IT][R];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = jl + LP * it;
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int t = j + m * NB;
      if constexpr (NS == 1) {
        int sl = rbase + t;
        if (sl >= RS) sl -= RS;
        v[it][m] = ring[sl];
      } else {
        v[it][m] = work[wpad(t)];
      }
    }
    if constexpr (NS > 1) {
      // stage table: entry (m, jm) at (NS - R1) + (m - 1) NS + jm, contiguous in jm
      constexpr int R1 = WarpPlan<T>::R1;
      const int jm = j % NS;
#pragma unroll
      for (int m = 1; m < R; ++m) v[it][m] = cmul(v[it][m], tw[(NS - R1) + (m - 1) * NS + jm]);
    }
  }
  if constexpr (NS * R == T) {
    if (lower) {
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        dft_lower<R>(v[it]);
#pragma unroll
        for (int m = 0; m < R / 2; ++m) acc.add<T>(jl + LP * it + m * NB, v[it][m]);
      }
    } else {
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        dft<R, -1>(v[it]);
#pragma unroll
        for (int m = 0; m < R; ++m) acc.add<T>(jl + LP * it + m * NB, v[it][m]);
      }
    }
  } else {
#pragma unroll
    for (int it = 0; it < IT; ++it) dft<R, -1>(v[it]);
    __syncwarp();
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int j = jl + LP * it;
      const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int m = 0; m < R; ++m) work[wpad(base + m * NS)] = v[it][m];
    }
    __syncwarp();
    warp_fft<T, NS * R, LP>(ring, rbase, RS, work, tw, jl, acc, lower);
  }
}

template <int T>
__host__ __device__ constexpr size_t warp_smem(uint32_t S) {
  using Lw = WarpLayout<T>;
  return (size_t(Lw::BT) * (T + (S < uint32_t(T) ? S : T) + 1) + T + size_t(Lw::BT) * Lw::WLD) *
         sizeof(float2);
}

template <int T>
__global__ void __launch_bounds__(WarpLayout<T>::NT, (T <= 512 ? 3 : 1)) k_stft_warp(StftArgs a) {
  using Lw = WarpLayout<T>;
  constexpr int BT = Lw::BT, NT = Lw::NT, LP = Lw::LP, PW = Lw::PW;
  extern __shared__ float2 smem[];
  const int S = int(a.S);
  const int RS = T + (S < T ? S : T);
  const int RLD = RS + 1;
  float2* ring = smem;
  float2* tw = ring + BT * RLD;
  float2* work = tw + T;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pl = lane / LP, jl = lane % LP;  // pixel within the warp, lane within the pixel
  const int px = warp * PW + pl;             // pixel within the CTA
  const size_t HW = size_t(a.W) * a.H;
  const uint32_t p0 = blockIdx.x * BT;
  const float2* tq = static_cast<const float2*>(a.tq.base);
  const bool lower = a.khi < uint32_t(T / 2);

  auto fetch = [&](int w) {  // issue the loads of window w's new frames
    int o0, n, s0;
    if (w == 0) {
      o0 = 0; n = T; s0 = 0;
    } else if (S < T) {
      o0 = w * S + T - S; n = S; s0 = o0 % RS;
    } else {
      o0 = w * S; n = T; s0 = (w & 1) * T;
    }
    for (int idx = tid; idx < n * BT; idx += NT) {
      const int b = idx % BT, f = idx / BT;
      int sl = s0 + f;
      if (sl >= RS) sl -= RS;
      const size_t g = (size_t(a.tq.slot0) + uint32_t(o0 + f)) % a.tq.cap;
      cp_async8(&ring[b * RLD + sl], &tq[g * HW + p0 + b]);
    }
    cp_async_commit();
  };

  // per-stage twiddle tables, laid out so that a warp's reads are contiguous:
  // stage of span NS and radix R keeps w_T^{jm m T/(NS R)} at (NS - R1) + (m-1) NS + jm
  {
    constexpr int R1 = WarpPlan<T>::R1;
    int NS = R1;
    while (NS < T) {
      const int rem = T / NS;
      const int R = WarpPlan<T>::R2 != 0 ? WarpPlan<T>::R2 : (rem % 8 == 0 ? 8 : (rem % 4 == 0 ? 4 : 2));
      for (int idx = tid; idx < (R - 1) * NS; idx += NT) {
        const int m = idx / NS + 1, jm = idx % NS;
        tw[(NS - R1) + idx] = a.tw_t[jm * m * (T / (NS * R))];
      }
      NS *= R;
    }
  }
  fetch(0);
  for (uint32_t w = 0; w < a.nwin; ++w) {
    cp_async_wait_all();
    __syncthreads();
    if (w + 1 < a.nwin) fetch(int(w) + 1);
    const int rbase = S < T ? int((size_t(w) * S) % RS) : int(w & 1) * T;
    MomAcc acc{a.klo, a.khi, a.fscale, 0.f, 0.f, 0.f};
    warp_fft<T, 1, LP>(ring + px * RLD, rbase, RS, work + px * Lw::WLD, tw, jl, acc, lower);
#pragma unroll
    for (int o = LP / 2; o > 0; o >>= 1) {  // reduce within the pixel's lane group
      acc.m0 += __shfl_xor_sync(0xffffffffu, acc.m0, o);
      acc.m1 += __shfl_xor_sync(0xffffffffu, acc.m1, o);
      acc.m2 += __shfl_xor_sync(0xffffffffu, acc.m2, o);
    }
    if (jl == 0) {
      float* o = a.out + size_t(w) * a.nout * HW + p0 + px;
      int q = 0;
      if (a.mask & HV_MOM_M0) o[HW * q++] = acc.m0;
      if (a.mask & HV_MOM_M1) o[HW * q++] = acc.m1;
      if (a.mask & HV_MOM_M2) o[HW * q++] = acc.m2;
      const double d0 = acc.m0;
      if (a.mask & HV_MOM_M1N) o[HW * q++] = d0 > 0.0 ? float(double(acc.m1) / d0) : 0.f;
      if (a.mask & HV_MOM_M2N) {
        const double r = d0 > 0.0 ? double(acc.m2) / d0 : 0.0;
        o[HW * q++] = float(sqrt(r > 0.0 ? r : 0.0));
      }
    }
  }
}

template <int T>
static cudaError_t launch_warp(const StftArgs& a, cudaStream_t s) {
  using Lw = WarpLayout<T>;
  const size_t hw = size_t(a.W) * a.H;
  if (hw % Lw::BT) return cudaErrorInvalidValue;
  const size_t smem = warp_smem<T>(a.S);
  cudaError_t e = cudaFuncSetAttribute(k_stft_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem));
  if (e != cudaSuccess) return e;
  k_stft_warp<T><<<unsigned(hw / Lw::BT), Lw::NT, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_stft(const StftArgs& a, cudaStream_t s, int* launches) {
  if (a.nwin == 0) return cudaSuccess;
  ++*launches;
  switch (a.T) {
    case 8: return launch_warp<8>(a, s);
    case 16: return launch_warp<16>(a, s);
    case 32: return launch_warp<32>(a, s);
    case 64: return launch_warp<64>(a, s);
    case 128: return launch_warp<128>(a, s);
    case 256: return launch_warp<256>(a, s);
    case 512: return launch_warp<512>(a, s);
    case 1024: return launch_warp<1024>(a, s);
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
