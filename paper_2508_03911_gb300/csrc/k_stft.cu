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
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <type_traits>

#include "fft_dev.cuh"
#include "hv_internal.h"
#include "../../include/hv.h"

namespace hv {

// ------------------------------------------------------------------------
// Kernel layout: 8 pixels per CTA; each pixel's FFT is carried by LP lanes of one
// warp (LP = 32 for T >= 256, fewer for short windows, a warp then holding
// PW = 32 / LP pixels). A warp runs on its own: it fetches its pixels' frames,
// transforms them and writes their moments with only __syncwarp between steps,
// so the warps of a CTA never wait on one another inside the window loop.
//
// Ring of a pixel in shared memory:
//  - overlapping windows (S < T): slots [0, T) hold the current window, frame o
//    of the launch at slot o mod T; the S frames the next window adds are staged
//    while the current window is transformed, and at the start of a window move
//    into the slots of the S frames that left. The FFT reads slots 0 .. T-1 in
//    order: a circular shift of the window, which leaves every |S_k|^2
//    unchanged, so the loads need no wrap-around. Staging:
//      TMA path: one cp.async.bulk.tensor load per window brings the CTA's S x BT
//      block (64-byte rows, 64-byte swizzle) into a staging tile, completing on
//      an mbarrier; the last warp to move a window's frames out issues the next
//      load. Each warp then reads only its own pixels' 16-byte column of the
//      tile, conflict-free thanks to the swizzle.
//      Fallback (S not dividing the queue, T < 64, S > 256): every warp stages
//      its own pixels with 8-byte cp.async into slots [T, T + S) of its rows.
//  - S >= T: windows alternate between the halves [0, T) and [T, 2T), filled by
//    CTA-wide cp.async (whole 64-byte frame segments per warp instruction) with
//    one CTA barrier per window.
// The FFT is a Stockham pass sequence through a padded work row (index i at
// i + i/16, two wavefronts per stage access of a pixel). When the band lies
// below T/2 the last stage only forms the lower half of its outputs.

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// all but the newest N committed groups complete
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ int wpad(int i) { return i + (i >> 4); }

// Band moments of one lane in units of bins. Its bins are k = kb + m NB (kb =
// jl + LP it for its butterflies it); the signed frequency index of bin k is
// kb + NB m' with m' = m below T/2 and m - R above. Per butterfly the lane sums
// P, m' P and m'^2 P over its in-band m (constant weights), and folds them into
// sum k' P and sum k'^2 P once.
struct MomAcc {
  uint32_t band;     // bit it R + m set: bin (it, m) of the last stage lies in [klo, khi]
  float m0, m1, m2;  // sum P, sum k' P, sum k'^2 P
};

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
  // radix of the last stage
  __host__ __device__ static constexpr int last() {
    if (R2 != 0) return R2;
    int ns = 1, r = 2;
    while (ns < T) {
      const int rem = T / ns;
      r = rem % 8 == 0 ? 8 : (rem % 4 == 0 ? 4 : 2);
      ns *= r;
    }
    return r;
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
  static constexpr int RL = WarpPlan<T>::last();                      // last-stage radix
  static constexpr int ITL = T / RL / LP;                             // last-stage butterflies per lane
  static_assert(ITL * RL <= 32, "band bits of a lane");
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
    // X_k = E_k + w32^k O_k with the twiddle product fused into the sum
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k == 0) {
        v[0] = cadd(e[0], o[0]);
      } else if (k == 8) {
        v[8] = cadd(e[8], mul_i<-1>(o[8]));
      } else {
        const float2 w = tw32<-1>(make_float2(1.f, 0.f), k);  // constants after unrolling
        v[k] = make_float2(fmaf(o[k].x, w.x, fmaf(-o[k].y, w.y, e[k].x)),
                           fmaf(o[k].x, w.y, fmaf(o[k].y, w.x, e[k].y)));
      }
    }
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

// Moment sums of butterfly it of the last stage (outputs m < MO in registers).
template <int R, int NB, int MO>
__device__ __forceinline__ void add_moments(const float2* v, int it, float kb, MomAcc& acc) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int m = 0; m < MO; ++m) {
    if (acc.band & (1u << (it * R + m))) {
      const float P = fmaf(v[m].x, v[m].x, v[m].y * v[m].y);
      const float mm = float(m < R / 2 ? m : m - R);
      s0 += P;
      if (m != 0) {
        s1 = fmaf(mm, P, s1);
        s2 = fmaf(mm * mm, P, s2);
      }
    }
  }
  // k' = kb + NB m': sum k' P = kb s0 + NB s1, sum k'^2 P = kb^2 s0 + 2 kb NB s1 + NB^2 s2
  acc.m0 += s0;
  acc.m1 = fmaf(kb, s0, fmaf(float(NB), s1, acc.m1));
  acc.m2 = fmaf(kb * kb, s0, fmaf(2.f * float(NB) * kb, s1, fmaf(float(NB * NB), s2, acc.m2)));
}

// Stockham stages of one pixel's length-T forward FFT, carried by the LP lanes
// of its group (jl = lane within the group): stage 1 reads the window (T
// samples from `win`, in order), later stages the pixel's work row; the last
// stage feeds the moment sums.
template <int T, int NS, int LP, bool WP = false>
__device__ __forceinline__ void warp_fft(const float2* win, float2* work, const float2* tw, int jl,
                                         MomAcc& acc, bool lower) {
  // WP: the window itself is stored padded (sample t at t + t / 16)
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
      if constexpr (NS == 1) v[it][m] = WP ? win[wpad(t)] : win[t];
      else v[it][m] = work[wpad(t)];
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
    const float kb0 = float(jl);
    if (lower) {
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        dft_lower<R>(v[it]);
        add_moments<R, NB, R / 2>(v[it], it, kb0 + float(LP * it), acc);
      }
    } else {
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        dft<R, -1>(v[it]);
        add_moments<R, NB, R>(v[it], it, kb0 + float(LP * it), acc);
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
    warp_fft<T, NS * R, LP, WP>(win, work, tw, jl, acc, lower);
  }
}

// Shared memory of the kernel (bytes): [1 KB alignment slack, staging tile]
// (TMA path), ring rows, work rows, twiddles.
template <int T>
struct WarpSmem {
  using Lw = WarpLayout<T>;
  static constexpr int WLD = T + T / 16;           // work row stride (wpad, bank skew between pixels)
  static constexpr int NTW = T - WarpPlan<T>::R1;   // twiddle entries of stages 2 ..
  __host__ __device__ static constexpr int rld(uint32_t S, bool tma) {
    return S >= uint32_t(T) ? 2 * T + 4 : (tma ? T : T + int(S) + 1);  // bank skew between pixels
  }
  __host__ __device__ static constexpr size_t staging(uint32_t S, bool tma) {
    return tma ? 1024 + size_t(S) * Lw::BT * 8 : 0;
  }
  __host__ __device__ static constexpr size_t bytes(uint32_t S, bool tma) {
    return staging(S, tma) + (size_t(Lw::BT) * rld(S, tma) + size_t(Lw::BT) * WLD + NTW) * sizeof(float2);
  }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// 2-D tiled TMA load (x innermost) completing on an mbarrier
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}
// Bounded wait (about 2^32 clocks) for phase `parity` of an mbarrier to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 32)) return false;
  }
}

// Post-processing fused into the moment epilogue: the moments of pixel `pix` for
// window w, from the lane group's reduced sums (held by its lane jl = 0, the
// writer) -- M0, M1, M2 (bins -> kHz), then M1N and M2N in float64, in that order
// among those the mask asks for -- to the image ring slot of the window (or to
// out [w][image][pixel] without a ring), adding each image's sum over the warp's
// pixels into one of the slot's partial sums. Called by every lane of the warp
// (the sums are reduced across it). The kernels take it in an instantiation of
// their own (POST) and keep their plain epilogue otherwise: routing renders
// without post-processing through this one measured 16 % slower for the walking
// kernel, and even an untaken branch to it 4 %.
__device__ __forceinline__ void emit_moments(const StftArgs& a, uint32_t w, size_t pix, const MomAcc& acc,
                                             bool writer, bool streaming) {
  const size_t HW = size_t(a.W) * a.H;
  float v[5];
  v[0] = acc.m0;
  v[1] = acc.m1 * a.fscale;
  v[2] = acc.m2 * (a.fscale * a.fscale);
  const double d0 = acc.m0;
  v[3] = 0.f;
  v[4] = 0.f;
  if (a.mask & HV_MOM_M1N) v[3] = d0 > 0.0 ? float(double(v[1]) / d0) : 0.f;
  if (a.mask & HV_MOM_M2N) {
    const double r = d0 > 0.0 ? double(v[2]) / d0 : 0.0;
    v[4] = float(sqrt(r > 0.0 ? r : 0.0));
  }
  uint32_t slot = 0;
  float* o;
  if (a.post_ring) {
    slot = uint32_t((a.post_count + w) % a.post_R);
    o = a.post_ring + size_t(slot) * a.nout * HW + pix;
  } else {
    o = a.out + size_t(w) * a.nout * HW + pix;
  }
  const uint32_t sub = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % kPostSub;
  int q = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if (!(a.mask & (1u << k))) continue;
    if (writer) {
      if (streaming) __stcs(&o[HW * q], v[k]);
      else o[HW * q] = v[k];
    }
    if (a.post_sums) {
      float t = writer ? v[k] : 0.f;
#pragma unroll
      for (int x = 16; x > 0; x >>= 1) t += __shfl_xor_sync(0xffffffffu, t, x);
      if ((threadIdx.x & 31) == 0)
        atomicAdd(&a.post_sums[(size_t(slot) * a.nout + q) * kPostSub + sub], double(t));
    }
    ++q;
  }
}

template <int T, bool POST>
__global__ void __launch_bounds__(WarpLayout<T>::NT, (T <= 512 ? 3 : 1))
    k_stft_warp(StftArgs a, const __grid_constant__ CUtensorMap qmap) {
  using Lw = WarpLayout<T>;
  using Sm = WarpSmem<T>;
  constexpr int NT = Lw::NT, LP = Lw::LP, PW = Lw::PW, NW = Lw::NW, BT = Lw::BT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long s_full;  // the staged frames of the next window landed
  __shared__ unsigned s_done;                         // warps that moved a window's staged frames out
  const uint32_t S = a.S;
  const bool overlap = S < uint32_t(T);
  const bool tma = a.tma != 0;  // only with overlap and BT = 8 (64-byte tile rows)
  const int RLD = Sm::rld(S, tma);
  const uint32_t align_pad = (1024u - (smem_addr(smem_raw) & 1023u)) & 1023u;
  unsigned char* staging = smem_raw + align_pad;  // 1024-byte aligned (swizzle atoms)
  float2* ring = reinterpret_cast<float2*>(smem_raw + Sm::staging(S, tma));
  float2* work = ring + BT * RLD;
  float2* tw = work + BT * Sm::WLD;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pl = lane / LP, jl = lane % LP;  // pixel within the warp, lane within the pixel
  const int px = warp * PW + pl;             // pixel within the CTA
  const size_t HW = size_t(a.W) * a.H;
  const uint32_t p0 = blockIdx.x * BT;
  const float2* tq = static_cast<const float2*>(a.tq.base);
  const uint32_t cap = a.tq.cap;
  const bool lower = a.khi < uint32_t(T / 2);
  const uint32_t mbar = smem_addr(&s_full);
  // the warp's pixels and its lanes' share of their frames: pixel fb, frames ff + k 32/PW
  float2* wring = ring + warp * PW * RLD;
  const int fb = lane % PW, ff = lane / PW;
  const float2* src = tq + p0 + warp * PW + fb;

  // queue slot of frame o of the launch (o < cap: the launch's frames fit the queue)
  auto slot_of = [&](uint32_t o) {
    const uint32_t g = a.tq.slot0 + o;
    return g >= cap ? g - cap : g;
  };
  // cp.async of n frames starting at frame o0 into slots s0 + f of the warp's pixels
  auto fetch_warp = [&](uint32_t o0, int n, int s0) {
    uint32_t g = slot_of(o0 + uint32_t(ff));
    for (int f = ff; f < n; f += 32 / PW) {
      cp_async8(&wring[fb * RLD + s0 + f], &src[size_t(g) * HW]);
      g += 32 / PW;
      if (g >= cap) g -= cap;
    }
    cp_async_commit();
  };
  // CTA-wide cp.async of n frames from frame o0 into slots s0 + f of all BT
  // pixels: a warp instruction covers 32 / BT whole frames of the CTA (full
  // sectors); the row stride 2T + 4 keeps those stores at two wavefronts
  auto fetch_cta = [&](uint32_t o0, int n, int s0) {
    constexpr int FS = NT / BT;  // frames per pass of the CTA
    const int b = tid % BT;
    int f = tid / BT;
    uint32_t g = slot_of(o0 + uint32_t(f));
    for (; f < n; f += FS) {
      cp_async8(&ring[b * RLD + s0 + f], &tq[size_t(g) * HW + p0 + b]);
      g += FS;
      if (g >= cap) g -= cap;
    }
    cp_async_commit();
  };
  // one thread: the CTA's S x BT block from frame o0 into the staging tile
  // (S consecutive queue slots; the host guarantees they do not wrap)
  auto fetch_tile = [&](uint32_t o0) {
    mbar_arrive_tx(mbar, S * uint32_t(BT * 8));
    tma_load_2d(smem_addr(staging), &qmap, int(p0), int(slot_of(o0)), mbar);
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
  // in-band bits of the lane's last-stage bins
  uint32_t band = 0;
  {
    constexpr int RL = Lw::RL, NBL = T / RL;
#pragma unroll
    for (int it = 0; it < Lw::ITL; ++it)
#pragma unroll
      for (int m = 0; m < RL; ++m) {
        const uint32_t k = uint32_t(jl + LP * it + m * NBL);
        if (k - a.klo <= a.khi - a.klo) band |= 1u << (it * RL + m);
      }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_done = 0;
  }
  __syncthreads();  // twiddles, mbarrier
  if (overlap) fetch_warp(0, T, 0);
  else fetch_cta(0, T, 0);
  if (overlap && a.nwin > 1) {  // window 1's new frames
    if (!tma) fetch_warp(uint32_t(T), int(S), T);
    else if (tid == 0) fetch_tile(uint32_t(T));
  }
  for (uint32_t w = 0; w < a.nwin; ++w) {
    const float2* win;
    if (overlap) {
      const uint32_t d = (w - 1) * S;  // ring slot of the first frame that left (w > 0)
      if (!tma) {
        cp_async_wait_all();
        __syncwarp();
        if (w > 0) {
          for (int f = ff; f < int(S); f += 32 / PW)
            wring[fb * RLD + int((d + uint32_t(f)) & uint32_t(T - 1))] = wring[fb * RLD + T + f];
          __syncwarp();
          if (w + 1 < a.nwin) fetch_warp((w + 1) * S + uint32_t(T) - S, int(S), T);
        }
      } else if (w == 0) {
        cp_async_wait_all();
        __syncwarp();
      } else {
        if (!mbar_wait(mbar, (w - 1) & 1)) {
          if (lane == 0) atomicOr(a.err, 2u);
          return;
        }
        // pixel q of tile row f: 16-byte chunk q / 2 of the 64-byte row is stored at
        // chunk (q / 2) ^ ((f >> 1) & 3) (64-byte swizzle), q % 2 selects its half
        for (uint32_t e = lane; e < S * PW; e += 32) {
          const uint32_t b = e % PW, f = e / PW, q = uint32_t(warp * PW) + b;
          const float2 v = *reinterpret_cast<const float2*>(staging + f * 64u + 16u * ((q >> 1) ^ ((f >> 1) & 3u)) +
                                                            8u * (q & 1u));
          wring[int(b) * RLD + int((d + f) & uint32_t(T - 1))] = v;
        }
        __syncwarp();
        // the last warp to finish issues the next window's load into the tile
        unsigned prev = 0;
        if (lane == 0) {
          __threadfence_block();
          prev = atomicAdd(&s_done, 1u);
          __threadfence_block();
          if (prev % NW == NW - 1 && w + 1 < a.nwin) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            fetch_tile((w + 1) * S + uint32_t(T) - S);
          }
        }
      }
      win = ring + px * RLD;
    } else {
      // every warp is done with window w - 1, whose half the next fetch refills
      cp_async_wait_all();
      __syncthreads();
      if (w + 1 < a.nwin) fetch_cta((w + 1) * S, T, int((w + 1) & 1) * T);
      win = ring + px * RLD + int(w & 1) * T;
    }
    MomAcc acc{band, 0.f, 0.f, 0.f};
    warp_fft<T, 1, LP>(win, work + px * Sm::WLD, tw, jl, acc, lower);
#pragma unroll
    for (int o = LP / 2; o > 0; o >>= 1) {  // reduce within the pixel's lane group
      acc.m0 += __shfl_xor_sync(0xffffffffu, acc.m0, o);
      acc.m1 += __shfl_xor_sync(0xffffffffu, acc.m1, o);
      acc.m2 += __shfl_xor_sync(0xffffffffu, acc.m2, o);
    }
    if constexpr (POST) {
      emit_moments(a, w, p0 + px, acc, jl == 0, false);
    } else if (jl == 0) {
      const float m1 = acc.m1 * a.fscale, m2 = acc.m2 * (a.fscale * a.fscale);  // bins -> kHz
      float* o = a.out + size_t(w) * a.nout * HW + p0 + px;
      int q = 0;
      if (a.mask & HV_MOM_M0) o[HW * q++] = acc.m0;
      if (a.mask & HV_MOM_M1) o[HW * q++] = m1;
      if (a.mask & HV_MOM_M2) o[HW * q++] = m2;
      const double d0 = acc.m0;
      if (a.mask & HV_MOM_M1N) o[HW * q++] = d0 > 0.0 ? float(double(m1) / d0) : 0.f;
      if (a.mask & HV_MOM_M2N) {
        const double r = d0 > 0.0 ? double(m2) / d0 : 0.0;
        o[HW * q++] = float(sqrt(r > 0.0 ? r : 0.0));
      }
    }
  }
}

// Windows that do not overlap (S >= T): one CTA per (window, tile of BT pixels),
// so that many windows are in flight per SM instead of one CTA walking all
// windows of its pixels. The window's T frames of the CTA's pixels land by
// cp.async straight in the pixels' padded work rows (sample t at t + t / 16; the
// row stride adds two more values so that the eight rows of a CTA start in
// different banks), and the FFT runs in place there: the first stage reads the
// whole row into registers before any lane of the pixel writes. A CTA holds one
// window, so its shared memory is a quarter of the walking kernel's and several
// CTAs share an SM.
template <int T, bool WIDE = false>
struct WinCfg {
  using Lw = WarpLayout<T>;
  // warps per CTA: 8 for short windows (a warp's fetch covers 32 pixels, 256
  // contiguous bytes of a frame), else the walking kernel's count; WIDE doubles
  // it (twice the pixels per CTA: longer contiguous runs of each frame)
  static constexpr int NW = (T <= 128 ? 8 : Lw::NW) * (WIDE ? 2 : 1);
  static constexpr int NT = 32 * NW;
  static constexpr int BT = NW * Lw::PW;  // pixels per CTA
  // row stride (float2): the padded row, rounded to 1 mod 16 so that the rows of
  // consecutive pixels start in consecutive bank pairs
  static constexpr int WR = (T + T / 16 + 15) / 16 * 16 + 1;
  static constexpr int OCC = WIDE ? (T >= 512 ? 2 : 2) : (T >= 1024 ? 1 : (T >= 512 ? 4 : (T >= 256 ? 6 : 4)));
  static constexpr size_t bytes() { return (size_t(BT) * WR + (T - WarpPlan<T>::R1)) * sizeof(float2); }
};

template <int T, bool WIDE, bool POST>
__global__ void __launch_bounds__(WinCfg<T, WIDE>::NT, WinCfg<T, WIDE>::OCC) k_stft_win(StftArgs a) {
  using Lw = WarpLayout<T>;
  using Wc = WinCfg<T, WIDE>;
  constexpr int NT = Wc::NT, LP = Lw::LP, PW = Lw::PW, BT = Wc::BT, WR = Wc::WR;
  extern __shared__ __align__(16) unsigned char smem_win[];
  float2* rows = reinterpret_cast<float2*>(smem_win);
  float2* tw = rows + BT * WR;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pl = lane / LP, jl = lane % LP;
  const int px = warp * PW + pl;
  const size_t HW = size_t(a.W) * a.H;
  const uint32_t ntile = uint32_t(HW / BT);
  const uint32_t w = blockIdx.x / ntile;
  const uint32_t p0 = (blockIdx.x % ntile) * BT;
  const float2* tq = static_cast<const float2*>(a.tq.base);
  const uint32_t cap = a.tq.cap;
  // the window's frames: queue slots slot0 + w S + f (one wrap at most)
  {
    constexpr int FS = NT / BT;  // frames per pass of the CTA
    const int b = tid % BT;
    int f = tid / BT;
    uint32_t g = a.tq.slot0 + w * a.S + uint32_t(f);
    while (g >= cap) g -= cap;
    for (; f < T; f += FS) {
      cp_async8(&rows[b * WR + wpad(f)], &tq[size_t(g) * HW + p0 + b]);
      g += FS;
      if (g >= cap) g -= cap;
    }
    cp_async_commit();
  }
  {  // stage twiddles (the walking kernel's table layout)
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
  uint32_t band = 0;
  {
    constexpr int RL = Lw::RL, NBL = T / RL;
#pragma unroll
    for (int it = 0; it < Lw::ITL; ++it)
#pragma unroll
      for (int m = 0; m < RL; ++m) {
        const uint32_t k = uint32_t(jl + LP * it + m * NBL);
        if (k - a.klo <= a.khi - a.klo) band |= 1u << (it * RL + m);
      }
  }
  cp_async_wait_all();
  __syncthreads();
  const bool lower = a.khi < uint32_t(T / 2);
  MomAcc acc{band, 0.f, 0.f, 0.f};
  float2* row = rows + px * WR;
  warp_fft<T, 1, LP, true>(row, row, tw, jl, acc, lower);
#pragma unroll
  for (int o = LP / 2; o > 0; o >>= 1) {
    acc.m0 += __shfl_xor_sync(0xffffffffu, acc.m0, o);
    acc.m1 += __shfl_xor_sync(0xffffffffu, acc.m1, o);
    acc.m2 += __shfl_xor_sync(0xffffffffu, acc.m2, o);
  }
  if constexpr (POST) {
    emit_moments(a, w, p0 + px, acc, jl == 0, true);
  } else if (jl == 0) {
    const float m1 = acc.m1 * a.fscale, m2 = acc.m2 * (a.fscale * a.fscale);  // bins -> kHz
    float* o = a.out + size_t(w) * a.nout * HW + p0 + px;
    int q = 0;
    if (a.mask & HV_MOM_M0) __stcs(&o[HW * q++], acc.m0);
    if (a.mask & HV_MOM_M1) __stcs(&o[HW * q++], m1);
    if (a.mask & HV_MOM_M2) __stcs(&o[HW * q++], m2);
    const double d0 = acc.m0;
    if (a.mask & HV_MOM_M1N) __stcs(&o[HW * q++], d0 > 0.0 ? float(double(m1) / d0) : 0.f);
    if (a.mask & HV_MOM_M2N) {
      const double r = d0 > 0.0 ? double(m2) / d0 : 0.0;
      __stcs(&o[HW * q++], float(sqrt(r > 0.0 ? r : 0.0)));
    }
  }
}

// The window-per-CTA kernel made persistent and double-buffered: CTA c takes the
// (window, pixel tile) items c, c + grid, ... and issues the cp.async copies of its
// next item's frames into the other buffer before it transforms the current one,
// so that its loads overlap its own FFT instead of only other CTAs'. Two padded
// buffers per CTA: fewer CTAs per SM than the one-item kernel (3 at T = 512).
template <int T, bool POST>
__global__ void __launch_bounds__(WinCfg<T, false>::NT, 1) k_stft_winp(StftArgs a) {
  using Lw = WarpLayout<T>;
  using Wc = WinCfg<T, false>;
  constexpr int NT = Wc::NT, LP = Lw::LP, PW = Lw::PW, BT = Wc::BT, WR = Wc::WR;
  extern __shared__ __align__(16) unsigned char smem_winp[];
  float2* rows0 = reinterpret_cast<float2*>(smem_winp);  // buffer b at rows0 + b BT WR
  float2* tw = rows0 + 2 * BT * WR;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pl = lane / LP, jl = lane % LP;
  const int px = warp * PW + pl;
  const size_t HW = size_t(a.W) * a.H;
  const uint32_t ntile = uint32_t(HW / BT);
  const uint32_t nitem = a.nwin * ntile;
  const float2* tq = static_cast<const float2*>(a.tq.base);
  const uint32_t cap = a.tq.cap;
  // item i: window i / ntile, pixels (i % ntile) BT ..; its frames into buffer b
  auto fetch = [&](uint32_t i, int b) {
    constexpr int FS = NT / BT;  // frames per pass of the CTA
    const uint32_t w = i / ntile, p0 = (i % ntile) * BT;
    float2* rows = rows0 + b * BT * WR;
    const int c = tid % BT;
    int f = tid / BT;
    uint32_t g = a.tq.slot0 + w * a.S + uint32_t(f);
    while (g >= cap) g -= cap;
    for (; f < T; f += FS) {
      cp_async8(&rows[c * WR + wpad(f)], &tq[size_t(g) * HW + p0 + c]);
      g += FS;
      if (g >= cap) g -= cap;
    }
    cp_async_commit();
  };
  uint32_t item = blockIdx.x;
  if (item < nitem) fetch(item, 0);
  {  // stage twiddles (the walking kernel's table layout)
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
  uint32_t band = 0;
  {
    constexpr int RL = Lw::RL, NBL = T / RL;
#pragma unroll
    for (int it = 0; it < Lw::ITL; ++it)
#pragma unroll
      for (int m = 0; m < RL; ++m) {
        const uint32_t k = uint32_t(jl + LP * it + m * NBL);
        if (k - a.klo <= a.khi - a.klo) band |= 1u << (it * RL + m);
      }
  }
  const bool lower = a.khi < uint32_t(T / 2);
  for (int b = 0; item < nitem; item += gridDim.x, b ^= 1) {
    const uint32_t next = item + gridDim.x;
    // the other buffer was released by the barrier that ended the previous item
    if (next < nitem) {
      fetch(next, b ^ 1);
      cp_async_wait_group<1>();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();  // every thread's copies of this item landed
    const uint32_t w = item / ntile, p0 = (item % ntile) * BT;
    MomAcc acc{band, 0.f, 0.f, 0.f};
    float2* row = rows0 + b * BT * WR + px * WR;
    warp_fft<T, 1, LP, true>(row, row, tw, jl, acc, lower);
#pragma unroll
    for (int o = LP / 2; o > 0; o >>= 1) {
      acc.m0 += __shfl_xor_sync(0xffffffffu, acc.m0, o);
      acc.m1 += __shfl_xor_sync(0xffffffffu, acc.m1, o);
      acc.m2 += __shfl_xor_sync(0xffffffffu, acc.m2, o);
    }
    if constexpr (POST) {
      emit_moments(a, w, p0 + px, acc, jl == 0, true);
    } else if (jl == 0) {
      const float m1 = acc.m1 * a.fscale, m2 = acc.m2 * (a.fscale * a.fscale);  // bins -> kHz
      float* o = a.out + size_t(w) * a.nout * HW + p0 + px;
      int q = 0;
      if (a.mask & HV_MOM_M0) __stcs(&o[HW * q++], acc.m0);
      if (a.mask & HV_MOM_M1) __stcs(&o[HW * q++], m1);
      if (a.mask & HV_MOM_M2) __stcs(&o[HW * q++], m2);
      const double d0 = acc.m0;
      if (a.mask & HV_MOM_M1N) __stcs(&o[HW * q++], d0 > 0.0 ? float(double(m1) / d0) : 0.f);
      if (a.mask & HV_MOM_M2N) {
        const double r = d0 > 0.0 ? double(m2) / d0 : 0.0;
        __stcs(&o[HW * q++], float(sqrt(r > 0.0 ? r : 0.0)));
      }
    }
    __syncthreads();  // every warp is done with this buffer before it is refilled
  }
}

// Windows that do not overlap at T = 512, frames by TMA: the window-per-CTA
// kernel's work (8 pixels of one window per CTA) with the window's frames brought
// in by two TMA tensor loads (8 pixels x 256 queue slots each, 64-byte swizzle)
// instead of one 8-byte cp.async per element, and the FFT run in place in that
// tile as a decimation in frequency, 512 = 16 x 32: with t = j + 32 m and
// k = k1 + 16 k2, X_k = sum_j w32^(j k2) w512^(j k1) sum_m x_t w16^(m k1).
// Stage 1: butterfly j (two per lane) reads the 16 samples t = j + 32 m, takes
// their 16-point DFT, multiplies output k1 by w512^(j k1) and writes it back to
// t = j + 32 k1; under the swizzle the 32 lanes of a warp (two pixels) then touch
// 16 different bank pairs. Stage 2: lane jl owns k1 = jl, a 32-point DFT over the
// contiguous positions 32 k1 + j. Read in order, the 16 lanes of a pixel would all
// hit one bank pair, so lane jl reads them rotated by r = jl mod 8 (sample m of its
// sequence is position 32 k1 + (m + r) mod 32) and multiplies output k2 by
// w32^(r k2): the DFT of a sequence rotated by r is the DFT of the sequence times
// w32^(-r k2). Bins come out as k = jl + 16 k2, the layout of the other kernels'
// last stage, and feed the same moment sums. The host checks that no window's
// slots wrap around the queue.
constexpr int WT_T = 512, WT_BT = 8, WT_NT = 128;
constexpr int WT_TW1 = 15 * 32;  // w512^(j k1) at (k1 - 1) 32 + j
constexpr int WT_TW2 = 31 * 8;   // w32^(r k2) at (k2 - 1) 8 + r
constexpr size_t WT_TILE = size_t(WT_T) * WT_BT;  // float2 per tile
constexpr size_t wt_smem(int tiles) { return 1024 + (tiles * WT_TILE + WT_TW1 + WT_TW2) * sizeof(float2); }

// Lanes of the TMA-fed window kernels: each half-warp holds 8 lanes of each of the
// warp's two pixels (lanes 0-7 and 16-23 the first, 8-15 and 24-31 the second), so
// that the 16 lanes of one 64-bit shared-memory access phase cover both halves of
// the 16-byte chunks and, under the swizzle, 16 different bank pairs.
__device__ __forceinline__ int wt_jl(int lane) { return (lane & 7) | ((lane & 16) >> 1); }

// Twiddle tables and band bits of the TMA-fed window kernels.
__device__ __forceinline__ uint32_t wt_setup(const StftArgs& a, float2* tw1, float2* tw2, int tid, int jl) {
  for (int e = tid; e < WT_TW1; e += WT_NT) tw1[e] = a.tw_t[(e % 32) * (e / 32 + 1)];
  for (int e = tid; e < WT_TW2; e += WT_NT) tw2[e] = a.tw_t[(16 * (e % 8) * (e / 8 + 1)) & (WT_T - 1)];
  uint32_t band = 0;
#pragma unroll
  for (int m = 0; m < 32; ++m) {
    const uint32_t k = uint32_t(jl + 16 * m);
    if (k - a.klo <= a.khi - a.klo) band |= 1u << m;
  }
  return band;
}

// One thread: the window's T frames of pixels p0 .. p0 + 7 into `tile` by two
// TMA tensor loads completing on `mbar`.
__device__ __forceinline__ void wt_load(const StftArgs& a, const CUtensorMap* qmap, float2* tile, uint32_t mbar,
                                        uint32_t w, uint32_t p0) {
  uint32_t slot = a.tq.slot0 + w * a.S;  // the host keeps slot + T within the queue
  while (slot >= a.tq.cap) slot -= a.tq.cap;
  mbar_arrive_tx(mbar, uint32_t(WT_T * WT_BT * 8));
  tma_load_2d(smem_addr(tile), qmap, int(p0), int(slot), mbar);
  tma_load_2d(smem_addr(tile + 256 * WT_BT), qmap, int(p0), int(slot + 256), mbar);
}

// The two FFT stages of the warp's two pixels in the landed tile, the moments,
// and the epilogue (pixel p0 + px of window w).
template <bool POST>
__device__ __forceinline__ void wt_window(const StftArgs& a, float2* tile, const float2* tw1, const float2* tw2,
                                          uint32_t band, int px, int jl, uint32_t w, uint32_t p0) {
  constexpr int T = WT_T;
  const size_t HW = size_t(a.W) * a.H;
  // sample t of pixel px: 16-byte chunk px / 2 of row t sits at chunk
  // (px / 2) ^ ((t >> 1) & 3), px % 2 selects its half
  auto at = [&](int t) -> float2* { return tile + 8 * t + (px ^ (((t >> 1) & 3) << 1)); };
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int j = jl + 16 * it;
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = *at(j + 32 * m);
    dft<16, -1>(v);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw1[(k1 - 1) * 32 + j]);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) *at(j + 32 * k1) = v[k1];
  }
  __syncwarp();
  const int r = jl & 7;
  const bool lower = a.khi < uint32_t(T / 2);
  float2 v[32];
#pragma unroll
  for (int m = 0; m < 32; ++m) v[m] = *at(32 * jl + ((m + r) & 31));
  MomAcc acc{band, 0.f, 0.f, 0.f};
  if (lower) {
    dft_lower<32>(v);
#pragma unroll
    for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmul(v[k2], tw2[(k2 - 1) * 8 + r]);
    add_moments<32, 16, 16>(v, 0, float(jl), acc);
  } else {
    dft<32, -1>(v);
#pragma unroll
    for (int k2 = 1; k2 < 32; ++k2) v[k2] = cmul(v[k2], tw2[(k2 - 1) * 8 + r]);
    add_moments<32, 16, 32>(v, 0, float(jl), acc);
  }
  // the pixel's 16 lanes: lane ^ 16, then within the group of 8
  auto fold = [&](int o) {
    acc.m0 += __shfl_xor_sync(0xffffffffu, acc.m0, o);
    acc.m1 += __shfl_xor_sync(0xffffffffu, acc.m1, o);
    acc.m2 += __shfl_xor_sync(0xffffffffu, acc.m2, o);
  };
  fold(16);
  fold(4);
  fold(2);
  fold(1);
  if constexpr (POST) {
    emit_moments(a, w, p0 + px, acc, jl == 0, true);
  } else if (jl == 0) {
    const float m1 = acc.m1 * a.fscale, m2 = acc.m2 * (a.fscale * a.fscale);  // bins -> kHz
    float* o = a.out + size_t(w) * a.nout * HW + p0 + px;
    int q = 0;
    if (a.mask & HV_MOM_M0) __stcs(&o[HW * q++], acc.m0);
    if (a.mask & HV_MOM_M1) __stcs(&o[HW * q++], m1);
    if (a.mask & HV_MOM_M2) __stcs(&o[HW * q++], m2);
    const double d0 = acc.m0;
    if (a.mask & HV_MOM_M1N) __stcs(&o[HW * q++], d0 > 0.0 ? float(double(m1) / d0) : 0.f);
    if (a.mask & HV_MOM_M2N) {
      const double rr = d0 > 0.0 ? double(m2) / d0 : 0.0;
      __stcs(&o[HW * q++], float(sqrt(rr > 0.0 ? rr : 0.0)));
    }
  }
}

// One CTA per (window, 8-pixel tile); five CTAs per SM (96 registers, no spills:
// 0.509 against 0.532 ms per 4,096 frames with four at 112).
template <bool POST>
__global__ void __launch_bounds__(WT_NT, 5) k_stft_wt(StftArgs a, const __grid_constant__ CUtensorMap qmap) {
  extern __shared__ __align__(16) unsigned char smem_wt[];
  __shared__ __align__(8) unsigned long long s_full;
  // the tile first, 1024-byte aligned (the swizzle pattern repeats every 512 bytes)
  float2* tile = reinterpret_cast<float2*>(smem_wt + ((1024u - (smem_addr(smem_wt) & 1023u)) & 1023u));
  float2* tw1 = tile + WT_TILE;
  float2* tw2 = tw1 + WT_TW1;
  const int tid = threadIdx.x, lane = tid & 31, jl = wt_jl(lane), px = (tid >> 5) * 2 + ((lane >> 3) & 1);
  const uint32_t ntile = uint32_t(size_t(a.W) * a.H / WT_BT);
  const uint32_t w = blockIdx.x / ntile, p0 = (blockIdx.x % ntile) * WT_BT;
  const uint32_t mbar = smem_addr(&s_full);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    wt_load(a, &qmap, tile, mbar, w, p0);
  }
  const uint32_t band = wt_setup(a, tw1, tw2, tid, jl);
  __syncthreads();  // mbarrier initialised, twiddles staged
  const bool landed = mbar_wait(mbar, 0);
  if (!__all_sync(0xffffffffu, landed)) {
    if (lane == 0) atomicOr(a.err, 2u);
    if (tid == 0) mbar_wait(mbar, 0);  // give the copy in flight a second bounded wait
    return;
  }
  wt_window<POST>(a, tile, tw1, tw2, band, px, jl, w, p0);
}

// Persistent and double-buffered: CTA c takes the (window, tile) items c, c + grid,
// ...; while it transforms one item, the next one's frames land in the other tile
// (one thread issues the loads as soon as every warp is done with that tile).
template <bool POST>
__global__ void __launch_bounds__(WT_NT, 3) k_stft_wtp(StftArgs a, const __grid_constant__ CUtensorMap qmap) {
  extern __shared__ __align__(16) unsigned char smem_wt[];
  __shared__ __align__(8) unsigned long long s_full[2];
  float2* tiles = reinterpret_cast<float2*>(smem_wt + ((1024u - (smem_addr(smem_wt) & 1023u)) & 1023u));
  float2* tw1 = tiles + 2 * WT_TILE;
  float2* tw2 = tw1 + WT_TW1;
  const int tid = threadIdx.x, lane = tid & 31, jl = wt_jl(lane), px = (tid >> 5) * 2 + ((lane >> 3) & 1);
  const uint32_t ntile = uint32_t(size_t(a.W) * a.H / WT_BT);
  const uint32_t items = a.nwin * ntile;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&s_full[b])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const uint32_t i0 = blockIdx.x;
    if (i0 < items) wt_load(a, &qmap, tiles, smem_addr(&s_full[0]), i0 / ntile, (i0 % ntile) * WT_BT);
  }
  const uint32_t band = wt_setup(a, tw1, tw2, tid, jl);
  uint32_t k = 0;
  for (uint32_t i = blockIdx.x; i < items; i += gridDim.x, ++k) {
    const int b = int(k & 1);
    // every warp is done with the other tile (item k - 1): its next load may start
    __syncthreads();
    const uint32_t nxt = i + gridDim.x;
    if (tid == 0 && nxt < items) {
      // the tile's generic reads and writes (item k - 1) before the async-proxy load
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      wt_load(a, &qmap, tiles + (b ^ 1) * WT_TILE, smem_addr(&s_full[b ^ 1]), nxt / ntile, (nxt % ntile) * WT_BT);
    }
    const bool landed = mbar_wait(smem_addr(&s_full[b]), (k >> 1) & 1);
    if (!__syncthreads_and(landed)) {
      if (tid == 0) {
        atomicOr(a.err, 2u);
        // second bounded waits for the copies in flight (this item's and the next one's)
        mbar_wait(smem_addr(&s_full[b]), (k >> 1) & 1);
        if (nxt < items) mbar_wait(smem_addr(&s_full[b ^ 1]), ((k + 1) >> 1) & 1);
      }
      return;
    }
    wt_window<POST>(a, tiles + b * WT_TILE, tw1, tw2, band, px, jl, i / ntile, (i % ntile) * WT_BT);
  }
}

// cuTensorMapEncodeTiled from the driver (resolved once through the runtime)
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of the time queue for the staged loads: 8-byte elements, {H W
// pixels, cap slots}, box {8 pixels, S slots}, 64-byte swizzle. False when the
// launch does not qualify: the staged S frames of a window must be S whole
// consecutive slots (the queue capacity, T and the first slot multiples of S).
static bool queue_map(const StftArgs& a, int BT, CUtensorMap* map) {
  if (BT != 8 || a.S == 0 || a.S >= a.T || a.S > 256 || a.tq.cap % a.S || a.T % a.S || a.tq.slot0 % a.S) return false;
  return encode_map_2d_u64(map, a.tq.base, uint64_t(a.W) * a.H, a.tq.cap, uint64_t(a.W) * a.H * 8, 8, a.S, true);
}

bool encode_map_2d(void* map, const void* base, int elem_bytes, uint64_t inner, uint64_t outer,
                   uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_outer) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const CUtensorMapDataType dt = elem_bytes == 1   ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                 : elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                 : elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                                   : CU_TENSOR_MAP_DATA_TYPE_UINT64;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {pitch_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return fn(static_cast<CUtensorMap*>(map), dt, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_map_2d_u64(void* map, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch_bytes,
                       uint32_t box_inner, uint32_t box_outer, bool swizzle64) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {pitch_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return fn(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dims,
            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The TMA-fed window kernel (T = 512, S >= T): cudaErrorNotSupported when a
// window's queue slots wrap around the queue or the tensor map cannot be made.
static cudaError_t launch_wt(const StftArgs& a, cudaStream_t s) {
  const size_t hw = size_t(a.W) * a.H;
  if (hw % WT_BT || a.T != uint32_t(WT_T) || a.S < a.T) return cudaErrorNotSupported;
  for (uint32_t w = 0; w < a.nwin; ++w) {
    const uint64_t slot = (uint64_t(a.tq.slot0) + uint64_t(w) * a.S) % a.tq.cap;
    if (slot + WT_T > a.tq.cap) return cudaErrorNotSupported;
  }
  CUtensorMap map{};
  if (!encode_map_2d_u64(&map, a.tq.base, hw, a.tq.cap, hw * 8, WT_BT, 256, true)) return cudaErrorNotSupported;
  const uint64_t items = uint64_t(a.nwin) * (hw / WT_BT);
  if (items >= (1ull << 31)) return cudaErrorInvalidValue;
  if (a.kernel == STFT_TMA_PIPE) {
    auto kern = a.post_ring ? k_stft_wtp<true> : k_stft_wtp<false>;
    const size_t smem = wt_smem(2);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int per_sm = 0, dev = 0, nsm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WT_NT, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorNotSupported;
    kern<<<unsigned(std::min<uint64_t>(items, uint64_t(per_sm) * nsm)), WT_NT, smem, s>>>(a, map);
    return cudaGetLastError();
  }
  auto kern = a.post_ring ? k_stft_wt<true> : k_stft_wt<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(wt_smem(1)));
  if (e != cudaSuccess) return e;
  kern<<<unsigned(items), WT_NT, wt_smem(1), s>>>(a, map);
  return cudaGetLastError();
}

template <int T>
static cudaError_t launch_warp(const StftArgs& a0, cudaStream_t s) {
  using Lw = WarpLayout<T>;
  const size_t hw = size_t(a0.W) * a0.H;
  if (hw % Lw::BT) return cudaErrorInvalidValue;
  // every frame of the launch is resident in the queue (no slot reduction beyond one wrap)
  if (a0.tq.slot0 >= a0.tq.cap || uint64_t(a0.nwin - 1) * a0.S + uint64_t(T) > a0.tq.cap)
    return cudaErrorInvalidValue;
  StftArgs a = a0;
  if constexpr (T == WT_T) {
    if (a.S >= uint32_t(T) && (a.kernel == STFT_TMA || a.kernel == STFT_TMA_PIPE)) {
      const cudaError_t e = launch_wt(a, s);
      if (e != cudaErrorNotSupported) return e;  // else a window wraps: the window-per-CTA kernel
    }
  }
  if (a.S >= uint32_t(T) && a.kernel != STFT_WALK) {
    // one CTA per (window, pixel tile)
    auto launch_win = [&](auto wide) -> cudaError_t {
      constexpr bool W = decltype(wide)::value;
      using Wc = WinCfg<T, W>;
      if (hw % Wc::BT) return cudaErrorNotSupported;
      const size_t smem = Wc::bytes();
      auto kern = a.post_ring ? k_stft_win<T, W, true> : k_stft_win<T, W, false>;
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
      const uint64_t grid = uint64_t(a.nwin) * (hw / Wc::BT);
      if (grid >= (1ull << 31)) return cudaErrorInvalidValue;
      kern<<<unsigned(grid), Wc::NT, smem, s>>>(a);
      return cudaGetLastError();
    };
    if (a.kernel == STFT_PIPE) {
      using Wc = WinCfg<T, false>;
      if (hw % Wc::BT == 0) {
        const size_t smem = 2 * size_t(Wc::BT) * Wc::WR * sizeof(float2) + (T - WarpPlan<T>::R1) * sizeof(float2);
        auto kern = a.post_ring ? k_stft_winp<T, true> : k_stft_winp<T, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        int per_sm = 0, dev = 0, nsm = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Wc::NT, smem);
        if (e != cudaSuccess) return e;
        if (per_sm >= 1) {
          cudaGetDevice(&dev);
          cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
          const uint64_t items = uint64_t(a.nwin) * (hw / Wc::BT);
          const uint64_t grid = std::min<uint64_t>(items, uint64_t(per_sm) * nsm);
          kern<<<unsigned(grid), Wc::NT, smem, s>>>(a);
          return cudaGetLastError();
        }
      }
    }
    const cudaError_t e = a.kernel == STFT_WIDE ? launch_win(std::true_type{}) : launch_win(std::false_type{});
    if (e != cudaErrorNotSupported) return e;
  }
  CUtensorMap map{};
  a.tma = queue_map(a, Lw::BT, &map) ? 1 : 0;
  const size_t smem = WarpSmem<T>::bytes(a.S, a.tma != 0);
  auto kern = a.post_ring ? k_stft_warp<T, true> : k_stft_warp<T, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  kern<<<unsigned(hw / Lw::BT), Lw::NT, smem, s>>>(a, map);
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
