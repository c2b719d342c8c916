// k_spatial_pp.cu -- the multi-pass spatial transform (same passes and layouts as
// k_spatial.cu, Sec. III-B.1) as persistent kernels that prefetch.
//
// A CTA stays resident and loops over work items (frame, strip of 16 lines).
// While it transforms one item, the input of its next item streams into the
// other buffer with cp.async, so global-load latency overlaps the FFT stages
// instead of stalling every short-lived CTA at its start:
//   P1  raw strip (uint8/uint16 rows) -> staging buffer; conversion (+ chirp)
//       into the FFT buffer; column FFT; transposed store -> S1[x][ky]
//   P2a S1 strip -> FFT buffer; row FFT, x H, row IFFT; transposed store -> S2
//   P3a S2 strip -> FFT buffer; column IFFT -> time queue
//   P2f S1 strip -> FFT buffer; row FFT; transposed store -> time queue
#include "fft_dev.cuh"
#include "hv_internal.h"
#include "../../include/hv.h"

namespace hv {

namespace {

constexpr int PP_BT = 16;
enum { PK_P1 = 0, PK_P2A = 1, PK_P3A = 2, PK_P2F = 3 };

template <int L>
struct PpCfg {
  static constexpr int BT = PP_BT;
  static constexpr int NT = FftThreads<L, BT>::value;
  static constexpr int LD = BT + 1;
  static constexpr size_t BUF = size_t(L) * LD * sizeof(float2);
  static constexpr size_t RAW = size_t(L) * BT * 2;  // one uint16 strip
};

__device__ __forceinline__ void cpa8(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(s))),
               "l"(g)
               : "memory");
}
__device__ __forceinline__ void cpa16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(s))),
               "l"(g)
               : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int LD>
struct MulHt {  // bin k of line b times the transposed transfer function
  float2* buf;
  const float2* ht;
  uint32_t H, b0;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const {
    buf[k * LD + b] = cmul(v, __ldg(&ht[size_t(k) * H + b0 + b]));
  }
};

struct ToGlobal {
  float2* out;
  uint32_t ld, b0;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const { out[size_t(k) * ld + b0 + b] = v; }
};

// Prefetch the input of item (frame i, lines b0 .. b0+BT) of pass PK into dst.
template <int L, int PK>
__device__ __forceinline__ void prefetch(const SpatialArgs& a, int i, int b0, void* dst) {
  using C = PpCfg<L>;
  if constexpr (PK == PK_P1) {
    const int bpp = a.in_kind == IN_U8 ? 1 : 2;
    const int chunks = C::BT * bpp / 16;  // 16-byte pieces per row segment
    const size_t rslot = (a.raw.slot0 + uint32_t(i)) % a.raw.cap;
    const unsigned char* src = static_cast<const unsigned char*>(a.raw.base) +
                               (rslot * size_t(a.W) * L + b0) * bpp;
    unsigned char* d = static_cast<unsigned char*>(dst);
    for (int e = threadIdx.x; e < L * chunks; e += C::NT) {
      const int y = e / chunks, q = e % chunks;
      cpa16(d + (y * C::BT * bpp) + q * 16, src + size_t(y) * a.W * bpp + q * 16);
    }
  } else {
    // complex strip: element (t, b) of the pass at src[t * ld + b0 + b]
    const float2* src;
    uint32_t ld;
    if constexpr (PK == PK_P3A) {
      src = a.scratch2 + size_t(i) * a.W * L;
      ld = a.W;
    } else {
      src = a.scratch1 + size_t(i) * a.H * L;
      ld = a.H;
    }
    float2* d = static_cast<float2*>(dst);
    for (int e = threadIdx.x; e < L * C::BT; e += C::NT) {
      const int b = e % C::BT, t = e / C::BT;
      cpa8(&d[t * C::LD + b], &src[size_t(t) * ld + b0 + b]);
    }
  }
  cpa_commit();
}

template <int L, int PK>
__global__ void __launch_bounds__(PpCfg<L>::NT, (L <= 256 ? 3 : 1)) k_pass_pp(SpatialArgs a, int nitems, int nstrips) {
  using C = PpCfg<L>;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* buf0 = reinterpret_cast<float2*>(smem);
  // P1: one FFT buffer and two raw staging buffers; other passes: two FFT buffers
  float2* buf1 = reinterpret_cast<float2*>(smem + C::BUF);
  unsigned char* raw0 = smem + C::BUF;
  unsigned char* raw1 = smem + C::BUF + C::RAW;
  const int tid = threadIdx.x;

  int item = blockIdx.x;
  if (item < nitems) prefetch<L, PK>(a, item / nstrips, (item % nstrips) * C::BT, PK == PK_P1 ? (void*)raw0 : (void*)buf0);
  for (int k = 0; item < nitems; ++k, item += gridDim.x) {
    const int cur = k & 1;
    const int i = item / nstrips, b0 = (item % nstrips) * C::BT;
    cpa_wait_all();
    __syncthreads();  // this item's input resident; the other buffer is free
    float2* buf = (PK == PK_P1 || cur == 0) ? buf0 : buf1;
    if constexpr (PK == PK_P1) {
      const unsigned char* raw = cur == 0 ? raw0 : raw1;
      const bool chirp = a.spatial == HV_SPATIAL_FRESNEL;
      const bool u8 = a.in_kind == IN_U8;
      for (int e = tid; e < L * C::BT; e += C::NT) {
        const int b = e % C::BT, y = e / C::BT;
        const float v = u8 ? float(raw[y * C::BT + b]) : float(reinterpret_cast<const uint16_t*>(raw)[y * C::BT + b]);
        float2 u = make_float2(v, 0.f);
        if (chirp) u = cscale(cmul(__ldg(&a.chirp_y[y]), __ldg(&a.chirp_x[b0 + b])), v);
        buf[y * C::LD + b] = u;
      }
      __syncthreads();
    }
    const int nxt = item + gridDim.x;
    if (nxt < nitems) {
      void* dst = PK == PK_P1 ? (void*)(cur == 0 ? raw1 : raw0) : (void*)(cur == 0 ? buf1 : buf0);
      prefetch<L, PK>(a, nxt / nstrips, (nxt % nstrips) * C::BT, dst);
    }
    StoreSmem<C::LD> st{buf};
    if constexpr (PK == PK_P1) {
      fft_lines<L, -1, C::BT, C::NT, C::LD>(buf, a.tw_h, st);
      __syncthreads();
      float2* s1 = a.scratch1 + size_t(i) * a.W * L;
      for (int e = tid; e < L * C::BT; e += C::NT) {
        const int kk = e % L, b = e / L;
        s1[size_t(b0 + b) * L + kk] = buf[kk * C::LD + b];
      }
    } else if constexpr (PK == PK_P2A) {
      MulHt<C::LD> mul{buf, a.asp_ht, a.H, uint32_t(b0)};
      fft_lines<L, -1, C::BT, C::NT, C::LD>(buf, a.tw_w, mul);
      __syncthreads();
      fft_lines<L, +1, C::BT, C::NT, C::LD>(buf, a.tw_w, st);
      __syncthreads();
      float2* s2 = a.scratch2 + size_t(i) * a.H * L;
      for (int e = tid; e < L * C::BT; e += C::NT) {
        const int x = e % L, b = e / L;
        s2[size_t(b0 + b) * L + x] = buf[x * C::LD + b];
      }
    } else if constexpr (PK == PK_P3A) {
      const size_t tslot = (a.tq.slot0 + uint32_t(i)) % a.tq.cap;
      ToGlobal out{static_cast<float2*>(a.tq.base) + tslot * size_t(a.W) * L, a.W, uint32_t(b0)};
      fft_lines<L, +1, C::BT, C::NT, C::LD>(buf, a.tw_h, out);
    } else {
      fft_lines<L, -1, C::BT, C::NT, C::LD>(buf, a.tw_w, st);
      __syncthreads();
      const size_t tslot = (a.tq.slot0 + uint32_t(i)) % a.tq.cap;
      float2* out = static_cast<float2*>(a.tq.base) + tslot * size_t(a.H) * L;
      for (int e = tid; e < L * C::BT; e += C::NT) {
        const int kk = e % L, b = e / L;
        out[size_t(b0 + b) * L + kk] = buf[kk * C::LD + b];
      }
    }
  }
  cpa_wait_all();
}

template <int L, int PK>
static cudaError_t launch_pp(const SpatialArgs& a, int nstrips, cudaStream_t s) {
  using C = PpCfg<L>;
  const size_t smem = PK == PK_P1 ? C::BUF + 2 * C::RAW : 2 * C::BUF;
  auto kern = k_pass_pp<L, PK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, nsm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, smem);
  if (e != cudaSuccess) return e;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int nitems = int(a.n) * nstrips;
  int grid = per_sm * nsm;
  if (grid > nitems) grid = nitems;
  if (grid < 1) grid = 1;
  kern<<<grid, C::NT, smem, s>>>(a, nitems, nstrips);
  return cudaGetLastError();
}

template <int LH, int LW>
static cudaError_t pp_fixed(const SpatialArgs& a, cudaStream_t s, int* launches) {
  cudaError_t e = launch_pp<LH, PK_P1>(a, int(a.W / PP_BT), s);
  if (e != cudaSuccess) return e;
  ++*launches;
  if (a.spatial == HV_SPATIAL_ASP) {
    e = launch_pp<LW, PK_P2A>(a, int(a.H / PP_BT), s);
    if (e != cudaSuccess) return e;
    e = launch_pp<LH, PK_P3A>(a, int(a.W / PP_BT), s);
    *launches += 2;
  } else {
    e = launch_pp<LW, PK_P2F>(a, int(a.H / PP_BT), s);
    ++*launches;
  }
  return e;
}

template <int LH>
static cudaError_t pp_w(const SpatialArgs& a, cudaStream_t s, int* launches) {
  switch (a.W) {
    case 64: return pp_fixed<LH, 64>(a, s, launches);
    case 128: return pp_fixed<LH, 128>(a, s, launches);
    case 256: return pp_fixed<LH, 256>(a, s, launches);
    case 512: return pp_fixed<LH, 512>(a, s, launches);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool spatial_pp_supported(const SpatialArgs& a) {
  auto ok = [](uint32_t v) { return v >= 64 && v <= 512; };  // two strip buffers must fit
  return ok(a.W) && ok(a.H) && (a.spatial == HV_SPATIAL_ASP || a.spatial == HV_SPATIAL_FRESNEL);
}

cudaError_t launch_spatial_pp(const SpatialArgs& a, cudaStream_t s, int* launches) {
  if (a.n == 0) return cudaSuccess;
  switch (a.H) {
    case 64: return pp_w<64>(a, s, launches);
    case 128: return pp_w<128>(a, s, launches);
    case 256: return pp_w<256>(a, s, launches);
    case 512: return pp_w<512>(a, s, launches);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hv
