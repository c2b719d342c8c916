// hv_static.cu -- a spatial-transform entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they want a
// hologram propagated: code running inside a memory-pool or allocator callback,
// plugins whose host framework owns every allocation and forbids cudaMalloc /
// cudaFree (they can synchronise the device or fail under a capture), or
// real-time loops that must not touch the allocator at all. hv_spatial_static
// serves them: the caller passes device pointers to the raw frames and to the
// output fields, and everything else the transform needs -- twiddle tables,
// the angular-spectrum transfer function or Fresnel chirp, and the two
// intermediate buffers of the 2-D FFT passes -- lives in one file-scope
// __device__ array of fixed size that every GPU loading this library holds
// until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents. Nothing in it has to start at zero: every call rewrites the tables
// and the intermediates it reads. Calls whose GPU work overlaps (different
// streams, no ordering between them) race on the array; order them on one
// stream or with events.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/hv.h"
#include "hv_internal.h"

namespace {

using namespace hv;

// Layout of the array (bytes): twiddles for L = 8..1024, chirp x/y factors,
// transfer function, then two intermediate buffers of HV_STATIC_MAX_PIXELS
// complex values each.
constexpr size_t kTwBytes = 16384;                        // 2040 float2 packed
constexpr size_t kChirpBytes = 2 * 512 * sizeof(float2);  // W + H <= 1024 factors
constexpr size_t kHBytes = size_t(512) * 512 * sizeof(float2);
constexpr size_t kInterBytes = size_t(HV_STATIC_MAX_PIXELS) * sizeof(float2);
constexpr size_t kScratchBytes = kTwBytes + kChirpBytes + kHBytes + 2 * kInterBytes;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Resolved address of the array per device, with the driver context it was
// resolved in: a different current context (after cudaDeviceReset, or a
// non-primary context made current by the caller) has its own copy of the
// module, so the address is resolved again there.
void* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// cuCtxGetCurrent from the driver, resolved once through the runtime (no link
// dependency on libcuda). NULL when the driver does not offer it.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  });
  return fn;
}

__host__ __device__ size_t packed_offset(uint32_t L) {  // twiddle tables packed by increasing length from 8
  size_t off = 0;
  for (uint32_t l = 8; l < L; l <<= 1) off += l;
  return off;
}

bool pow2_in(uint32_t v, uint32_t lo, uint32_t hi) { return v >= lo && v <= hi && !(v & (v - 1)); }

struct TableArgs {
  float2* tw;
  float2* chirp;
  float2* h;
  int spatial, fftshift;
  uint32_t W, H;
  double z, lam, dx, dy;
  double highpass;  // cutoff in cycles per pixel, 0 = off
};

// Twiddles, chirp factors and the transposed transfer function, in float64 on
// the device (same definitions as the tables the handle path builds on the host).
__global__ void k_static_tables(TableArgs a) {
  const size_t ntw = packed_offset(2048);
  const size_t nh = size_t(a.W) * a.H;
  const size_t total = ntw + a.W + a.H + nh;
  for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < total;
       e += size_t(gridDim.x) * blockDim.x) {
    if (e < ntw) {
      uint32_t L = 8;
      size_t off = 0;
      while (e >= off + L) {
        off += L;
        L <<= 1;
      }
      double s, c;
      sincospi(-2.0 * double(e - off) / double(L), &s, &c);
      a.tw[e] = make_float2(float(c), float(s));
    } else if (e < ntw + a.W + a.H) {
      const size_t j = e - ntw;
      float2 v = make_float2(1.f, 0.f);
      if (a.spatial == HV_SPATIAL_FRESNEL) {
        const bool isx = j < a.W;
        const uint32_t i = isx ? uint32_t(j) : uint32_t(j - a.W);
        const uint32_t n = isx ? a.W : a.H;
        const double d = isx ? a.dx : a.dy;
        const double x = (double(i) - n / 2.0) * d;
        double ph = M_PI * x * x / (a.lam * a.z) + ((a.fftshift && (i & 1)) ? M_PI : 0.0);
        double s, c;
        sincos(ph, &s, &c);
        v = make_float2(float(c), float(s));
      }
      a.chirp[j] = v;
    } else if (a.spatial == HV_SPATIAL_ASP) {
      const size_t q = e - ntw - a.W - a.H;  // [kx][ky]
      const uint32_t kx = uint32_t(q / a.H), ky = uint32_t(q % a.H);
      const double k = 2.0 * M_PI / a.lam;
      const double mx = kx < a.W / 2 ? double(kx) : double(kx) - a.W;
      const double my = ky < a.H / 2 ? double(ky) : double(ky) - a.H;
      const double fx = 2.0 * M_PI * mx / (a.W * a.dx);
      const double fy = 2.0 * M_PI * my / (a.H * a.dy);
      const double kz2 = k * k - fx * fx - fy * fy;
      // the high-pass filter after propagation zeroes the spectrum below the cutoff radius
      const double rx = mx / a.W, ry = my / a.H;
      const bool passed = !(a.highpass > 0.0) || rx * rx + ry * ry >= a.highpass * a.highpass;
      float2 v = make_float2(0.f, 0.f);
      if (kz2 >= 0 && passed) {
        const double scale = 1.0 / (double(a.W) * double(a.H));
        double s, c;
        sincos(a.z * sqrt(kz2), &s, &c);
        v = make_float2(float(c * scale), float(s * scale));
      }
      a.h[q] = v;
    }
  }
}

}  // namespace

extern "C" hv_status hv_spatial_static(const void* frames, uint32_t pixel_bits, uint32_t n,
                                       const hv_params* p, float* out, void* stream) {
  if (!frames || !out || !p || n == 0) return HV_ERR_ARG;
  if (p->struct_size != sizeof(hv_params)) return HV_ERR_ARG;
  if (pixel_bits != 8 && pixel_bits != 16) return HV_ERR_ARG;
  // the kernels store complex values as 8-byte pairs and read 16-bit pixels as
  // 2-byte words: a misaligned pointer would fault on the device
  if ((reinterpret_cast<uintptr_t>(out) & 7u) != 0) return HV_ERR_ARG;
  if (pixel_bits == 16 && (reinterpret_cast<uintptr_t>(frames) & 1u) != 0) return HV_ERR_ARG;
  const uint32_t W = p->width, H = p->height;
  if (!pow2_in(W, 16, 512) || !pow2_in(H, 16, 512)) return HV_ERR_ARG;
  if (uint64_t(n) * W * H > HV_STATIC_MAX_PIXELS) return HV_ERR_ARG;
  if (p->spatial != HV_SPATIAL_NONE && p->spatial != HV_SPATIAL_ASP && p->spatial != HV_SPATIAL_FRESNEL)
    return HV_ERR_ARG;
  if (p->spatial != HV_SPATIAL_NONE) {
    if (!(p->lambda_m > 0) || !(p->pitch_x_m > 0) || !(p->pitch_y_m > 0) || !std::isfinite(p->z_m))
      return HV_ERR_ARG;
    if (p->spatial == HV_SPATIAL_FRESNEL && p->z_m == 0.0) return HV_ERR_ARG;
  }
  if (!(p->highpass_cpp >= 0.0) || (p->highpass_cpp > 0.0 && p->spatial != HV_SPATIAL_ASP)) return HV_ERR_ARG;
  // an error left pending by the caller's earlier runtime calls is theirs: report
  // it without clearing it rather than mistake it for a failure of this call
  if (cudaPeekAtLastError() != cudaSuccess) return HV_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HV_ERR_CUDA;
  // Set-up, once per device (and driver context) with that device current: the
  // host cannot use the array's name as a device address, so resolve the address
  // the kernels get.
  CUcontext ctx = nullptr;
  if (CtxGetCurrentFn f = ctx_get_current()) {
    if (f(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return HV_ERR_CUDA;
      g_scratch_addr[dev] = ptr;
      g_scratch_ctx[dev] = ctx;
    }
    base = g_scratch_addr[dev];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  float2* tw = reinterpret_cast<float2*>(b);
  float2* chirp = reinterpret_cast<float2*>(b + kTwBytes);
  float2* htab = reinterpret_cast<float2*>(b + kTwBytes + kChirpBytes);
  float2* s1 = reinterpret_cast<float2*>(b + kTwBytes + kChirpBytes + kHBytes);
  float2* s2 = reinterpret_cast<float2*>(b + kTwBytes + kChirpBytes + kHBytes + kInterBytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  TableArgs ta{tw, chirp, htab, p->spatial, p->fftshift, W, H, p->z_m, p->lambda_m, p->pitch_x_m,
               p->pitch_y_m, p->highpass_cpp};
  k_static_tables<<<256, 256, 0, s>>>(ta);
  // no error was pending before the launch, so one now is this launch's
  if (cudaGetLastError() != cudaSuccess) return HV_ERR_CUDA;

  SpatialArgs sa{};
  sa.spatial = p->spatial;
  sa.in_kind = pixel_bits == 8 ? IN_U8 : IN_U16;
  sa.W = W;
  sa.H = H;
  sa.n = n;
  sa.raw = RingRef{const_cast<void*>(frames), n, 0};
  sa.tq = RingRef{out, n, 0};
  sa.scratch1 = s1;
  sa.scratch2 = s2;
  sa.tw_w = tw + packed_offset(W);
  sa.tw_h = tw + packed_offset(H);
  sa.asp_ht = htab;
  sa.chirp_x = chirp;
  sa.chirp_y = chirp + W;
  int launches = 0;
  if (launch_spatial(sa, s, &launches) != cudaSuccess) return HV_ERR_CUDA;
  return HV_OK;
}
