// k_spatial_cluster.cu -- whole-frame spatial transform in one kernel, the frame
// held in the distributed shared memory of a thread-block cluster.
//
// Same operations as the multi-pass kernels (Sec. III-B.1): angular-spectrum
// propagation IFFT2(FFT2(u) H) or the Fresnel transform FFT2(u chirp). A cluster
// of CL CTAs owns one N x N frame at a time; CTA c holds a strip of SB = N / CL
// lines (128 KB of complex64 at most). Per frame:
//   1. CTA c loads raw columns [c SB, c SB + SB) (conversion and Fresnel chirp
//      fused), FFT along y for its SB columns;
//   2. cluster barrier; each CTA gathers the rows [c SB, c SB + SB) of every
//      CTA's strip through DSMEM into registers, barrier, stores them
//      transposed (x along the FFT axis) in its own shared memory;
//   3. FFT along x for its SB rows. Fresnel: store the rows to the time queue.
//      ASP: multiply by H (1/(N N) folded in), inverse FFT along x, exchange back
//      to column strips as in 2, inverse FFT along y, store columns to the queue.
// Raw frames are read from HBM once and fields written once; nothing goes
// through global scratch. The next frame's raw strip is fetched with cp.async
// while the current one is transformed. Clusters are persistent over frames.
#include <cooperative_groups.h>

#include "fft_dev.cuh"
#include "hv_internal.h"
#include "../../include/hv.h"

namespace cg = cooperative_groups;

namespace hv {

template <int N>
struct ClCfg {
  static constexpr int CL = N <= 64 ? 1 : (N <= 256 ? N / 64 : 16);
  static constexpr int SB = N / CL;          // lines per CTA
  static constexpr int LD = SB + 1;          // padded: transposed accesses conflict-free
  static constexpr int NT = 1024;
  static constexpr size_t DATA = size_t(N) * LD * sizeof(float2);
  static constexpr size_t RAW = size_t(N) * SB * 2;  // uint16 worst case
  static constexpr size_t SMEM = DATA + RAW;
  static constexpr int EXCH = SB * N / NT;    // complex values per thread per exchange
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Fetch this CTA's raw strip (N rows x SB pixels) of frame slot `rslot`.
template <int N>
__device__ __forceinline__ void fetch_raw(const SpatialArgs& a, unsigned char* raw, size_t rslot,
                                          int c, int bpp) {
  using C = ClCfg<N>;
  const int row_bytes = C::SB * bpp;           // 64..128 bytes
  const int chunks = row_bytes / 16;
  const unsigned char* src = static_cast<const unsigned char*>(a.raw.base) +
                             rslot * size_t(N) * N * bpp + size_t(c) * C::SB * bpp;
  for (int e = threadIdx.x; e < N * chunks; e += C::NT) {
    const int y = e / chunks, q = e % chunks;
    cp_async16(raw + y * row_bytes + q * 16, src + size_t(y) * N * bpp + q * 16);
  }
  cpa_commit();
}

template <int LD>
struct AspMulStore {  // multiply bin kx of row b by H^T[kx][ky0 + b], store
  float2* buf;
  const float2* ht;
  uint32_t H, ky0;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const {
    buf[k * LD + b] = cmul(v, __ldg(&ht[size_t(k) * H + ky0 + b]));
  }
};

struct StoreTqCols {  // column strip to the queue: element (y, x0 + b)
  float2* out;
  uint32_t N, x0;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const {
    out[size_t(k) * N + x0 + b] = v;
  }
};

// Move the frame between strip layouts. Source CTA r holds lines [r SB, r SB + SB)
// of the "from" orientation as buf[t * LD + b]; this CTA gathers, for its own
// SB lines of the other orientation, element t' = r SB + b_src of every source
// line t' ... see the kernel comment: we read src[t_own * LD + b] for t_own in
// this CTA's range and write dst[(r SB + b) * LD + t_own - own0].
template <int N>
__device__ __forceinline__ void exchange(cg::cluster_group& cluster, float2* buf, int c) {
  using C = ClCfg<N>;
  float2 stage[C::EXCH];
  const int own0 = c * C::SB;
#pragma unroll
  for (int i = 0; i < C::EXCH; ++i) {
    const int e = threadIdx.x + i * C::NT;     // over CL * SB * SB elements
    const int b = e % C::SB;                    // source column within its strip
    const int tl = (e / C::SB) % C::SB;         // my line index (0..SB)
    const int r = e / (C::SB * C::SB);          // source CTA
    const float2* src = cluster.map_shared_rank(buf, r);
    stage[i] = src[(own0 + tl) * C::LD + b];
  }
  cluster.sync();
#pragma unroll
  for (int i = 0; i < C::EXCH; ++i) {
    const int e = threadIdx.x + i * C::NT;
    const int b = e % C::SB;
    const int tl = (e / C::SB) % C::SB;
    const int r = e / (C::SB * C::SB);
    buf[(r * C::SB + b) * C::LD + tl] = stage[i];
  }
  __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(ClCfg<N>::NT, 1) k_spatial_cluster(SpatialArgs a) {
  using C = ClCfg<N>;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  unsigned char* raw = smem_raw + C::DATA;
  const int c = int(cluster.block_rank());
  const int ncl = gridDim.x / C::CL;
  const int cid = blockIdx.x / C::CL;
  const int bpp = a.in_kind == IN_U8 ? 1 : 2;
  const bool fresnel = a.spatial == HV_SPATIAL_FRESNEL;
  const int x0 = c * C::SB;

  if (cid < int(a.n)) fetch_raw<N>(a, raw, (a.raw.slot0 + cid) % a.raw.cap, c, bpp);
  for (int f = cid; f < int(a.n); f += ncl) {
    cpa_wait();
    __syncthreads();
    // 1. convert (+ chirp) into buf[y][b], b = column within the strip
    for (int e = threadIdx.x; e < N * C::SB; e += C::NT) {
      const int y = e / C::SB, b = e % C::SB;
      const float v = bpp == 1 ? float(raw[y * C::SB + b])
                               : float(reinterpret_cast<const uint16_t*>(raw)[y * C::SB + b]);
      float2 u = make_float2(v, 0.f);
      if (fresnel) u = cscale(cmul(__ldg(&a.chirp_y[y]), __ldg(&a.chirp_x[x0 + b])), v);
      buf[y * C::LD + b] = u;
    }
    __syncthreads();
    // prefetch the next frame's raw strip (raw buffer is free now)
    if (f + ncl < int(a.n)) fetch_raw<N>(a, raw, (a.raw.slot0 + f + ncl) % a.raw.cap, c, bpp);
    StoreSmem<C::LD> st{buf};
    fft_lines<N, -1, C::SB, C::NT, C::LD>(buf, a.tw_h, st);
    __syncthreads();
    cluster.sync();
    exchange<N>(cluster, buf, c);  // now buf[x][b] = F[ky = x0 + b][x]
    float2* tq = static_cast<float2*>(a.tq.base) + ((a.tq.slot0 + f) % a.tq.cap) * size_t(N) * N;
    if (fresnel) {
      fft_lines<N, -1, C::SB, C::NT, C::LD>(buf, a.tw_w, st);
      __syncthreads();
      // rows ky = x0 + b to the queue, coalesced along kx
      for (int e = threadIdx.x; e < N * C::SB; e += C::NT) {
        const int k = e % N, b = e / N;
        tq[size_t(x0 + b) * N + k] = buf[k * C::LD + b];
      }
    } else {
      AspMulStore<C::LD> mul{buf, a.asp_ht, uint32_t(N), uint32_t(x0)};
      fft_lines<N, -1, C::SB, C::NT, C::LD>(buf, a.tw_w, mul);
      __syncthreads();
      fft_lines<N, +1, C::SB, C::NT, C::LD>(buf, a.tw_w, st);
      __syncthreads();
      cluster.sync();
      exchange<N>(cluster, buf, c);  // buf[ky][b] = G[ky][x = x0 + b]
      StoreTqCols out{tq, uint32_t(N), uint32_t(x0)};
      fft_lines<N, +1, C::SB, C::NT, C::LD>(buf, a.tw_h, out);
    }
    // No barrier needed here: remote buffers are read only inside the next
    // frame's exchange, which every CTA reaches after a cluster barrier.
  }
  cpa_wait();
}

template <int N>
static cudaError_t launch_cl(const SpatialArgs& a, cudaStream_t s, int* launches) {
  using C = ClCfg<N>;
  auto kern = k_spatial_cluster<N>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM));
  if (e != cudaSuccess) return e;
  if (C::CL > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C::CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(C::NT);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int max_clusters = 0;
  cfg.gridDim = dim3(C::CL);
  e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (max_clusters < 1) return cudaErrorInvalidConfiguration;
  const int ncl = int(a.n) < max_clusters ? int(a.n) : max_clusters;
  cfg.gridDim = dim3(ncl * C::CL);
  e = cudaLaunchKernelEx(&cfg, kern, a);
  ++*launches;
  return e;
}

bool spatial_cluster_supported(const SpatialArgs& a) {
  return a.W == a.H && (a.spatial == HV_SPATIAL_ASP || a.spatial == HV_SPATIAL_FRESNEL) &&
         (a.W == 128 || a.W == 256 || a.W == 512);
}

cudaError_t launch_spatial_cluster(const SpatialArgs& a, cudaStream_t s, int* launches) {
  if (a.n == 0) return cudaSuccess;
  switch (a.W) {
    case 128: return launch_cl<128>(a, s, launches);
    case 256: return launch_cl<256>(a, s, launches);
    case 512: return launch_cl<512>(a, s, launches);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hv
