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
  // N <= 256: two strip buffers per CTA (exchange reads remote rows straight
  // into the other buffer); N = 512: one buffer, exchange staged in registers.
  static constexpr bool DB = N <= 256;
  static constexpr int CL = N == 128 ? 2 : (N == 256 ? 8 : 16);
  static constexpr int SB = N / CL;          // lines per CTA
  static constexpr int LD = SB + 1;          // padded: transposed accesses conflict-free
  static constexpr int NT = 512;
  static constexpr size_t DATA = size_t(N) * LD * sizeof(float2);
  static constexpr size_t RAW = size_t(N) * SB * 2;  // uint16 worst case
  static constexpr size_t SMEM = (DB ? 2 : 1) * DATA + RAW;
};

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

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

// Move the frame between strip layouts (a transpose across the cluster). Every
// CTA holds its SB lines as buf[t * LD + b]; afterwards CTA c holds, as its SB
// lines of the other orientation, element t = c SB + tl of line r SB + b of
// CTA r, at buf[(r SB + b) * LD + tl]. All remote reads go to registers first,
// then a cluster barrier, then the local writes (the buffer is reused in place).
// 32-bit address of `p` (this CTA's shared memory) in CTA `rank`'s shared window.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, int rank) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 ld_cluster(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}

template <int N>
__device__ __forceinline__ void exchange(cg::cluster_group& cluster, const float2* src_buf,
                                         float2* dst_buf, int c) {
  using C = ClCfg<N>;
  constexpr int QN = C::NT / C::SB;   // thread groups per source column
  constexpr int PER = C::SB / QN;     // lines gathered per thread per source CTA
  static_assert(C::NT % C::SB == 0 && C::SB % QN == 0, "exchange layout");
  const int b = threadIdx.x % C::SB, q = threadIdx.x / C::SB;
  const int own0 = c * C::SB;
  const float2* mine = src_buf + (own0 + q) * C::LD + b;
  float2* dst = dst_buf + b * C::LD + q;
  cluster.sync();  // every CTA's source strip is complete
  if constexpr (C::DB) {
    // separate destination: copy through registers one value at a time
#pragma unroll
    for (int r = 0; r < C::CL; ++r) {
      const uint32_t src = cluster_addr(mine, r);
#pragma unroll
      for (int s = 0; s < PER; ++s)
        dst[r * C::SB * C::LD + s * QN] = ld_cluster(src + uint32_t(s * QN * C::LD * sizeof(float2)));
    }
  } else {
    float2 stage[C::CL][PER];
#pragma unroll
    for (int r = 0; r < C::CL; ++r) {
      const uint32_t src = cluster_addr(mine, r);
#pragma unroll
      for (int s = 0; s < PER; ++s) stage[r][s] = ld_cluster(src + uint32_t(s * QN * C::LD * sizeof(float2)));
    }
    cluster.sync();  // all reads of the (shared) buffer done before it is overwritten
#pragma unroll
    for (int r = 0; r < C::CL; ++r)
#pragma unroll
      for (int s = 0; s < PER; ++s) dst[r * C::SB * C::LD + s * QN] = stage[r][s];
  }
  __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(ClCfg<N>::NT, 1) k_spatial_cluster(SpatialArgs a) {
  using C = ClCfg<N>;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);                     // column strips
  float2* buf2 = C::DB ? reinterpret_cast<float2*>(smem_raw + C::DATA) : buf;  // row strips
  unsigned char* raw = smem_raw + (C::DB ? 2 : 1) * C::DATA;
  const int c = int(cluster.block_rank());
  const int ncl = gridDim.x / C::CL;
  const int cid = blockIdx.x / C::CL;
  const int bpp = a.in_kind == IN_U8 ? 1 : 2;
  const bool fresnel = a.spatial == HV_SPATIAL_FRESNEL;
  const int x0 = c * C::SB;

  if (cid < int(a.n)) fetch_raw<N>(a, raw, (a.raw.slot0 + cid) % a.raw.cap, c, bpp);
  // Double-buffered strips: a CTA may refill `buf` for the next frame only after
  // every CTA has finished reading it remotely (split barrier: arrive after the
  // last exchange of a frame, wait before the next frame's conversion).
  if constexpr (C::DB) cluster_arrive();
  for (int f = cid; f < int(a.n); f += ncl) {
    cpa_wait();
    if constexpr (C::DB) cluster_wait();
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
    exchange<N>(cluster, buf, buf2, c);  // buf2[x][b] = F[ky = x0 + b][x]
    float2* tq = static_cast<float2*>(a.tq.base) + ((a.tq.slot0 + f) % a.tq.cap) * size_t(N) * N;
    StoreSmem<C::LD> st2{buf2};
    if (fresnel) {
      if constexpr (C::DB) cluster_arrive();  // done reading remote column strips
      fft_lines<N, -1, C::SB, C::NT, C::LD>(buf2, a.tw_w, st2);
      __syncthreads();
      // rows ky = x0 + b to the queue, coalesced along kx
      for (int e = threadIdx.x; e < N * C::SB; e += C::NT) {
        const int k = e % N, b = e / N;
        tq[size_t(x0 + b) * N + k] = buf2[k * C::LD + b];
      }
    } else {
      AspMulStore<C::LD> mul{buf2, a.asp_ht, uint32_t(N), uint32_t(x0)};
      fft_lines<N, -1, C::SB, C::NT, C::LD>(buf2, a.tw_w, mul);
      __syncthreads();
      fft_lines<N, +1, C::SB, C::NT, C::LD>(buf2, a.tw_w, st2);
      __syncthreads();
      exchange<N>(cluster, buf2, buf, c);  // buf[ky][b] = G[ky][x = x0 + b]
      if constexpr (C::DB) cluster_arrive();  // done reading remote row strips
      StoreTqCols out{tq, uint32_t(N), uint32_t(x0)};
      fft_lines<N, +1, C::SB, C::NT, C::LD>(buf, a.tw_h, out);
    }
  }
  // no CTA may exit while another can still read its shared memory
  if constexpr (C::DB) cluster_wait();
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
