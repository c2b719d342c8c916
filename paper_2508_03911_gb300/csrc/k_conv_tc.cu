// k_conv_tc.cu -- the 3 x 3, stride-2 convolutions of the autofocus network with
// 16 or more input channels, on the 5th-generation tensor cores (tcgen05.mma,
// accumulator in tensor memory): an implicit GEMM per tile of 128 output pixels.
//
//   D[p][o] = sum_k A[p][k] B[o][k],  k = t CI + c  (tap t = 3 di + dj, channel c),
//   A[p][k] = x[n][c][2i+di-1][2j+dj-1] (0 outside the image), B[o][k] = w[o][c][t],
//   y[n][o][i][j] = bf16(relu(D[p][o] + b[o])),  p = (n, i, j) flattened.
//
// bfloat16 operands, float32 accumulation (as the CUDA-core forward). A CTA keeps
// all weights (B, CO x 9 CI) in shared memory and walks tiles of 128 output
// pixels; per tile it gathers the 9 taps one at a time (128 pixels x CI channels,
// no-swizzle K-major core matrices) into two alternating buffers, and one thread
// issues the tap's K = CI / 16 MMAs and commits them to the buffer's mbarrier,
// so gathering tap t + 1 overlaps the MMAs of tap t. Every mbarrier wait is
// bounded; on timeout the kernel records an error, stops and releases its tensor
// memory.
#include <cuda_bf16.h>

#include "cnn_internal.h"

namespace hv {
namespace cnn {

namespace {

constexpr int CT_NT = 128;  // 4 warps; in the epilogue warp w reads TMEM lanes 32 w .. 32 w + 31
constexpr int CT_M = 128;   // output pixels per tile (MMA M)

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// no-swizzle K-major descriptor: start >> 4, LBO = 128 B (next core matrix along K)
// at bit 16, SBO (next 8-row group) at bit 32, version 1 at bit 46
__device__ __forceinline__ uint64_t kdesc(uint32_t addr, uint32_t sbo) {
  return uint64_t((addr & 0x3FFFF) >> 4) | (uint64_t(128 >> 4) << 16) | (uint64_t(sbo >> 4) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: F32 accumulator, BF16 A and B, both K-major
__device__ __forceinline__ uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

// Bounded wait (about 2^32 clocks) for the completion of phase `parity` of an mbarrier.
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity) {
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

__device__ __forceinline__ uint32_t pack(uint16_t lo, uint16_t hi) { return uint32_t(lo) | (uint32_t(hi) << 16); }

// core-matrix offset of element (row, k) in a K-major tile whose 8-row groups are sbo apart
__device__ __forceinline__ int cm_off(int row, int kgroup, int sbo) { return (row >> 3) * sbo + kgroup * 128 + (row & 7) * 16; }

template <int CI, int CO, int HI>
struct ConvTc {
  static_assert(CI % 16 == 0 && CO % 16 == 0 && CO >= 16 && CO <= 256, "tensor-core shapes");
  static constexpr int HO = HI / 2, K = 9 * CI;
  static constexpr int SBO_A = (CI / 8) * 128, SBO_B = (K / 8) * 128;
  static constexpr int A_BYTES = CT_M * CI * 2;  // one tap of a tile
  static constexpr int B_BYTES = CO * K * 2;     // all weights
  static constexpr int SMEM = B_BYTES + 2 * A_BYTES;
  static constexpr uint32_t TMEM_COLS = CO <= 32 ? 32 : (CO <= 64 ? 64 : (CO <= 128 ? 128 : 256));
};

template <int CI, int CO, int HI>
__global__ void __launch_bounds__(CT_NT) k_conv_tc(const __nv_bfloat16* __restrict__ x,
                                                   const __nv_bfloat16* __restrict__ w,
                                                   const float* __restrict__ bias, __nv_bfloat16* __restrict__ y,
                                                   int npix, unsigned* err) {
  using G = ConvTc<CI, CO, HI>;
  constexpr int HO = G::HO;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_ok;
  unsigned char* Bs = sm;
  unsigned char* As0 = sm + G::B_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint16_t* xr = reinterpret_cast<const uint16_t*>(x);
  const uint16_t* wr = reinterpret_cast<const uint16_t*>(w);

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_slot)),
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  // weights: B[o][k = t CI + c] = w[o][c][t], 8 consecutive k (channels of one tap) per 16 bytes
  for (int e = tid; e < CO * (G::K / 8); e += CT_NT) {
    const int o = e / (G::K / 8), kg = e % (G::K / 8);
    const int t = (kg * 8) / CI, c0 = (kg * 8) % CI;
    uint16_t v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = wr[(size_t(o) * CI + c0 + q) * 9 + t];
    *reinterpret_cast<uint4*>(Bs + cm_off(o, kg, G::SBO_B)) =
        make_uint4(pack(v[0], v[1]), pack(v[2], v[3]), pack(v[4], v[5]), pack(v[6], v[7]));
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t id = idesc(CT_M, CO);
  const uint32_t bs = su32(Bs), as0 = su32(As0);
  bool ok = true;
  uint32_t q = 0;  // taps issued so far: tap q used buffer q & 1 and completes phase q >> 1 of its mbarrier
  const int ntiles = (npix + CT_M - 1) / CT_M;

  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int p = tile * CT_M + tid;  // this thread's output pixel = row of A and D
    const bool valid = p < npix;
    const int n = p / (HO * HO), rem = p % (HO * HO), i = rem / HO, j = rem % HO;
    for (int t = 0; t < 9; ++t, ++q) {
      const uint32_t b = q & 1;
      if (q >= 2) {  // the MMAs that last read this buffer are done
        if (tid == 0) s_ok = wait_phase(su32(&mbar[b]), ((q >> 1) - 1) & 1) ? 1 : 0;
        __syncthreads();
        ok = s_ok != 0;
        if (!ok) break;
      }
      const int yy = 2 * i + t / 3 - 1, xx = 2 * j + t % 3 - 1;
      const bool in = valid && yy >= 0 && yy < HI && xx >= 0 && xx < HI;
      const uint16_t* src = xr + ((size_t(n) * CI) * HI + (in ? yy : 0)) * HI + (in ? xx : 0);
      unsigned char* At = As0 + b * G::A_BYTES;
#pragma unroll
      for (int cg = 0; cg < CI / 8; ++cg) {
        uint16_t v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = in ? src[size_t(cg * 8 + c) * HI * HI] : uint16_t(0);
        *reinterpret_cast<uint4*>(At + cm_off(tid, cg, G::SBO_A)) =
            make_uint4(pack(v[0], v[1]), pack(v[2], v[3]), pack(v[4], v[5]), pack(v[6], v[7]));
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t at = as0 + b * G::A_BYTES;
#pragma unroll
        for (int s = 0; s < CI / 16; ++s)
          mma(tmem, kdesc(at + 256 * s, G::SBO_A), kdesc(bs + (t * CI / 8 + 2 * s) * 128, G::SBO_B), id,
              (t > 0 || s > 0) ? 1u : 0u);
        commit(su32(&mbar[b]));
      }
    }
    if (!ok) break;
    // the last tap's commit covers every MMA of the tile
    if (tid == 0) s_ok = wait_phase(su32(&mbar[(q - 1) & 1]), ((q - 1) >> 1) & 1) ? 1 : 0;
    __syncthreads();
    ok = s_ok != 0;
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
    for (int c0 = 0; c0 < CO; c0 += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
          "%12, %13, %14, %15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + (uint32_t(32 * warp) << 16) + uint32_t(c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (valid) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int o = c0 + k;
          const float r = fmaxf(__uint_as_float(v[k]) + __ldg(&bias[o]), 0.f);
          y[((size_t(n) * CO + o) * HO + i) * HO + j] = __float2bfloat16_rn(r);
        }
      }
    }
    // every thread's TMEM reads are done before the next tile's first MMA overwrites D
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
  }
  if (!ok && tid == 0) atomicOr(err, 4u);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(G::TMEM_COLS) : "memory");
  }
}

}  // namespace

template <int CI, int CO, int HI>
cudaError_t conv_tc(const __nv_bfloat16* x, const __nv_bfloat16* w, const float* bias, __nv_bfloat16* y,
                    uint32_t n, unsigned* err, cudaStream_t s) {
  using G = ConvTc<CI, CO, HI>;
  auto kern = k_conv_tc<CI, CO, HI>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // CTAs per SM: as many as shared memory holds (the hardware places them), at most
  // as many as share the SM's 512 tensor-memory columns
  const int by_smem = int((228 * 1024) / (G::SMEM + 2048));
  const int by_tmem = int(512 / G::TMEM_COLS);
  const int per_sm = by_smem < by_tmem ? by_smem : by_tmem;
  const int npix = int(n) * G::HO * G::HO;
  const int ntiles = (npix + CT_M - 1) / CT_M;
  int grid = (per_sm > 0 ? per_sm : 1) * nsm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  kern<<<grid, CT_NT, G::SMEM, s>>>(x, w, bias, y, npix, err);
  return cudaGetLastError();
}

template cudaError_t conv_tc<16, 32, 64>(const __nv_bfloat16*, const __nv_bfloat16*, const float*, __nv_bfloat16*,
                                         uint32_t, unsigned*, cudaStream_t);
template cudaError_t conv_tc<32, 64, 32>(const __nv_bfloat16*, const __nv_bfloat16*, const float*, __nv_bfloat16*,
                                         uint32_t, unsigned*, cudaStream_t);
template cudaError_t conv_tc<64, 64, 16>(const __nv_bfloat16*, const __nv_bfloat16*, const float*, __nv_bfloat16*,
                                         uint32_t, unsigned*, cudaStream_t);

}  // namespace cnn
}  // namespace hv
