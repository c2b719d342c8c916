// k_cov_tc.cu -- PCA covariance C = X^H X on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), BF16 or split-BF16 inputs with
// FP32 accumulation (covariance of the window, Sec. III-B.1).
//
// The complex Gram matrix is a real one: with Y the 2T x P matrix whose rows
// 2a and 2a+1 are the real and imaginary parts of frame a, G = Y Y^T and
//   Re C[a][b] = G[2a][2b] + G[2a+1][2b+1],  Im C[a][b] = G[2a][2b+1] - G[2a+1][2b].
// A CTA computes one 128 x N tile of G (rows: 64 frames, columns: N/2 frames,
// N = 2 min(T, 128)) over one pixel chunk; tiles wholly below the diagonal are
// skipped; chunk partials are summed in float64 by k_cov_tc_reduce.
//
// A first kernel converts the window once: each value v becomes hi = bf16(v) and
// lo = bf16(v - hi), stored in a staging buffer in the no-swizzle K-major
// canonical layout of the MMA operands (8 x 16-byte core matrices, element (r, k)
// of a 64-pixel step at (r/8)*1024 + (k/8)*128 + (r%8)*16 + (k%8)*2 bytes:
// leading-dimension byte offset 128 along K, stride-dimension byte offset 1024
// along rows), so every tile of consecutive rows of a step is one contiguous
// chunk. The covariance kernel then streams those chunks into shared memory with
// 1-D bulk copies (one thread, two stages on mbarriers) while another thread
// issues four K = 16 MMAs per product -- hi.hi (BF16), plus hi.lo and lo.hi
// (split-BF16) -- per step. Every mbarrier wait is bounded; on timeout the kernel
// records an error, stops issuing, releases its tensor memory and returns.
#include <cuda_bf16.h>

#include "hv_internal.h"
#include "../../include/hv.h"

namespace hv {

namespace {

constexpr int TC_NT = 512;
constexpr int TC_KS = 64;                          // pixels per step
constexpr int TC_M = 128;                          // G rows per tile (64 frames)
constexpr int A_BYTES = TC_M * TC_KS * 2;          // 16 KB per A tile (hi or lo)
constexpr int B_BYTES_MAX = 256 * TC_KS * 2;       // 32 KB per B tile (hi or lo)
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES_MAX;  // 96 KB
constexpr int TC_SMEM = 2 * STAGE_BYTES;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// no-swizzle K-major descriptor: start >> 4, LBO >> 4 at 16, SBO >> 4 at 32, version 1 at 46
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return uint64_t((addr & 0x3FFFF) >> 4) | (uint64_t(128 >> 4) << 16) | (uint64_t(1024 >> 4) << 32) |
         (1ull << 46);
}

// kind::f16 instruction descriptor: F32 accumulator, BF16 A and B, both K-major
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

// Bounded wait for the completion of phase `parity` of an mbarrier.
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

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return uint32_t(__bfloat16_as_ushort(a)) | (uint32_t(__bfloat16_as_ushort(b)) << 16);
}

__device__ __forceinline__ int tile_off(int r, int kb) { return (r >> 3) * 1024 + kb * 128 + (r & 7) * 16; }

// Load 8 consecutive pixels of `frame` (zero past p_end), split into bf16 hi/lo,
// and store rows 2f (re) and 2f+1 (im) of the hi and lo tiles.
__device__ __forceinline__ void convert8(const float2* frame, size_t p, size_t p_end, int f, int kb,
                                         unsigned char* hi_tile, unsigned char* lo_tile) {
  float re[8], im[8];
  if (p + 8 <= p_end) {
    const float4* q = reinterpret_cast<const float4*>(frame + p);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 v = __ldg(q + i);
      re[2 * i] = v.x;
      im[2 * i] = v.y;
      re[2 * i + 1] = v.z;
      im[2 * i + 1] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 v = p + i < p_end ? frame[p + i] : make_float2(0.f, 0.f);
      re[i] = v.x;
      im[i] = v.y;
    }
  }
  uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat16 a0 = __float2bfloat16_rn(re[2 * i]), a1 = __float2bfloat16_rn(re[2 * i + 1]);
    const __nv_bfloat16 b0 = __float2bfloat16_rn(im[2 * i]), b1 = __float2bfloat16_rn(im[2 * i + 1]);
    rh[i] = pack2(a0, a1);
    ih[i] = pack2(b0, b1);
    rl[i] = pack2(__float2bfloat16_rn(re[2 * i] - __bfloat162float(a0)),
                  __float2bfloat16_rn(re[2 * i + 1] - __bfloat162float(a1)));
    il[i] = pack2(__float2bfloat16_rn(im[2 * i] - __bfloat162float(b0)),
                  __float2bfloat16_rn(im[2 * i + 1] - __bfloat162float(b1)));
  }
  const int o_re = tile_off(2 * f, kb), o_im = tile_off(2 * f + 1, kb);
  *reinterpret_cast<uint4*>(hi_tile + o_re) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
  *reinterpret_cast<uint4*>(hi_tile + o_im) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
  if (lo_tile) {
    *reinterpret_cast<uint4*>(lo_tile + o_re) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
    *reinterpret_cast<uint4*>(lo_tile + o_im) = make_uint4(il[0], il[1], il[2], il[3]);
  }
}

// The window as BF16 operands in the staging buffer: item (step, frame, k block)
// converts 8 pixels of one frame (zero past the last pixel) into rows 2f (re) and
// 2f + 1 (im) of the step's core-matrix block -- the layout of an MMA tile in
// shared memory, so a tile of consecutive rows is one contiguous chunk. A warp
// covers 4 frames x 8 k blocks: 2 KB of reads, 1 KB contiguous per part written.
__global__ void __launch_bounds__(256) k_cov_stage(PcaArgs a) {
  const size_t hw = size_t(a.W) * a.H;
  const uint32_t T = a.T;
  const size_t nsteps = (hw + TC_KS - 1) / TC_KS;
  const size_t total = nsteps * T * 8;
  const bool split = a.precision == HV_PREC_SPLIT_BF16;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total;
       idx += size_t(gridDim.x) * blockDim.x) {
    const int kb = int(idx & 7);
    const uint32_t f = uint32_t((idx >> 3) % T);
    const size_t st = (idx >> 3) / T;
    uint32_t slot = a.tq.slot0 + f;  // slot0 < cap, f < T <= cap
    if (slot >= a.tq.cap) slot -= a.tq.cap;
    const float2* fp = static_cast<const float2*>(a.tq.base) + size_t(slot) * hw;
    unsigned char* hi = reinterpret_cast<unsigned char*>(a.tc_stage + st * 2 * T * TC_KS);
    unsigned char* lo = split ? reinterpret_cast<unsigned char*>(a.tc_stage + a.tc_stage_part + st * 2 * T * TC_KS)
                              : nullptr;
    convert8(fp, st * TC_KS + size_t(kb) * 8, hw, int(f), kb, hi, lo);
  }
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// One 128 x N tile of G over one pixel chunk. Warp 0 (one thread) streams each
// 64-pixel step's operand tiles from the staging buffer into one of two stages
// with 1-D bulk copies completing on the stage's `full` mbarrier; warp 1 (one
// thread) waits for a stage, issues its MMAs and commits them to the stage's
// `empty` mbarrier, which the copies of the stage's next step wait for.
__global__ void __launch_bounds__(TC_NT, 1) k_cov_tc(PcaArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t full[2], empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_ok;  // outcome of the waits, one value every thread agrees on
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ti = a.tc_tile_i[blockIdx.x], tj = a.tc_tile_j[blockIdx.x];
  const int BF = int(a.T) < 128 ? int(a.T) : 128;  // frames per B block
  const int N = 2 * BF;                             // G columns per tile
  const uint32_t B_BYTES = uint32_t(N) * TC_KS * 2;
  const bool split = a.precision == HV_PREC_SPLIT_BF16;
  const size_t hw = size_t(a.W) * a.H;
  const size_t p_begin = size_t(blockIdx.y) * a.tc_chunk;
  const size_t p_end = p_begin + a.tc_chunk < hw ? p_begin + a.tc_chunk : hw;
  const int nsteps = int((p_end - p_begin + TC_KS - 1) / TC_KS);
  const size_t step0 = p_begin / TC_KS;
  const size_t step_elems = size_t(2) * a.T * TC_KS;

  if (tid == 0) {
    for (int st = 0; st < 2; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[st])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[st])) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_ok = 1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(
                     smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t id = idesc_bf16(TC_M, N);

  if (tid == 0) {
    // copies: A rows 128 ti .., B rows N tj .. of each step, hi and (split) lo parts
    const uint32_t bytes = (uint32_t(A_BYTES) + B_BYTES) * (split ? 2u : 1u);
    for (int it = 0; it < nsteps; ++it) {
      const int st = it & 1;
      if (it >= 2 && !mbar_wait(smem_u32(&empty[st]), uint32_t(((it >> 1) - 1) & 1))) {
        atomicOr(a.err, 1u);
        s_ok = 0;
        break;
      }
      unsigned char* stg = sm + st * STAGE_BYTES;
      const uint32_t fb = smem_u32(&full[st]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(bytes) : "memory");
      const uint16_t* hi = a.tc_stage + (step0 + size_t(it)) * step_elems;
      bulk_load(smem_u32(stg), hi + size_t(ti) * TC_M * TC_KS, A_BYTES, fb);
      bulk_load(smem_u32(stg + 2 * A_BYTES), hi + size_t(tj) * N * TC_KS, B_BYTES, fb);
      if (split) {
        const uint16_t* lo = hi + a.tc_stage_part;
        bulk_load(smem_u32(stg + A_BYTES), lo + size_t(ti) * TC_M * TC_KS, A_BYTES, fb);
        bulk_load(smem_u32(stg + 2 * A_BYTES + B_BYTES_MAX), lo + size_t(tj) * N * TC_KS, B_BYTES, fb);
      }
    }
  } else if (tid == 32) {
    bool ok = true;
    for (int it = 0; it < nsteps; ++it) {
      const int st = it & 1;
      if (!mbar_wait(smem_u32(&full[st]), uint32_t((it >> 1) & 1))) {
        atomicOr(a.err, 1u);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      unsigned char* stg = sm + st * STAGE_BYTES;
      const uint32_t ahi = smem_u32(stg), alo = smem_u32(stg + A_BYTES), bhi = smem_u32(stg + 2 * A_BYTES),
                     blo = smem_u32(stg + 2 * A_BYTES + B_BYTES_MAX);
#pragma unroll
      for (int k = 0; k < TC_KS / 16; ++k) {
        const uint32_t kofs = uint32_t(k * 256);  // two core matrices along K
        mma_bf16(tmem, smem_desc(ahi + kofs), smem_desc(bhi + kofs), id, (it > 0 || k > 0) ? 1u : 0u);
        if (split) {
          mma_bf16(tmem, smem_desc(ahi + kofs), smem_desc(blo + kofs), id, 1u);
          mma_bf16(tmem, smem_desc(alo + kofs), smem_desc(bhi + kofs), id, 1u);
        }
      }
      mma_commit(smem_u32(&empty[st]));
    }
    // the last commit covers every MMA issued before it
    if (ok && nsteps > 0 &&
        !mbar_wait(smem_u32(&empty[(nsteps - 1) & 1]), uint32_t(((nsteps - 1) >> 1) & 1))) {
      atomicOr(a.err, 1u);
      ok = false;
    }
    if (!ok) s_ok = 0;
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok) {
    // warp w reads TMEM lanes 32 (w % 4) .. +31 (G rows), columns chunk (w / 4) of N/4
    const int sub = warp & 3, q = warp >> 2;
    const int row = 32 * sub + lane;
    const int ncol = N / 4;
    float* out = a.tc_partials + (size_t(blockIdx.y) * gridDim.x + blockIdx.x) * TC_M * 256 + size_t(row) * 256;
    for (int c0 = q * ncol; c0 < (q + 1) * ncol; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + (uint32_t(32 * sub) << 16) + uint32_t(c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
          "%12, %13, %14, %15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
            "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int i = 0; i < 16; i += 4)
        *reinterpret_cast<float4*>(out + c0 + i) =
            make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]), __uint_as_float(v[i + 2]),
                        __uint_as_float(v[i + 3]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem) : "memory");
  }
}

// C from the chunk partials of G (float64 sums); V = I; largest diagonal.
__global__ void k_cov_tc_reduce(PcaArgs a) {
  const int T = int(a.T), BF = T < 128 ? T : 128, ntiles = int(a.tc_ntiles);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < T * T; e += gridDim.x * blockDim.x) {
    const int r = e / T, c = e % T;
    a.V[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    if (r > c) continue;
    const int ti = r / 64, tj = c / BF;
    int t = 0;
    while (t < ntiles && !(a.tc_tile_i[t] == ti && a.tc_tile_j[t] == tj)) ++t;
    if (t == ntiles) continue;  // unreachable: every upper-triangle (r, c) lies in a listed tile
    const int lr = 2 * (r - 64 * ti), lc = 2 * (c - BF * tj);
    double g00 = 0, g11 = 0, g01 = 0, g10 = 0;
    for (uint32_t k = 0; k < a.tc_nchunks; ++k) {
      const float* P = a.tc_partials + (size_t(k) * ntiles + t) * TC_M * 256;
      g00 += P[lr * 256 + lc];
      g11 += P[(lr + 1) * 256 + lc + 1];
      g01 += P[lr * 256 + lc + 1];
      g10 += P[(lr + 1) * 256 + lc];
    }
    const double re = g00 + g11;
    const double im = r == c ? 0.0 : g01 - g10;
    if (r == c)
      atomicMax(reinterpret_cast<unsigned long long*>(a.cmax),
                static_cast<unsigned long long>(__double_as_longlong(re > 0.0 ? re : 0.0)));
    a.C[r * T + c] = make_double2(re, im);
    a.C[c * T + r] = make_double2(re, -im);
  }
}

}  // namespace

size_t cov_tc_partials_floats(uint32_t ntiles, uint32_t nchunks) { return size_t(ntiles) * nchunks * TC_M * 256; }

// Tile list of the upper triangle: A blocks of 64 frames, B blocks of min(T, 128).
uint32_t cov_tc_tiles(uint32_t T, uint8_t* ti, uint8_t* tj) {
  const uint32_t BF = T < 128 ? T : 128;
  uint32_t n = 0;
  for (uint32_t i = 0; i < T / 64; ++i)
    for (uint32_t j = 0; j < T / BF; ++j)
      if (64 * i <= BF * j + BF - 1) {
        ti[n] = uint8_t(i);
        tj[n] = uint8_t(j);
        ++n;
      }
  return n;
}

cudaError_t launch_cov_tc(PcaArgs& a, cudaStream_t s, int* launches) {
  if (!a.tc_stage) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_cov_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  k_cov_stage<<<unsigned(nsm) * 8, 256, 0, s>>>(a);
  k_cov_tc<<<dim3(a.tc_ntiles, a.tc_nchunks), TC_NT, TC_SMEM, s>>>(a);
  k_cov_tc_reduce<<<(a.T * a.T + 255) / 256, 256, 0, s>>>(a);
  *launches += 3;
  return cudaGetLastError();
}

}  // namespace hv
