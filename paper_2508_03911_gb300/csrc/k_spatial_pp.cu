// k_spatial_pp.cu -- the spatial transform (Sec. III-B.1) as persistent kernels, one
// per pass, that prefetch their next work item and keep the integer work per
// pixel small.
//
// A CTA stays resident and loops over work items (frame, strip of 16 lines of
// the pass; 8 at line length 1024). While it transforms one item, the input of its next item streams
// into a second buffer with cp.async. Each pass reads its input in whatever
// order makes the global loads coalesced and writes its output straight from
// the registers of the last FFT stage; the intermediate layouts are chosen so
// that those stores are coalesced too (lanes of a warp hold 16 neighbouring
// lines):
//   P1  column FFT (length H) of 16 columns: the first FFT stage reads the raw
//       strip (uint8/uint16, staged by cp.async) and converts it in registers
//       (Fresnel: times the chirp) -> S1[ky][x]
//   P2a row FFT (length W) of 16 rows ky of S1, x H^T (1/(WH) and the optional
//       high-pass folded in), row IFFT -> S2[x][ky]
//   P3a column IFFT (length H) of 16 columns x of S2 -> time queue [y][x]
//   P2f row FFT of 16 rows ky of S1 -> time queue [ky][kx]; its last stage maps
//       threads along kx (twiddles from a per-stage table), so the store of
//       each row is coalesced straight from registers
//   P3t as P3a, but instead of storing the field it adds sum |u| and sum |u|^2 of
//       the strip to the frame's two float64 accumulators (focus sweep)
// Twiddles of the pass length are copied to shared memory once per CTA. In the
// full transform the intermediates S1 and S2 are read exactly once: once a strip
// is staged, its L2 lines are discarded (no write-back of dead data when a
// chunk's intermediates fit in L2). Single passes (the focus sweep re-reads S1
// for every distance) keep them.
#include <cuda.h>

#include "fft_dev.cuh"
#include "hv_internal.h"
#include "../../include/hv.h"

namespace hv {

namespace {

constexpr int PP_BT = 16;
enum { PK_P1 = PASS_COL_FFT, PK_P2A = PASS_ROW_ASP, PK_P3A = PASS_COL_IFFT, PK_P2F = PASS_ROW_FFT,
       PK_P3T = PASS_COL_IFFT_TAMURA, PK_P2C = PASS_ROW_CELLS };

// Lines per strip: 16, or 8 at L = 1024 (two buffers of 16 lines would not fit).
template <int L>
struct PpCfg {
  static constexpr int BT = L >= 1024 ? 8 : PP_BT;
  static constexpr int NT = FftThreads<L, BT>::value;  // L for 64 <= L <= 512, 512 at 1024
  static constexpr int LD = BT + 1;
  static constexpr size_t BUF = size_t(L) * LD * sizeof(float2);
  static constexpr size_t RAW = size_t(L) * BT * 2;    // one uint16 strip
  static constexpr size_t TW = size_t(L) * sizeof(float2);
  static_assert(L % NT == 0 && NT % BT == 0, "threads cover the elements of a line");
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

// ------------------------------------------------ stage inputs and epilogues

// Element t of line b from the FFT buffer.
template <int LD>
struct SmemSrc {
  static constexpr bool kAliasesBuf = true;
  const float2* buf;
  __device__ __forceinline__ float2 operator()(int t, int b) const { return buf[t * LD + b]; }
};

// Element t (row y) of column b from a staged raw strip [y][BT], converted to
// complex; with the Fresnel chirp cy[y] * cx (cx: this thread's column factor).
template <bool U8, bool CHIRP, int BT, bool ALIAS = false>
struct RawSrc {
  static constexpr bool kAliasesBuf = ALIAS;  // staged inside the FFT buffer: read all before writing
  const unsigned char* raw;
  const float2* cy;
  float2 cx;
  __device__ __forceinline__ float2 operator()(int t, int b) const {
    const float v = U8 ? float(raw[t * BT + b]) : float(reinterpret_cast<const uint16_t*>(raw)[t * BT + b]);
    if constexpr (CHIRP) return cscale(cmul(cy[t], cx), v);
    return make_float2(v, 0.f);
  }
};

// Two real raw columns as one complex line: line b of the strip is columns 2b
// (real part) and 2b + 1 (imaginary part); 32 columns staged, rows 32 pixels apart.
template <bool U8>
struct PackedRawSrc {
  static constexpr bool kAliasesBuf = true;  // staged inside the FFT buffer: read all before writing
  const unsigned char* raw;
  __device__ __forceinline__ float2 operator()(int t, int b) const {
    if constexpr (U8) {
      const uint16_t p = reinterpret_cast<const uint16_t*>(raw)[t * 16 + b];
      return make_float2(float(p & 0xffu), float(p >> 8));
    } else {
      const uint32_t p = reinterpret_cast<const uint32_t*>(raw)[t * 16 + b];
      return make_float2(float(p & 0xffffu), float(p >> 16));
    }
  }
};

// Bin k of line b to the buffer at buf[k * LD + b] (after every read of it).
template <int LD>
struct SmemOut {
  static constexpr bool kSyncFirst = true;
  static constexpr bool kJFast = false;
  float2* buf;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const { buf[k * LD + b] = v; }
};

// Bin k of line b straight to global memory at out[k * stride + b].
struct GlobalOut {
  static constexpr bool kSyncFirst = false;
  static constexpr bool kJFast = false;
  float2* out;
  uint32_t stride;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const { out[size_t(k) * stride + b] = v; }
};

// Sum of |v| and |v|^2 over the bins this thread holds (Tamura accumulation).
struct AmpSums {
  static constexpr bool kSyncFirst = false;
  static constexpr bool kJFast = false;
  float* s;  // s[0] += |v|, s[1] += |v|^2
  __device__ __forceinline__ void operator()(int, int, float2 v) const {
    const float q = fmaf(v.x, v.x, v.y * v.y);
    s[0] += sqrtf(q);
    s[1] += q;
  }
};

// Bin k of line b times the transposed transfer function, back to the buffer.
template <int LD>
struct MulHtSmem {
  static constexpr bool kSyncFirst = true;
  static constexpr bool kJFast = false;
  float2* buf;
  const float2* ht;  // ht[k * H + line] of this strip's first line
  uint32_t H;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const {
    buf[k * LD + b] = cmul(v, __ldg(&ht[size_t(k) * H + b]));
  }
};

// Bin k of line b straight to global memory at out[b * stride + k], with the
// last stage's threads laid out along the bins (consecutive lanes hold
// consecutive bins of one line, so the stores are coalesced).
struct RowOut {
  static constexpr bool kSyncFirst = false;
  static constexpr bool kJFast = true;
  float2* out;
  uint32_t stride;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const { out[size_t(b) * stride + k] = v; }
};

// Network-input cells from bins handed out bin-fastest with 16 butterflies per
// line (lanes 0-15: row b, lanes 16-31: row b + 1; bins j + 16 m): the 2 x 2 block
// of unshifted bins (even ky, even kx) sits in lanes j, j ^ 1, j ^ 16, j ^ 17. The
// lane with even j of the even row writes log1p(mean |F|) (DC bin as 0) at the
// block's centred position and adds it to its running (sum v, sum v^2).
struct CellsOut {
  static constexpr bool kSyncFirst = false;
  static constexpr bool kJFast = true;
  float* cells;      // this frame's [H/2][W/2]
  uint32_t ky0;      // unshifted row of the strip's first line
  uint32_t W, H;
  float* s;          // s[0] += v, s[1] += v^2
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const {
    const uint32_t ky = ky0 + uint32_t(b);
    float a = (ky | uint32_t(k)) ? sqrtf(fmaf(v.x, v.x, v.y * v.y)) : 0.f;
    a += __shfl_xor_sync(0xffffffffu, a, 1);
    a += __shfl_xor_sync(0xffffffffu, a, 16);
    if (((threadIdx.x & 31) & 17) == 0) {  // even bin, even row
      const float c = log1pf(0.25f * a);
      const uint32_t r = ((ky + H / 2) & (H - 1)) >> 1, q = ((uint32_t(k) + W / 2) & (W - 1)) >> 1;
      cells[size_t(r) * (W / 2) + q] = c;
      s[0] += c;
      s[1] = fmaf(c, c, s[1]);
    }
  }
};

// Span NS and radix R of the last stage of the pass (the BlockRadix chain).
template <int L, int BT, int NT>
struct LastStage {
  static constexpr int radix(int rem) {
    return (rem % 16 == 0 && (BT * (L / 16)) % NT == 0 && BT * (L / 16) >= NT) ? 16
           : (rem % 8 == 0 ? 8 : (rem % 4 == 0 ? 4 : 2));
  }
  static constexpr int ns() {
    int ns = 1;
    while (ns * radix(L / ns) < L) ns *= radix(L / ns);
    return ns;
  }
  static constexpr int NS = ns();
  static constexpr int R = L / NS;
};

// One Stockham stage of span NS over the PP_BT lines (thread layout and index
// rules of fft_dev.cuh), and recursively the rest. The first stage reads
// through `src`, later ones the buffer; twiddles come from the shared table
// tws[e] = exp(-2 pi i e / L). The last stage hands bin k of line b to epi.
// With an epilogue of kJFast, the last stage maps threads bin-fastest (b = idx / NB,
// j = idx % NB) and takes its twiddles from twl[(m - 1) NS + j] (contiguous in j).
// Barrier between stages: the whole CTA (BAR = 0), or named barrier BAR over the
// pass's NT threads (warp-specialised kernels whose other warps do not take part).
template <int BAR, int NT>
__device__ __forceinline__ void pp_sync() {
  if constexpr (BAR == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;\n" ::"n"(BAR), "n"(NT) : "memory");
}

template <int L, int NS, int DIR, class Src, class Epi, int LDX = 0, int BAR = 0>
__device__ __forceinline__ void pp_stages(const Src& src, float2* buf, const float2* tws, const Epi& epi,
                                          const float2* twl = nullptr) {
  using C = PpCfg<L>;
  // LDX > 0: buffer row stride other than the padded one (16 for TMA-staged strips:
  // with lines fastest, a warp's stage accesses are two contiguous 128-byte runs)
  constexpr int NT = C::NT, BT = C::BT, LD = LDX > 0 ? LDX : C::LD;
  constexpr int REM = L / NS;
  constexpr int R = BlockRadix<REM, L, BT, NT>::value;
  constexpr int NB = L / R;
  static_assert((BT * NB) % NT == 0, "thread count must divide the butterflies");
  constexpr int ITEMS = BT * NB / NT;
  constexpr bool LAST = NS * R == L;
  constexpr bool JF = LAST && Epi::kJFast;
  float2 v[ITEMS][R];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int idx = threadIdx.x + it * NT;
    const int b = JF ? idx / NB : idx % BT, j = JF ? idx % NB : idx / BT;
#pragma unroll
    for (int m = 0; m < R; ++m) v[it][m] = src(j + m * NB, b);
    if constexpr (NS > 1) {
      const int jm = j % NS;
#pragma unroll
      for (int m = 1; m < R; ++m) {
        float2 w = JF ? twl[(m - 1) * NS + jm] : tws[jm * m * (L / (NS * R))];
        if constexpr (DIR > 0) w.y = -w.y;
        v[it][m] = cmul(v[it][m], w);
      }
    }
    dft<R, DIR>(v[it]);
  }
  if constexpr (LAST) {
    if constexpr (Epi::kSyncFirst) pp_sync<BAR, NT>();  // every read of buf is done
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int idx = threadIdx.x + it * NT;
      const int b = JF ? idx / NB : idx % BT, j = JF ? idx % NB : idx / BT;
#pragma unroll
      for (int m = 0; m < R; ++m) epi(b, j + m * NB, v[it][m]);
    }
  } else {
    if constexpr (Src::kAliasesBuf) pp_sync<BAR, NT>();
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int idx = threadIdx.x + it * NT;
      const int b = idx % BT, j = idx / BT;
      const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int m = 0; m < R; ++m) buf[(base + m * NS) * LD + b] = v[it][m];
    }
    pp_sync<BAR, NT>();
    SmemSrc<LD> s{buf};
    pp_stages<L, NS * R, DIR, SmemSrc<LD>, Epi, LDX, BAR>(s, buf, tws, epi, twl);
  }
}

// ------------------------------------------------------------- prefetch

// Raw strip of pass P1: rows 0..H-1, columns s0..s0+BT-1 of frame i -> raw_s[y][BT],
// in 16-byte pieces (8-byte ones when a row segment is shorter: uint8 at BT = 8).
template <int L>
__device__ __forceinline__ void prefetch_raw(const SpatialArgs& a, int i, int s0, unsigned char* dst) {
  using C = PpCfg<L>;
  const int bpp = a.in_kind == IN_U8 ? 1 : 2;
  const int seg = C::BT * bpp;  // bytes of one row segment: 8, 16 or 32
  const size_t rslot = (a.raw.slot0 + uint32_t(i)) % a.raw.cap;
  const unsigned char* src = static_cast<const unsigned char*>(a.raw.base) + (rslot * size_t(a.W) * L + s0) * bpp;
  const size_t row = size_t(a.W) * bpp;
  if (seg >= 16) {
    const int pieces = seg / 16;
    for (int e = threadIdx.x; e < L * pieces; e += C::NT) {
      const int y = e / pieces, q = e % pieces;
      cpa16(dst + y * seg + q * 16, src + y * row + q * 16);
    }
  } else {
    for (int y = threadIdx.x; y < L; y += C::NT) cpa8(dst + y * seg, src + y * row);
  }
  cpa_commit();
}

// Complex strip: line b of the strip is src[b * L + t], t = 0..L-1 -> buf[t][b].
template <int L>
__device__ __forceinline__ void prefetch_lines(const float2* src, float2* dst) {
  using C = PpCfg<L>;
#pragma unroll
  for (int t = threadIdx.x; t < L; t += C::NT)
#pragma unroll
    for (int b = 0; b < C::BT; ++b) cpa8(&dst[t * C::LD + b], &src[b * L + t]);
  cpa_commit();
}

// ---------------------------------------------------------------- kernel

template <int L, int PK>
__global__ void __launch_bounds__(PpCfg<L>::NT, (L <= 256 ? 768 / L : 1))
    k_pass_pp(SpatialArgs a, int nitems, int strip_log2) {
  using C = PpCfg<L>;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tws = reinterpret_cast<float2*>(smem);
  float2* cys = reinterpret_cast<float2*>(smem + C::TW);  // P1 Fresnel: chirp along y
  float2* twl = cys;                                      // P2f: last-stage twiddles by (m, j)
  unsigned char* body = smem + ((PK == PK_P1 || PK == PK_P2F || PK == PK_P2C) ? 2 * C::TW : C::TW);
  float2* buf0 = reinterpret_cast<float2*>(body);
  // P1: one FFT buffer and two raw staging buffers; other passes: two FFT buffers
  float2* buf1 = reinterpret_cast<float2*>(body + C::BUF);
  unsigned char* raw0 = body + C::BUF;
  unsigned char* raw1 = body + C::BUF + C::RAW;
  const int tid = threadIdx.x;
  const int smask = (1 << strip_log2) - 1;
  const bool fresnel = a.spatial == HV_SPATIAL_FRESNEL;
  const bool u8 = a.in_kind == IN_U8;
  // the pass length: P1 and P3a run along y (length H), P2a and P2f along x
  const float2* twg = (PK == PK_P1 || PK == PK_P3A || PK == PK_P3T) ? a.tw_h : a.tw_w;
  for (int e = tid; e < L; e += C::NT) {
    tws[e] = __ldg(&twg[e]);
    if (PK == PK_P1 && fresnel) cys[e] = __ldg(&a.chirp_y[e]);
  }
  if constexpr (PK == PK_P2F || PK == PK_P2C) {
    using LS = LastStage<L, C::BT, C::NT>;
    for (int e = tid; e < (LS::R - 1) * LS::NS; e += C::NT) {
      const int m = e / LS::NS + 1, jm = e % LS::NS;
      twl[e] = __ldg(&twg[jm * m * (L / (LS::NS * LS::R))]);
    }
  }
  // lines per frame of the other axis: W columns (P1, P3a) or H rows (P2a, P2f)
  const uint32_t LO = (PK == PK_P1 || PK == PK_P3A || PK == PK_P3T) ? a.W : a.H;

  auto issue = [&](int it, int cur) {
    const int i = it >> strip_log2, s0 = (it & smask) * C::BT;
    if constexpr (PK == PK_P1) {
      prefetch_raw<L>(a, i, s0, cur == 0 ? raw0 : raw1);
    } else {
      const float2* base = (PK == PK_P3A || PK == PK_P3T) ? a.scratch2 : a.scratch1;
      prefetch_lines<L>(base + size_t(i) * L * LO + size_t(s0) * L, cur == 0 ? buf0 : buf1);
    }
  };

  int item = blockIdx.x;
  if (item < nitems) issue(item, 0);
  for (int k = 0; item < nitems; ++k, item += gridDim.x) {
    const int cur = k & 1;
    const int i = item >> strip_log2, s0 = (item & smask) * C::BT;
    cpa_wait_all();
    __syncthreads();  // this item's input resident; the other buffer is free
    const int nxt = item + gridDim.x;
    if (nxt < nitems) issue(nxt, cur ^ 1);
    if (PK != PK_P1 && a.discard_inputs) {
      // the strip's intermediate is dead once staged: drop its L2 lines unwritten
      const float2* base = (PK == PK_P3A || PK == PK_P3T) ? a.scratch2 : a.scratch1;
      const char* st = reinterpret_cast<const char*>(base + size_t(i) * L * LO + size_t(s0) * L);
      for (int e = tid; e < C::BT * L * 8 / 128; e += C::NT)
        asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(st + size_t(e) * 128) : "memory");
    }
    if constexpr (PK == PK_P1) {
      // S1[ky][x]: bin ky of column s0 + b at s1[ky * W + s0 + b]
      const GlobalOut out{a.scratch1 + size_t(i) * a.H * a.W + s0, a.W};
      const unsigned char* raw = cur == 0 ? raw0 : raw1;
      const int b = tid % C::BT;
      if (fresnel) {
        const float2 cx = __ldg(&a.chirp_x[s0 + b]);
        if (u8) pp_stages<L, 1, -1>(RawSrc<true, true, C::BT>{raw, cys, cx}, buf0, tws, out);
        else pp_stages<L, 1, -1>(RawSrc<false, true, C::BT>{raw, cys, cx}, buf0, tws, out);
      } else {
        if (u8) pp_stages<L, 1, -1>(RawSrc<true, false, C::BT>{raw, cys, make_float2(0.f, 0.f)}, buf0, tws, out);
        else pp_stages<L, 1, -1>(RawSrc<false, false, C::BT>{raw, cys, make_float2(0.f, 0.f)}, buf0, tws, out);
      }
    } else if constexpr (PK == PK_P2A) {
      float2* buf = cur == 0 ? buf0 : buf1;
      const SmemSrc<C::LD> src{buf};
      pp_stages<L, 1, -1>(src, buf, tws, MulHtSmem<C::LD>{buf, a.asp_ht + s0, a.H});
      __syncthreads();
      // S2[x][ky]: sample x of row s0 + b at s2[x * H + s0 + b]
      pp_stages<L, 1, +1>(src, buf, tws, GlobalOut{a.scratch2 + size_t(i) * a.H * a.W + s0, a.H});
    } else if constexpr (PK == PK_P3A) {
      float2* buf = cur == 0 ? buf0 : buf1;
      const size_t tslot = (a.tq.slot0 + uint32_t(i)) % a.tq.cap;
      // time queue [y][x]: sample y of column s0 + b at tq[y * W + s0 + b]
      pp_stages<L, 1, +1>(SmemSrc<C::LD>{buf}, buf, tws,
                          GlobalOut{static_cast<float2*>(a.tq.base) + tslot * size_t(a.W) * a.H + s0, a.W});
    } else if constexpr (PK == PK_P3T) {
      float2* buf = cur == 0 ? buf0 : buf1;
      float acc[2] = {0.f, 0.f};
      pp_stages<L, 1, +1>(SmemSrc<C::LD>{buf}, buf, tws, AmpSums{acc});
      // block sums: warp shuffles, then one partial per warp in shared memory
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
        acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], o);
      }
      __shared__ float red[2][C::NT / 32];
      if ((tid & 31) == 0) {
        red[0][tid >> 5] = acc[0];
        red[1][tid >> 5] = acc[1];
      }
      __syncthreads();
      if (tid < 2) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < C::NT / 32; ++w) t += red[tid][w];
        atomicAdd(&a.tam_acc[size_t(i) * a.tam_stride + tid], double(t));
      }
    } else if constexpr (PK == PK_P2C) {
      float2* buf = cur == 0 ? buf0 : buf1;
      float acc[2] = {0.f, 0.f};
      pp_stages<L, 1, -1>(SmemSrc<C::LD>{buf}, buf, tws,
                          CellsOut{a.cells + size_t(i) * (a.H / 2) * (a.W / 2), uint32_t(s0), a.W, a.H, acc}, twl);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
        acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], o);
      }
      __shared__ float redc[2][C::NT / 32];
      if ((tid & 31) == 0) {
        redc[0][tid >> 5] = acc[0];
        redc[1][tid >> 5] = acc[1];
      }
      __syncthreads();
      if (tid < 2) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < C::NT / 32; ++w) t += redc[tid][w];
        atomicAdd(&a.tam_acc[size_t(i) * a.tam_stride + tid], t);
      }
    } else {
      float2* buf = cur == 0 ? buf0 : buf1;
      // time queue [ky][kx]: bin kx of row s0 + b, stored from the registers of the
      // last stage (threads along kx there)
      const size_t tslot = (a.tq.slot0 + uint32_t(i)) % a.tq.cap;
      float2* out = static_cast<float2*>(a.tq.base) + tslot * size_t(a.H) * a.W + size_t(s0) * a.W;
      pp_stages<L, 1, -1>(SmemSrc<C::LD>{buf}, buf, tws, RowOut{out, a.W}, twl);
    }
  }
  cpa_wait_all();
}

template <int L, int PK>
static cudaError_t launch_pp(const SpatialArgs& a, uint32_t lines, cudaStream_t s) {
  using C = PpCfg<L>;
  const size_t smem = PK == PK_P1 ? 2 * C::TW + C::BUF + 2 * C::RAW
                                   : ((PK == PK_P2F || PK == PK_P2C) ? 2 * C::TW : C::TW) + 2 * C::BUF;
  auto kern = k_pass_pp<L, PK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, nsm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, smem);
  if (e != cudaSuccess) return e;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int strip_log2 = 0;
  while ((uint32_t(C::BT) << strip_log2) < lines) ++strip_log2;
  const int nitems = int(a.n) << strip_log2;
  int grid = per_sm * nsm;
  if (grid > nitems) grid = nitems;
  if (grid < 1) grid = 1;
  kern<<<grid, C::NT, smem, s>>>(a, nitems, strip_log2);
  return cudaGetLastError();
}

// ------------------------------------------------- row FFT, one warp per 2 rows
//
// The Fresnel row pass at L = 256 with the STFT's warp-private layout: 16 lanes
// carry one row, so the 256-point FFT (16 x 16 Stockham) needs only __syncwarp
// between its stages. A CTA of 8 warps takes strips of 16 rows of S1 [ky][x]; one
// TMA tensor load per strip (16 x 256 complex64, dense rows) lands in one of two
// tiles and completes on the tile's mbarrier, the next strip's load in flight
// while the current one is transformed. Stage 1 reads samples jl + 16 m
// (consecutive lanes) and writes its output m back into the row at 16 jl +
// (m ^ jl) (an XOR swizzle: conflict-free without padding); stage 2 reads
// 16 m + (jl ^ m), applies w_256^(jl m) from a table laid out by (m, jl) and leaves
// bin jl + 16 m in lane jl, stored to the time queue row (coalesced).
constexpr int RW_L = 256, RW_BT = 16, RW_NT = 256;

__device__ __forceinline__ uint32_t rw_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait (about 2^32 clocks) for phase `parity` of an mbarrier.
__device__ __forceinline__ bool rw_wait(uint32_t mbar, uint32_t parity) {
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

__global__ void __launch_bounds__(RW_NT, 3)
    k_row_warp(SpatialArgs a, int nitems, int strip_log2, const __grid_constant__ CUtensorMap s1map) {
  extern __shared__ __align__(128) unsigned char smem_tma[];  // TMA destinations: 128-byte aligned
  __shared__ __align__(8) unsigned long long full[2];
  float2* tile0 = reinterpret_cast<float2*>(smem_tma);
  float2* tile1 = tile0 + RW_BT * RW_L;
  float2* tw2 = tile1 + RW_BT * RW_L;  // stage 2: w_256^(j m) at (m - 1) 16 + j
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = 2 * warp + (lane >> 4), jl = lane & 15;  // row of the strip, lane within the row
  const int smask = (1 << strip_log2) - 1;
  for (int e = tid; e < 15 * 16; e += RW_NT) {
    const int m = e / 16 + 1, j = e % 16;
    tw2[e] = __ldg(&a.tw_w[j * m]);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(rw_smem(&full[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(rw_smem(&full[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // one thread: the strip of item `it` (rows i H + s0 .. + 15 of S1) into tile `k`
  auto issue = [&](int it, int k) {
    const int i = it >> strip_log2, s0 = (it & smask) * RW_BT;
    const uint32_t mb = rw_smem(&full[k]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(RW_BT * RW_L * 8)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(rw_smem(k ? tile1 : tile0)),
        "l"(reinterpret_cast<uint64_t>(&s1map)), "r"(0), "r"(int(i * a.H + s0)), "r"(mb)
        : "memory");
  };
  int item = blockIdx.x;
  if (tid == 0 && item < nitems) issue(item, 0);
  bool ok = true;
  for (int k = 0; item < nitems && ok; ++k, item += gridDim.x) {
    const int cur = k & 1;
    float2* tile = cur ? tile1 : tile0;
    const int i = item >> strip_log2, s0 = (item & smask) * RW_BT;
    ok = rw_wait(rw_smem(&full[cur]), uint32_t(k >> 1) & 1u);
    // every warp is done with the other tile (two strips ago) and sees this one
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    const int nxt = item + gridDim.x;
    if (tid == 0 && nxt < nitems) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(nxt, cur ^ 1);
    }
    if (a.discard_inputs) {
      const char* st = reinterpret_cast<const char*>(a.scratch1 + (size_t(i) * a.H + s0) * RW_L);
      for (int e = tid; e < RW_BT * RW_L * 8 / 128; e += RW_NT)
        asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(st + size_t(e) * 128) : "memory");
    }
    float2* row = tile + b * RW_L;
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = row[jl + 16 * m];
    dft<16, -1>(v);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) row[16 * jl + (m ^ jl)] = v[m];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      v[m] = row[16 * m + (jl ^ m)];
      if (m > 0) v[m] = cmul(v[m], tw2[(m - 1) * 16 + jl]);
    }
    dft<16, -1>(v);
    // time queue [ky][kx]: bin kx = jl + 16 m of row s0 + b
    const size_t tslot = (a.tq.slot0 + uint32_t(i)) % a.tq.cap;
    float2* out = static_cast<float2*>(a.tq.base) + (tslot * a.H + s0 + b) * size_t(RW_L);
#pragma unroll
    for (int m = 0; m < 16; ++m) out[jl + 16 * m] = v[m];
  }
  if (!ok && tid == 0 && a.err) atomicOr(a.err, 8u);
}

static cudaError_t launch_row_warp(const SpatialArgs& a, cudaStream_t s) {
  const size_t smem = (2 * size_t(RW_BT) * RW_L + 15 * 16) * sizeof(float2);
  CUtensorMap map{};
  if (!encode_map_2d_u64(&map, a.scratch1, RW_L, uint64_t(a.n) * a.H, RW_L * 8, RW_L, RW_BT, false))
    return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(k_row_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, nsm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_row_warp, RW_NT, smem);
  if (e != cudaSuccess) return e;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int strip_log2 = 0;
  while ((uint32_t(RW_BT) << strip_log2) < a.H) ++strip_log2;
  const int nitems = int(a.n) << strip_log2;
  int grid = per_sm * nsm;
  if (grid > nitems) grid = nitems;
  if (grid < 1) grid = 1;
  k_row_warp<<<grid, RW_NT, smem, s>>>(a, nitems, strip_log2, map);
  return cudaGetLastError();
}

// ASP row pass at W = 256, warp-private like k_row_warp: forward row FFT, bins
// times the transfer function H[ky][kx] (row-major copy, 1/(W H) folded in), then
// the inverse row FFT, whose first stage takes the bins the forward FFT left in
// the lane's registers (butterfly jl of the inverse is bins jl + 16 m). S2 is
// written row-major [ky][x], coalesced.
__global__ void __launch_bounds__(RW_NT, 3)
    k_row_asp(SpatialArgs a, int nitems, int strip_log2, const __grid_constant__ CUtensorMap s1map) {
  extern __shared__ __align__(128) unsigned char smem_tma[];  // TMA destinations: 128-byte aligned
  __shared__ __align__(8) unsigned long long full[2];
  float2* tile0 = reinterpret_cast<float2*>(smem_tma);
  float2* tile1 = tile0 + RW_BT * RW_L;
  float2* tw2 = tile1 + RW_BT * RW_L;  // w_256^(j m) at (m - 1) 16 + j
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = 2 * warp + (lane >> 4), jl = lane & 15;
  const int smask = (1 << strip_log2) - 1;
  for (int e = tid; e < 15 * 16; e += RW_NT) {
    const int m = e / 16 + 1, j = e % 16;
    tw2[e] = __ldg(&a.tw_w[j * m]);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(rw_smem(&full[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(rw_smem(&full[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int it, int k) {
    const int i = it >> strip_log2, s0 = (it & smask) * RW_BT;
    const uint32_t mb = rw_smem(&full[k]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(RW_BT * RW_L * 8)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(rw_smem(k ? tile1 : tile0)),
        "l"(reinterpret_cast<uint64_t>(&s1map)), "r"(0), "r"(int(i * a.H + s0)), "r"(mb)
        : "memory");
  };
  int item = blockIdx.x;
  if (tid == 0 && item < nitems) issue(item, 0);
  bool ok = true;
  for (int k = 0; item < nitems && ok; ++k, item += gridDim.x) {
    const int cur = k & 1;
    float2* tile = cur ? tile1 : tile0;
    const int i = item >> strip_log2, s0 = (item & smask) * RW_BT;
    ok = rw_wait(rw_smem(&full[cur]), uint32_t(k >> 1) & 1u);
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    const int nxt = item + gridDim.x;
    if (tid == 0 && nxt < nitems) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(nxt, cur ^ 1);
    }
    if (a.discard_inputs) {
      const char* st = reinterpret_cast<const char*>(a.scratch1 + (size_t(i) * a.H + s0) * RW_L);
      for (int e = tid; e < RW_BT * RW_L * 8 / 128; e += RW_NT)
        asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(st + size_t(e) * 128) : "memory");
    }
    float2* row = tile + b * RW_L;
    const int ky = s0 + b;
    float2 v[16];
    // forward row FFT
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = row[jl + 16 * m];
    dft<16, -1>(v);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) row[16 * jl + (m ^ jl)] = v[m];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      v[m] = row[16 * m + (jl ^ m)];
      if (m > 0) v[m] = cmul(v[m], tw2[(m - 1) * 16 + jl]);
    }
    dft<16, -1>(v);
    // bins kx = jl + 16 m times H[ky][kx]
    const float2* hrow = a.asp_h + size_t(ky) * RW_L;
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = cmul(v[m], __ldg(&hrow[jl + 16 * m]));
    // inverse row FFT: its first butterfly jl takes the inputs jl + 16 m, here already
    dft<16, +1>(v);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) row[16 * jl + (m ^ jl)] = v[m];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      v[m] = row[16 * m + (jl ^ m)];
      if (m > 0) {
        float2 w = tw2[(m - 1) * 16 + jl];
        w.y = -w.y;
        v[m] = cmul(v[m], w);
      }
    }
    dft<16, +1>(v);
    // S2 [ky][x]: sample x = jl + 16 m of row ky
    float2* out = a.scratch2 + (size_t(i) * a.H + ky) * RW_L;
#pragma unroll
    for (int m = 0; m < 16; ++m) out[jl + 16 * m] = v[m];
  }
  if (!ok && tid == 0 && a.err) atomicOr(a.err, 8u);
}

// Column IFFT (length L = H <= 256) of 16-column strips of a row-major S2 [ky][x]:
// one TMA tensor load per strip (H rows x 16 columns, dense: the block-wide FFT's
// lines-fastest layout with row stride 16), the next strip in flight; samples
// stored to the time queue [y][x] from the last stage's registers.
template <int L>
__global__ void __launch_bounds__(PpCfg<L>::NT, (L <= 256 ? 768 / L : 1))
    k_col_ifft_tma(SpatialArgs a, int nitems, int strip_log2, const __grid_constant__ CUtensorMap s2map) {
  using C = PpCfg<L>;
  static_assert(C::BT == 16, "16-column strips");
  extern __shared__ __align__(128) unsigned char smem_tma[];  // TMA destinations: 128-byte aligned
  __shared__ __align__(8) unsigned long long full[2];
  float2* buf0 = reinterpret_cast<float2*>(smem_tma);
  float2* buf1 = buf0 + L * 16;
  float2* tws = buf1 + L * 16;
  const int tid = threadIdx.x;
  const int smask = (1 << strip_log2) - 1;
  for (int e = tid; e < L; e += C::NT) tws[e] = __ldg(&a.tw_h[e]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(rw_smem(&full[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(rw_smem(&full[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int it, int k) {
    const int i = it >> strip_log2, s0 = (it & smask) * 16;
    const uint32_t mb = rw_smem(&full[k]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(L * 16 * 8) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(rw_smem(k ? buf1 : buf0)),
        "l"(reinterpret_cast<uint64_t>(&s2map)), "r"(s0), "r"(int(i * L)), "r"(mb)
        : "memory");
  };
  int item = blockIdx.x;
  if (tid == 0 && item < nitems) issue(item, 0);
  bool ok = true;
  for (int k = 0; item < nitems && ok; ++k, item += gridDim.x) {
    const int cur = k & 1;
    float2* buf = cur ? buf1 : buf0;
    const int i = item >> strip_log2, s0 = (item & smask) * 16;
    ok = rw_wait(rw_smem(&full[cur]), uint32_t(k >> 1) & 1u);
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    const int nxt = item + gridDim.x;
    if (tid == 0 && nxt < nitems) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(nxt, cur ^ 1);
    }
    if (a.discard_inputs)  // the strip's 128-byte row segments of S2 are dead once staged
      for (int y = tid; y < L; y += C::NT)
        asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(a.scratch2 + (size_t(i) * L + y) * a.W + s0)
                     : "memory");
    const size_t tslot = (a.tq.slot0 + uint32_t(i)) % a.tq.cap;
    // time queue [y][x]: sample y of column s0 + b at tq[y W + s0 + b]
    pp_stages<L, 1, +1, SmemSrc<16>, GlobalOut, 16>(
        SmemSrc<16>{buf}, buf, tws, GlobalOut{static_cast<float2*>(a.tq.base) + tslot * size_t(a.W) * L + s0, a.W});
  }
  if (!ok && tid == 0 && a.err) atomicOr(a.err, 8u);
}

template <int LH>
static cudaError_t launch_asp_rows(const SpatialArgs& a, cudaStream_t s, int* launches) {
  CUtensorMap m1{}, m2{};
  if (!encode_map_2d_u64(&m1, a.scratch1, RW_L, uint64_t(a.n) * a.H, RW_L * 8, RW_L, RW_BT, false) ||
      !encode_map_2d_u64(&m2, a.scratch2, RW_L, uint64_t(a.n) * a.H, RW_L * 8, 16, LH, false))
    return cudaErrorNotSupported;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // row pass
  {
    const size_t smem = (2 * size_t(RW_BT) * RW_L + 15 * 16) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_row_asp, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_row_asp, RW_NT, smem);
    if (e != cudaSuccess) return e;
    int sl = 0;
    while ((uint32_t(RW_BT) << sl) < a.H) ++sl;
    const int nitems = int(a.n) << sl;
    int grid = per_sm * nsm;
    grid = grid > nitems ? nitems : (grid < 1 ? 1 : grid);
    k_row_asp<<<grid, RW_NT, smem, s>>>(a, nitems, sl, m1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // column IFFT
  {
    using C = PpCfg<LH>;
    const size_t smem = (2 * size_t(LH) * 16 + LH) * sizeof(float2);
    auto kern = k_col_ifft_tma<LH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, smem);
    if (e != cudaSuccess) return e;
    int sl = 0;
    while ((16u << sl) < a.W) ++sl;
    const int nitems = int(a.n) << sl;
    int grid = per_sm * nsm;
    grid = grid > nitems ? nitems : (grid < 1 ? 1 : grid);
    kern<<<grid, C::NT, smem, s>>>(a, nitems, sl, m2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  *launches += 2;
  return cudaSuccess;
}

template <int LH, int LW>
static cudaError_t pp_fixed(const SpatialArgs& a, cudaStream_t s, int* launches) {
  cudaError_t e = launch_pp<LH, PK_P1>(a, a.W, s);
  if (e != cudaSuccess) return e;
  ++*launches;
  if (a.spatial == HV_SPATIAL_ASP) {
    // rows of 256 with the row-major transfer function: warp-private row pass and
    // TMA-staged column IFFT (the block-wide passes when a tensor map cannot be built)
    if constexpr (LW == RW_L && LH <= 256) {
      if (a.asp_h) {
        e = launch_asp_rows<LH>(a, s, launches);
        if (e != cudaErrorNotSupported) return e;
      }
    }
    e = launch_pp<LW, PK_P2A>(a, a.H, s);
    if (e != cudaSuccess) return e;
    e = launch_pp<LH, PK_P3A>(a, a.W, s);
    *launches += 2;
  } else {
    // rows of 256: the warp-private row pass (H a multiple of its 16-row strips;
    // the block-wide pass when the tensor map cannot be encoded)
    e = (LW == RW_L && a.H % RW_BT == 0) ? launch_row_warp(a, s) : cudaErrorNotSupported;
    if (e == cudaErrorNotSupported) e = launch_pp<LW, PK_P2F>(a, a.H, s);
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
    case 1024: return pp_fixed<LH, 1024>(a, s, launches);
  }
  return cudaErrorInvalidValue;
}

template <int PK>
static cudaError_t pass_by_len(const SpatialArgs& a, cudaStream_t s) {
  // pass length and number of lines: columns (length H, W lines) or rows (length W, H lines)
  const bool cols = PK == PK_P1 || PK == PK_P3A || PK == PK_P3T;
  const uint32_t L = cols ? a.H : a.W, lines = cols ? a.W : a.H;
  switch (L) {
    case 64: return launch_pp<64, PK>(a, lines, s);
    case 128: return launch_pp<128, PK>(a, lines, s);
    case 256: return launch_pp<256, PK>(a, lines, s);
    case 512: return launch_pp<512, PK>(a, lines, s);
    case 1024: return launch_pp<1024, PK>(a, lines, s);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------- fused transform, 256 x 256 frames
//
// Every pass of every frame of a launch in one persistent kernel. The passes
// above each run as a launch of their own over a chunk of frames, so their
// intermediates (S1, S2: 512 KB per frame) go through HBM once written and once
// read. Here work items come in a fixed global order from an atomic ticket
// counter: row r of the order holds the column items of frame r and the items of
// each later pass of frame r - (the lags up to that pass). A Fresnel frame takes two passes of 16
// items: 16 chirped (complex) columns per column item, 16 rows per row item,
// the row FFT writing the time queue. ASP takes four passes, using that the
// hologram is real:
//   1. 8 column items of 32 real columns, packed in pairs as the real and
//      imaginary parts of 16 complex lines whose spectra Z are separated after
//      the transform (for real a and b, z = a + i b: A(k) = (Z(k) + conj Z(-k)) / 2,
//      B(k) = (Z(k) - conj Z(-k)) / 2i). Only bins ky = 1 .. 127 are stored, row
//      by row, with the real rows ky = 0 and 128 packed into row 0 as
//      S1(0, x) + i S1(128, x): the other half is their conjugate.
//   2. 8 row items over S1 rows 0 .. 127: the forward row FFT W(ky, .) is kept
//      in the second half of the S1 slot (S3), then x H(ky) and the inverse row
//      FFT give S2 rows 0 .. 127 (row 0 takes W(0) = (Wp(k) + conj Wp(-k)) / 2
//      from the packed row's transform Wp).
//   3. 8 mirror items: the spectrum of row ky in 128 .. 255 is
//      conj W(256 - ky, -kx) (row 128: (Wp(k) - conj Wp(-k)) / 2i), read from S3;
//      x H(ky) and the inverse row FFT give S2 rows 128 .. 255. A frame takes
//      128 forward row FFTs instead of 256.
//   4. 16 column-IFFT items of 16 columns of S2 write the time queue.
// S1 (with S3) and S2 are rings of RING frames that stay in L2. An item may start
// once the counters that make its input complete and its output slot free have
// been published (P1 .. P4 the ASP passes above; each chain of release adds and
// acquire loads orders what it covers, so a condition implied through an
// earlier item's wait is not checked again):
//   P1 of f: the P2 items of f - RING have read S1 slot f mod RING
//   P2 of f: P1 of f wrote S1; the P4 items of f - RING have read S2 (and so the
//            P3 items of f - RING have read S3)
//   P3 of f: P2 of f wrote S3 (and so P4 of f - RING has read S2)
//   P4 of f: P3 of f wrote S2 (and so P2 of f did)
// and for Fresnel: column items of f after the row items of f - RING, row items
// of f after the column items of f.
// A CTA is warp-specialised: one producer thread takes the tickets, waits (bounded
// spin on acquire loads) for each item's counters, stages its input strip into
// one of two buffers with one copy (a TMA tensor copy, or a 1-D bulk copy)
// completing on the buffer's mbarrier, and publishes every finished item, in
// order (release add on its slot counter); eight consumer warps transform the
// staged strip while the next one streams in. The producer readies the following
// item (ticket and counters) while the consumers still hold both buffers, so its
// copy starts as soon as one frees. Every wait is on an item with a smaller
// ticket (RING > 2 LAG), a CTA takes its items in ticket order, and the producer
// publishes finished items from inside each of its waits, so the item with the
// smallest unfinished ticket always completes: the launch ends. Raw frames are read with an evict-first L2
// policy and the propagated frames stored with streaming stores, so that the two
// rings keep their L2 lines.
constexpr int FZ_NT = 256;       // consumer threads (one pass's thread layout)
constexpr int FZ_THREADS = FZ_NT + 32;
// rows of tickets between a frame's passes: at least the tickets in flight (3 per
// CTA: the transformed item, the staged one, the one waiting for its buffer) over
// the items per row, so that an item's inputs are usually published when it is
// staged. A ticket is fetched only when the producer is ready to handle it: every
// ticket held but not worked on delays the frames that wait for it (fetching one
// ahead measured 1.5 % slower, lags of 40 and 56 rows 1-2 % slower)
constexpr int FZ_LAG = 48;
// ASP runs four passes of 8, 8, 8 and 16 items per frame (the row pass split into
// the rows it transforms forward and the rows it takes as mirrors), so 40 items
// per ticket row; FZ_LAG_ASP1 rows from the column pass to the row pass, then
// FZ_LAG_ASP between the later passes. The rings must outlast the two later lags
// (the row pass of frame f + R waits for the column IFFT of f)
constexpr int FZ_LAG_ASP1 = 36;
constexpr int FZ_LAG_ASP = 36;
constexpr int FZ_BAR = 1;        // named barrier of the consumer warps
constexpr size_t FZ_FRAME = size_t(RW_L) * RW_L;  // complex values per frame
constexpr size_t FZ_BUF = size_t(256) * 16;       // complex values per buffer
constexpr size_t FZ_RAW = 256 * 64;               // bytes of a raw strip (32 uint16 columns), in the buffer's tail
// every wait is on a smaller ticket when the rings are longer than the lag; the
// headroom above it keeps column items from waiting for a slot to be freed
static_assert(kFusedRing > FZ_LAG && kFusedRing > FZ_LAG_ASP1 && kFusedRing > 2 * FZ_LAG_ASP,
              "the rings must outlast the lags between passes");
// shared memory: pass twiddles (256), row-FFT stage-2 twiddles (240), Fresnel
// chirp along y (256), two buffers of 16 lines x 256 (the column passes' lines
// fastest with row stride 16, the row tile 16 x 256; a raw strip lands in the
// tail of its buffer and is read whole by the first FFT stage before it writes)
constexpr size_t FZ_SMEM = 1024 + (256 + 240 + 256 + 2 * FZ_BUF) * sizeof(float2);  // + alignment slack
constexpr uint32_t FZ_STOP = 0xffffffffu;

// Bin k of line b to global memory at out[k * stride + b] with a streaming store.
struct GlobalOutCs {
  static constexpr bool kSyncFirst = false;
  static constexpr bool kJFast = false;
  float2* out;
  uint32_t stride;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const { __stcs(&out[size_t(k) * stride + b], v); }
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

struct FzItem {
  uint32_t pass, frame, strip;
};

// 256-point FFT of a row held by 16 lanes (lane jl: elements jl + 16 m in v[m]) as
// 16 x 16: the 16-point DFTs over m, a transpose through the row's shared buffer
// (XOR-swizzled), twiddles, the 16-point DFTs over the lanes' first digits. Bin
// jl + 16 m ends in v[m]. DIR -1 forward, +1 inverse (unscaled).
template <int DIR>
__device__ __forceinline__ void row_fft16x16(float2 (&v)[16], float2* rowp, const float2* tw2, int jl) {
  dft<16, DIR>(v);
  __syncwarp();
#pragma unroll
  for (int m = 0; m < 16; ++m) rowp[16 * jl + (m ^ jl)] = v[m];
  __syncwarp();
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    v[m] = rowp[16 * m + (jl ^ m)];
    if (m > 0) {
      float2 w = tw2[(m - 1) * 16 + jl];
      if (DIR > 0) w.y = -w.y;
      v[m] = cmul(v[m], w);
    }
  }
  dft<16, DIR>(v);
}

__global__ void __launch_bounds__(FZ_THREADS, 3)
    k_spatial_fused(SpatialArgs a, uint32_t nticket, const __grid_constant__ CUtensorMap raw_map,
                    const __grid_constant__ CUtensorMap s2_map) {
  extern __shared__ __align__(16) unsigned char smem[];
  // the two buffers first, 1024-byte aligned (bulk-copy destinations), then the tables
  unsigned char* base = smem + ((1024u - (rw_smem(smem) & 1023u)) & 1023u);
  float2* bufs = reinterpret_cast<float2*>(base);  // buffer b at bufs + b FZ_BUF
  float2* tws = bufs + 2 * FZ_BUF;
  float2* tw2 = tws + 256;
  float2* cys = tw2 + 240;
  // raw strip of buffer b: its last FZ_RAW bytes
  auto raw_of = [&](int b) {
    return reinterpret_cast<unsigned char*>(bufs + (b + 1) * FZ_BUF) - FZ_RAW;
  };
  __shared__ __align__(8) unsigned long long full[2], freed[2];
  __shared__ FzItem desc[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool asp = a.spatial == HV_SPATIAL_ASP;
  const bool u8 = a.in_kind == IN_U8;
  // items per ticket row (ASP: 8 + 8 + 8 + 16, Fresnel: 16 + 16), rows between passes
  const uint32_t ipr = asp ? 40u : 32u, R = a.ring;
  for (int e = tid; e < 256; e += FZ_THREADS) {
    tws[e] = __ldg(&a.tw_h[e]);
    cys[e] = asp ? make_float2(1.f, 0.f) : __ldg(&a.chirp_y[e]);
  }
  for (int e = tid; e < 240; e += FZ_THREADS) {
    const int m = e / 16 + 1, j = e % 16;
    tw2[e] = __ldg(&a.tw_w[j * m]);
  }
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      // full: the producer's arrival with the item's byte count, completed by its copy
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(rw_smem(&full[b])) : "memory");
      // freed: one arrival per consumer warp
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(rw_smem(&freed[b])), "n"(FZ_NT / 32) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  float2* const tq = static_cast<float2*>(a.tq.base);
  unsigned* const done = a.fused_ctr + 1;  // done[pass * R + slot]

  if (warp == FZ_NT / 32) {
    // ------------------------------------------------------------ producer (lane 0)
    if (lane != 0) return;
    uint64_t pol_first;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol_first));
    const long long limit = 1ll << 31;
    bool stuck = false;  // a wait for the consumers gave up
    // items are staged in order, item k into buffer k & 1; `issued` items were staged,
    // the first `published` of them transformed and counted. The counter of item k
    // sits at done[cnt0] or done[cnt1] (by k & 1) until it is published.
    uint32_t issued = 0, published = 0, cnt0 = 0, cnt1 = 0;
    // publish, in order, the items below `upto` whose transform is done; block: wait
    // for each (false when a wait gave up). Release-add: the consumers' stores, ordered
    // before this thread by the buffer's mbarrier, are visible at GPU scope before the
    // count; nothing waits on a reply.
    auto drain = [&](uint32_t upto, bool block) -> bool {
      const long long t0 = clock64();
      while (published < upto) {
        if (mbar_test(rw_smem(&freed[published & 1]), (published >> 1) & 1)) {
          const uint32_t c = (published & 1) ? cnt1 : cnt0;
          asm volatile("red.release.gpu.global.add.u32 [%0], 1;\n" ::"l"(&done[c]) : "memory");
          ++published;
        } else if (!block) {
          return true;
        } else if (clock64() - t0 > limit) {
          return false;
        }
      }
      return true;
    };
    // the next item with its counters satisfied, publishing finished items meanwhile;
    // false when the tickets are used up or a wait gave up
    auto prepare = [&](FzItem& it) -> bool {
      uint32_t pass, f, strip;
      while (true) {
        const uint32_t t = atomicAdd(a.fused_ctr, 1u);
        if (t >= nticket) return false;
        const uint32_t row = t / ipr, kk = t % ipr;
        pass = asp ? (kk < 24u ? kk >> 3 : 3u) : kk >> 4;
        strip = asp ? (kk < 24u ? kk & 7u : kk - 24u) : kk & 15u;
        const uint32_t off = !asp ? pass * FZ_LAG : pass == 0 ? 0u : FZ_LAG_ASP1 + (pass - 1) * FZ_LAG_ASP;
        const long long fl = (long long)row - (long long)off;
        if (fl >= 0 && fl < (long long)a.n) {
          f = uint32_t(fl);
          break;
        }
      }
      const uint32_t slot = f % R, gen = f / R;
      const long long t0 = clock64();
      while (true) {
        bool ready;
        if (!asp) ready = pass == 0 ? ld_acquire_u32(&done[R + slot]) >= 16u * gen
                                    : ld_acquire_u32(&done[slot]) >= 16u * (gen + 1);
        else if (pass == 0) ready = ld_acquire_u32(&done[R + slot]) >= 8u * gen;
        else if (pass == 1) ready = ld_acquire_u32(&done[slot]) >= 8u * (gen + 1) &&
                                    ld_acquire_u32(&done[3 * R + slot]) >= 16u * gen;
        else ready = ld_acquire_u32(&done[(pass - 1) * R + slot]) >= 8u * (gen + 1);
        if (a.stall && pass == 1) ready = false;  // fault injection: a condition nothing sets
        drain(issued, false);
        if (ready) break;
        if ((*reinterpret_cast<const volatile unsigned*>(a.err) & 16u) || clock64() - t0 > limit) {
          atomicOr(a.err, 16u);
          return false;
        }
        __nanosleep(32);
      }
      it = FzItem{pass, f, strip};
      return true;
    };
    // the next item is ready before its buffer frees, so that its copy starts the
    // moment the consumers are done with the item two before it
    FzItem it{0, 0, 0};
    bool more = prepare(it);
    while (more) {
      const uint32_t k = issued, b = k & 1;
      // buffer b is free once item k - 2 is transformed (published here, in order)
      if (k >= 2 && !drain(k - 1, true)) {
        stuck = true;
        atomicOr(a.err, 16u);
        break;
      }
      // one copy per item: the raw strip (256 rows x 16 pixels) and the column-IFFT
      // strip (256 rows x 16 complex) by a TMA tensor copy, the row pass's 16 rows
      // (contiguous) by a 1-D bulk copy. The rings were written by other CTAs'
      // generic stores, fenced for the async proxy before their publication; this
      // thread acquired the counters that published them.
      const uint32_t s0 = it.strip * (it.pass == 0 && asp ? 32u : 16u), slot = it.frame % R;
      const float2* s1 = a.scratch1 + size_t(slot) * FZ_FRAME;
      desc[b] = it;
      const uint32_t fb = rw_smem(&full[b]);
      if (it.pass == 0) {
        const uint32_t bytes = 256u * (asp ? 32u : 16u) * (u8 ? 1u : 2u);
        const uint32_t rslot = uint32_t((a.raw.slot0 + it.frame) % a.raw.cap);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint "
            "[%0], [%1, {%2, %3}], [%4], %5;\n" ::"r"(rw_smem(raw_of(b))),
            "l"(reinterpret_cast<uint64_t>(&raw_map)), "r"(int(s0)), "r"(int(rslot * 256u)), "r"(fb),
            "l"(pol_first)
            : "memory");
      } else if (it.pass == 1 || (asp && it.pass == 2)) {
        // 16 rows of S1 (row pass), or (mirror pass) the S3 rows 256 - r of its
        // output rows r = 143 + s0 - b, b = 0 .. 15: rows 113 - s0 .. 128 - s0; the
        // first strip's last row (r = 128) is the packed row S3(0)
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(32768u) : "memory");
        const float2* src = it.pass == 1 ? s1 + size_t(s0) * 256 : s1 + size_t(128 + 113 - s0) * 256;
        const uint32_t bytes = it.pass == 2 && s0 == 0 ? 15u * 2048u : 32768u;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                rw_smem(bufs + b * FZ_BUF)),
            "l"(src), "r"(bytes), "r"(fb)
            : "memory");
        if (bytes != 32768u)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                  rw_smem(bufs + b * FZ_BUF + 15 * 256)),
              "l"(s1 + size_t(128) * 256), "r"(2048u), "r"(fb)
              : "memory");
      } else {
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(32768u) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];\n" ::"r"(rw_smem(bufs + b * FZ_BUF)),
            "l"(reinterpret_cast<uint64_t>(&s2_map)), "r"(int(s0)), "r"(int(slot * 256u)), "r"(fb)
            : "memory");
      }
      const uint32_t c = it.pass * R + slot;
      if (b) cnt1 = c;
      else cnt0 = c;
      issued = k + 1;
      more = prepare(it);
    }
    // publish the rest as it finishes, then tell the consumers to stop (item `issued`,
    // whose buffer the last drain freed); if a wait gave up, the consumers' own
    // bounded waits end them
    if (!stuck && drain(issued, true)) {
      const int b = int(issued & 1);
      desc[b] = FzItem{FZ_STOP, 0, 0};
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(rw_smem(&full[b])) : "memory");
    } else {
      atomicOr(a.err, 16u);
    }
    return;
  }

  // ------------------------------------------------------------- consumers
  const int rb = 2 * warp + (lane >> 4), jl = lane & 15;  // row pass: row of the strip, lane in the row
  for (uint32_t k = 0;; ++k) {
    const int b = int(k & 1);
    if (!rw_wait(rw_smem(&full[b]), (k >> 1) & 1)) {
      if (tid == 0) atomicOr(a.err, 16u);
      break;
    }
    const FzItem it = desc[b];
    if (it.pass == FZ_STOP) break;
    const uint32_t pass = it.pass, f = it.frame, s0 = it.strip * (pass == 0 && asp ? 32u : 16u), slot = f % R;
    float2* buf = bufs + b * FZ_BUF;
    float2* s1 = a.scratch1 + size_t(slot) * FZ_FRAME;
    float2* s2 = a.scratch2 + size_t(slot) * FZ_FRAME;
    const size_t tslot = (a.tq.slot0 + f) % a.tq.cap;
    if (pass == 0) {
      const unsigned char* raw = raw_of(b);
      const GlobalOut out{s1 + s0, 256u};
      if (asp) {
        // column FFT of 32 real raw columns, packed in pairs (conversion in the first
        // stage), spectra Z of the 16 lines into the buffer [k][line]; then the two
        // columns' spectra A, B at bins 1 .. 127 -> S1 [ky][x], and at the real bins 0
        // and 128 packed as A(0) + i A(128), B(0) + i B(128) -> S1 row 0
        if (u8) pp_stages<256, 1, -1, PackedRawSrc<true>, SmemOut<16>, 16, FZ_BAR>(PackedRawSrc<true>{raw}, buf,
                                                                                    tws, SmemOut<16>{buf});
        else pp_stages<256, 1, -1, PackedRawSrc<false>, SmemOut<16>, 16, FZ_BAR>(PackedRawSrc<false>{raw}, buf,
                                                                                  tws, SmemOut<16>{buf});
        pp_sync<FZ_BAR, FZ_NT>();
        const int line = tid % 16;
        float4* o = reinterpret_cast<float4*>(s1 + s0 + 2 * line);  // columns 2 line, 2 line + 1
#pragma unroll
        for (int k = tid / 16; k < 128; k += FZ_NT / 16) {
          const float2 z = buf[k * 16 + line];  // Z(k)
          if (k == 0) {
            const float2 h = buf[128 * 16 + line];  // Z(128): A(128) = Re, B(128) = Im
            o[0] = make_float4(z.x, h.x, z.y, h.y);
          } else {
            const float2 w = buf[(256 - k) * 16 + line];                    // Z(-k)
            const float ax = 0.5f * (z.x + w.x), ay = 0.5f * (z.y - w.y);  // A(k) = (Z + conj W) / 2
            const float bx = 0.5f * (z.y + w.y), by = 0.5f * (w.x - z.x);  // B(k) = (Z - conj W) / 2i
            o[size_t(k) * 128] = make_float4(ax, ay, bx, by);
          }
        }
      } else {
        // column FFT of 16 raw columns (conversion and chirp in the first stage) -> S1 [ky][x]
        const float2 cx = __ldg(&a.chirp_x[s0 + (tid % 16)]);
        if (u8) pp_stages<256, 1, -1, RawSrc<true, true, 16, true>, GlobalOut, 16, FZ_BAR>(
                    RawSrc<true, true, 16, true>{raw, cys, cx}, buf, tws, out);
        else pp_stages<256, 1, -1, RawSrc<false, true, 16, true>, GlobalOut, 16, FZ_BAR>(
                 RawSrc<false, true, 16, true>{raw, cys, cx}, buf, tws, out);
      }
    } else if (pass == 3 || (pass == 1 && !asp)) {
      if (asp) {
        // column IFFT of 16 columns x = s0 .. s0 + 15 of S2 -> time queue [y][x]
        asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(s2 + s0 + size_t(tid) * 256) : "memory");
        pp_stages<256, 1, +1, SmemSrc<16>, GlobalOutCs, 16, FZ_BAR>(SmemSrc<16>{buf}, buf, tws,
                                                                    GlobalOutCs{tq + tslot * FZ_FRAME + s0, 256u});
      } else {
        // 16 rows ky = s0 .. s0 + 15 of S1 -> row FFT -> time queue [ky][kx]
        asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(s1 + size_t(s0) * 256 + size_t(tid) * 16) : "memory");
        float2* rowp = buf + rb * 256;
        float2 v[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = rowp[jl + 16 * m];
        row_fft16x16<-1>(v, rowp, tw2, jl);
        float2* out = tq + (tslot * 256 + size_t(s0 + rb)) * 256;
#pragma unroll
        for (int m = 0; m < 16; ++m) __stcs(&out[jl + 16 * m], v[m]);
      }
    } else {
      float2* rowp = buf + rb * 256;
      float2 v[16];
      int ky;
      if (pass == 1) {
        // rows ky = s0 .. s0 + 15 of S1 (row 0 packed with row 128): forward row FFT,
        // kept in S3 for the mirror pass; the staged strip of S1 is dead: drop its
        // L2 lines unwritten
        asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(s1 + size_t(s0) * 256 + size_t(tid) * 16) : "memory");
        ky = int(s0) + rb;
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = rowp[jl + 16 * m];
        row_fft16x16<-1>(v, rowp, tw2, jl);
        float2* w3 = s1 + size_t(128 + ky) * 256;
#pragma unroll
        for (int m = 0; m < 16; ++m) w3[jl + 16 * m] = v[m];
        if (s0 == 0 && warp == 0) {
          // row 0: W(0, k) = (Wp(k) + conj Wp(-k)) / 2 through the row's buffer
          __syncwarp();
#pragma unroll
          for (int m = 0; m < 16; ++m) rowp[jl + 16 * m] = v[m];
          __syncwarp();
          if (rb == 0) {
#pragma unroll
            for (int m = 0; m < 16; ++m) {
              const float2 w = rowp[(256 - jl - 16 * m) & 255];
              v[m] = make_float2(0.5f * (v[m].x + w.x), 0.5f * (v[m].y - w.y));
            }
          }
        }
      } else {
        // mirror rows ky = 143 + s0 - b of buffer row b, spectrum conj W(256 - ky, -kx);
        // row 128 from the packed row: W(128, k) = (Wp(k) - conj Wp(-k)) / 2i. The
        // staged rows of S3 are dead (16 threads a row; the first strip's last 16
        // threads reach S3 row 0 from 15 rows before it)
        const float2* w3 = s1 + size_t(s0 == 0 && tid >= 240 ? 128 - 15 : 128 + 113 - s0) * 256;
        asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(w3 + size_t(tid) * 16) : "memory");
        ky = 143 + int(s0) - rb;
        if (ky == 128) {
#pragma unroll
          for (int m = 0; m < 16; ++m) {
            const float2 z = rowp[jl + 16 * m], w = rowp[(256 - jl - 16 * m) & 255];
            v[m] = make_float2(0.5f * (z.y + w.y), 0.5f * (w.x - z.x));
          }
        } else {
#pragma unroll
          for (int m = 0; m < 16; ++m) {
            const float2 w = rowp[(256 - jl - 16 * m) & 255];
            v[m] = make_float2(w.x, -w.y);
          }
        }
      }
      // x H(ky), inverse row FFT -> S2 [ky][x]
      const float2* hrow = a.asp_h + size_t(ky) * 256;
#pragma unroll
      for (int m = 0; m < 16; ++m) v[m] = cmul(v[m], __ldg(&hrow[jl + 16 * m]));
      row_fft16x16<+1>(v, rowp, tw2, jl);
      float2* out = s2 + size_t(ky) * 256;
#pragma unroll
      for (int m = 0; m < 16; ++m) out[jl + 16 * m] = v[m];
    }
    // the ring stores are read back by bulk copies (the async proxy) of other CTAs
    if (pass == 0 || (asp && pass < 3)) asm volatile("fence.proxy.async.global;\n" ::: "memory");
    // this warp is done with the buffer and has issued its stores: each warp releases
    // the buffer on its own and goes on to the next staged item (a column pass's
    // named barriers keep the warps in step within an item)
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(rw_smem(&freed[b])) : "memory");
  }
}

}  // namespace

cudaError_t launch_pp_pass(const SpatialArgs& a, int pass, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (!spatial_pp_supported(a)) return cudaErrorInvalidValue;
  switch (pass) {
    case PASS_COL_FFT: return pass_by_len<PK_P1>(a, s);
    case PASS_ROW_ASP: return pass_by_len<PK_P2A>(a, s);
    case PASS_COL_IFFT: return pass_by_len<PK_P3A>(a, s);
    case PASS_ROW_FFT: return pass_by_len<PK_P2F>(a, s);
    case PASS_COL_IFFT_TAMURA: return pass_by_len<PK_P3T>(a, s);
    case PASS_ROW_CELLS:
      // the cell epilogue pairs rows and bins across lanes: 16 butterflies per line in the last stage
      if (a.W > 256 || a.H > 1024) return cudaErrorInvalidValue;
      return pass_by_len<PK_P2C>(a, s);
  }
  return cudaErrorInvalidValue;
}

bool spatial_pp_supported(const SpatialArgs& a) {
  auto ok = [](uint32_t v) { return v >= 64 && v <= 1024; };  // two strip buffers must fit
  return ok(a.W) && ok(a.H) && (a.spatial == HV_SPATIAL_ASP || a.spatial == HV_SPATIAL_FRESNEL);
}

cudaError_t launch_spatial_pp(const SpatialArgs& a0, cudaStream_t s, int* launches) {
  if (a0.n == 0) return cudaSuccess;
  SpatialArgs a = a0;
  a.discard_inputs = 1;  // the full transform reads each intermediate exactly once
  switch (a.H) {
    case 64: return pp_w<64>(a, s, launches);
    case 128: return pp_w<128>(a, s, launches);
    case 256: return pp_w<256>(a, s, launches);
    case 512: return pp_w<512>(a, s, launches);
    case 1024: return pp_w<1024>(a, s, launches);
  }
  return cudaErrorInvalidValue;
}

bool spatial_fused_supported(const SpatialArgs& a) {
  return a.W == RW_L && a.H == RW_L && (a.spatial == HV_SPATIAL_ASP || a.spatial == HV_SPATIAL_FRESNEL) &&
         a.ring >= kFusedRing && a.fused_ctr && a.err && a.scratch1 &&
         (a.spatial == HV_SPATIAL_FRESNEL || (a.scratch2 && a.asp_h));
}

cudaError_t launch_spatial_fused(const SpatialArgs& a, cudaStream_t s, int* launches) {
  if (a.n == 0) return cudaSuccess;
  if (!spatial_fused_supported(a)) return cudaErrorInvalidValue;
  const bool asp = a.spatial == HV_SPATIAL_ASP;
  // ticket rows: one per frame plus the lags of the last pass; items per row
  const uint64_t nt = (uint64_t(a.n) + (asp ? FZ_LAG_ASP1 + 2u * FZ_LAG_ASP : FZ_LAG)) * (asp ? 40u : 32u);
  if (nt >= (1ull << 31)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.fused_ctr, 0, (1 + kFusedPasses * size_t(a.ring)) * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_spatial_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, int(FZ_SMEM));
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, nsm = 0;
  // tensor maps: the raw ring (256 x cap 256 pixels, boxes of 32 (ASP) or 16 x 256) and
  // the S2 ring (256 x ring 256 complex, boxes of 16 x 256)
  CUtensorMap raw_map{}, s2_map{};
  const int bpp = a.in_kind == IN_U8 ? 1 : 2;
  if (!encode_map_2d(&raw_map, a.raw.base, bpp, RW_L, uint64_t(a.raw.cap) * RW_L, uint64_t(RW_L) * bpp,
                     a.spatial == HV_SPATIAL_ASP ? 32 : 16, 256))
    return cudaErrorNotSupported;
  if (a.spatial == HV_SPATIAL_ASP &&
      !encode_map_2d(&s2_map, a.scratch2, 8, RW_L, uint64_t(a.ring) * RW_L, uint64_t(RW_L) * 8, 16, 256))
    return cudaErrorNotSupported;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spatial_fused, FZ_THREADS, FZ_SMEM);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  uint64_t grid = uint64_t(per_sm) * nsm;  // every CTA resident: the items' waits rely on it
  if (grid > nt) grid = nt;
  k_spatial_fused<<<unsigned(grid), FZ_THREADS, FZ_SMEM, s>>>(a, uint32_t(nt), raw_map, s2_map);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace hv
