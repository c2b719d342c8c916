// fft_dev.cuh -- device building blocks for batched complex FFTs in shared memory.
//
// The spatial transforms (FFT2 of every frame, Sec. III-B.1) and the temporal
// transform (FFT along the frame axis of every pixel) are both many independent
// 1-D FFTs of one power-of-two length L. A CTA holds BT of them side by side in
// shared memory with the batch index fastest: element t of line b lives at
// buf[t * LD + b]. Batch-fastest means every global load and store of a line
// segment is coalesced and every shared-memory stage access by a warp is a
// contiguous run along b (conflict-free).
//
// Algorithm: Stockham autosort decimation in time, radix 16 where the thread
// layout allows it, else radix 8 while the remaining length allows, then 4 or 2. Stage with span NS (product of the
// radices already applied) and radix R: butterfly j in [0, L/R) reads the R
// inputs j + m L/R, multiplies input m by w_L^{(j mod NS) m L/(NS R)}, applies an
// R-point DFT, and writes output m to (j / NS) NS R + (j mod NS) + m NS. The
// last stage leaves bin k = j + m L/R of butterfly j in registers and hands it
// to an epilogue. Twiddles come from a per-length table w_L^e = exp(-2 pi i e/L)
// computed in float64 on the host and rounded to float.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hv {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// v * (DIR * i): DIR = -1 is the forward transform's -i, DIR = +1 the inverse's +i.
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 v) {
  if constexpr (DIR < 0) return make_float2(v.y, -v.x);
  else return make_float2(-v.y, v.x);
}

// v * exp(DIR 2 pi i e / 16) for the exponents a 16-point DFT uses.
template <int E, int DIR>
__device__ __forceinline__ float2 tw16(float2 v) {
  constexpr float C1 = 0.92387953251128675613f;  // cos(pi/8)
  constexpr float S1 = 0.38268343236508977173f;  // sin(pi/8)
  constexpr float R2 = 0.70710678118654752440f;  // cos(pi/4)
  constexpr float c = E == 1 ? C1 : E == 2 ? R2 : E == 3 ? S1 : E == 6 ? -R2 : -C1;
  constexpr float s = E == 1 ? S1 : E == 2 ? R2 : E == 3 ? C1 : E == 6 ? R2 : -S1;
  if constexpr (E == 4) return mul_i<DIR>(v);
  else return make_float2(fmaf(v.x, c, -v.y * (DIR * s)), fmaf(v.y, c, v.x * (DIR * s)));
}

// v * exp(DIR 2 pi i k / 32), k = 0..15 (k a compile-time constant after unrolling).
template <int DIR>
__device__ __forceinline__ float2 tw32(float2 v, int k) {
  constexpr float C[16] = {
      1.00000000000000000000f,
      0.98078528040323043058f,
      0.92387953251128673848f,
      0.83146961230254523567f,
      0.70710678118654757274f,
      0.55557023301960228867f,
      0.38268343236508983729f,
      0.19509032201612833135f,
      0.00000000000000006123f,
      -0.19509032201612819257f,
      -0.38268343236508972627f,
      -0.55557023301960195560f,
      -0.70710678118654746172f,
      -0.83146961230254534669f,
      -0.92387953251128673848f,
      -0.98078528040323043058f};
  constexpr float S[16] = {
      0.00000000000000000000f,
      0.19509032201612824808f,
      0.38268343236508978178f,
      0.55557023301960217765f,
      0.70710678118654746172f,
      0.83146961230254523567f,
      0.92387953251128673848f,
      0.98078528040323043058f,
      1.00000000000000000000f,
      0.98078528040323043058f,
      0.92387953251128673848f,
      0.83146961230254545772f,
      0.70710678118654757274f,
      0.55557023301960217765f,
      0.38268343236508989280f,
      0.19509032201612860891f};
  const float c = C[k], s = DIR * S[k];
  return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.y, c, v.x * s));
}

// Packed FP32x2 arithmetic (sm_100 and later): a complex addition or
// subtraction is one instruction on the (re, im) register pair.
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, exact product by -1
}

// In-register R-point DFT, X_k = sum_m v_m exp(DIR 2 pi i m k / R), R in {2, 4, 8, 16, 32}.
// Complex sums and differences use the packed additions; products by twiddles
// (and by +-i, a swap of the pair) stay per component.
template <int R, int DIR>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = padd(a, b);
    v[1] = psub(a, b);
  } else if constexpr (R == 4) {
    const float2 t0 = padd(v[0], v[2]), t1 = psub(v[0], v[2]);
    const float2 t2 = padd(v[1], v[3]), d = psub(v[1], v[3]);
    v[0] = padd(t0, t2);
    v[2] = psub(t0, t2);
    // X1 = t1 + (DIR i) d, X3 = t1 - (DIR i) d; (DIR i) d = (-DIR d.y, DIR d.x)
    if constexpr (DIR < 0) {
      v[1] = make_float2(t1.x + d.y, t1.y - d.x);
      v[3] = make_float2(t1.x - d.y, t1.y + d.x);
    } else {
      v[1] = make_float2(t1.x - d.y, t1.y + d.x);
      v[3] = make_float2(t1.x + d.y, t1.y - d.x);
    }
  } else if constexpr (R == 16) {
    // 16 = 4 x 4: DFT4 over n1 of x[4 n1 + n2], twiddle w16^(n2 k1), DFT4 over n2
    float2 a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      a[n2][0] = v[n2];
      a[n2][1] = v[4 + n2];
      a[n2][2] = v[8 + n2];
      a[n2][3] = v[12 + n2];
      dft<4, DIR>(a[n2]);
    }
    a[1][1] = tw16<1, DIR>(a[1][1]);
    a[1][2] = tw16<2, DIR>(a[1][2]);
    a[1][3] = tw16<3, DIR>(a[1][3]);
    a[2][1] = tw16<2, DIR>(a[2][1]);
    a[2][2] = tw16<4, DIR>(a[2][2]);
    a[2][3] = tw16<6, DIR>(a[2][3]);
    a[3][1] = tw16<3, DIR>(a[3][1]);
    a[3][2] = tw16<6, DIR>(a[3][2]);
    a[3][3] = tw16<9, DIR>(a[3][3]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
      dft<4, DIR>(b);
      v[k1] = b[0];
      v[k1 + 4] = b[1];
      v[k1 + 8] = b[2];
      v[k1 + 12] = b[3];
    }
  } else if constexpr (R == 32) {
    // 32 = 2 x 16: DFT16 of even and odd samples, X_k = E_k + w32^k O_k, X_{k+16} = E_k - w32^k O_k
    float2 e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    dft<16, DIR>(e);
    dft<16, DIR>(o);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 t = tw32<DIR>(o[k], k);
      v[k] = padd(e[k], t);
      v[k + 16] = psub(e[k], t);
    }
  } else {
    static_assert(R == 8, "radix");
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft<4, DIR>(e);
    dft<4, DIR>(o);
    const float c = 0.70710678118654752440f;
    // o_k *= exp(DIR 2 pi i k / 8)
    const float2 o1 = make_float2(c * (o[1].x - DIR * o[1].y), c * (o[1].y + DIR * o[1].x));
    const float2 o2 = mul_i<DIR>(o[2]);
    const float2 o3 = make_float2(c * (-o[3].x - DIR * o[3].y), c * (-o[3].y + DIR * o[3].x));
    v[0] = padd(e[0], o[0]);
    v[4] = psub(e[0], o[0]);
    v[1] = padd(e[1], o1);
    v[5] = psub(e[1], o1);
    v[2] = padd(e[2], o2);
    v[6] = psub(e[2], o2);
    v[3] = padd(e[3], o3);
    v[7] = psub(e[3], o3);
  }
}

// Radix 8 while the remaining length allows it, then 4 or 2.
template <int REM>
struct RadixOf {
  static constexpr int value = (REM % 8 == 0) ? 8 : ((REM % 4 == 0) ? 4 : 2);
};

// Radix of a block-wide stage: 16 where every thread gets whole butterflies
// (fewer passes through shared memory), else as RadixOf.
template <int REM, int L, int BT, int NT>
struct BlockRadix {
  static constexpr bool r16 = REM % 16 == 0 && (BT * (L / 16)) % NT == 0 && BT * (L / 16) >= NT;
  static constexpr int value = r16 ? 16 : RadixOf<REM>::value;
};

// Threads per CTA for BT lines of length L: one radix-8 butterfly pair per
// thread (<= 16 complex values in registers per stage), clamped to [32, 1024].
template <int L, int BT>
struct FftThreads {
  static constexpr int raw = BT * L / 16;
  static constexpr int value = raw < 32 ? 32 : (raw > 1024 ? 1024 : raw);
};

// One Stockham stage and (recursively) the rest. `src` holds the stage input
// with leading dimension src_ld (it may alias buf); intermediate stages write
// buf (leading dimension LD). The last stage calls epi(b, k, value) for every
// output bin, after a barrier (so the epilogue may overwrite buf).
template <int L, int NS, int DIR, int BT, int NT, int LD, class Epi>
__device__ __forceinline__ void fft_stages(const float2* src, int src_ld, float2* buf,
                                           const float2* __restrict__ tw, Epi& epi) {
  constexpr int REM = L / NS;
  constexpr int R = BlockRadix<REM, L, BT, NT>::value;
  constexpr int NB = L / R;
  static_assert((BT * NB) % NT == 0, "thread count must divide the butterflies");
  constexpr int ITEMS = BT * NB / NT;
  static_assert(ITEMS >= 1, "too many threads");
  float2 v[ITEMS][R];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int idx = threadIdx.x + it * NT;
    const int b = idx % BT, j = idx / BT;
#pragma unroll
    for (int m = 0; m < R; ++m) v[it][m] = src[(j + m * NB) * src_ld + b];
    if constexpr (NS > 1) {
      const int jm = j % NS;
#pragma unroll
      for (int m = 1; m < R; ++m) {
        float2 w = __ldg(&tw[jm * m * (L / (NS * R))]);
        if constexpr (DIR > 0) w.y = -w.y;
        v[it][m] = cmul(v[it][m], w);
      }
    }
    dft<R, DIR>(v[it]);
  }
  __syncthreads();
  if constexpr (NS * R == L) {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int idx = threadIdx.x + it * NT;
      const int b = idx % BT, j = idx / BT;
#pragma unroll
      for (int m = 0; m < R; ++m) epi(b, j + m * NB, v[it][m]);
    }
  } else {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int idx = threadIdx.x + it * NT;
      const int b = idx % BT, j = idx / BT;
      const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int m = 0; m < R; ++m) buf[(base + m * NS) * LD + b] = v[it][m];
    }
    __syncthreads();
    fft_stages<L, NS * R, DIR, BT, NT, LD, Epi>(buf, LD, buf, tw, epi);
  }
}

// Full FFT of the BT lines in buf (in place through registers).
template <int L, int DIR, int BT, int NT, int LD, class Epi>
__device__ __forceinline__ void fft_lines(float2* buf, const float2* __restrict__ tw, Epi& epi) {
  fft_stages<L, 1, DIR, BT, NT, LD, Epi>(buf, LD, buf, tw, epi);
}

// Epilogue that stores bin k of line b back to buf in natural order.
template <int LD>
struct StoreSmem {
  float2* buf;
  __device__ __forceinline__ void operator()(int b, int k, float2 v) const { buf[k * LD + b] = v; }
};

}  // namespace hv
