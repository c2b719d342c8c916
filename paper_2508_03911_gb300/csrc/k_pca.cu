// k_pca.cu -- PCA temporal analysis of one window (Sec. III-B.1: a covariance
// matrix of the window, its eigendecomposition, projection onto a sub-basis).
//
// With X the P x T matrix whose column t is propagated frame t (P = W H):
//   C = X^H X                      (T x T Hermitian, unnormalised)
//   C = V diag(lam) V^H            (cyclic complex Jacobi, float64)
//   E(p) = sum_{j = lo..hi} |(X v_j)_p|^2, eigenvectors ranked by descending lam.
//
// Kernels (all on the handle's stream; windows of T <= 64 frames are batched,
// blockIdx.z / blockIdx.y / blockIdx.x selecting the window where noted):
//   k_cov_fp32     split-K covariance: each CTA multiplies a 64 x 64 tile of the
//                  upper triangle over one pixel chunk (float32 FMA), partials
//                  written per chunk (deterministic, no atomics)
//   k_cov_reduce   sums the chunk partials in float64 -> C (full Hermitian), V = I
//   k_jacobi_cluster, k_jacobi_f32
//                  float32 phase of the long-window eigensolver (T > 64, one
//                  window): parallel cyclic (round-robin) two-sided Jacobi on one
//                  16-CTA cluster, or cooperative on a quarter of the SMs
//   k_gemm_c64     float64 congruence C' = Vf^H C Vf
//   k_jacobi_refine cooperative refinement sweeps on C' over all SMs: float64
//                  diagonal and V, float32 off-diagonal entries
//   k_jacobi_small both phases for T <= 64, one CTA per window, C and V in
//                  shared memory, selection of the sub-basis fused
//   k_pca_select   ranks eigenvalues (descending) and gathers the sub-basis
//   k_project      Y = X V_s for 64-pixel tiles and E(p) = sum_j |Y_pj|^2
#include <cooperative_groups.h>

#include "fft_dev.cuh"
#include "hv_internal.h"
#include "../../include/hv.h"

namespace cg = cooperative_groups;

namespace hv {

// ----------------------------------------------------------------- covariance

constexpr int COV_TS = 64;   // output tile (frames x frames)
constexpr int COV_KS = 32;   // pixels per smem stage

// Frame t of the ring from slot0 on. slot0 < cap and t < cap (launch_pca checks
// both for every window of a launch), so one conditional subtraction wraps it.
__device__ __forceinline__ const float2* frame_ptr(const RingRef& r, uint32_t t, size_t hw) {
  uint32_t slot = r.slot0 + t;
  if (slot >= r.cap) slot -= r.cap;
  return static_cast<const float2*>(r.base) + size_t(slot) * hw;
}

// Frame t of window w (windows start S frames apart).
__device__ __forceinline__ const float2* win_frame(const PcaArgs& a, uint32_t w, uint32_t t, size_t hw) {
  return frame_ptr(a.tq, w * a.wstride + t, hw);
}

// grid (n_upper_tiles, n_chunks), 256 threads; thread (ty, tx) owns rows
// a0 + ty + 16 i and columns b0 + tx + 16 j of the TS x TS tile (TS = min(T, 64)).
__global__ void __launch_bounds__(256) k_cov_fp32(PcaArgs a) {
  __shared__ float2 As[COV_KS][COV_TS + 1];
  __shared__ float2 Bs[COV_KS][COV_TS + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int TS = a.T < COV_TS ? int(a.T) : COV_TS;
  const int nI = TS / 16;
  const int nT = a.T / TS;
  int u = blockIdx.x, ta = 0;
  while (u >= nT - ta) {
    u -= nT - ta;
    ++ta;
  }
  const int tb = ta + u;
  const size_t hw = size_t(a.W) * a.H;
  const size_t p_begin = size_t(blockIdx.y) * a.chunk;
  const size_t p_end = p_begin + a.chunk < hw ? p_begin + a.chunk : hw;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (size_t p0 = p_begin; p0 < p_end; p0 += COV_KS) {
    for (int e = tid; e < TS * COV_KS; e += 256) {
      const int k = e % COV_KS, f = e / COV_KS;
      const size_t p = p0 + k;
      float2 va = make_float2(0.f, 0.f), vb = va;
      if (p < p_end) {
        va = win_frame(a, blockIdx.z, ta * TS + f, hw)[p];
        vb = win_frame(a, blockIdx.z, tb * TS + f, hw)[p];
      }
      As[k][f] = va;
      Bs[k][f] = vb;
    }
    __syncthreads();
    if (ty < TS && tx < TS) {
#pragma unroll 4
      for (int k = 0; k < COV_KS; ++k) {
        float2 x[4], y[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = i < nI ? As[k][ty + 16 * i] : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] = j < nI ? Bs[k][tx + 16 * j] : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // conj(x) * y
            acc[i][j].x = fmaf(x[i].x, y[j].x, fmaf(x[i].y, y[j].y, acc[i][j].x));
            acc[i][j].y = fmaf(x[i].x, y[j].y, fmaf(-x[i].y, y[j].x, acc[i][j].y));
          }
      }
    }
    __syncthreads();
  }
  const int ntile_up = nT * (nT + 1) / 2;
  float2* out = a.partials + ((size_t(blockIdx.z) * a.nchunks + blockIdx.y) * ntile_up + blockIdx.x) * TS * TS;
  for (int i = 0; i < nI; ++i)
    for (int j = 0; j < nI; ++j) out[(ty + 16 * i) * TS + tx + 16 * j] = acc[i][j];
}

// C[a][b] = sum over chunks (float64), mirrored to the lower triangle; V = I.
__global__ void k_cov_reduce(PcaArgs a) {
  const int T = a.T, TS = T < COV_TS ? T : COV_TS, nT = T / TS, ntile_up = nT * (nT + 1) / 2;
  for (int ew = blockIdx.x * blockDim.x + threadIdx.x; ew < int(a.nwin) * T * T; ew += gridDim.x * blockDim.x) {
    const int w = ew / (T * T), e = ew % (T * T);
    const int r = e / T, c = e % T;
    double2* Cw = a.C + size_t(w) * T * T;
    const float2* Pw = a.partials + size_t(w) * a.nchunks * ntile_up * TS * TS;
    if (w == 0) a.V[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    if (r > c) continue;
    const int ta = r / TS, tb = c / TS;
    const int up = ta * nT - ta * (ta - 1) / 2 + (tb - ta);
    const int off = (r % TS) * TS + (c % TS);
    double sx = 0.0, sy = 0.0;
    for (uint32_t k = 0; k < a.nchunks; ++k) {
      const float2 v = Pw[(size_t(k) * ntile_up + up) * TS * TS + off];
      sx += v.x;
      sy += v.y;
    }
    if (r == c) {
      sy = 0.0;
      // non-negative doubles order like their bit patterns
      atomicMax(reinterpret_cast<unsigned long long*>(a.cmax),
                static_cast<unsigned long long>(__double_as_longlong(sx > 0.0 ? sx : 0.0)));
    }
    Cw[r * T + c] = make_double2(sx, sy);
    Cw[c * T + r] = make_double2(sx, -sy);
  }
}

// ------------------------------------------------------------------ Jacobi

// Round robin (circle method): position 0 holds index 0, position k >= 1 holds
// ((k - 1 + r) mod (T - 1)) + 1; pair p of round r is (pos p, pos T-1-p).
__device__ __forceinline__ int rr_elem(int k, int r, int T) {
  return k == 0 ? 0 : ((k - 1 + r) % (T - 1)) + 1;
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Rotation J = [[c, -s], [conj(ph) s, conj(ph) c]] (c, s real, |ph| = 1) that
// zeroes the off-diagonal of the Hermitian 2 x 2 block [[al, g], [conj(g), be]]:
// J = P R, P = diag(1, conj(g)/|g|), R a real rotation with tan(2 theta) =
// 2|g| / (al - be); identity when |g| is below either bound.
struct RotF {
  float c, s, px, py;
};

__device__ __forceinline__ bool jacobi_rot_f(float al, float be, float2 g, float tol, float floor_abs, RotF& q) {
  const float ag = sqrtf(g.x * g.x + g.y * g.y);
  q = RotF{1.f, 0.f, 1.f, 0.f};
  if (!(ag > tol * sqrtf(fabsf(al * be)) && ag > floor_abs && ag > 0.f)) return false;
  const float zeta = (be - al) / (2.f * ag);
  const float t = -(zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  const float c = 1.f / sqrtf(1.f + t * t);
  q = RotF{c, t * c, g.x / ag, g.y / ag};
  return true;
}

// B <- Jp^H B Jq for the 2 x 2 block of rows (i0, i1) and columns (j0, j1) of the
// row-major T x T matrix, read from Cs and written to C (may be the same); `own`
// marks the pair's own diagonal block, whose off-diagonal is set to zero.
__device__ __forceinline__ void jacobi_block_f2(const float2* Cs, float2* C, int T, int i0, int i1, int j0, int j1,
                                                const RotF& Jp, const RotF& Jq, bool own) {
  const float2 b00 = Cs[i0 * T + j0], b01 = Cs[i0 * T + j1], b10 = Cs[i1 * T + j0], b11 = Cs[i1 * T + j1];
  const float2 q10 = make_float2(Jq.px * Jq.s, -Jq.py * Jq.s), q11 = make_float2(Jq.px * Jq.c, -Jq.py * Jq.c);
  const float2 m00 = cadd(cscale(b00, Jq.c), cmul(b01, q10)), m01 = cadd(cscale(b00, -Jq.s), cmul(b01, q11));
  const float2 m10 = cadd(cscale(b10, Jq.c), cmul(b11, q10)), m11 = cadd(cscale(b10, -Jq.s), cmul(b11, q11));
  const float2 p01 = make_float2(Jp.px * Jp.s, Jp.py * Jp.s), p11 = make_float2(Jp.px * Jp.c, Jp.py * Jp.c);
  float2 c00 = cadd(cscale(m00, Jp.c), cmul(p01, m10)), c01 = cadd(cscale(m01, Jp.c), cmul(p01, m11));
  float2 c10 = cadd(cscale(m00, -Jp.s), cmul(p11, m10)), c11 = cadd(cscale(m01, -Jp.s), cmul(p11, m11));
  if (own) {
    c01 = make_float2(0.f, 0.f);
    c10 = make_float2(0.f, 0.f);
    c00.y = 0.f;
    c11.y = 0.f;
  }
  C[i0 * T + j0] = c00;
  C[i0 * T + j1] = c01;
  C[i1 * T + j0] = c10;
  C[i1 * T + j1] = c11;
}

__device__ __forceinline__ void jacobi_block_f(float2* C, int T, int i0, int i1, int j0, int j1, const RotF& Jp,
                                               const RotF& Jq, bool own) {
  jacobi_block_f2(C, C, T, i0, i1, j0, j1, Jp, Jq, own);
}

// Columns (j0, j1) of row `row` of V times Jq.
__device__ __forceinline__ void jacobi_vrow_f(float2* V, int T, int row, int j0, int j1, const RotF& Jq) {
  const float2 v0 = V[row * T + j0], v1 = V[row * T + j1];
  const float2 q10 = make_float2(Jq.px * Jq.s, -Jq.py * Jq.s), q11 = make_float2(Jq.px * Jq.c, -Jq.py * Jq.c);
  V[row * T + j0] = cadd(cscale(v0, Jq.c), cmul(v1, q10));
  V[row * T + j1] = cadd(cscale(v0, -Jq.s), cmul(v1, q11));
}

// Float64 rotation of the refinement sweeps with its column factors
// q10 = conj(ph) s and q11 = conj(ph) c precomputed (J = [[c, -s], [q10, q11]]).
struct RotV {
  double c, s;
  double2 q10, q11;
};

// Columns (j0, j1) of row `row` of the float64 V times Jq.
__device__ __forceinline__ void refine_vrow(double2* V, int T, int row, int j0, int j1, const RotV& Jq) {
  const double2 v0 = V[row * T + j0], v1 = V[row * T + j1];
  V[row * T + j0] = make_double2(fma(Jq.c, v0.x, fma(Jq.q10.x, v1.x, -Jq.q10.y * v1.y)),
                                 fma(Jq.c, v0.y, fma(Jq.q10.x, v1.y, Jq.q10.y * v1.x)));
  V[row * T + j1] = make_double2(fma(-Jq.s, v0.x, fma(Jq.q11.x, v1.x, -Jq.q11.y * v1.y)),
                                 fma(-Jq.s, v0.y, fma(Jq.q11.x, v1.y, Jq.q11.y * v1.x)));
}

// Rotation of a refinement sweep for the pair (i, j): the diagonal d in float64,
// the off-diagonal entry g in float32 (ag = |g|). The angle (tan theta = t, the root of
// t^2 - 2 zeta t - 1 = 0 of smaller magnitude, zeta = (d_j - d_i) / (2 |g|)) is
// taken in float32; the float64 factors c = (1 + t^2)^(-1/2) and ph = g / |g|
// come from the float32 inverse square roots refined by one Newton step each,
// so that J is unitary to about 1e-13 whatever the angle's own rounding. The
// diagonal moves by t |g| (d_i + t |g|, d_j - t |g|, the exact result of the
// rotation that zeroes g; an angle off by a relative 1e-7 changes it only in
// the second order and leaves 1e-7 |g| behind in the zeroed entry).
__device__ __forceinline__ bool refine_rot(double* d, int i, int j, float2 g, float ag, float tol, float floor_abs,
                                           RotF& qf, RotV& qv) {
  qf = RotF{1.f, 0.f, 1.f, 0.f};
  qv = RotV{1.0, 0.0, make_double2(0.0, 0.0), make_double2(1.0, 0.0)};
  const double al = d[i], be = d[j];
  if (!(ag > tol * sqrtf(fabsf(float(al))) * sqrtf(fabsf(float(be))) && ag > floor_abs && ag > 0.f)) return false;
  const float zeta = float(be - al) / (2.f * ag);
  const float az = fabsf(zeta);
  const float den = az > 1e18f ? 2.f * az : az + sqrtf(fmaf(az, az, 1.f));
  const float t = (zeta >= 0.f ? -1.f : 1.f) / den;
  if (t == 0.f) return false;
  const double td = t;
  const double x = fma(td, td, 1.0);
  double c = rsqrtf(float(x));
  c = fma(0.5 * c, fma(-x * c, c, 1.0), c);  // c <- c (3 - x c^2) / 2
  const double s = td * c;
  const double gx = g.x, gy = g.y, g2 = fma(gx, gx, gy * gy);
  double rg = 1.f / ag;
  rg = fma(0.5 * rg, fma(-g2 * rg, rg, 1.0), rg);  // rg -> g2^(-1/2)
  const double px = gx * rg, py = gy * rg;
  const double tg = td * (g2 * rg);
  d[i] = al + tg;
  d[j] = be - tg;
  qv = RotV{c, s, make_double2(px * s, -py * s), make_double2(px * c, -py * c)};
  qf = RotF{float(c), float(s), float(px), float(py)};
  return true;
}

// The rotation of refine_rot for the cluster's refinement, whose rotations are
// applied in float32 (the float64 refinement of c and ph would be rounded away):
// the angle and the factors in float32 (approximate reciprocals, a few ulp), the
// diagonal moved by t |g| in float64.
__device__ __forceinline__ void refine_rot_f(double* d, int i, int j, float2 g, float ag, float tol,
                                             float floor_abs, RotF& q) {
  q = RotF{1.f, 0.f, 1.f, 0.f};
  const double al = d[i], be = d[j];
  if (!(ag > tol * sqrtf(fabsf(float(al))) * sqrtf(fabsf(float(be))) && ag > floor_abs && ag > 0.f)) return;
  const float rg = __fdividef(1.f, ag);
  const float zeta = float(be - al) * (0.5f * rg);
  const float az = fabsf(zeta);
  const float den = az > 1e18f ? 2.f * az : az + sqrtf(fmaf(az, az, 1.f));
  const float t = __fdividef(zeta >= 0.f ? -1.f : 1.f, den);
  if (t == 0.f) return;
  const float c = rsqrtf(fmaf(t, t, 1.f));
  const double tg = double(t * ag);
  d[i] = al + tg;
  d[j] = be - tg;
  q = RotF{c, t * c, g.x * rg, g.y * rg};
}

// Refinement of the long-window eigensolver (T >= 128), cooperative over all SMs
// with one grid barrier per round, on C' = Vf^H C Vf: the diagonal in float64 (a
// copy in every CTA's shared memory, updated identically by every CTA), the
// off-diagonal entries in float32 alternating between Cf and Cf2 (every entry is
// rewritten each round), V in float64 -- the arithmetic of the short-window
// refinement (refine_rot). Every CTA computes all rotations itself, a deterministic
// function of the same data, so all agree; the rotation count and the largest
// off-diagonal entry of a sweep, identical in every CTA, end the loop without a
// further barrier. C' is scaled by a power of two near 1 / max C'_ii first; the
// unscaled diagonal goes back into a.C for the eigenvalue selection.
__global__ void __launch_bounds__(256) k_jacobi_refine(PcaArgs a) {
  cg::grid_group grid = cg::this_grid();
  const int T = a.T, NP = T / 2;
  __shared__ RotF rf[256];
  __shared__ RotV rv[256];
  __shared__ double d[512];
  __shared__ unsigned cnt, offbits;
  __shared__ double scale_s, cmax_s, trace_s;
  const size_t gtid = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t gsz = size_t(gridDim.x) * blockDim.x;
  for (int i = threadIdx.x; i < T; i += blockDim.x) d[i] = a.C[size_t(i) * T + i].x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0, t = 0.0;
    for (int i = 0; i < T; ++i) {
      m = fmax(m, d[i]);
      t += d[i];
    }
    int ex = 0;
    frexp(m, &ex);
    scale_s = m > 0.0 ? ldexp(1.0, -ex) : 1.0;
    cmax_s = m * scale_s;
    trace_s = t * scale_s;
  }
  __syncthreads();
  const double scale = scale_s;
  for (int i = threadIdx.x; i < T; i += blockDim.x) d[i] *= scale;
  for (size_t e = gtid; e < size_t(T) * T; e += gsz) {  // Hermitian by construction
    const int r = int(e / T), c = int(e % T);
    const double2 v = a.C[size_t(r < c ? r : c) * T + (r < c ? c : r)];
    a.Cf[e] = make_float2(float(v.x * scale), r == c ? 0.f : (r < c ? float(v.y * scale) : -float(v.y * scale)));
  }
  grid.sync();
  const float rtol = float(a.tol), rfloor = float(a.tol_abs * cmax_s);
  float2* Cs = a.Cf;
  float2* Cd = a.Cf2;
  int sweeps = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    if (threadIdx.x == 0) {
      cnt = 0;
      offbits = 0u;
    }
    for (int r = 0; r < T - 1; ++r) {
      __syncthreads();  // rotations of the previous round fully used; cnt reset visible
      for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        const int i = rr_elem(p, r, T), j = rr_elem(T - 1 - p, r, T);
        const float2 g = Cs[size_t(i) * T + j];
        const float ag = hypotf(g.x, g.y);
        atomicMax(&offbits, __float_as_uint(ag));  // non-negative floats order like their bits
        if (refine_rot(d, i, j, g, ag, rtol, rfloor, rf[p], rv[p])) atomicAdd(&cnt, 1u);
      }
      __syncthreads();
      const size_t nblk = size_t(NP) * NP;
      for (size_t e = gtid; e < nblk + size_t(T) * NP; e += gsz) {
        if (e < nblk) {
          const int p = int(e / NP), q = int(e % NP);
          jacobi_block_f2(Cs, Cd, T, rr_elem(p, r, T), rr_elem(T - 1 - p, r, T), rr_elem(q, r, T),
                          rr_elem(T - 1 - q, r, T), rf[p], rf[q], p == q);
        } else {
          const size_t f = e - nblk;
          const int row = int(f / NP), q = int(f % NP);
          if (rf[q].s == 0.f) continue;
          refine_vrow(a.V, T, row, rr_elem(q, r, T), rr_elem(T - 1 - q, r, T), rv[q]);
        }
      }
      grid.sync();
      float2* t = Cs;
      Cs = Cd;
      Cd = t;
    }
    sweeps = sweep + 1;
    __syncthreads();
    // a sweep without any rotation, or below the early-end bound: converged (same in every CTA)
    const bool done = cnt == 0 || (a.stop_rel > 0.0 && double(__uint_as_float(offbits)) <= a.stop_rel * trace_s);
    __syncthreads();  // every thread has read cnt and offbits before the next sweep resets them
    if (done) break;
  }
  if (blockIdx.x == 0)  // the Rayleigh numerators (V^H C V)_ii, unscaled, for the selection
    for (int i = threadIdx.x; i < T; i += blockDim.x) a.C[size_t(i) * T + i] = make_double2(d[i] / scale, 0.0);
  if (gtid == 0) atomicAdd(&a.counters[2], unsigned(sweeps));  // refinement sweeps
}

// Power of two near 1 / max_i C_ii (exact scaling): the float32 phase works on
// C times this, so no product of two entries can overflow float32 whatever the
// frames' range (a 16-bit full-range window of a large frame reaches diagonal
// entries above 1e19, whose products exceed the float32 range). Every thread
// computes the same value from the float64 diagonal.
__device__ __forceinline__ double pow2_diag_scale(const double2* C, int T) {
  double m = 0.0;
  for (int i = 0; i < T; ++i) m = fmax(m, C[size_t(i) * T + i].x);
  int ex = 0;
  frexp(m, &ex);
  return m > 0.0 ? ldexp(1.0, -ex) : 1.0;
}

// First phase of the large-window eigensolver: the same cooperative cyclic
// Jacobi in float32 (on a quarter of the SMs: the arithmetic is cheap, so the
// grid barrier sets the pace of a round, and a smaller grid makes it cheaper),
// Cf alternating with Cf2, rotations accumulated in Vf, until a sweep rotates
// nothing at 1e-6 relative.
__global__ void __launch_bounds__(256) k_jacobi_f32(PcaArgs a) {
  cg::grid_group grid = cg::this_grid();
  const int T = a.T, NP = T / 2;
  __shared__ RotF rot[256];
  __shared__ unsigned cnt;
  const size_t gtid = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t gsz = size_t(gridDim.x) * blockDim.x;
  const double scale = pow2_diag_scale(a.C, T);  // the rotations do not depend on it
  for (size_t e = gtid; e < size_t(T) * T; e += gsz) {
    const double2 v = a.C[e];
    a.Cf[e] = make_float2(float(v.x * scale), float(v.y * scale));
    a.Vf[e] = make_float2(e / T == e % T ? 1.f : 0.f, 0.f);
  }
  grid.sync();
  // scales: the trace (>= the largest eigenvalue); float32 rounding leaves
  // off-diagonal entries near 6e-8 of the largest eigenvalue
  float trace = 0.f;
  for (int i = 0; i < T; ++i) trace += float(a.C[size_t(i) * T + i].x * scale);
  const float ftol = 1e-6f, ffloor = 2e-7f * trace;
  __shared__ unsigned offbits;  // largest |C_ij| met in the sweep (non-negative float bits)
  float2* Cs = a.Cf;
  float2* Cd = a.Cf2;
  int sweeps = 0;
  for (int sweep = 0; sweep < 20; ++sweep) {
    if (threadIdx.x == 0) {
      cnt = 0;
      offbits = 0;
    }
    for (int r = 0; r < T - 1; ++r) {
      __syncthreads();
      for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        const int i = rr_elem(p, r, T), j = rr_elem(T - 1 - p, r, T);
        RotF q;
        const float2 g = Cs[i * T + j];
        if (jacobi_rot_f(Cs[i * T + i].x, Cs[j * T + j].x, g, ftol, ffloor, q)) atomicAdd(&cnt, 1u);
        atomicMax(&offbits, __float_as_uint(sqrtf(g.x * g.x + g.y * g.y)));
        rot[p] = q;
      }
      __syncthreads();
      const size_t nblk = size_t(NP) * NP;
      for (size_t e = gtid; e < nblk + size_t(T) * NP; e += gsz) {
        if (e < nblk) {
          const int p = int(e / NP), q = int(e % NP);
          const int i0 = rr_elem(p, r, T), i1 = rr_elem(T - 1 - p, r, T), j0 = rr_elem(q, r, T),
                    j1 = rr_elem(T - 1 - q, r, T);
          // copy the 2 x 2 block into the other buffer, then rotate it there
          Cd[i0 * T + j0] = Cs[i0 * T + j0];
          Cd[i0 * T + j1] = Cs[i0 * T + j1];
          Cd[i1 * T + j0] = Cs[i1 * T + j0];
          Cd[i1 * T + j1] = Cs[i1 * T + j1];
          if (rot[p].s != 0.f || rot[q].s != 0.f) jacobi_block_f(Cd, T, i0, i1, j0, j1, rot[p], rot[q], p == q);
        } else {
          const size_t f = e - nblk;
          const int row = int(f / NP), q = int(f % NP);
          if (rot[q].s == 0.f) continue;
          jacobi_vrow_f(a.Vf, T, row, rr_elem(q, r, T), rr_elem(T - 1 - q, r, T), rot[q]);
        }
      }
      grid.sync();
      float2* t = Cs;
      Cs = Cd;
      Cd = t;
    }
    sweeps = sweep + 1;
    __syncthreads();
    const bool done = cnt == 0 || __uint_as_float(offbits) <= 1e-6f * trace;  // same in every CTA
    __syncthreads();
    if (done) break;
  }
  if (gtid == 0) atomicAdd(&a.counters[1], unsigned(sweeps));  // float32 sweeps
}

// Both phases of the long-window eigensolver on one thread-block cluster (JC CTAs,
// the matrix in their shared memory; T = 128 or 256). The cyclic order is the
// round-robin one (rr_elem): in round r position k holds index rr_elem(k, r) and
// pair p joins positions p and T-1-p; from one round to the next the index at
// position k moves to k - 1 (position 1 to T-1, position 0 stays). CTA c owns
// pairs c PPC .. c PPC + PPC - 1: the rows at their positions sit in its shared
// memory (slot l for position c PPC + l, slot R-1-l for position T-1-(c PPC + l)),
// so the left rotation of a row mixes it with a local row. Rows are double
// buffered: round r reads buffer r & 1 and writes each new row straight into the
// slot of its next position in buffer (r + 1) & 1 -- of the same CTA, except for
// two rows a round that go to a neighbour's shared memory. A round: (1) every CTA
// reads each pair's off-diagonal entry (and in the float32 phase both diagonal
// entries) from the owners' shared memory and computes all rotations itself (a
// deterministic function of the same data, so all CTAs agree); (2) it rotates the
// 2 x 2 blocks of its pairs' rows (left by the pair's rotation, right by each
// column pair's) and the column pairs of its rows of V (CTA c owns rows c R ..
// c R + R - 1 of V, which do not move); (3) one cluster barrier. Float32 phase
// (REFINE false): C scaled by a power of two near 1 / max C_ii, rotations
// J = [[c, -s], [conj(ph) s, conj(ph) c]] accumulated in Vf (from the identity),
// until a sweep rotates nothing at 1e-6 of the trace. Refinement (REFINE true) on
// C' = Vf^H C Vf: the diagonal in float64, a copy in every CTA updated
// identically, the off-diagonal entries in float32, the angles of refine_rot; at
// most max_sweeps sweeps, fewer when every entry met in a sweep is below stop_rel
// of the trace; the unscaled diagonal goes back into a.C for the eigenvalue
// selection. Its rotations take the form J = [[c, -s u], [s conj(u), c]] (u = g / |g|;
// the same diagonal as the form with the phase on the second column,
// P R = diag(1, conj(u)) R, since J = P R P^H), so that their product Q = I + D stays
// near the identity: D (|D| ~ the off-diagonal size, 1e-6 of the trace) is
// accumulated in float32 as D <- D J + (J - I), with c - 1 = -s^2 / (1 + c), and
// written to a.Cf; V = Vf + Vf D follows in k_vcorr, the float32 product exact to
// ~1e-13 against the entries of V. (Owning rows rather than pairs, each round read
// the 32 KB of partner rows through the cluster's shared-memory network, about
// 14 bytes a clock per SM, and V rotated in float64 on 16 SMs was bound by their
// float64 rate: 4.5 us a round against about 1 us here.)
constexpr int JC = 16;
constexpr int JC_NT = 512;

template <int T, bool REFINE>
struct JclSmem {
  static constexpr int NP = T / 2, PPC = NP / JC, R = 2 * PPC;
  // C buffers (2), Vf or D rows, the rotation table, (REFINE) the diagonal
  static constexpr size_t c_bytes = size_t(R) * T * sizeof(float2);
  static constexpr size_t bytes() { return 3 * c_bytes + NP * sizeof(RotF) + (REFINE ? T * sizeof(double) : 0); }
};

// Owner CTA and slot of position k (pairs PPC to a CTA, R = 2 PPC slots)
__device__ __forceinline__ void jc_place(int k, int T, int PPC, int& cta, int& slot) {
  if (k < T / 2) {
    cta = k / PPC;
    slot = k % PPC;
  } else {
    const int p = T - 1 - k;
    cta = p / PPC;
    slot = 2 * PPC - 1 - p % PPC;
  }
}

template <int T, bool REFINE>
__global__ void __launch_bounds__(JC_NT) k_jacobi_cluster(PcaArgs a) {
  using Sm = JclSmem<T, REFINE>;
  constexpr int NP = Sm::NP, PPC = Sm::PPC, R = Sm::R;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = int(cl.block_rank()), tid = threadIdx.x, row0 = rank * R;
  extern __shared__ float4 jcs[];
  float2* C0 = reinterpret_cast<float2*>(jcs);  // buffer b at C0 + b R T, slot s at + s T
  float2* Vr = C0 + 2 * R * T;                  // own rows of Vf (float32 phase) or of D
  RotF* rot = reinterpret_cast<RotF*>(Vr + R * T);
  double* d = reinterpret_cast<double*>(rot + NP);  // REFINE: the scaled diagonal
  __shared__ float gabs[NP];  // |C_ij| of each pair when its rotation was decided
  __shared__ unsigned s_nrot;
  __shared__ float s_offmax;
  __shared__ double s_trace;
  const double scale = pow2_diag_scale(a.C, T);  // the same in every CTA
  // round 0: position k holds index k
  for (int e = tid; e < R * T; e += JC_NT) {
    const int sl = e / T, c = e % T;
    const int k = sl < PPC ? rank * PPC + sl : T - 1 - (rank * PPC + (R - 1 - sl));
    if (REFINE) {  // Hermitian by construction: the upper triangle, a real zero diagonal
      const double2 v = a.C[size_t(k < c ? k : c) * T + (k < c ? c : k)];
      C0[e] = make_float2(float(v.x * scale), k == c ? 0.f : (k < c ? float(v.y * scale) : -float(v.y * scale)));
      Vr[e] = make_float2(0.f, 0.f);  // D = 0
    } else {
      const double2 v = a.C[size_t(k) * T + c];
      C0[e] = make_float2(float(v.x * scale), float(v.y * scale));
      Vr[e] = make_float2(row0 + sl == c ? 1.f : 0.f, 0.f);
    }
  }
  if (tid == 0) {
    double t = 0.0;
    for (int i = 0; i < T; ++i) t += a.C[size_t(i) * T + i].x * scale;
    s_trace = t;
  }
  if (REFINE)
    for (int i = tid; i < T; i += JC_NT) d[i] = a.C[size_t(i) * T + i].x * scale;
  cl.sync();
  const double trace = s_trace;
  // float32 phase: the trace bounds the largest eigenvalue; float32 rounding leaves
  // off-diagonal entries near 6e-8 of it. Refinement: the caller's bounds, relative
  // to the largest diagonal entry (scaled to [0.5, 1))
  double cmax = 0.0;
  if (REFINE)
    for (int i = 0; i < T; ++i) cmax = fmax(cmax, a.C[size_t(i) * T + i].x * scale);
  const float tol = REFINE ? float(a.tol) : 1e-6f;
  const float floor_abs = REFINE ? float(a.tol_abs * cmax) : 2e-7f * float(trace);
  const int max_sweeps = REFINE ? a.max_sweeps : 20;
  // a thread's column pair q is the same in every round, and so is its pair row l
  // (at most one: JC_NT >= PPC NP) with the slots of the pair rows' next positions
  constexpr int NB = (PPC * NP + JC_NT - 1) / JC_NT;  // pair blocks per thread: pair rows l0 + k JC_NT / NP
  static_assert(JC_NT % NP == 0 && NB <= 2, "pair blocks per thread");
  const int q = tid % NP, l0 = tid / NP;
  float2* nlo[NB];  // buffer 0 of the slot of the next position of each pair row
  float2* nhi[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int l = l0 + k * (JC_NT / NP);
    nlo[k] = nhi[k] = nullptr;
    if (l >= PPC) continue;
    const int p = rank * PPC + l, klo = p, khi = T - 1 - p;
    int cta, slot;
    jc_place(klo == 0 ? 0 : (klo == 1 ? T - 1 : klo - 1), T, PPC, cta, slot);
    nlo[k] = (cta == rank ? C0 : cl.map_shared_rank(C0, cta)) + slot * T;
    jc_place(khi - 1, T, PPC, cta, slot);
    nhi[k] = (cta == rank ? C0 : cl.map_shared_rank(C0, cta)) + slot * T;
  }
  // indices of the thread's pair (rotation phase) and column pair in round 0; from one
  // round to the next each moves to the following index of 1 .. T-1 (0 stays)
  auto next_idx = [](int x) { return x == 0 ? 0 : (x == T - 1 ? 1 : x + 1); };
  int ri = tid < NP ? rr_elem(tid, 0, T) : 0, rj = tid < NP ? rr_elem(T - 1 - tid, 0, T) : 0;
  int ca = rr_elem(q, 0, T), cb = rr_elem(T - 1 - q, 0, T);
  int sweeps = 0, cur = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    unsigned nrot = 0;  // warp 0's running totals of the sweep
    float offmax = 0.f;
    for (int r = 0; r < T - 1; ++r) {
      const float2* Cs = C0 + cur * R * T;
      // (1) every pair's rotation, from its owner's rows
      if (tid < NP) {
        const int p = tid, i = ri, j = rj;
        const float2* own = cl.map_shared_rank(Cs, p / PPC);
        const float2* lo = own + (p % PPC) * T;
        const float2 g = lo[j];
        float ci = 0.f, cj = 0.f;
        if (!REFINE) {
          ci = lo[i].x;
          cj = own[(R - 1 - p % PPC) * T + j].x;
        }
        const float ag = sqrtf(g.x * g.x + g.y * g.y);
        if (REFINE) {
          refine_rot_f(d, i, j, g, ag, tol, floor_abs, rot[p]);
        } else {
          jacobi_rot_f(ci, cj, g, tol, floor_abs, rot[p]);
        }
        gabs[p] = ag;
      }
      __syncthreads();
      // (2) the 2 x 2 blocks (pair rows x column pair q) of the CTA's pairs, written
      // to the slots of the rows' next positions
      const RotF Jq = rot[q];
      const float2 uq = cscale(make_float2(Jq.px, Jq.py), Jq.s);  // u_q s (REFINE), ph_q s
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        const int l = l0 + k * (JC_NT / NP), p = rank * PPC + l;
        if (l >= PPC) continue;
        const RotF Jp = rot[p];
        const float2* lo = Cs + l * T;
        const float2* hi = Cs + (R - 1 - l) * T;
        const float2 b00 = lo[ca], b01 = lo[cb], b10 = hi[ca], b11 = hi[cb];
        float2 c00, c01, c10, c11;
        if (REFINE) {
          // right by J_q = [[c, -s u], [s conj(u), c]], then left by J_p^H
          const float2 cuq = make_float2(uq.x, -uq.y);
          const float2 m00 = cadd(cscale(b00, Jq.c), cmul(b01, cuq)), m01 = csub(cscale(b01, Jq.c), cmul(b00, uq));
          const float2 m10 = cadd(cscale(b10, Jq.c), cmul(b11, cuq)), m11 = csub(cscale(b11, Jq.c), cmul(b10, uq));
          const float2 up = cscale(make_float2(Jp.px, Jp.py), Jp.s), cup = make_float2(up.x, -up.y);
          c00 = cadd(cscale(m00, Jp.c), cmul(up, m10));
          c01 = cadd(cscale(m01, Jp.c), cmul(up, m11));
          c10 = csub(cscale(m10, Jp.c), cmul(cup, m00));
          c11 = csub(cscale(m11, Jp.c), cmul(cup, m01));
        } else {
          // right by J_q = [[c, -s], [conj(ph) s, conj(ph) c]], then left by J_p^H
          const float2 q10 = make_float2(Jq.px * Jq.s, -Jq.py * Jq.s), q11 = make_float2(Jq.px * Jq.c, -Jq.py * Jq.c);
          const float2 m00 = cadd(cscale(b00, Jq.c), cmul(b01, q10)), m01 = cadd(cscale(b00, -Jq.s), cmul(b01, q11));
          const float2 m10 = cadd(cscale(b10, Jq.c), cmul(b11, q10)), m11 = cadd(cscale(b10, -Jq.s), cmul(b11, q11));
          const float2 p01 = make_float2(Jp.px * Jp.s, Jp.py * Jp.s), p11 = make_float2(Jp.px * Jp.c, Jp.py * Jp.c);
          c00 = cadd(cscale(m00, Jp.c), cmul(p01, m10));
          c01 = cadd(cscale(m01, Jp.c), cmul(p01, m11));
          c10 = cadd(cscale(m00, -Jp.s), cmul(p11, m10));
          c11 = cadd(cscale(m01, -Jp.s), cmul(p11, m11));
        }
        if (q == p) {  // the pair's own block: exactly diagonal, real diagonal
          c01 = make_float2(0.f, 0.f);
          c10 = make_float2(0.f, 0.f);
          c00.y = 0.f;
          c11.y = 0.f;
        }
        // into the slots of the rows' next positions, buffer cur ^ 1
        float2* dlo = nlo[k] + (cur ^ 1) * R * T;
        float2* dhi = nhi[k] + (cur ^ 1) * R * T;
        dlo[ca] = c00;
        dlo[cb] = c01;
        dhi[ca] = c10;
        dhi[cb] = c11;
      }
      // (3) this CTA's new rows are written (some into a neighbour) and its reads of the
      // round done: arrive on the cluster barrier, rotate the local rows of V while
      // the others finish, then wait
      asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
      // the CTA's rows of V (or D): right rotation of the column pair q
      if (Jq.s != 0.f) {
        const float2 cuq = make_float2(uq.x, -uq.y);
        const float2 q10 = make_float2(Jq.px * Jq.s, -Jq.py * Jq.s), q11 = make_float2(Jq.px * Jq.c, -Jq.py * Jq.c);
#pragma unroll
        for (int li = tid / NP; li < R; li += JC_NT / NP) {
          const float2 va = Vr[li * T + ca], vb = Vr[li * T + cb];
          if (REFINE) {  // D <- D J + (J - I)
            float2 na = cadd(cscale(va, Jq.c), cmul(vb, cuq));
            float2 nb = csub(cscale(vb, Jq.c), cmul(va, uq));
            const int i = row0 + li;
            if (i == ca || i == cb) {
              const float cm1 = -Jq.s * Jq.s / (1.f + Jq.c);
              if (i == ca) {
                na.x += cm1;
                nb = csub(nb, uq);
              } else {
                na = cadd(na, cuq);
                nb.x += cm1;
              }
            }
            Vr[li * T + ca] = na;
            Vr[li * T + cb] = nb;
          } else {
            Vr[li * T + ca] = cadd(cscale(va, Jq.c), cmul(vb, q10));
            Vr[li * T + cb] = cadd(cscale(va, -Jq.s), cmul(vb, q11));
          }
        }
      }
      if (tid < 32)  // the table is the same in every CTA
        for (int p = tid; p < NP; p += 32) {
          nrot += rot[p].s != 0.f;
          offmax = fmaxf(offmax, gabs[p]);
        }
      asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
      cur ^= 1;
      ri = next_idx(ri);
      rj = next_idx(rj);
      ca = next_idx(ca);
      cb = next_idx(cb);
    }
    sweeps = sweep + 1;
    if (tid < 32) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        nrot += __shfl_xor_sync(0xffffffffu, nrot, o);
        offmax = fmaxf(offmax, __shfl_xor_sync(0xffffffffu, offmax, o));
      }
      if (tid == 0) {
        s_nrot = nrot;
        s_offmax = offmax;
      }
    }
    __syncthreads();
    const bool done = s_nrot == 0 || (REFINE ? (a.stop_rel > 0.0 && double(s_offmax) <= a.stop_rel * trace)
                                             : s_offmax <= 1e-6f * float(trace));
    __syncthreads();  // s_nrot / s_offmax read by every thread before the next sweep writes them
    if (done) break;  // float32 phase: the refinement takes it from 1e-6 of the trace
  }
  if (REFINE) {
    for (int e = tid; e < R * T; e += JC_NT) a.Cf[size_t(row0) * T + e] = Vr[e];  // D
    if (rank == 0)  // the Rayleigh numerators (V^H C V)_ii, unscaled, for the selection
      for (int i = tid; i < T; i += JC_NT) a.C[size_t(i) * T + i] = make_double2(d[i] / scale, 0.0);
  } else {
    for (int e = tid; e < R * T; e += JC_NT) a.Vf[size_t(row0) * T + e] = Vr[e];
  }
  if (rank == 0 && tid == 0) atomicAdd(&a.counters[REFINE ? 2 : 1], unsigned(sweeps));
}

template <int T, bool REFINE>
static cudaError_t launch_jacobi_cluster(const PcaArgs& a, cudaStream_t s, bool* ok) {
  *ok = false;
  const size_t smem = JclSmem<T, REFINE>::bytes();
  auto kern = k_jacobi_cluster<T, REFINE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;  // not available: the caller uses the cooperative kernel
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(JC);
  cfg.blockDim = dim3(JC_NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = JC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  if (e != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return cudaSuccess;
  }
  e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e == cudaSuccess) *ok = true;
  return e;
}

// out = op(A) B for T x T complex matrices: A float64 (op = identity) or the
// float32 Vf (op = conjugate transpose, transA = 1); B float64 or Vf as float64.
// 16 x 16 output tiles, 16-wide k stages in shared memory, float64 accumulation.
__global__ void __launch_bounds__(256) k_gemm_c64(int T, const double2* A, const float2* Af, int transA,
                                                  const double2* B, const float2* Bf, double2* out) {
  __shared__ double2 As[16][17], Bs[16][17];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r = blockIdx.y * 16 + ty, c = blockIdx.x * 16 + tx;
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < T; k0 += 16) {
    // A element (r, k): A[r][k], or conj(Vf[k][r]) when transposed
    const int ar = blockIdx.y * 16 + ty, ak = k0 + tx;
    if (transA) {
      const float2 v = Af[size_t(ak) * T + ar];
      As[ty][tx] = make_double2(v.x, -v.y);
    } else {
      As[ty][tx] = A[size_t(ar) * T + ak];
    }
    const int bk = k0 + ty, bc = blockIdx.x * 16 + tx;
    if (Bf) {
      const float2 v = Bf[size_t(bk) * T + bc];
      Bs[ty][tx] = make_double2(v.x, v.y);
    } else {
      Bs[ty][tx] = B[size_t(bk) * T + bc];
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 16; ++k) acc = zadd(acc, zmul(As[ty][k], Bs[k][tx]));
    __syncthreads();
  }
  out[size_t(r) * T + c] = acc;
}

// V = Vf + Vf D in float64 (D in a.Cf, the refinement's correction): the product
// in float32 (its entries ~1e-6 of V's, so float32 leaves ~1e-13), added to Vf
// exactly in float64. 16 x 16 output tiles, 16-wide k stages in shared memory.
__global__ void __launch_bounds__(256) k_vcorr(PcaArgs a) {
  __shared__ float2 As[16][17], Bs[16][17];
  const int T = a.T, tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r = blockIdx.y * 16 + ty, c = blockIdx.x * 16 + tx;
  float2 acc = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < T; k0 += 16) {
    As[ty][tx] = a.Vf[size_t(r) * T + k0 + tx];
    Bs[ty][tx] = a.Cf[size_t(k0 + ty) * T + c];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = cadd(acc, cmul(As[ty][k], Bs[k][tx]));
    __syncthreads();
  }
  const float2 v = a.Vf[size_t(r) * T + c];
  a.V[size_t(r) * T + c] = make_double2(double(v.x) + double(acc.x), double(v.y) + double(acc.y));
}

// Rayleigh quotient and inverse norm of every column of V (the columns are unitary
// only to the float32 phase's accuracy): lam_i = (V^H C V)_ii / |v_i|^2 with the
// numerators on the diagonal of a.C, into scratch [lam_0 .. lam_T-1, 1/|v_0| ..].
// 16 columns per CTA, 16 threads per column, float64 sums.
__global__ void __launch_bounds__(256) k_pca_norms(PcaArgs a, double* scratch) {
  const int T = a.T, i = blockIdx.x * 16 + threadIdx.x / 16, part = threadIdx.x % 16;
  double n2 = 0.0;
  for (int t = part; t < T; t += 16) {
    const double2 v = a.V[size_t(t) * T + i];
    n2 = fma(v.x, v.x, fma(v.y, v.y, n2));
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  if (part == 0) {
    scratch[i] = a.C[size_t(i) * T + i].x / n2;
    scratch[T + i] = 1.0 / sqrt(n2);
  }
}

// Ranks the eigenvalues (descending, ties by index), writes lam sorted and the
// sub-basis columns lo..hi of V, normalised, as float32 (zero padding to Mpad).
__global__ void __launch_bounds__(1024) k_pca_select(PcaArgs a, const double* scratch) {
  const int T = a.T;
  __shared__ double lamv[512];
  __shared__ int col_of[512];  // column of V of each rank
  for (int i = threadIdx.x; i < T; i += blockDim.x) lamv[i] = scratch[i];
  __syncthreads();
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    const double li = lamv[i];
    int rank = 0;
    for (int j = 0; j < T; ++j) {
      const double lj = lamv[j];
      rank += (lj > li) || (lj == li && j < i);
    }
    a.lam[rank] = li;
    col_of[rank] = i;
  }
  __syncthreads();
  const int Mp = int(a.Mpad), lo = int(a.lo) - 1;
  for (int e = threadIdx.x; e < T * Mp; e += blockDim.x) {
    const int t = e / Mp, m = e % Mp;
    float2 v = make_float2(0.f, 0.f);
    if (m < int(a.M)) {
      const int i = col_of[lo + m];
      const double2 x = a.V[size_t(t) * T + i];
      const double r = scratch[T + i];
      v = make_float2(float(x.x * r), float(x.y * r));
    }
    a.Vs[e] = v;
  }
}

// One sweep's rounds of the CTA-local cyclic Jacobi on C (T x T) and V. The
// rotation of the pair (i, j) in slot k is made by rotfn(i, j, k), which stores
// it in rc[k] (applied to C) and rv[k] (applied to V; may be the same array);
// returns the rotations performed.
template <int T, class CM, class VM, class RC, class RV, class RotFn, class BlockFn, class RowFn>
__device__ __forceinline__ unsigned local_sweep(CM* C, VM* V, const RC* rc, const RV* rv, unsigned* cnt, RotFn rotfn,
                                                BlockFn blockfn, RowFn rowfn) {
  constexpr int NP = T / 2;
  const int tid = threadIdx.x;
  if (tid == 0) *cnt = 0;
  __syncthreads();
  for (int r = 0; r < T - 1; ++r) {
    if (tid < NP) {
      const int i = rr_elem(tid, r, T), j = rr_elem(T - 1 - tid, r, T);
      if (rotfn(i, j, tid)) atomicAdd(cnt, 1u);
    }
    __syncthreads();
    for (int e = tid; e < NP * NP + T * NP; e += blockDim.x) {
      if (e < NP * NP) {
        const int p = e / NP, q = e % NP;
        if (rc[p].s == 0 && rc[q].s == 0) continue;
        blockfn(C, T, rr_elem(p, r, T), rr_elem(T - 1 - p, r, T), rr_elem(q, r, T), rr_elem(T - 1 - q, r, T), rc[p],
                rc[q], p == q);
      } else {
        const int f = e - NP * NP, row = f / NP, q = f % NP;
        if (rc[q].s == 0) continue;
        rowfn(V, T, row, rr_elem(q, r, T), rr_elem(T - 1 - q, r, T), rv[q]);
      }
    }
    __syncthreads();
  }
  const unsigned n = *cnt;
  __syncthreads();
  return n;
}

// Short windows (T <= 64): one CTA per window, the eigendecomposition in shared
// memory in two phases, on C scaled by a power of two near 1 / max C_ii (exact,
// and no float32 overflow whatever the data's range).
// (1) Float32 cyclic Jacobi on a float copy of C, with the rotations accumulated
// in Vf, until a sweep rotates nothing at 1e-6 relative.
// (2) Refinement: C' = Vf^H C Vf in float64 from the float64 C, whose
// off-diagonal entries are then about 1e-6 of its diagonal; Jacobi sweeps on C'
// with the diagonal d in float64, the off-diagonal entries in float32 (every
// float32 operation of a sweep combines off-diagonal entries only, so its
// rounding is relative to them: ~1e-7 of 1e-6, far below the float32
// covariance's own error) and V = Vf rotated further in float64 by J unitary to
// ~1e-13 (refine_rot), until a sweep rotates nothing at 1e-14 or meets
// no off-diagonal entry above 1e-12 of the trace. V's columns are then
// C-orthogonal to the refinement's accuracy; Vf is unitary to about 1e-6 only,
// so each eigenvalue is the Rayleigh quotient d_i / |v_i|^2 and the vectors are
// normalised. Then the ranking and the sub-basis. GB300's float64 rate is 1/64
// of float32, which is why only the diagonal, the rotation factors and V are
// float64.
template <int T>
__global__ void __launch_bounds__(256) k_jacobi_small(PcaArgs a) {
  extern __shared__ double2 jsm[];
  double2* RA = jsm;            // Cf (float) in phase 1, then M = C Vf, then V (float64)
  double2* C = jsm + T * T;     // C' (float64)
  float2* Vf = reinterpret_cast<float2*>(jsm + 2 * T * T);
  float2* Cf = reinterpret_cast<float2*>(RA);
  float2* Co = Vf;              // the refinement's float32 off-diagonal entries (Vf is dead by then)
  __shared__ RotV rotv[T / 2];
  __shared__ RotF rotf[T / 2];
  __shared__ double d[T];
  __shared__ unsigned cnt, offbits;
  __shared__ double scale_s, cmax_s, trace_s;
  const int w = blockIdx.x, tid = threadIdx.x;
  const double2* Cg = a.C + size_t(w) * T * T;
  if (tid == 0) {
    double m = 0.0, t = 0.0;
    for (int i = 0; i < T; ++i) {
      m = fmax(m, Cg[i * T + i].x);
      t += Cg[i * T + i].x;
    }
    int ex = 0;
    frexp(m, &ex);
    scale_s = m > 0.0 ? ldexp(1.0, -ex) : 1.0;  // scaled max C_ii in [0.5, 1)
    cmax_s = m * scale_s;
    trace_s = t * scale_s;
  }
  __syncthreads();
  const double scale = scale_s, cmax = cmax_s;  // of the scaled C
  for (int e = tid; e < T * T; e += blockDim.x) {
    const double2 v = Cg[e];
    Cf[e] = make_float2(float(v.x * scale), float(v.y * scale));
    Vf[e] = make_float2(e / T == e % T ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  // (1) float32 sweeps until one rotates nothing at 1e-6 (relative, and of the
  // largest diagonal entry)
  const float ftol = 1e-6f, ffloor = 1e-6f * float(cmax);
  int sweeps_f = 0;
  for (int sw = 0; sw < 20; ++sw) {
    const unsigned n = local_sweep<T>(
        Cf, Vf, rotf, rotf, &cnt,
        [&](int i, int j, int k) {
          return jacobi_rot_f(Cf[i * T + i].x, Cf[j * T + j].x, Cf[i * T + j], ftol, ffloor, rotf[k]);
        },
        jacobi_block_f, jacobi_vrow_f);
    sweeps_f = sw + 1;
    if (n == 0) break;
  }
  // (2) C' = Vf^H (C Vf) in float64 (scaled): M = C Vf into RA (Cf is dead), then
  // the upper triangle of C' into C
  for (int e = tid; e < T * T; e += blockDim.x) {
    const int r = e / T, c = e % T;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < T; ++k) {
      const float2 v = Vf[k * T + c];
      acc = zadd(acc, zmul(Cg[r * T + k], make_double2(v.x, v.y)));
    }
    RA[e] = make_double2(acc.x * scale, acc.y * scale);
  }
  __syncthreads();
  for (int u = tid; u < T * (T + 1) / 2; u += blockDim.x) {
    int r = 0, rem = u;
    while (rem >= T - r) {
      rem -= T - r;
      ++r;
    }
    const int c = r + rem;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < T; ++k) {
      const float2 v = Vf[k * T + r];
      acc = zadd(acc, zmul(make_double2(v.x, -v.y), RA[k * T + c]));
    }
    C[r * T + c] = acc;
  }
  __syncthreads();
  double2* V = RA;  // V = Vf in float64, rotated further below
  for (int e = tid; e < T * T; e += blockDim.x) V[e] = make_double2(Vf[e].x, Vf[e].y);
  __syncthreads();  // Vf read for the last time: its storage takes the off-diagonal entries
  for (int e = tid; e < T * T; e += blockDim.x) {
    const int r = e / T, c = e % T;
    const double2 v = C[(r < c ? r : c) * T + (r < c ? c : r)];
    Co[e] = r == c ? make_float2(float(v.x), 0.f) : make_float2(float(v.x), r < c ? float(v.y) : -float(v.y));
    if (r == c) d[r] = v.x;
  }
  __syncthreads();
  const double trace64 = trace_s;
  const float rtol = float(a.tol), rfloor = float(a.tol_abs * cmax);
  int sweeps_d = 0;
  for (int sw = 0; sw < a.max_sweeps; ++sw) {
    if (tid == 0) offbits = 0u;
    const unsigned n = local_sweep<T>(
        Co, V, rotf, rotv, &cnt,
        [&](int i, int j, int k) {
          const float2 g = Co[i * T + j];
          const float ag = hypotf(g.x, g.y);
          atomicMax(&offbits, __float_as_uint(ag));  // non-negative floats order like their bits
          return refine_rot(d, i, j, g, ag, rtol, rfloor, rotf[k], rotv[k]);
        },
        jacobi_block_f, refine_vrow);
    sweeps_d = sw + 1;
    const bool done = n == 0 || double(__uint_as_float(offbits)) <= 1e-12 * trace64;
    __syncthreads();
    if (done) break;
  }
  if (tid == 0) {  // summed over the launch's windows
    atomicAdd(&a.counters[1], unsigned(sweeps_f));
    atomicAdd(&a.counters[2], unsigned(sweeps_d));
  }
  // eigenvalues as Rayleigh quotients, vectors normalised; rank and sub-basis
  __shared__ double lamv[T], inrm[T];
  for (int i = tid; i < T; i += blockDim.x) {
    double n2 = 0.0;
    for (int t = 0; t < T; ++t) n2 += V[t * T + i].x * V[t * T + i].x + V[t * T + i].y * V[t * T + i].y;
    lamv[i] = d[i] / (n2 * scale);
    inrm[i] = 1.0 / sqrt(n2);
  }
  __syncthreads();
  double* lam = a.lam + size_t(w) * T;
  float2* Vs = a.Vs + size_t(w) * T * a.Mpad;
  for (int i = tid; i < T; i += blockDim.x) {
    const double li = lamv[i];
    int rank = 0;
    for (int j = 0; j < T; ++j) {
      const double lj = lamv[j];
      rank += (lj > li) || (lj == li && j < i);
    }
    lam[rank] = li;
    const int m = rank - int(a.lo - 1);
    if (m >= 0 && m < int(a.M))
      for (int t = 0; t < T; ++t)
        Vs[size_t(t) * a.Mpad + m] = make_float2(float(V[t * T + i].x * inrm[i]), float(V[t * T + i].y * inrm[i]));
  }
  for (int e = tid; e < T * int(a.Mpad); e += blockDim.x)
    if (e % int(a.Mpad) >= int(a.M)) Vs[e] = make_float2(0.f, 0.f);
}

// ---------------------------------------------------------------- projection

constexpr int PRJ_KS = 16;  // frames per stage

// Y = X V_s and E(p) = sum_j |Y_pj|^2. A CTA of 256 threads covers PB = 4096 / MB
// pixels and MB sub-basis columns per pass (MB = 16, 32 or 64; the sub-basis is
// padded to a multiple of 16); thread (tx, ty) owns pixels tx + (PB/4) i and
// columns 4 ty .. 4 ty + 3. Stages of PRJ_KS frames of the pixel strip are
// fetched with 16-byte cp.async into one of two buffers while the other is used.
template <int MB>
__global__ void __launch_bounds__(256) k_project(PcaArgs a, float* out) {
  constexpr int PB = 4096 / MB, PG = PB / 4, LDX = PB + 2;  // row stride keeps 16-byte alignment
  extern __shared__ float2 psm[];
  float2* Xs = psm;                      // 2 x [PRJ_KS][LDX]
  float2* Vss = psm + 2 * PRJ_KS * LDX;  // [PRJ_KS][MB]
  __shared__ float Er[MB / 4][PB];
  const int tid = threadIdx.x, tx = tid % PG, ty = tid / PG;
  const size_t hw = size_t(a.W) * a.H;
  const size_t pb = size_t(blockIdx.x) * PB;
  const int nst = int(a.T) / PRJ_KS;
  auto issue = [&](int st, int buf) {
    float2* d = Xs + buf * PRJ_KS * LDX;
    for (int e = tid; e < PRJ_KS * PB / 2; e += 256) {
      const int k = e / (PB / 2), q = e % (PB / 2);
      const float2* src = win_frame(a, blockIdx.y, st * PRJ_KS + k, hw) + pb + 2 * q;
      const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(&d[k * LDX + 2 * q]));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  float e_acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (uint32_t m0 = 0; m0 < a.Mpad; m0 += MB) {
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    issue(0, 0);
    for (int st = 0; st < nst; ++st) {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();  // stage st resident; the other buffer and Vss free
      if (st + 1 < nst) issue(st + 1, (st + 1) & 1);
      for (int e = tid; e < PRJ_KS * MB; e += 256) {
        const int k = e / MB, m = e % MB;
        Vss[k * MB + m] = a.Vs[(size_t(blockIdx.y) * a.T + st * PRJ_KS + k) * a.Mpad + m0 + m];
      }
      __syncthreads();
      const float2* X = Xs + (st & 1) * PRJ_KS * LDX;
#pragma unroll 4
      for (int k = 0; k < PRJ_KS; ++k) {
        float2 x[4], v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = X[k * LDX + tx + PG * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = Vss[k * MB + ty * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j].x = fmaf(x[i].x, v[j].x, fmaf(-x[i].y, v[j].y, acc[i][j].x));
            acc[i][j].y = fmaf(x[i].x, v[j].y, fmaf(x[i].y, v[j].x, acc[i][j].y));
          }
      }
    }
    __syncthreads();  // Vss and the buffers are reused by the next pass
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) e_acc[i] = fmaf(acc[i][j].x, acc[i][j].x, fmaf(acc[i][j].y, acc[i][j].y, e_acc[i]));
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) Er[ty][tx + PG * i] = e_acc[i];
  __syncthreads();
  for (int px = tid; px < PB; px += 256) {
    float s = 0.f;
#pragma unroll
    for (int g = 0; g < MB / 4; ++g) s += Er[g][px];
    out[size_t(blockIdx.y) * hw + pb + px] = s;
  }
}

template <int MB>
static cudaError_t launch_project(const PcaArgs& a, float* out, cudaStream_t s) {
  constexpr int PB = 4096 / MB;
  const size_t hw = size_t(a.W) * a.H;
  if (hw % PB) return cudaErrorInvalidValue;
  const size_t smem = (size_t(2) * PRJ_KS * (PB + 2) + size_t(PRJ_KS) * MB) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_project<MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  k_project<MB><<<dim3(unsigned(hw / PB), a.nwin), 256, smem, s>>>(a, out);
  return cudaGetLastError();
}

// -------------------------------------------------- covariance of short windows
//
// T <= 64: a group of (T/4)^2 threads covers the whole T x T matrix with 4 x 4
// complex tiles (thread (ta, tb): rows 4 ta.., columns 4 tb..); the CTA's
// 256 / (T/4)^2 groups take alternate pixels of each staged strip. A strip is
// SP pixels of all T frames of the window, [t][p] in shared memory (row stride
// SP + 1), fetched with cp.async into one of two buffers while the other is
// used. The groups' sums are added in shared memory and each CTA writes its
// partial matrix part[window][cta][T][T]; a second kernel sums them in float64.
constexpr int CS_SP = 64;

// Groups of k_cov_small<T> (tiles per group: the upper triangle's for T = 32) and
// its dynamic shared memory: two strip buffers, or the groups' partial matrices
// at the end, whichever is larger.
__host__ __device__ constexpr int cov_small_groups(int T) {
  return 256 / (T == 32 ? (T / 4) * (T / 4 + 1) / 2 : (T / 4) * (T / 4));
}
__host__ __device__ constexpr size_t cov_small_smem(int T) {
  const size_t strips = size_t(2) * T * (CS_SP + 1), red = size_t(cov_small_groups(T)) * T * T;
  return (strips > red ? strips : red) * sizeof(float2);
}

template <int T>
__global__ void __launch_bounds__(256) k_cov_small(PcaArgs a) {
  // T = 32: only the 36 tiles on or above the diagonal (ta <= tb), 7 groups in 252
  // threads; T = 64: all 256 tiles, one group (the reduction reads the upper triangle)
  constexpr bool UPPER = T == 32;
  constexpr int TG = T / 4, GT = UPPER ? TG * (TG + 1) / 2 : TG * TG, G = 256 / GT, LDX = CS_SP + 1;
  static_assert(G == cov_small_groups(T), "groups");
  extern __shared__ float2 xs[];  // cov_small_smem(T): 2 buffers of T x LDX, later G x T x T
  const int tid = threadIdx.x, g = tid / GT, r = tid % GT;
  const bool active = g < G;
  int ta = r / TG, tb = r % TG;
  if constexpr (UPPER) {  // r-th tile of the upper triangle, row by row
    int rr = r;
    ta = 0;
    while (rr >= TG - ta) {
      rr -= TG - ta;
      ++ta;
    }
    tb = ta + rr;
  }
  const size_t hw = size_t(a.W) * a.H;
  const uint32_t z = blockIdx.y;
  const size_t p_begin = size_t(blockIdx.x) * a.chunk;
  const size_t p_end = p_begin + a.chunk < hw ? p_begin + a.chunk : hw;
  const int nstrips = int((p_end - p_begin + CS_SP - 1) / CS_SP);
  auto issue = [&](int sidx, int buf) {
    float2* d = xs + buf * T * LDX;
    const size_t q0 = p_begin + size_t(sidx) * CS_SP;
    for (int e = tid; e < T * CS_SP; e += 256) {
      const int t = e / CS_SP, p = e % CS_SP;
      if (q0 + p < p_end) {
        const float2* src = win_frame(a, z, t, hw) + q0 + p;
        const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(&d[t * LDX + p]));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
      } else {
        d[t * LDX + p] = make_float2(0.f, 0.f);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  if (nstrips > 0) issue(0, 0);
  for (int sidx = 0; sidx < nstrips; ++sidx) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();  // strip sidx resident, the other buffer free
    if (sidx + 1 < nstrips) issue(sidx + 1, (sidx + 1) & 1);
    const float2* x = xs + (sidx & 1) * T * LDX;
#pragma unroll 4
    for (int p = active ? g : CS_SP; p < CS_SP; p += G) {
      float2 u[4], v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) u[i] = x[(4 * ta + i) * LDX + p];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = x[(4 * tb + j) * LDX + p];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // conj(u) * v
          acc[i][j].x = fmaf(u[i].x, v[j].x, fmaf(u[i].y, v[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(u[i].x, v[j].y, fmaf(-u[i].y, v[j].x, acc[i][j].y));
        }
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  // groups' sums in shared memory (reusing the strip buffers: G x T x T <= 2 x T x LDX)
  float2* red = xs;
  if (active)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) red[(size_t(g) * T + 4 * ta + i) * T + 4 * tb + j] = acc[i][j];
  __syncthreads();
  float2* out = a.partials + (size_t(z) * gridDim.x + blockIdx.x) * T * T;
  for (int e = tid; e < T * T; e += 256) {
    float2 s = red[e];
    for (int q = 1; q < G; ++q) {
      const float2 v = red[size_t(q) * T * T + e];
      s.x += v.x;
      s.y += v.y;
    }
    out[e] = s;
  }
}

// C[w] = sum over the CTAs' partials in float64 (upper triangle, mirrored).
__global__ void k_cov_small_reduce(PcaArgs a, uint32_t nparts) {
  const int T = a.T;
  for (int ew = blockIdx.x * blockDim.x + threadIdx.x; ew < int(a.nwin) * T * T; ew += gridDim.x * blockDim.x) {
    const int w = ew / (T * T), e = ew % (T * T), rr = e / T, cc = e % T;
    if (rr > cc) continue;
    const float2* P = a.partials + size_t(w) * nparts * T * T + e;
    double sx = 0.0, sy = 0.0;
    for (uint32_t k = 0; k < nparts; ++k) {
      const float2 v = P[size_t(k) * T * T];
      sx += v.x;
      sy += v.y;
    }
    if (rr == cc) sy = 0.0;
    double2* Cw = a.C + size_t(w) * T * T;
    Cw[rr * T + cc] = make_double2(sx, sy);
    Cw[cc * T + rr] = make_double2(sx, -sy);
  }
}

// V = Vf in float64; the diagonal of C' made exactly real.
__global__ void k_vf_to_v(PcaArgs a) {
  const int T = a.T;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < T * T; e += gridDim.x * blockDim.x) {
    a.V[e] = make_double2(a.Vf[e].x, a.Vf[e].y);
    if (e / T == e % T) a.C[e].y = 0.0;
  }
}

template <int T>
static cudaError_t launch_jacobi_small(const PcaArgs& a, cudaStream_t s) {
  const size_t smem = size_t(2) * T * T * sizeof(double2) + size_t(T) * T * sizeof(float2);  // RA, C', Vf
  cudaError_t e = cudaFuncSetAttribute(k_jacobi_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  k_jacobi_small<T><<<a.nwin, 256, smem, s>>>(a);
  return cudaGetLastError();
}

size_t pca_partials_floats2(uint32_t T, uint32_t nchunks) {
  const uint32_t TS = T < uint32_t(COV_TS) ? T : COV_TS, nT = T / TS;
  return size_t(nchunks) * (nT * (nT + 1) / 2) * TS * TS;
}

cudaError_t launch_pca_cov(PcaArgs& a, cudaStream_t s, int* launches) {
  const size_t hw = size_t(a.W) * a.H;
  const int TS = a.T < uint32_t(COV_TS) ? int(a.T) : COV_TS;
  if (a.T % TS || TS % 16 || hw % 256 || a.T % PRJ_KS) return cudaErrorInvalidValue;
  if (a.nwin == 0 || a.tq.slot0 >= a.tq.cap || uint64_t(a.nwin - 1) * a.wstride + a.T > a.tq.cap)
    return cudaErrorInvalidValue;  // the frame addressing (frame_ptr) relies on both
  const int nT = a.T / TS;
  const dim3 g1(nT * (nT + 1) / 2, a.nchunks, a.nwin);
  cudaError_t e0 = cudaMemsetAsync(a.counters, 0, 4 * sizeof(unsigned) + sizeof(double), s);
  if (e0 != cudaSuccess) return e0;
  if (a.precision == HV_PREC_FP32 && (a.T == 32 || a.T == 64)) {
    const size_t smem = cov_small_smem(int(a.T));
    const dim3 gs(a.nchunks, a.nwin);
    if (a.T == 32) {
      cudaFuncSetAttribute(k_cov_small<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      k_cov_small<32><<<gs, 256, smem, s>>>(a);
    } else {
      cudaFuncSetAttribute(k_cov_small<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      k_cov_small<64><<<gs, 256, smem, s>>>(a);
    }
    k_cov_small_reduce<<<unsigned((size_t(a.nwin) * a.T * a.T + 255) / 256), 256, 0, s>>>(a, a.nchunks);
    *launches += 2;
  } else if (a.precision == HV_PREC_FP32) {
    k_cov_fp32<<<g1, 256, 0, s>>>(a);
    k_cov_reduce<<<(a.T * a.T + 255) / 256, 256, 0, s>>>(a);
    *launches += 2;
  } else {
    cudaError_t et = launch_cov_tc(a, s, launches);
    if (et != cudaSuccess) return et;
  }
  return cudaGetLastError();
}

cudaError_t launch_pca_eig(PcaArgs& a, cudaStream_t s, int* launches) {
  cudaError_t e = cudaSuccess;
  if (a.T == 32) {
    e = launch_jacobi_small<32>(a, s);
  } else if (a.T == 64) {
    e = launch_jacobi_small<64>(a, s);
  } else {
    if (a.nwin != 1) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_refine, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    void* args[] = {&a};
    // (1) float32 sweeps: on one 16-CTA cluster (T = 128, 256), else cooperative on a
    // quarter of the SMs
    bool on_cluster = false;
    if (a.T == 256) e = launch_jacobi_cluster<256, false>(a, s, &on_cluster);
    else if (a.T == 128) e = launch_jacobi_cluster<128, false>(a, s, &on_cluster);
    if (e != cudaSuccess) return e;
    if (!on_cluster) {
      const int nf = nsm / 4 > 0 ? nsm / 4 : 1;
      e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_jacobi_f32), dim3(nf), dim3(256), args, 0, s);
      if (e != cudaSuccess) return e;
    }
    // (2) C' = Vf^H (C Vf) and V = Vf in float64
    const dim3 gg(a.T / 16, a.T / 16);
    k_gemm_c64<<<gg, 256, 0, s>>>(int(a.T), a.C, nullptr, 0, nullptr, a.Vf, a.C2);     // M = C Vf
    k_gemm_c64<<<gg, 256, 0, s>>>(int(a.T), nullptr, a.Vf, 1, a.C2, nullptr, a.C);     // C' = Vf^H M
    *launches += 3;
    // (3) float64 sweeps on C' (off-diagonals ~1e-6 of the trace): at most two, fewer
    // when every entry met in a sweep is below 1e-12 of the trace. Two leave the
    // energy image within ~2e-5 of the float64 reference and the eigenvalues within
    // ~3e-8 of the largest (a third and fourth sweep halve the first figure only;
    // the covariance itself carries float32 accumulation error). On the cluster when
    // the float32 phase ran there, else cooperative over all SMs (V = Vf first).
    PcaArgs b = a;
    b.max_sweeps = 2;
    b.stop_rel = 1e-12;
    bool ref_cluster = false;
    if (on_cluster && a.T == 256) e = launch_jacobi_cluster<256, true>(b, s, &ref_cluster);
    else if (on_cluster && a.T == 128) e = launch_jacobi_cluster<128, true>(b, s, &ref_cluster);
    if (e != cudaSuccess) return e;
    if (ref_cluster) {
      k_vcorr<<<gg, 256, 0, s>>>(a);  // V = Vf (I + D)
      *launches += 1;
    } else {
      k_vf_to_v<<<(a.T * a.T + 255) / 256, 256, 0, s>>>(a);
      void* bargs[] = {&b};
      e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_jacobi_refine), dim3(nsm), dim3(256), bargs, 0, s);
      if (e != cudaSuccess) return e;
      *launches += 1;
    }
    // the cooperative paths' rotation table is free by now: lam and 1/|v| of every column
    double* scratch = a.rot;
    k_pca_norms<<<a.T / 16, 256, 0, s>>>(a, scratch);
    k_pca_select<<<1, 1024, 0, s>>>(a, scratch);
    *launches += 3;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_pca_proj(PcaArgs& a, float* out, cudaStream_t s, int* launches) {
  cudaError_t e;
  if (a.Mpad % 64 == 0) e = launch_project<64>(a, out, s);
  else if (a.Mpad % 32 == 0) e = launch_project<32>(a, out, s);
  else e = launch_project<16>(a, out, s);
  if (e != cudaSuccess) return e;
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_pca(PcaArgs& a, float* out, cudaStream_t s, int* launches, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], s);
  cudaError_t e = launch_pca_cov(a, s, launches);
  if (e != cudaSuccess) return e;
  if (ev) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
  }
  e = launch_pca_eig(a, s, launches);
  if (e != cudaSuccess) return e;
  if (ev) {
    cudaEventRecord(ev[3], s);
    cudaEventRecord(ev[4], s);
  }
  e = launch_pca_proj(a, out, s, launches);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[5], s);
  return cudaSuccess;
}

// total[0] += float32 sweeps, total[1] += refinement sweeps of the last window
__global__ void k_pca_sweeps_add(const unsigned* counters, unsigned long long* total) {
  total[0] += counters[1];
  total[1] += counters[2];
}

cudaError_t launch_pca_sweeps_add(const unsigned* counters, unsigned long long* total, cudaStream_t s) {
  k_pca_sweeps_add<<<1, 1, 0, s>>>(counters, total);
  return cudaGetLastError();
}

}  // namespace hv
