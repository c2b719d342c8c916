// hv_api.cu -- the C ABI (include/hv.h): handle, input ring, time-transformation
// queue, delayed settings and the render scheduler.
//
// Buffers follow Sec. II-B.1: fixed-size device buffers allocated once per
// setting (Sec. VII-C: allocate up front, never in the per-batch loop) and a
// ring FIFO for input frames with backpressure instead of frame drops. Compute
// settings are "delayed" (Sec. IV-B): hv_set_params validates and stores them;
// they take effect at the next window boundary (start of the next hv_render).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <deque>
#include <vector>

#include "../../include/hv.h"
#include "hv_internal.h"

using namespace hv;

struct hv_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_pushed = nullptr, ev_consumed = nullptr;
  // raw-ring consumption: event k is recorded on the stream after a spatial stage
  // that had propagated every frame below cons_hi[k] (oldest first, circular)
  static constexpr int NCONS = 32;
  cudaEvent_t cons_ev[NCONS] = {};
  uint64_t cons_hi[NCONS] = {};
  int cons_head = 0, cons_n = 0;
  // frames pushed with HV_MEM_DEVICE_ASYNC are read in place: frames first .. first
  // + n - 1 at ptr (oldest first); entries below the next window are dropped
  struct Borrowed {
    uint64_t first;
    uint32_t n;
    const void* ptr;
  };
  std::deque<Borrowed> borrowed;
  uint32_t max_w = 0, max_h = 0, bits = 8, cap = 0, tq_req = 0;
  void* raw = nullptr;
  // settings
  bool has_params = false, pending = false;
  hv_params cur{}, pend{};
  uint32_t W = 0, H = 0, T = 1, S = 1, klo = 0, khi = 0, nout = 0;
  size_t win_floats = 0;
  // device workspace
  float2* tq = nullptr;
  uint32_t Q = 0;
  size_t tq_bytes = 0;
  float2* s1 = nullptr;
  float2* s2 = nullptr;
  size_t s1_bytes = 0, s2_bytes = 0;
  uint32_t chunk = 0;
  int sp_cluster = 0;         // 1: whole-frame cluster kernel
  int sp_pp = 0;              // 1: persistent multi-pass kernels
  int sp_fused = 0;           // 1: fused transform (s1 / s2 are rings of kFusedRing frames)
  int inject = HV_INJECT_NONE;  // pending fault injection (hv_debug_inject)
  int stft_kernel = STFT_AUTO;  // STFT kernel for windows that do not overlap (autotuner's choice)
  unsigned* fused_ctr = nullptr;  // its ticket and per-slot counters
  size_t fused_ctr_bytes = 0;
  hv_tuning tuning{};
  float2* tw = nullptr;  // all twiddle tables, length 8..1024 packed
  unsigned* dev_err = nullptr;  // sticky device flags: a kernel's bounded wait gave up
  float2* asp_ht = nullptr;
  float2* chirp = nullptr;  // [W] x factors then [H] y factors
  size_t table_bytes = 0;
  float* staging = nullptr;
  size_t staging_bytes = 0;
  // stream state (frame indices since open)
  uint64_t pushed = 0, next_win = 0, propagated = 0;
  hv_stats st{};
  std::string err;
  // PCA workspace
  void* pca_ws = nullptr;
  size_t pca_ws_bytes = 0;
  PcaArgs pca{};
  bool pca_has_lam = false;
  bool pca_batched = false;   // T <= 64 with FP32 covariance: many windows per launch
  uint32_t pca_last_nwin = 1;
  // long windows, several per render: the eigensolver of one window (16 SMs) runs on
  // eig_stream while the handle's stream runs the next window's covariance and the
  // previous window's projection; windows alternate between two sets of C, counters,
  // eigenvalues and sub-basis (set 0 is the one in `pca`)
  cudaStream_t eig_stream = nullptr;
  cudaEvent_t ev_cov[2] = {}, ev_eig[2] = {};
  double2* pca_C[2] = {};
  unsigned* pca_cnt[2] = {};
  double* pca_lam[2] = {};
  float2* pca_Vs[2] = {};
  const double* pca_lam_last = nullptr;  // eigenvalues of the last window rendered
  // stage timing
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev;  // triples: before spatial, after spatial, after temporal
  size_t prof_used = 0;
  hv_profile prof_acc{};
  std::vector<cudaEvent_t> pca_ev;   // groups of 8 per recorded PCA window (start, end of spatial
                                     // chunk -- pipelined windows only --, covariance, eigensolver,
                                     // projection)
  size_t pca_ev_used = 0;
  unsigned long long* pca_sweeps_dev = nullptr;  // float32 and refinement sweeps while profiling
  // focus sweep: transfer functions of the swept distances (DC bin zero), cached
  float2* sw_tables = nullptr;
  size_t sw_bytes = 0;
  std::vector<double> sw_key;        // W, H, lambda, pitches, then the distances
  double* sw_acc = nullptr;
  size_t sw_acc_bytes = 0;
  // post-processing: settings (current, pending), kernel weights, image ring
  hv_post post_cur{}, post_pend{};
  std::vector<float> post_k_cur, post_k_pend;
  bool post_pending = false, post_active = false, post_dirty = true;
  float* post_kdev = nullptr;
  size_t post_kdev_bytes = 0;
  float* post_ring = nullptr;
  size_t post_ring_bytes = 0;
  double* post_sums = nullptr;
  size_t post_sums_bytes = 0;
  uint32_t post_R = 0;
  uint64_t post_count = 0;
};

// A group of handles stepped together (hv_render_group).
struct hv_group {
  std::vector<hv_handle*> hs;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool use_graph = false;
  cudaEvent_t ev_fork = nullptr, ev_done = nullptr;
  std::vector<cudaEvent_t> ev_pre, ev_join;  // per member
  cudaGraphExec_t exec = nullptr;
  hv_group_stats st{};
  std::string err;
};

namespace {

thread_local std::string g_open_err;

constexpr int kMinLog = 3, kMaxLog = 10;  // twiddle tables for L = 8 .. 1024

size_t tw_offset(uint32_t L) {  // tables packed by increasing length
  size_t off = 0;
  for (uint32_t l = 1u << kMinLog; l < L; l <<= 1) off += l;
  return off;
}

bool is_pow2(uint32_t v) { return v && !(v & (v - 1)); }

hv_status fail(hv_handle* h, hv_status s, const std::string& msg) {
  if (h) h->err = msg;
  else g_open_err = msg;
  return s;
}

hv_status cuda_fail(hv_handle* h, cudaError_t e, const char* what) {
  return fail(h, HV_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define HV_CU(h, call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

template <class Tp>
void dfree(Tp*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

uint32_t popcount5(uint32_t m) {
  uint32_t n = 0;
  for (int i = 0; i < 5; ++i) n += (m >> i) & 1u;
  return n;
}

// Derived quantities of a settings block; also the validation.
struct Derived {
  uint32_t T, S, klo, khi, nout;
  size_t win_floats;
};

hv_status validate(const hv_handle* h, const hv_params& p, Derived& d, std::string& why) {
  if (p.struct_size != sizeof(hv_params)) { why = "hv_params.struct_size mismatch"; return HV_ERR_ARG; }
  if (!is_pow2(p.width) || !is_pow2(p.height) || p.width < 16 || p.height < 16 || p.width > 1024 ||
      p.height > 1024) {
    why = "width and height must be powers of two in [16, 1024]";
    return HV_ERR_ARG;
  }
  if (p.width > h->max_w || p.height > h->max_h) { why = "frame larger than the handle's maximum"; return HV_ERR_ARG; }
  if (p.spatial != HV_SPATIAL_NONE && p.spatial != HV_SPATIAL_ASP && p.spatial != HV_SPATIAL_FRESNEL) {
    why = "unknown spatial transform";
    return HV_ERR_ARG;
  }
  if (p.spatial_kernel > HV_SK_FUSED) { why = "unknown spatial_kernel"; return HV_ERR_ARG; }
  if (p.stft_kernel != 0 && p.stft_kernel != HV_STFT_WALK && p.stft_kernel != HV_STFT_WINDOW &&
      p.stft_kernel != HV_STFT_WINDOW_WIDE && p.stft_kernel != HV_STFT_WINDOW_PIPELINED &&
      p.stft_kernel != HV_STFT_WINDOW_TMA && p.stft_kernel != HV_STFT_WINDOW_TMA_PIPELINED) {
    why = "unknown stft_kernel";
    return HV_ERR_ARG;
  }
  if (p.spatial_kernel == HV_SK_FUSED &&
      (p.width != 256 || p.height != 256 || (p.spatial != HV_SPATIAL_ASP && p.spatial != HV_SPATIAL_FRESNEL))) {
    why = "the fused spatial transform needs 256 x 256 frames and ASP or Fresnel";
    return HV_ERR_UNSUPPORTED;
  }
  if (p.spatial_kernel == HV_SK_PERSISTENT &&
      !(p.width >= 64 && p.height >= 64 && (p.spatial == HV_SPATIAL_ASP || p.spatial == HV_SPATIAL_FRESNEL))) {
    why = "the persistent multi-pass kernels need sides in [64, 1024] and ASP or Fresnel";
    return HV_ERR_UNSUPPORTED;
  }
  if (p.spatial_kernel == HV_SK_CLUSTER &&
      !(p.width == p.height && (p.width == 128 || p.width == 256 || p.width == 512) &&
        (p.spatial == HV_SPATIAL_ASP || p.spatial == HV_SPATIAL_FRESNEL))) {
    why = "the cluster kernel needs square 128, 256 or 512 frames and ASP or Fresnel";
    return HV_ERR_UNSUPPORTED;
  }
  if (p.spatial != HV_SPATIAL_NONE) {
    if (!(p.lambda_m > 0) || !(p.pitch_x_m > 0) || !(p.pitch_y_m > 0) || !std::isfinite(p.z_m)) {
      why = "lambda, pitches must be > 0 and z finite";
      return HV_ERR_ARG;
    }
    if (p.spatial == HV_SPATIAL_FRESNEL && p.z_m == 0.0) { why = "Fresnel needs z != 0"; return HV_ERR_ARG; }
  }
  if (!(p.highpass_cpp >= 0.0) || p.highpass_cpp > 1.0) { why = "highpass_cpp must be in [0, 1]"; return HV_ERR_ARG; }
  if (p.highpass_cpp > 0.0 && p.spatial != HV_SPATIAL_ASP) {
    why = "the high-pass filter is applied with angular-spectrum propagation only";
    return HV_ERR_ARG;
  }
  const size_t hw = size_t(p.width) * p.height;
  if (p.temporal == HV_TEMPORAL_NONE) {
    d = Derived{1, 1, 0, 0, 0, 2 * hw};
    return HV_OK;
  }
  if (p.temporal == HV_TEMPORAL_PCA) {
    if (!is_pow2(p.T) || p.T < 32 || p.T > 512) { why = "PCA needs T a power of two in [32, 512]"; return HV_ERR_ARG; }
    if (p.stride < 1) { why = "stride must be >= 1"; return HV_ERR_ARG; }
    if (p.pca_lo < 1 || p.pca_hi < p.pca_lo || p.pca_hi > p.T) {
      why = "PCA sub-basis must satisfy 1 <= pca_lo <= pca_hi <= T";
      return HV_ERR_ARG;
    }
    if (p.precision != HV_PREC_FP32 && p.precision != HV_PREC_BF16 && p.precision != HV_PREC_SPLIT_BF16) {
      why = "unknown precision";
      return HV_ERR_ARG;
    }
    if (p.precision != HV_PREC_FP32 && p.T < 64) {
      why = "tensor-core covariance needs T >= 64";
      return HV_ERR_UNSUPPORTED;
    }
    d = Derived{p.T, p.stride, 0, 0, 1, hw};
    return HV_OK;
  }
  if (p.temporal != HV_TEMPORAL_STFT) { why = "unknown temporal transform"; return HV_ERR_ARG; }
  if (!is_pow2(p.T) || p.T < 8 || p.T > 1024) { why = "T must be a power of two in [8, 1024]"; return HV_ERR_ARG; }
  if (p.stride < 1) { why = "stride must be >= 1"; return HV_ERR_ARG; }
  if (!(p.fs_hz > 0)) { why = "fs_hz must be > 0"; return HV_ERR_ARG; }
  uint32_t klo = p.band_lo_bin, khi = p.band_hi_bin;
  if (p.band_lo_hz > 0 && p.band_hi_hz > 0) {
    const double a = std::ceil(p.band_lo_hz * p.T / p.fs_hz - 1e-12);
    const double b = std::floor(p.band_hi_hz * p.T / p.fs_hz + 1e-12);
    if (a < 0 || b < a || b >= p.T) { why = "band in Hz selects no bin inside [0, T)"; return HV_ERR_ARG; }
    klo = uint32_t(a);
    khi = uint32_t(b);
  }
  if (klo > khi || khi >= p.T) { why = "band bins must satisfy lo <= hi < T"; return HV_ERR_ARG; }
  if (p.moments_mask == 0 || p.moments_mask > 31) { why = "moments_mask must select M0..M2N bits"; return HV_ERR_ARG; }
  const uint32_t nout = popcount5(p.moments_mask);
  d = Derived{p.T, p.stride, klo, khi, nout, size_t(nout) * hw};
  return HV_OK;
}

// exp(i a) in float64, rounded to float
float2 cis(double a) { return make_float2(float(std::cos(a)), float(std::sin(a))); }

// Build ASP / Fresnel tables for p in float64 and upload them.
hv_status build_tables(hv_handle* h, const hv_params& p) {
  const uint32_t W = p.width, H = p.height;
  // [Hᵀ: W H][chirp x: W][chirp y: H][H row-major: W H]
  const size_t need = (2 * size_t(W) * H + W + H) * sizeof(float2);
  if (need > h->table_bytes) {
    dfree(h->asp_ht);
    HV_CU(h, cudaMalloc(&h->asp_ht, need));
    h->table_bytes = need;
  }
  h->chirp = h->asp_ht + size_t(W) * H;
  std::vector<float2> host(2 * size_t(W) * H + W + H, make_float2(0.f, 0.f));
  const size_t rowmajor = size_t(W) * H + W + H;
  if (p.spatial == HV_SPATIAL_ASP) {
    // H(kx, ky) = exp(i z sqrt(k^2 - kx^2 - ky^2)), zero where evanescent; stored
    // transposed [kx][ky] with the inverse transform's 1/(W H) folded in.
    const double k = 2.0 * M_PI / p.lambda_m;
    const double scale = 1.0 / (double(W) * double(H));
    for (uint32_t kx = 0; kx < W; ++kx) {
      const double mx = kx < W / 2 ? double(kx) : double(kx) - W;
      const double fx = 2.0 * M_PI * mx / (W * p.pitch_x_m);
      for (uint32_t ky = 0; ky < H; ++ky) {
        const double my = ky < H / 2 ? double(ky) : double(ky) - H;
        const double fy = 2.0 * M_PI * my / (H * p.pitch_y_m);
        const double kz2 = k * k - fx * fx - fy * fy;
        float2 v = make_float2(0.f, 0.f);
        // high-pass filter after propagation = mask on the propagated spectrum
        const double rx = mx / W, ry = my / H;
        const bool passed = !(p.highpass_cpp > 0.0) || rx * rx + ry * ry >= p.highpass_cpp * p.highpass_cpp;
        if (kz2 >= 0 && passed) {
          const double ph = p.z_m * std::sqrt(kz2);
          v = make_float2(float(std::cos(ph) * scale), float(std::sin(ph) * scale));
        }
        host[size_t(kx) * H + ky] = v;
        host[rowmajor + size_t(ky) * W + kx] = v;
      }
    }
  } else if (p.spatial == HV_SPATIAL_FRESNEL) {
    // chirp exp(i pi (x^2 + y^2) / (lam z)) = cx(x) cy(y), x = (j - W/2) dx; the
    // fftshift of the output is the input modulation (-1)^(j + l).
    const double c = M_PI / (p.lambda_m * p.z_m);
    for (uint32_t j = 0; j < W; ++j) {
      const double x = (double(j) - W / 2.0) * p.pitch_x_m;
      double ph = c * x * x + ((p.fftshift && (j & 1)) ? M_PI : 0.0);
      host[size_t(W) * H + j] = cis(ph);
    }
    for (uint32_t l = 0; l < H; ++l) {
      const double y = (double(l) - H / 2.0) * p.pitch_y_m;
      double ph = c * y * y + ((p.fftshift && (l & 1)) ? M_PI : 0.0);
      host[size_t(W) * H + W + l] = cis(ph);
    }
  }
  HV_CU(h, cudaMemcpyAsync(h->asp_ht, host.data(), need, cudaMemcpyHostToDevice, h->stream));
  HV_CU(h, cudaStreamSynchronize(h->stream));
  return HV_OK;
}

hv_status ensure(hv_handle* h, void** p, size_t* have, size_t need) {
  if (need <= *have) return HV_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(p, need);
  if (e != cudaSuccess) return fail(h, HV_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  *have = need;
  return HV_OK;
}

hv_status tune_spatial(hv_handle* h);
hv_status tune_temporal(hv_handle* h);

// Apply the pending settings (window boundary).
hv_status apply_pending(hv_handle* h) {
  if (!h->pending) return HV_OK;
  const hv_params& p = h->pend;
  Derived d{};
  std::string why;
  hv_status s = validate(h, p, d, why);
  if (s != HV_OK) return fail(h, s, why);
  // make sure earlier work that used the old workspace is finished
  HV_CU(h, cudaStreamSynchronize(h->stream));
  const uint32_t W = p.width, H = p.height;
  const size_t fbytes = size_t(W) * H * sizeof(float2);
  // time-transformation queue: T frames plus room for many windows per launch
  uint32_t Q = h->tq_req;
  if (Q == 0) {
    // room for about 4096 new frames (and at least 64 windows) per temporal launch
    const uint64_t target = uint64_t(d.T) + uint64_t(d.S) * std::max<uint64_t>(63, 4095 / d.S);
    const uint64_t cap_frames = std::max<uint64_t>(d.T, (size_t(4) << 30) / fbytes);
    Q = uint32_t(std::min<uint64_t>(target, cap_frames));
  }
  Q = std::max(Q, d.T);
  s = ensure(h, reinterpret_cast<void**>(&h->tq), &h->tq_bytes, size_t(Q) * fbytes);
  if (s != HV_OK) return s;
  uint32_t chunk = p.spatial_chunk ? p.spatial_chunk : std::max<uint32_t>(1, uint32_t((size_t(32) << 20) / fbytes));
  chunk = std::min<uint32_t>(chunk, 1024);
  const bool fused = p.spatial_kernel == HV_SK_FUSED;
  const size_t sbytes = size_t(fused ? std::max(chunk, kFusedRing) : chunk) * fbytes;
  if (fused) {
    s = ensure(h, reinterpret_cast<void**>(&h->fused_ctr), &h->fused_ctr_bytes,
               (1 + kFusedPasses * size_t(kFusedRing)) * sizeof(unsigned));
    if (s != HV_OK) return s;
  }
  if (p.spatial != HV_SPATIAL_NONE) {
    s = ensure(h, reinterpret_cast<void**>(&h->s1), &h->s1_bytes, sbytes);
    if (s != HV_OK) return s;
    if (p.spatial == HV_SPATIAL_ASP) {
      s = ensure(h, reinterpret_cast<void**>(&h->s2), &h->s2_bytes, sbytes);
      if (s != HV_OK) return s;
    }
  }
  s = build_tables(h, p);
  if (s != HV_OK) return s;
  if (p.temporal == HV_TEMPORAL_PCA) {
    const size_t hw = size_t(W) * H;
    const bool batched = d.T <= 64 && p.precision == HV_PREC_FP32;
    const uint32_t NW = batched ? 128 : 1;  // windows per launch
    // batched (T <= 64): 2048-pixel chunks, one partial T x T matrix per chunk and window;
    // otherwise up to 64 chunks of the tiled covariance
    uint32_t nchunks = batched ? uint32_t(std::max<size_t>(1, hw / 2048))
                               : uint32_t(std::min<size_t>(64, std::max<size_t>(1, hw / 1024)));
    uint32_t chunk = uint32_t((hw + nchunks - 1) / nchunks);
    chunk = (chunk + 63) / 64 * 64;
    nchunks = uint32_t((hw + chunk - 1) / chunk);
    const uint32_t T = d.T, M = p.pca_hi - p.pca_lo + 1, Mpad = (M + 15) / 16 * 16;
    const size_t b_part = (batched ? size_t(nchunks) * T * T : pca_partials_floats2(T, nchunks)) * sizeof(float2) * NW;
    const size_t b_mat = size_t(T) * T * sizeof(double2);
    const size_t b_rot = size_t(T / 2) * 4 * sizeof(double);
    const size_t b_cnt = 64;
    const size_t b_lam = size_t(T) * sizeof(double) * NW;
    const size_t b_vs = size_t(T) * Mpad * sizeof(float2) * NW;
    // tensor-core covariance tiles and chunks (about one CTA per SM)
    uint8_t ti[32] = {}, tj[32] = {};
    uint32_t ntiles = 0, tc_nchunks = 0, tc_chunk = 0;
    size_t b_tc = 0;
    if (p.precision != HV_PREC_FP32) {
      ntiles = cov_tc_tiles(T, ti, tj);
      int dev = 0, nsm = 152;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      tc_nchunks = std::max<uint32_t>(1, uint32_t(nsm) / ntiles);
      tc_chunk = uint32_t((hw + tc_nchunks - 1) / tc_nchunks);
      tc_chunk = (tc_chunk + 63) / 64 * 64;
      tc_nchunks = uint32_t((hw + tc_chunk - 1) / tc_chunk);
      b_tc = cov_tc_partials_floats(ntiles, tc_nchunks) * sizeof(float);
    }
    // BF16 operand staging: 64-pixel steps x 2T rows x 64 values per part
    const size_t stage_part = p.precision != HV_PREC_FP32 ? (hw + 63) / 64 * 64 * 2 * size_t(T) : 0;
    const size_t b_stage = stage_part * sizeof(uint16_t) * (p.precision == HV_PREC_SPLIT_BF16 ? 2 : 1);
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t b_matf = size_t(T) * T * sizeof(float2);
    // the second window set of the pipelined long windows: C, counters, lam, Vs
    const size_t b_set2 = batched ? 0 : al(b_mat) + al(b_cnt) + al(b_lam) + al(b_vs);
    const size_t total = al(b_part) + (NW + 2) * al(b_mat) + 3 * al(b_matf) + al(b_rot) + al(b_cnt) + al(b_lam) +
                         al(b_vs) + al(b_tc) + al(b_stage) + b_set2;
    s = ensure(h, &h->pca_ws, &h->pca_ws_bytes, total);
    if (s != HV_OK) return s;
    char* b = static_cast<char*>(h->pca_ws);
    PcaArgs& a = h->pca;
    a = PcaArgs{};
    a.W = W;
    a.H = H;
    a.T = T;
    a.chunk = chunk;
    a.nchunks = nchunks;
    a.lo = p.pca_lo;
    a.M = M;
    a.Mpad = Mpad;
    a.max_sweeps = 30;
    // skip a rotation when |C_ab| <= 1e-14 sqrt(C_aa C_bb) or <= 1e-13 max_i C_ii: the
    // second bound sits above the rounding noise that rotations leave in small
    // entries (~1e-16 max C_ii), so sweeps stop once only noise is left
    a.tol = 1e-14;
    a.tol_abs = 1e-13;
    a.partials = reinterpret_cast<float2*>(b);
    b += al(b_part);
    a.C = reinterpret_cast<double2*>(b);
    b += NW * al(b_mat);
    a.V = reinterpret_cast<double2*>(b);
    b += al(b_mat);
    a.C2 = reinterpret_cast<double2*>(b);
    b += al(b_mat);
    a.Cf = reinterpret_cast<float2*>(b);
    b += al(b_matf);
    a.Cf2 = reinterpret_cast<float2*>(b);
    b += al(b_matf);
    a.Vf = reinterpret_cast<float2*>(b);
    b += al(b_matf);
    a.rot = reinterpret_cast<double*>(b);
    b += al(b_rot);
    a.counters = reinterpret_cast<unsigned*>(b);
    a.cmax = reinterpret_cast<double*>(a.counters + 4);
    b += al(b_cnt);
    a.lam = reinterpret_cast<double*>(b);
    b += al(b_lam);
    a.Vs = reinterpret_cast<float2*>(b);
    b += al(b_vs);
    a.precision = p.precision;
    a.tc_partials = b_tc ? reinterpret_cast<float*>(b) : nullptr;
    b += al(b_tc);
    a.tc_stage = b_stage ? reinterpret_cast<uint16_t*>(b) : nullptr;
    a.tc_stage_part = stage_part;
    a.tc_chunk = tc_chunk;
    a.tc_nchunks = tc_nchunks;
    a.tc_ntiles = ntiles;
    std::memcpy(a.tc_tile_i, ti, sizeof(ti));
    std::memcpy(a.tc_tile_j, tj, sizeof(tj));
    b += al(b_stage);
    h->pca_C[0] = a.C;
    h->pca_cnt[0] = a.counters;
    h->pca_lam[0] = a.lam;
    h->pca_Vs[0] = a.Vs;
    h->pca_C[1] = nullptr;
    if (!batched) {
      h->pca_C[1] = reinterpret_cast<double2*>(b);
      b += al(b_mat);
      h->pca_cnt[1] = reinterpret_cast<unsigned*>(b);
      b += al(b_cnt);
      h->pca_lam[1] = reinterpret_cast<double*>(b);
      b += al(b_lam);
      h->pca_Vs[1] = reinterpret_cast<float2*>(b);
    }
    a.err = h->dev_err;
    a.nwin = 1;
    a.wstride = d.S;
    h->pca_batched = batched;
    h->pca_has_lam = false;
    h->pca_lam_last = nullptr;
  }
  h->cur = p;
  h->has_params = true;
  h->pending = false;
  h->post_dirty = true;  // ring sizes depend on the settings
  h->W = W;
  h->H = H;
  h->T = d.T;
  h->S = d.S;
  h->klo = d.klo;
  h->khi = d.khi;
  h->nout = d.nout;
  h->win_floats = d.win_floats;
  h->Q = Q;
  h->chunk = chunk;
  h->sp_cluster = p.spatial_kernel == HV_SK_CLUSTER ? 1 : 0;
  h->sp_pp = p.spatial_kernel == HV_SK_PERSISTENT ? 1 : 0;
  h->sp_fused = fused ? 1 : 0;
  h->tuning = hv_tuning{};
  h->tuning.spatial_chunk = chunk;
  h->tuning.spatial_kernel = p.spatial_kernel == HV_SK_AUTO ? HV_SK_MULTIPASS : int32_t(p.spatial_kernel);
  // STFT kernel for windows that do not overlap: the caller's, the autotuner's (tuned),
  // else the walking kernel launched once per window (the plain form)
  h->stft_kernel = p.stft_kernel == HV_STFT_WINDOW ? STFT_AUTO
                   : p.stft_kernel == HV_STFT_WINDOW_WIDE     ? STFT_WIDE
                   : p.stft_kernel == HV_STFT_WINDOW_PIPELINED ? STFT_PIPE
                   : p.stft_kernel == HV_STFT_WINDOW_TMA       ? STFT_TMA
                   : p.stft_kernel == HV_STFT_WINDOW_TMA_PIPELINED ? STFT_TMA_PIPE
                                                               : STFT_WALK;
  if (p.tuned && p.spatial_kernel == HV_SK_AUTO) {
    s = tune_spatial(h);  // rewrites the tuning record
    if (s != HV_OK) return s;
  }
  h->tuning.stft_kernel = p.stft_kernel == 0 ? HV_STFT_WALK : p.stft_kernel;
  if (p.tuned && p.stft_kernel == 0 && p.temporal == HV_TEMPORAL_STFT && d.S >= d.T) {
    s = tune_temporal(h);
    if (s != HV_OK) return s;
  }
  // queue flush: the next window starts at the first unconsumed frame and is
  // propagated entirely with the new settings
  h->propagated = h->next_win;
  return HV_OK;
}

// Fold the completed event triples into the accumulator.
hv_status prof_flush(hv_handle* h) {
  if (h->prof_used == 0 && h->pca_ev_used == 0) return HV_OK;
  HV_CU(h, cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i < h->pca_ev_used; i += 8) {
    float sp = 0.f, a = 0.f, b = 0.f, c = 0.f;
    HV_CU(h, cudaEventElapsedTime(&sp, h->pca_ev[i], h->pca_ev[i + 1]));
    HV_CU(h, cudaEventElapsedTime(&a, h->pca_ev[i + 2], h->pca_ev[i + 3]));
    HV_CU(h, cudaEventElapsedTime(&b, h->pca_ev[i + 4], h->pca_ev[i + 5]));
    HV_CU(h, cudaEventElapsedTime(&c, h->pca_ev[i + 6], h->pca_ev[i + 7]));
    // a pipelined window's spatial chunk runs inside the render's temporal span
    h->prof_acc.spatial_ms += sp;
    h->prof_acc.temporal_ms -= sp;
    h->prof_acc.pca_cov_ms += a;
    h->prof_acc.pca_eig_ms += b;
    h->prof_acc.pca_proj_ms += c;
  }
  h->pca_ev_used = 0;
  for (size_t i = 0; i + 2 < h->prof_used; i += 3) {
    float a = 0.f, b = 0.f;
    HV_CU(h, cudaEventElapsedTime(&a, h->prof_ev[i], h->prof_ev[i + 1]));
    HV_CU(h, cudaEventElapsedTime(&b, h->prof_ev[i + 1], h->prof_ev[i + 2]));
    h->prof_acc.spatial_ms += a;
    h->prof_acc.temporal_ms += b;
  }
  // an incomplete triple (flush called inside a render) stays for the next flush
  const size_t keep = h->prof_used % 3;
  for (size_t k = 0; k < keep; ++k) std::swap(h->prof_ev[k], h->prof_ev[h->prof_used - keep + k]);
  h->prof_used = keep;
  return HV_OK;
}

hv_status prof_mark(hv_handle* h, int which) {
  if (!h->prof) return HV_OK;
  if (which == 0 && h->prof_used + 3 > h->prof_ev.size()) {
    hv_status s = prof_flush(h);
    if (s != HV_OK) return s;
  }
  HV_CU(h, cudaEventRecord(h->prof_ev[h->prof_used++], h->stream));
  return HV_OK;
}

bool cluster_ok(const hv_handle* h) {
  return h->W == h->H && (h->W == 128 || h->W == 256 || h->W == 512) &&
         (h->cur.spatial == HV_SPATIAL_ASP || h->cur.spatial == HV_SPATIAL_FRESNEL);
}

// Spatial transform of frames r0 .. r1 - 1, whose raw frames are at `raw` (frame
// r0 at slot raw.slot0); the time queue slots follow the frame numbers.
hv_status propagate_run(hv_handle* h, uint64_t r0, uint64_t r1, RingRef raw) {
  // the cluster kernel needs no scratch, the fused transform keeps its intermediates
  // in rings: one persistent launch for all frames
  const bool whole = (h->sp_cluster && cluster_ok(h)) || h->sp_fused;
  const uint64_t step = whole ? r1 - r0 : h->chunk;
  for (uint64_t a = r0; a < r1; a += step) {
    const uint32_t n = uint32_t(std::min<uint64_t>(step, r1 - a));
    SpatialArgs sa{};
    sa.err = h->dev_err;
    sa.spatial = h->cur.spatial;
    sa.in_kind = h->bits == 8 ? IN_U8 : IN_U16;
    sa.W = h->W;
    sa.H = h->H;
    sa.n = n;
    sa.raw = RingRef{raw.base, raw.cap, uint32_t((raw.slot0 + (a - r0)) % raw.cap)};
    sa.tq = RingRef{h->tq, h->Q, uint32_t(a % h->Q)};
    sa.scratch1 = h->s1;
    sa.scratch2 = h->s2;
    sa.tw_w = h->tw + tw_offset(h->W);
    sa.tw_h = h->tw + tw_offset(h->H);
    sa.asp_ht = h->asp_ht;
    // the row-major copy follows the transposed table and the two chirp vectors
    sa.asp_h = h->cur.spatial == HV_SPATIAL_ASP ? h->asp_ht + size_t(h->W) * h->H + h->W + h->H : nullptr;
    sa.chirp_x = h->chirp;
    sa.chirp_y = h->chirp + h->W;
    sa.use_cluster = h->sp_cluster;
    sa.use_pp = h->sp_pp;
    sa.use_fused = h->sp_fused;
    sa.ring = kFusedRing;
    sa.fused_ctr = h->fused_ctr;
    if (h->inject == HV_INJECT_FUSED_STALL && sa.use_fused && spatial_fused_supported(sa)) {
      sa.stall = 1;
      h->inject = HV_INJECT_NONE;
    }
    int launches = 0;
    cudaError_t e = launch_spatial(sa, h->stream, &launches);
    h->st.kernel_launches += launches;
    if (e != cudaSuccess) return cuda_fail(h, e, "spatial transform launch");
    h->st.frames_propagated += n;
  }
  return HV_OK;
}

// Spatial transform of frames f0 .. f1 - 1: runs of frames read in place from the
// caller's memory (HV_MEM_DEVICE_ASYNC) and runs in the input ring, one after the
// other. ring_only: the input ring whatever its contents (the autotuner's timing).
hv_status propagate(hv_handle* h, uint64_t f0, uint64_t f1, bool ring_only = false) {
  uint64_t a = f0;
  while (a < f1) {
    uint64_t end = f1;
    RingRef raw{h->raw, h->cap, uint32_t(a % h->cap)};
    if (!ring_only) {
      for (const auto& b : h->borrowed) {
        if (b.first + b.n <= a) continue;
        if (b.first <= a) {  // a lies in this caller buffer
          end = std::min<uint64_t>(f1, b.first + b.n);
          raw = RingRef{const_cast<void*>(b.ptr), b.n, uint32_t(a - b.first)};
        } else {  // the ring up to the next caller buffer
          end = std::min<uint64_t>(f1, b.first);
        }
        break;
      }
    }
    hv_status s = propagate_run(h, a, end, raw);
    if (s != HV_OK) return s;
    a = end;
  }
  return HV_OK;
}

// Autotuner of the tuned form: times the spatial-kernel candidates (multi-pass
// with several frames per launch, and the whole-frame cluster kernel) on the
// handle's own buffers and keeps the fastest. Runs when tuned settings are
// applied; the time queue is being flushed then, so its contents may be used.
hv_status tune_spatial(hv_handle* h) {
  hv_tuning t{};
  if (h->cur.spatial == HV_SPATIAL_NONE) {
    h->tuning = t;
    return HV_OK;
  }
  const size_t fbytes = size_t(h->W) * h->H * sizeof(float2);
  // frames per timed run: a render's worth where the rings allow (the fused
  // transform's pipeline fill and drain weigh on short runs)
  const uint32_t n = std::min<uint32_t>(2048, std::min(h->Q, h->cap));
  cudaEvent_t e0, e1;
  HV_CU(h, cudaEventCreate(&e0));
  HV_CU(h, cudaEventCreate(&e1));
  struct Cand { int kind; uint32_t chunk; };  // kind: 1 multi-pass, 3 persistent, 2 cluster, 4 fused
  static const Cand cands[] = {{1, 16}, {1, 32}, {1, 64}, {1, 128}, {1, 256},
                               {3, 64}, {3, 128}, {3, 256}, {3, 512}, {2, 0}, {4, 0}};
  SpatialArgs probe{};
  probe.spatial = h->cur.spatial;
  probe.W = h->W;
  probe.H = h->H;
  const bool pp_ok = spatial_pp_supported(probe);
  const bool fused_ok = h->W == 256 && h->H == 256;  // ASP or Fresnel (checked above)
  float best = 1e30f;
  int best_kind = 1;
  uint32_t best_chunk = h->chunk;
  for (int ci = 0; ci < 11; ++ci) {
    const Cand c = cands[ci];
    if (c.kind == 2 && !cluster_ok(h)) continue;
    if (c.kind == 3 && !pp_ok) continue;
    if (c.kind == 4 && !fused_ok) continue;
    const uint32_t ch = (c.kind == 2 || c.kind == 4) ? n : std::min(c.chunk, n);
    if (c.kind == 4 && ensure(h, reinterpret_cast<void**>(&h->fused_ctr), &h->fused_ctr_bytes,
                              (1 + kFusedPasses * size_t(kFusedRing)) * sizeof(unsigned)) != HV_OK)
      continue;
    if (c.kind != 2) {
      const size_t need = size_t(c.kind == 4 ? kFusedRing : ch) * fbytes;
      if (ensure(h, reinterpret_cast<void**>(&h->s1), &h->s1_bytes, need) != HV_OK) continue;
      if (h->cur.spatial == HV_SPATIAL_ASP &&
          ensure(h, reinterpret_cast<void**>(&h->s2), &h->s2_bytes, need) != HV_OK)
        continue;
    }
    h->sp_cluster = c.kind == 2;
    h->sp_pp = c.kind == 3;
    h->sp_fused = c.kind == 4;
    h->chunk = (c.kind == 2 || c.kind == 4) ? h->chunk : ch;
    const uint64_t before = h->st.frames_propagated;
    hv_status st = propagate(h, 0, n, true);  // warm-up
    if (st != HV_OK) return st;
    HV_CU(h, cudaEventRecord(e0, h->stream));
    for (int rep = 0; rep < 2; ++rep) {
      st = propagate(h, 0, n, true);
      if (st != HV_OK) return st;
    }
    HV_CU(h, cudaEventRecord(e1, h->stream));
    HV_CU(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    HV_CU(h, cudaEventElapsedTime(&ms, e0, e1));
    h->st.frames_propagated = before;  // tuning work is not rendering work
    const float us_per_frame = 1000.f * ms / (2.f * n);
    t.candidate_us_per_frame[ci] = us_per_frame;
    if (us_per_frame < best) {
      best = us_per_frame;
      best_kind = c.kind;
      best_chunk = (c.kind == 2 || c.kind == 4) ? best_chunk : ch;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->sp_cluster = best_kind == 2;
  h->sp_pp = best_kind == 3;
  h->sp_fused = best_kind == 4;
  h->chunk = best_chunk;
  // the chosen kernels' scratch: chunk frames (multi-pass), the rings (fused)
  if (best_kind != 2) {
    const size_t need = size_t(best_kind == 4 ? std::max(best_chunk, kFusedRing) : best_chunk) * fbytes;
    if (ensure(h, reinterpret_cast<void**>(&h->s1), &h->s1_bytes, need) != HV_OK ||
        (h->cur.spatial == HV_SPATIAL_ASP && ensure(h, reinterpret_cast<void**>(&h->s2), &h->s2_bytes, need) != HV_OK))
      return HV_ERR_NOMEM;
  }
  t.spatial_kernel = best_kind == 2 ? HV_SK_CLUSTER
                     : (best_kind == 3 ? HV_SK_PERSISTENT : (best_kind == 4 ? HV_SK_FUSED : HV_SK_MULTIPASS));
  t.spatial_chunk = best_chunk;
  t.tuned = 1;
  h->tuning = t;
  return HV_OK;
}

// Autotuner of the STFT for windows that do not overlap (S >= T): times the
// walking kernel (CTAs walk every window of their pixels), the kernels with one
// CTA per (window, pixel tile) (plain, wide, persistent double-buffered) and, at
// T = 512, the TMA-fed ones (one CTA per item, persistent double-buffered) on the
// handle's time queue (its contents are being flushed, so any values do) and
// keeps the fastest.
hv_status tune_temporal(hv_handle* h) {
  const uint32_t T = h->T, S = h->S;
  const uint32_t nwin = std::min<uint32_t>(16, (h->Q - T) / S + 1);
  const size_t hw = size_t(h->W) * h->H;
  float* out = nullptr;
  HV_CU(h, cudaMalloc(&out, size_t(nwin) * h->nout * hw * sizeof(float)));
  cudaEvent_t e0, e1;
  HV_CU(h, cudaEventCreate(&e0));
  HV_CU(h, cudaEventCreate(&e1));
  StftArgs sa{};
  sa.W = h->W;
  sa.H = h->H;
  sa.T = T;
  sa.S = S;
  sa.nwin = nwin;
  sa.tq = RingRef{h->tq, h->Q, 0};
  sa.tw_t = h->tw + tw_offset(T);
  sa.klo = h->klo;
  sa.khi = h->khi;
  sa.fscale = float(h->cur.fs_hz / double(T) / 1000.0);
  sa.mask = h->cur.moments_mask;
  sa.nout = h->nout;
  sa.out = out;
  sa.err = h->dev_err;
  const int kinds[6] = {STFT_WALK, STFT_AUTO, STFT_WIDE, STFT_PIPE, STFT_TMA, STFT_TMA_PIPE};
  float best = 1e30f;
  int best_kind = STFT_AUTO;
  hv_status st = HV_OK;
  for (int ci = 0; ci < 6 && st == HV_OK; ++ci) {
    // the TMA-fed kernels exist for T = 512 only (elsewhere they would time the
    // window-per-CTA kernel again)
    if ((kinds[ci] == STFT_TMA || kinds[ci] == STFT_TMA_PIPE) && T != 512) continue;
    sa.kernel = kinds[ci];
    int launches = 0;
    cudaError_t e = launch_stft(sa, h->stream, &launches);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) e = launch_stft(sa, h->stream, &launches);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      st = cuda_fail(h, e, "STFT autotuning");
      break;
    }
    const float us = 1000.f * ms / (3.f * nwin);
    h->tuning.stft_us_per_window[ci] = us;
    if (us < best) {
      best = us;
      best_kind = kinds[ci];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (st != HV_OK) return st;
  h->stft_kernel = best_kind;
  h->tuning.stft_kernel = best_kind == STFT_WALK       ? HV_STFT_WALK
                          : best_kind == STFT_WIDE     ? HV_STFT_WINDOW_WIDE
                          : best_kind == STFT_PIPE     ? HV_STFT_WINDOW_PIPELINED
                          : best_kind == STFT_TMA      ? HV_STFT_WINDOW_TMA
                          : best_kind == STFT_TMA_PIPE ? HV_STFT_WINDOW_TMA_PIPELINED
                                                       : HV_STFT_WINDOW;
  h->tuning.tuned = 1;
  return HV_OK;
}

// Applies pending post-processing settings, and (re)sizes the image ring when
// they or the compute settings changed; the accumulation history restarts then.
hv_status post_apply(hv_handle* h) {
  if (h->post_pending) {
    h->post_cur = h->post_pend;
    h->post_k_cur = h->post_k_pend;
    h->post_pending = false;
    h->post_dirty = true;
  }
  if (!h->post_dirty) return HV_OK;
  const hv_post& q = h->post_cur;
  h->post_active = q.struct_size != 0 && (q.kernel_size > 0 || q.renormalize || q.accumulate > 1);
  h->post_count = 0;
  if (h->post_active) {
    if (h->cur.temporal == HV_TEMPORAL_NONE)
      return fail(h, HV_ERR_UNSUPPORTED, "post-processing needs rendered images (STFT or PCA)");
    const uint32_t by_q = (h->Q - h->T) / h->S + 1;  // most windows one render emits
    h->post_R = q.accumulate - 1 + by_q;
    const size_t hw = size_t(h->W) * h->H;
    hv_status s = ensure(h, reinterpret_cast<void**>(&h->post_ring), &h->post_ring_bytes,
                         size_t(h->post_R) * h->nout * hw * sizeof(float));
    if (s == HV_OK)
      s = ensure(h, reinterpret_cast<void**>(&h->post_sums), &h->post_sums_bytes,
                 size_t(h->post_R) * h->nout * kPostSub * sizeof(double));
    if (s == HV_OK && q.kernel_size > 0) {
      s = ensure(h, reinterpret_cast<void**>(&h->post_kdev), &h->post_kdev_bytes,
                 h->post_k_cur.size() * sizeof(float));
      if (s == HV_OK) {
        HV_CU(h, cudaMemcpyAsync(h->post_kdev, h->post_k_cur.data(), h->post_k_cur.size() * sizeof(float),
                                 cudaMemcpyHostToDevice, h->stream));
        HV_CU(h, cudaStreamSynchronize(h->stream));
      }
    }
    if (s != HV_OK) return s;
  }
  h->post_dirty = false;
  return HV_OK;
}

// Settings and post-processing settings in force for the next windows.
hv_status settle(hv_handle* h) {
  hv_status s = apply_pending(h);
  return s == HV_OK ? post_apply(h) : s;
}

// Records that every raw frame below h->propagated has been read once the
// handle's stream reaches this point (pushes that overwrite those slots wait
// for it, and only for it).
hv_status note_consumed(hv_handle* h) {
  const int k = (h->cons_head + h->cons_n) % hv_handle::NCONS;
  if (h->cons_n == hv_handle::NCONS) h->cons_head = (h->cons_head + 1) % hv_handle::NCONS;
  else ++h->cons_n;
  HV_CU(h, cudaEventRecord(h->cons_ev[k], h->stream));
  h->cons_hi[k] = h->propagated;
  return HV_OK;
}

// The copy stream waits until the raw frames that a push of n frames overwrites
// have been consumed: the oldest recorded spatial stage that covered them.
hv_status wait_slots_free(hv_handle* h, uint32_t n) {
  if (h->pushed + n <= h->cap) return HV_OK;  // nothing overwritten yet
  const uint64_t need = h->pushed + n - h->cap;  // frames below this are overwritten
  for (int i = 0; i < h->cons_n; ++i) {
    const int k = (h->cons_head + i) % hv_handle::NCONS;
    if (h->cons_hi[k] >= need) {
      HV_CU(h, cudaStreamWaitEvent(h->copy_stream, h->cons_ev[k], 0));
      return HV_OK;
    }
  }
  HV_CU(h, cudaStreamWaitEvent(h->copy_stream, h->ev_consumed, 0));  // everything rendered so far
  return HV_OK;
}

// Copies n frames from device memory into the input ring on the handle's stream
// (one copy, or two where the ring wraps). The caller has checked the capacity.
hv_status enqueue_push_device(hv_handle* h, const void* frames, uint32_t n) {
  const hv_params& p = h->pending ? h->pend : h->cur;
  const size_t fb = size_t(p.width) * p.height * (h->bits / 8);
  const uint32_t slot = uint32_t(h->pushed % h->cap);
  const uint32_t n1 = std::min(n, h->cap - slot);
  const char* src = static_cast<const char*>(frames);
  char* ring = static_cast<char*>(h->raw);
  HV_CU(h, cudaMemcpyAsync(ring + slot * fb, src, n1 * fb, cudaMemcpyDeviceToDevice, h->stream));
  if (n1 < n) HV_CU(h, cudaMemcpyAsync(ring, src + n1 * fb, (n - n1) * fb, cudaMemcpyDeviceToDevice, h->stream));
  h->pushed += n;
  h->st.frames_pushed += n;
  return HV_OK;
}

// Number of complete windows that one render can emit into cap_floats floats.
uint32_t windows_ready(const hv_handle* h, size_t cap_floats) {
  const uint32_t T = h->T, S = h->S;
  uint64_t avail = 0;
  if (h->pushed >= h->next_win + T) avail = (h->pushed - h->next_win - T) / S + 1;
  const uint64_t by_q = (h->Q - T) / S + 1;
  const uint64_t by_out = cap_floats / h->win_floats;
  return uint32_t(std::min({avail, by_q, by_out}));
}

// Enqueues the spatial transform of the frames these nw windows still need and
// the temporal analysis of the windows into dst (device memory), all on the
// handle's stream. Makes no synchronising call unless profiling is on, so it
// may run inside a stream capture (capturing = true; profiling must be off).
hv_status enqueue_windows(hv_handle* h, float* dst, uint32_t nw, bool capturing) {
  const bool none = h->cur.temporal == HV_TEMPORAL_NONE;
  const uint32_t T = h->T, S = h->S;
  hv_status s = HV_OK;
  const uint64_t prop_before = h->st.frames_propagated;
  // long PCA windows, several in this render: window by window, each window's
  // spatial chunk and covariance on the handle's stream while the previous window's
  // eigensolver runs on eig_stream (below)
  const bool pca_pipe = h->cur.temporal == HV_TEMPORAL_PCA && !h->pca_batched && !capturing && nw >= 2 &&
                        h->pca_C[1] != nullptr;
  s = prof_mark(h, 0);
  if (s != HV_OK) return s;
  // spatial transform of every frame of these windows not yet in the queue: one
  // contiguous range when windows overlap or touch (S <= T), else per window
  if (pca_pipe) {
  } else if (S <= T) {
    const uint64_t lo = std::max(h->next_win, h->propagated);
    const uint64_t hi = h->next_win + uint64_t(nw - 1) * S + T;
    if (lo < hi) {
      s = propagate(h, lo, hi);
      if (s != HV_OK) return s;
      h->propagated = hi;
    }
  } else {
    for (uint32_t w = 0; w < nw; ++w) {
      const uint64_t a = h->next_win + uint64_t(w) * S;
      const uint64_t lo = std::max(a, h->propagated);
      if (lo < a + T) {
        s = propagate(h, lo, a + T);
        if (s != HV_OK) return s;
        h->propagated = a + T;
      }
    }
  }
  s = prof_mark(h, 1);
  if (s != HV_OK) return s;
  if (!capturing && !pca_pipe) {
    s = note_consumed(h);
    if (s != HV_OK) return s;
  }
  int launches = 0;
  cudaError_t e;
  const RingRef tq{h->tq, h->Q, uint32_t(h->next_win % h->Q)};
  PostArgs pa{};
  if (h->post_active) {
    pa.W = h->W;
    pa.H = h->H;
    pa.nout = h->nout;
    pa.K = int(h->post_cur.kernel_size);
    pa.kern = h->post_kdev;
    pa.renorm = h->post_cur.renormalize ? 1 : 0;
    pa.A = h->post_cur.accumulate;
    pa.R = h->post_R;
    pa.count = h->post_count;
    pa.ring = h->post_ring;
    pa.sums = h->post_sums;
    // without a convolution the STFT epilogue writes the image ring and its sums
    pa.fused = !none && h->cur.temporal != HV_TEMPORAL_PCA && pa.K == 0 ? 1 : 0;
  }
  if (none) {
    e = launch_copy_frames(tq, nw, h->W * h->H, dst, h->stream, &launches);
  } else if (pca_pipe) {
    // pipelined long windows: spatial chunk(w), covariance(w) and projection(w - 1)
    // on the handle's stream around eigensolver(w - 1, then w) on eig_stream; every
    // frame of the render's windows fits in the time queue at once
    e = cudaSuccess;
    auto window_args = [&](uint32_t w) {
      PcaArgs a = h->pca;
      const int k = int(w & 1);
      a.nwin = 1;
      a.wstride = S;
      a.tq = RingRef{h->tq, h->Q, uint32_t((h->next_win + uint64_t(w) * S) % h->Q)};
      a.C = h->pca_C[k];
      a.counters = h->pca_cnt[k];
      a.cmax = reinterpret_cast<double*>(a.counters + 4);
      a.lam = h->pca_lam[k];
      a.Vs = h->pca_Vs[k];
      return a;
    };
    // stage profiling: each window's eight events (start and end of its spatial
    // chunk, covariance, eigensolver and projection) on the stream that runs the
    // stage; room for all windows of the render first (the flush synchronises,
    // before anything is queued)
    cudaEvent_t* evw[2] = {nullptr, nullptr};
    if (h->prof && h->pca_ev_used + 8 * size_t(nw) > h->pca_ev.size()) {
      s = prof_flush(h);
      if (s != HV_OK) return s;
      while (h->pca_ev.size() < 8 * size_t(nw)) {
        cudaEvent_t x = nullptr;
        HV_CU(h, cudaEventCreate(&x));
        h->pca_ev.push_back(x);
      }
    }
    for (uint32_t w = 0; w <= nw && e == cudaSuccess; ++w) {
      if (w < nw) {
        PcaArgs a = window_args(w);
        cudaEvent_t* ev = nullptr;
        if (h->prof) {
          ev = evw[w & 1] = &h->pca_ev[h->pca_ev_used];
          h->pca_ev_used += 8;
        }
        // the window's frames not yet in the time queue
        const uint64_t a0 = h->next_win + uint64_t(w) * S, lo = std::max(a0, h->propagated);
        if (ev) HV_CU(h, cudaEventRecord(ev[0], h->stream));
        if (lo < a0 + T) {
          s = propagate(h, lo, a0 + T);
          if (s != HV_OK) return s;
          h->propagated = a0 + T;
          s = note_consumed(h);
          if (s != HV_OK) return s;
        }
        if (ev) HV_CU(h, cudaEventRecord(ev[1], h->stream));
        ev = ev ? ev + 2 : nullptr;
        if (ev) e = cudaEventRecord(ev[0], h->stream);
        if (e == cudaSuccess) e = launch_pca_cov(a, h->stream, &launches);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_cov[w & 1], h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->eig_stream, h->ev_cov[w & 1], 0);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], h->eig_stream);
        if (e == cudaSuccess) e = launch_pca_eig(a, h->eig_stream, &launches);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3], h->eig_stream);
        if (e == cudaSuccess && h->prof) e = launch_pca_sweeps_add(a.counters, h->pca_sweeps_dev, h->eig_stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_eig[w & 1], h->eig_stream);
      }
      if (w >= 1 && e == cudaSuccess) {
        PcaArgs a = window_args(w - 1);
        cudaEvent_t* ev = evw[(w - 1) & 1] ? evw[(w - 1) & 1] + 2 : nullptr;
        e = cudaStreamWaitEvent(h->stream, h->ev_eig[(w - 1) & 1], 0);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[4], h->stream);
        if (e == cudaSuccess) e = launch_pca_proj(a, dst + size_t(w - 1) * h->win_floats, h->stream, &launches);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[5], h->stream);
      }
    }
    h->pca_last_nwin = 1;
    h->pca_lam_last = h->pca_lam[(nw - 1) & 1];
    h->pca_has_lam = true;
  } else if (h->cur.temporal == HV_TEMPORAL_PCA) {
    e = cudaSuccess;
    for (uint32_t w = 0; w < nw && e == cudaSuccess;) {
      const uint32_t k = h->pca_batched ? std::min<uint32_t>(nw - w, 128) : 1;
      h->pca.nwin = k;
      h->pca.wstride = S;
      h->pca.tq = RingRef{h->tq, h->Q, uint32_t((h->next_win + uint64_t(w) * S) % h->Q)};
      h->pca_last_nwin = k;
      cudaEvent_t* ev = nullptr;
      if (h->prof) {
        if (h->pca_ev_used + 8 > h->pca_ev.size()) {
          s = prof_flush(h);
          if (s != HV_OK) return s;
        }
        ev = &h->pca_ev[h->pca_ev_used];
        h->pca_ev_used += 8;
        HV_CU(h, cudaEventRecord(ev[0], h->stream));  // no spatial chunk of its own
        HV_CU(h, cudaEventRecord(ev[1], h->stream));
        ev += 2;
      }
      e = launch_pca(h->pca, dst + size_t(w) * h->win_floats, h->stream, &launches, ev);
      h->pca_lam_last = h->pca.lam + size_t(k - 1) * h->T;
      w += k;
      if (h->prof && e == cudaSuccess) e = launch_pca_sweeps_add(h->pca.counters, h->pca_sweeps_dev, h->stream);
    }
    h->pca_has_lam = true;
  } else {
    StftArgs sa{};
    sa.W = h->W;
    sa.H = h->H;
    sa.T = T;
    sa.S = S;
    sa.nwin = nw;
    sa.tq = tq;
    sa.tw_t = h->tw + tw_offset(T);
    sa.klo = h->klo;
    sa.khi = h->khi;
    sa.fscale = float(h->cur.fs_hz / double(T) / 1000.0);
    sa.mask = h->cur.moments_mask;
    sa.nout = h->nout;
    sa.out = dst;
    sa.err = h->dev_err;
    sa.kernel = h->stft_kernel;
    e = cudaSuccess;
    if (pa.fused) {
      sa.post_ring = pa.ring;
      sa.post_R = pa.R;
      sa.post_count = pa.count;
      sa.post_sums = pa.renorm ? pa.sums : nullptr;
      e = launch_post_zero(pa, nw, h->stream);
    }
    if (e == cudaSuccess && (h->cur.tuned || h->cur.stft_kernel != 0)) {
      e = launch_stft(sa, h->stream, &launches);
    } else if (e == cudaSuccess) {
      // plain form: the walking kernel, one launch per window
      sa.nwin = 1;
      for (uint32_t w = 0; w < nw && e == cudaSuccess; ++w) {
        sa.tq = RingRef{h->tq, h->Q, uint32_t((h->next_win + uint64_t(w) * S) % h->Q)};
        sa.out = dst + size_t(w) * h->win_floats;
        sa.post_count = pa.count + w;
        e = launch_stft(sa, h->stream, &launches);
      }
    }
  }
  if (e == cudaSuccess && h->post_active) {
    e = launch_post(dst, nw, pa, h->stream, &launches);
    h->post_count += nw;
  }
  h->st.kernel_launches += launches;
  if (e != cudaSuccess) return cuda_fail(h, e, "temporal transform launch");
  s = prof_mark(h, 2);
  if (s != HV_OK) return s;
  if (h->prof) {
    h->prof_acc.renders += 1;
    h->prof_acc.frames += h->st.frames_propagated - prop_before;
    h->prof_acc.windows += nw;
  }
  // an event recorded inside a stream capture cannot be waited on from outside the
  // graph: the group step records it after launching the graph instead
  if (!capturing) HV_CU(h, cudaEventRecord(h->ev_consumed, h->stream));
  h->next_win += uint64_t(nw) * S;
  // caller buffers whose frames no window will read again
  while (!h->borrowed.empty() && h->borrowed.front().first + h->borrowed.front().n <= h->next_win)
    h->borrowed.pop_front();
  h->st.windows_rendered += nw;
  return HV_OK;
}

}  // namespace

extern "C" {

hv_status hv_open(const hv_open_desc* desc, hv_handle** out) {
  if (!out) return fail(nullptr, HV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!desc || desc->struct_size != sizeof(hv_open_desc)) return fail(nullptr, HV_ERR_ARG, "bad hv_open_desc");
  if (desc->pixel_bits != 8 && desc->pixel_bits != 16) return fail(nullptr, HV_ERR_ARG, "pixel_bits must be 8 or 16");
  if (desc->max_width < 16 || desc->max_height < 16 || desc->max_width > 1024 || desc->max_height > 1024)
    return fail(nullptr, HV_ERR_ARG, "max frame size must be within [16, 1024]");
  if (desc->queue_capacity_frames < 1) return fail(nullptr, HV_ERR_ARG, "queue capacity must be >= 1");
  hv_handle* h = new hv_handle();
  h->device = desc->device;
  h->max_w = desc->max_width;
  h->max_h = desc->max_height;
  h->bits = desc->pixel_bits;
  h->cap = desc->queue_capacity_frames;
  h->tq_req = desc->time_queue_frames;
  auto bail = [&](hv_status s, const std::string& m) {
    g_open_err = m;
    hv_close(h);
    return s;
  };
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return bail(HV_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  if (desc->stream) {
    h->stream = static_cast<cudaStream_t>(desc->stream);
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(HV_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    h->own_stream = true;
  }
  e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->eig_stream, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&h->ev_cov[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_eig[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_pushed, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_consumed, cudaEventDisableTiming);
  for (int i = 0; i < hv_handle::NCONS && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&h->cons_ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(HV_ERR_CUDA, std::string("stream/event: ") + cudaGetErrorString(e));
  const size_t raw_bytes = size_t(h->cap) * h->max_w * h->max_h * (h->bits / 8);
  e = cudaMalloc(&h->raw, raw_bytes);
  if (e != cudaSuccess) return bail(HV_ERR_NOMEM, std::string("input ring: ") + cudaGetErrorString(e));
  // twiddle tables exp(-2 pi i e / L), L = 8..1024, computed in float64
  std::vector<float2> tw(tw_offset(1u << (kMaxLog + 1)));
  for (uint32_t L = 1u << kMinLog; L <= (1u << kMaxLog); L <<= 1)
    for (uint32_t i = 0; i < L; ++i) tw[tw_offset(L) + i] = cis(-2.0 * M_PI * double(i) / double(L));
  e = cudaMalloc(&h->tw, tw.size() * sizeof(float2));
  if (e == cudaSuccess) e = cudaMemcpy(h->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(HV_ERR_NOMEM, std::string("twiddles: ") + cudaGetErrorString(e));
  e = cudaMalloc(&h->dev_err, 16);
  if (e == cudaSuccess) e = cudaMemset(h->dev_err, 0, 16);
  if (e == cudaSuccess) e = cudaMalloc(&h->pca_sweeps_dev, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(h->pca_sweeps_dev, 0, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) return bail(HV_ERR_NOMEM, std::string("error flags: ") + cudaGetErrorString(e));
  *out = h;
  return HV_OK;
}

hv_status hv_set_params(hv_handle* h, const hv_params* p) {
  if (!h || !p) return fail(h, HV_ERR_ARG, "NULL argument");
  Derived d{};
  std::string why;
  hv_status s = validate(h, *p, d, why);
  if (s != HV_OK) return fail(h, s, why);
  const hv_params& ref = h->pending ? h->pend : h->cur;
  const bool have = h->pending || h->has_params;
  if (have && (ref.width != p->width || ref.height != p->height)) {
    // a new frame size cannot reuse queued frames of the old size
    const uint64_t queued = h->pushed - h->next_win;
    h->st.frames_dropped += queued;
    h->next_win = h->pushed;
    h->propagated = h->pushed;
    h->borrowed.clear();
  }
  h->pend = *p;
  h->pending = true;
  return HV_OK;
}

hv_status hv_get_params(const hv_handle* h, hv_params* p) {
  if (!h || !p) return HV_ERR_ARG;
  if (!h->has_params && !h->pending) return HV_ERR_STATE;
  *p = h->pending ? h->pend : h->cur;
  return HV_OK;
}

hv_status hv_push_frames(hv_handle* h, const void* frames, uint32_t n, int mem_kind) {
  if (!h) return HV_ERR_ARG;
  if (n == 0) return HV_OK;
  if (!frames) return fail(h, HV_ERR_ARG, "frames is NULL");
  if (mem_kind != HV_MEM_HOST && mem_kind != HV_MEM_DEVICE && mem_kind != HV_MEM_HOST_ASYNC &&
      mem_kind != HV_MEM_DEVICE_ASYNC)
    return fail(h, HV_ERR_ARG, "bad mem_kind");
  if (!h->has_params && !h->pending) return fail(h, HV_ERR_STATE, "hv_set_params must come first");
  const hv_params& p = h->pending ? h->pend : h->cur;
  if (h->pushed + n - h->next_win > h->cap) {
    h->st.frames_rejected += n;
    return fail(h, HV_ERR_QUEUE_FULL, "input queue full");
  }
  HV_CU(h, cudaSetDevice(h->device));
  if (mem_kind == HV_MEM_DEVICE) return enqueue_push_device(h, frames, n);
  if (mem_kind == HV_MEM_DEVICE_ASYNC && (reinterpret_cast<uintptr_t>(frames) & 15) == 0) {
    // read in place by the spatial stage (16-byte aligned, as its bulk copies need)
    h->borrowed.push_back(hv_handle::Borrowed{h->pushed, n, frames});
    h->pushed += n;
    h->st.frames_pushed += n;
    return HV_OK;
  }
  const size_t fb = size_t(p.width) * p.height * (h->bits / 8);
  const uint32_t slot = uint32_t(h->pushed % h->cap);
  const uint32_t n1 = std::min(n, h->cap - slot);
  const char* src = static_cast<const char*>(frames);
  char* ring = static_cast<char*>(h->raw);
  {
    // copy stream: wait until the slots being overwritten have been consumed
    hv_status sw = wait_slots_free(h, n);
    if (sw != HV_OK) return sw;
    const cudaMemcpyKind dir = mem_kind == HV_MEM_DEVICE_ASYNC ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    HV_CU(h, cudaMemcpyAsync(ring + slot * fb, src, n1 * fb, dir, h->copy_stream));
    if (n1 < n) HV_CU(h, cudaMemcpyAsync(ring, src + n1 * fb, (n - n1) * fb, dir, h->copy_stream));
    HV_CU(h, cudaEventRecord(h->ev_pushed, h->copy_stream));
    if (mem_kind == HV_MEM_HOST) HV_CU(h, cudaEventSynchronize(h->ev_pushed));  // host buffer consumed on return
    HV_CU(h, cudaStreamWaitEvent(h->stream, h->ev_pushed, 0));
  }
  h->pushed += n;
  h->st.frames_pushed += n;
  return HV_OK;
}

hv_status hv_window_floats(const hv_handle* h, size_t* f) {
  if (!h || !f) return HV_ERR_ARG;
  if (h->pending) {
    Derived d{};
    std::string why;
    hv_status s = validate(h, h->pend, d, why);
    if (s != HV_OK) return s;
    *f = d.win_floats;
    return HV_OK;
  }
  if (!h->has_params) return HV_ERR_STATE;
  *f = h->win_floats;
  return HV_OK;
}

hv_status hv_render(hv_handle* h, float* out, size_t cap_floats, int out_kind, uint32_t* n_windows) {
  if (!h || !n_windows) return fail(h, HV_ERR_ARG, "NULL argument");
  *n_windows = 0;
  if (out_kind != HV_MEM_HOST && out_kind != HV_MEM_DEVICE && out_kind != HV_MEM_HOST_ASYNC)
    return fail(h, HV_ERR_ARG, "bad mem_kind");
  const bool host_out = out_kind != HV_MEM_DEVICE;
  if (!h->has_params && !h->pending) return fail(h, HV_ERR_STATE, "no settings");
  HV_CU(h, cudaSetDevice(h->device));
  hv_status s = settle(h);
  if (s != HV_OK) return s;
  const uint32_t nw = out ? windows_ready(h, cap_floats) : 0;
  if (nw == 0) return HV_OK;
  float* dst = out;
  if (host_out) {
    s = ensure(h, reinterpret_cast<void**>(&h->staging), &h->staging_bytes, size_t(nw) * h->win_floats * sizeof(float));
    if (s != HV_OK) return s;
    dst = h->staging;
  }
  s = enqueue_windows(h, dst, nw, false);
  if (s != HV_OK) return s;
  if (host_out) {
    HV_CU(h, cudaMemcpyAsync(out, dst, size_t(nw) * h->win_floats * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (out_kind == HV_MEM_HOST) HV_CU(h, cudaStreamSynchronize(h->stream));
  }
  *n_windows = nw;
  return HV_OK;
}

hv_status hv_pca_eigenvalues(const hv_handle* h, double* out, uint32_t n) {
  if (!h || !out) return HV_ERR_ARG;
  if (!h->pca_has_lam || h->cur.temporal != HV_TEMPORAL_PCA) return HV_ERR_STATE;
  if (n > h->T) return HV_ERR_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return HV_ERR_CUDA;
  const double* lam = h->pca_lam_last;
  if (!lam) return HV_ERR_STATE;
  if (cudaMemcpyAsync(out, lam, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return HV_ERR_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HV_ERR_CUDA;
  return HV_OK;
}

hv_status hv_get_tuning(const hv_handle* h, hv_tuning* t) {
  if (!h || !t) return HV_ERR_ARG;
  if (!h->has_params) return HV_ERR_STATE;
  *t = h->tuning;
  return HV_OK;
}

hv_status hv_get_stats(const hv_handle* h, hv_stats* s) {
  if (!h || !s) return HV_ERR_ARG;
  *s = h->st;
  return HV_OK;
}

hv_status hv_profile_enable(hv_handle* h, int on) {
  if (!h) return HV_ERR_ARG;
  HV_CU(h, cudaSetDevice(h->device));
  if (on && h->prof_ev.empty()) {
    h->prof_ev.resize(3 * 256, nullptr);
    for (auto& e : h->prof_ev) HV_CU(h, cudaEventCreate(&e));
    h->pca_ev.resize(8 * 64, nullptr);
    for (auto& e : h->pca_ev) HV_CU(h, cudaEventCreate(&e));
  }
  if (on) {
    HV_CU(h, cudaStreamSynchronize(h->stream));
    h->prof_used = 0;
    h->pca_ev_used = 0;
    h->prof_acc = hv_profile{};
    HV_CU(h, cudaMemset(h->pca_sweeps_dev, 0, 2 * sizeof(unsigned long long)));
  }
  h->prof = on != 0;
  return HV_OK;
}

hv_status hv_profile_read(hv_handle* h, hv_profile* out) {
  if (!h || !out) return HV_ERR_ARG;
  HV_CU(h, cudaSetDevice(h->device));
  hv_status s = prof_flush(h);
  if (s != HV_OK) return s;
  unsigned long long sw[2] = {0, 0};  // accumulated on the device by every profiled window
  HV_CU(h, cudaMemcpy(sw, h->pca_sweeps_dev, sizeof(sw), cudaMemcpyDeviceToHost));
  h->prof_acc.pca_sweeps_f32 = sw[0];
  h->prof_acc.pca_sweeps = sw[1];
  *out = h->prof_acc;
  return HV_OK;
}

hv_status hv_synchronize(hv_handle* h) {
  if (!h) return HV_ERR_ARG;
  HV_CU(h, cudaSetDevice(h->device));
  HV_CU(h, cudaStreamSynchronize(h->copy_stream));
  HV_CU(h, cudaStreamSynchronize(h->stream));
  unsigned flags = 0;
  HV_CU(h, cudaMemcpy(&flags, h->dev_err, sizeof(flags), cudaMemcpyDeviceToHost));
  if (flags != 0)
    return fail(h, HV_ERR_CUDA, "a kernel's bounded wait gave up (device flags " + std::to_string(flags) + ")");
  return HV_OK;
}

hv_status hv_debug_inject(hv_handle* h, int what) {
  if (!h) return HV_ERR_ARG;
  if (what != HV_INJECT_NONE && what != HV_INJECT_FUSED_STALL) return fail(h, HV_ERR_ARG, "bad injection");
  h->inject = what;
  return HV_OK;
}

hv_status hv_close(hv_handle* h) {
  if (!h) return HV_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->copy_stream) {
    cudaStreamSynchronize(h->copy_stream);
    cudaStreamDestroy(h->copy_stream);
  }
  if (h->eig_stream) {
    cudaStreamSynchronize(h->eig_stream);
    cudaStreamDestroy(h->eig_stream);
  }
  for (int i = 0; i < 2; ++i) {
    if (h->ev_cov[i]) cudaEventDestroy(h->ev_cov[i]);
    if (h->ev_eig[i]) cudaEventDestroy(h->ev_eig[i]);
  }
  if (h->ev_pushed) cudaEventDestroy(h->ev_pushed);
  if (h->ev_consumed) cudaEventDestroy(h->ev_consumed);
  for (auto& e : h->cons_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->prof_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->pca_ev)
    if (e) cudaEventDestroy(e);
  dfree(h->tq);
  dfree(h->s1);
  dfree(h->s2);
  dfree(h->tw);
  dfree(h->dev_err);
  dfree(h->pca_sweeps_dev);
  dfree(h->fused_ctr);
  dfree(h->asp_ht);
  dfree(h->staging);
  if (h->pca_ws) cudaFree(h->pca_ws);
  if (h->sw_tables) cudaFree(h->sw_tables);
  if (h->post_kdev) cudaFree(h->post_kdev);
  if (h->post_ring) cudaFree(h->post_ring);
  if (h->post_sums) cudaFree(h->post_sums);
  if (h->sw_acc) cudaFree(h->sw_acc);
  if (h->raw) cudaFree(h->raw);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return HV_OK;
}

hv_status hv_set_postprocess(hv_handle* h, const hv_post* p) {
  if (!h || !p) return fail(h, HV_ERR_ARG, "NULL argument");
  if (p->struct_size != sizeof(hv_post)) return fail(h, HV_ERR_ARG, "hv_post.struct_size mismatch");
  const uint32_t K = p->kernel_size;
  if (K > HV_POST_MAX_KERNEL || (K > 0 && K % 2 == 0)) return fail(h, HV_ERR_ARG, "kernel_size must be 0 or odd <= 31");
  if (p->accumulate < 1 || p->accumulate > HV_POST_MAX_ACCUMULATE)
    return fail(h, HV_ERR_ARG, "accumulate must be in [1, 64]");
  if (p->renormalize != 0 && p->renormalize != 1) return fail(h, HV_ERR_ARG, "renormalize must be 0 or 1");
  std::vector<float> k(size_t(K) * K);
  if (K > 0) {
    if (p->kernel) {
      std::memcpy(k.data(), p->kernel, k.size() * sizeof(float));
    } else {
      if (!(p->gauss_sigma > 0.f) || !std::isfinite(p->gauss_sigma))
        return fail(h, HV_ERR_ARG, "gauss_sigma must be > 0 without a kernel");
      // exp(-(dx^2 + dy^2) / (2 sigma^2)), normalised to sum 1, in float64
      std::vector<double> g(k.size());
      double tot = 0.0;
      const double s2 = 2.0 * double(p->gauss_sigma) * double(p->gauss_sigma);
      const int c = int(K / 2);
      for (int a = 0; a < int(K); ++a)
        for (int b = 0; b < int(K); ++b) {
          g[a * K + b] = std::exp(-double((a - c) * (a - c) + (b - c) * (b - c)) / s2);
          tot += g[a * K + b];
        }
      for (size_t e = 0; e < k.size(); ++e) k[e] = float(g[e] / tot);
    }
  }
  h->post_pend = *p;
  h->post_pend.kernel = nullptr;  // the weights live in post_k_pend
  h->post_k_pend = std::move(k);
  h->post_pending = true;
  return HV_OK;
}

// ------------------------------------------------------------- autofocus

// Frames [n][H][W] in device memory as a ring for the pass kernels.
static SpatialArgs af_args(const hv_handle* h, const void* frames, uint32_t n) {
  SpatialArgs sa{};
  sa.err = h->dev_err;
  sa.spatial = HV_SPATIAL_ASP;  // no chirp in the column pass
  sa.in_kind = h->bits == 8 ? IN_U8 : IN_U16;
  sa.W = h->W;
  sa.H = h->H;
  sa.raw = RingRef{const_cast<void*>(frames), n, 0};
  sa.scratch1 = h->s1;
  sa.scratch2 = h->s2;
  sa.tw_w = h->tw + tw_offset(h->W);
  sa.tw_h = h->tw + tw_offset(h->H);
  return sa;
}

static hv_status af_prepare(hv_handle* h, const void* frames, uint32_t n, uint32_t chunk) {
  if (!frames || n == 0) return fail(h, HV_ERR_ARG, "frames is NULL or n = 0");
  if (!h->has_params && !h->pending) return fail(h, HV_ERR_STATE, "no settings");
  HV_CU(h, cudaSetDevice(h->device));
  hv_status s = apply_pending(h);
  if (s != HV_OK) return s;
  SpatialArgs probe{};
  probe.spatial = HV_SPATIAL_ASP;
  probe.W = h->W;
  probe.H = h->H;
  if (!spatial_pp_supported(probe)) return fail(h, HV_ERR_UNSUPPORTED, "autofocus needs sides in [64, 1024]");
  const size_t need = size_t(chunk) * h->W * h->H * sizeof(float2);
  s = ensure(h, reinterpret_cast<void**>(&h->s1), &h->s1_bytes, need);
  if (s == HV_OK) s = ensure(h, reinterpret_cast<void**>(&h->s2), &h->s2_bytes, need);
  return s;
}

hv_status hv_focus_sweep(hv_handle* h, const void* frames, uint32_t n, const double* z, uint32_t nz, float* metric) {
  if (!h) return HV_ERR_ARG;
  if (!z || !metric || nz == 0 || nz > 1024) return fail(h, HV_ERR_ARG, "bad distances or output");
  const uint32_t chunk = 64;
  hv_status s = af_prepare(h, frames, n, std::min(n, chunk));
  if (s != HV_OK) return s;
  const uint32_t W = h->W, H = h->H;
  const hv_params& p = h->cur;
  // transfer functions H_j (transposed [kx][ky], 1/(W H) folded in, DC bin zero)
  std::vector<double> key = {double(W), double(H), p.lambda_m, p.pitch_x_m, p.pitch_y_m};
  key.insert(key.end(), z, z + nz);
  if (key != h->sw_key) {
    const size_t per = size_t(W) * H;
    s = ensure(h, reinterpret_cast<void**>(&h->sw_tables), &h->sw_bytes, per * nz * sizeof(float2));
    if (s != HV_OK) return s;
    std::vector<float2> host(per * nz);
    const double k = 2.0 * M_PI / p.lambda_m, scale = 1.0 / (double(W) * double(H));
    for (uint32_t kx = 0; kx < W; ++kx) {
      const double fx = 2.0 * M_PI * (kx < W / 2 ? double(kx) : double(kx) - W) / (W * p.pitch_x_m);
      for (uint32_t ky = 0; ky < H; ++ky) {
        const double fy = 2.0 * M_PI * (ky < H / 2 ? double(ky) : double(ky) - H) / (H * p.pitch_y_m);
        const double kz2 = k * k - fx * fx - fy * fy;
        for (uint32_t j = 0; j < nz; ++j) {
          float2 v = make_float2(0.f, 0.f);
          if (kz2 >= 0 && (kx | ky)) {
            const double ph = z[j] * std::sqrt(kz2);
            v = make_float2(float(std::cos(ph) * scale), float(std::sin(ph) * scale));
          }
          host[j * per + size_t(kx) * H + ky] = v;
        }
      }
    }
    HV_CU(h, cudaMemcpyAsync(h->sw_tables, host.data(), host.size() * sizeof(float2), cudaMemcpyHostToDevice,
                             h->stream));
    HV_CU(h, cudaStreamSynchronize(h->stream));
    h->sw_key = key;
  }
  s = ensure(h, reinterpret_cast<void**>(&h->sw_acc), &h->sw_acc_bytes, size_t(n) * nz * 2 * sizeof(double));
  if (s != HV_OK) return s;
  HV_CU(h, cudaMemsetAsync(h->sw_acc, 0, size_t(n) * nz * 2 * sizeof(double), h->stream));
  for (uint32_t a = 0; a < n; a += chunk) {
    SpatialArgs sa = af_args(h, frames, n);
    sa.raw.slot0 = a;
    sa.n = std::min(chunk, n - a);
    cudaError_t e = launch_pp_pass(sa, PASS_COL_FFT, h->stream);
    for (uint32_t j = 0; j < nz && e == cudaSuccess; ++j) {
      sa.asp_ht = h->sw_tables + size_t(j) * W * H;
      e = launch_pp_pass(sa, PASS_ROW_ASP, h->stream);
      sa.tam_acc = h->sw_acc + (size_t(a) * nz + j) * 2;
      sa.tam_stride = nz * 2;
      if (e == cudaSuccess) e = launch_pp_pass(sa, PASS_COL_IFFT_TAMURA, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "focus sweep passes");
    h->st.kernel_launches += 1 + 2 * nz;
  }
  cudaError_t e = launch_tamura_finish(h->sw_acc, n * nz, W * H, metric, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "tamura");
  h->st.kernel_launches += 1;
  return HV_OK;
}

hv_status hv_af_features(hv_handle* h, const void* frames, uint32_t n, void* out_bf16) {
  if (!h) return HV_ERR_ARG;
  if (!out_bf16) return fail(h, HV_ERR_ARG, "output is NULL");
  // frames per pass: the feature kernel runs one CTA per frame, so a chunk
  // should cover every SM several times (512 frames: 512 MB of spectra at 256^2)
  const uint32_t chunk = std::max<uint32_t>(64, std::min<uint32_t>(512, uint32_t((size_t(256) << 20) / (size_t(h->W) * h->H * sizeof(float2)))));
  hv_status s = af_prepare(h, frames, n, std::min(n, chunk));
  if (s != HV_OK) return s;
  const size_t cells = size_t(h->W / 2) * (h->H / 2);
  // widths up to 256: the row pass forms the cells in its epilogue (no spectrum in
  // memory); wider frames store the spectra and bin them in a second kernel
  const bool fused = h->W <= 256;
  for (uint32_t a = 0; a < n; a += chunk) {
    SpatialArgs sa = af_args(h, frames, n);
    sa.raw.slot0 = a;
    sa.n = std::min(chunk, n - a);
    sa.discard_inputs = 1;  // the column pass output is read once
    cudaError_t e = launch_pp_pass(sa, PASS_COL_FFT, h->stream);
    uint16_t* dst = static_cast<uint16_t*>(out_bf16) + a * cells;
    if (fused) {
      // s2 holds this chunk's cells [n][H/2][W/2] (floats), then its (sum, sum of squares)
      sa.cells = reinterpret_cast<float*>(h->s2);
      sa.tam_acc = reinterpret_cast<double*>(h->s2 + (size_t(sa.n) * cells + 1) / 2);
      sa.tam_stride = 2;
      if (e == cudaSuccess) e = cudaMemsetAsync(sa.tam_acc, 0, size_t(sa.n) * 2 * sizeof(double), h->stream);
      if (e == cudaSuccess) e = launch_pp_pass(sa, PASS_ROW_CELLS, h->stream);
      if (e == cudaSuccess)
        e = launch_af_standardize(sa.cells, sa.tam_acc, 2, sa.n, uint32_t(cells), dst, h->stream);
    } else {
      sa.tq = RingRef{h->s2, sa.n, 0};  // spectra [ky][kx] of this chunk
      if (e == cudaSuccess) e = launch_pp_pass(sa, PASS_ROW_FFT, h->stream);
      if (e == cudaSuccess) e = launch_af_features(h->s2, sa.n, h->W, h->H, dst, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "feature passes");
    h->st.kernel_launches += 3;
  }
  return HV_OK;
}

// ---------------------------------------------------------------------- groups

static hv_status gfail(hv_group* g, hv_status s, const std::string& msg) {
  g->err = msg;
  return s;
}

#define HV_GCU(g, call)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return gfail(g, HV_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

hv_status hv_group_close(hv_group* g) {
  if (!g) return HV_OK;
  cudaSetDevice(g->device);
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_done) cudaEventDestroy(g->ev_done);
  for (auto e : g->ev_pre)
    if (e) cudaEventDestroy(e);
  for (auto e : g->ev_join)
    if (e) cudaEventDestroy(e);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
  return HV_OK;
}

hv_status hv_group_open(hv_handle* const* handles, uint32_t n, void* stream, int use_graph, hv_group** out) {
  if (!out) return HV_ERR_ARG;
  *out = nullptr;
  if (!handles || n == 0) return HV_ERR_ARG;
  for (uint32_t i = 0; i < n; ++i) {
    if (!handles[i] || handles[i]->device != handles[0]->device) return HV_ERR_ARG;
    for (uint32_t j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return HV_ERR_ARG;
  }
  hv_group* g = new hv_group();
  g->hs.assign(handles, handles + n);
  g->device = handles[0]->device;
  g->use_graph = use_graph != 0;
  auto bail = [&](cudaError_t e) {
    hv_group_close(g);
    (void)e;
    return HV_ERR_CUDA;
  };
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return bail(e);
  if (stream) {
    g->stream = static_cast<cudaStream_t>(stream);
  } else {
    e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(e);
    g->own_stream = true;
  }
  e = cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_done, cudaEventDisableTiming);
  g->ev_pre.assign(n, nullptr);
  g->ev_join.assign(n, nullptr);
  for (uint32_t i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&g->ev_pre[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_join[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) return bail(e);
  *out = g;
  return HV_OK;
}

hv_status hv_render_group(hv_group* g, const void* const* frames, const uint32_t* n_frames, float* const* outs,
                          const size_t* out_capacity_floats, uint32_t* n_windows) {
  if (!g) return HV_ERR_ARG;
  if (!outs || !out_capacity_floats || !n_windows) return gfail(g, HV_ERR_ARG, "NULL argument");
  const uint32_t n = uint32_t(g->hs.size());
  HV_GCU(g, cudaSetDevice(g->device));
  // 1. settle every member's settings and check the batch before issuing work
  for (uint32_t i = 0; i < n; ++i) {
    hv_handle* h = g->hs[i];
    n_windows[i] = 0;
    if (!h->has_params && !h->pending) return gfail(g, HV_ERR_STATE, "member " + std::to_string(i) + ": no settings");
    hv_status s = settle(h);
    if (s != HV_OK) return gfail(g, s, "member " + std::to_string(i) + ": " + h->err);
    if (h->prof) return gfail(g, HV_ERR_STATE, "member " + std::to_string(i) + ": profiling is on");
    if (h->cur.temporal == HV_TEMPORAL_PCA && h->T > 64)
      return gfail(g, HV_ERR_UNSUPPORTED, "member " + std::to_string(i) + ": PCA over T > 64 frames");
    const uint32_t nf = n_frames ? n_frames[i] : 0;
    if (nf && (!frames || !frames[i])) return gfail(g, HV_ERR_ARG, "member " + std::to_string(i) + ": frames is NULL");
    if (h->pushed + nf - h->next_win > h->cap) {
      h->st.frames_rejected += nf;
      return gfail(g, HV_ERR_QUEUE_FULL, "member " + std::to_string(i) + ": input queue full");
    }
  }
  // 2. the group's stream follows every member's earlier work
  for (uint32_t i = 0; i < n; ++i) {
    HV_GCU(g, cudaEventRecord(g->ev_pre[i], g->hs[i]->stream));
    HV_GCU(g, cudaStreamWaitEvent(g->stream, g->ev_pre[i], 0));
  }
  const bool graph = g->use_graph;
  const auto t0 = std::chrono::steady_clock::now();
  if (graph) {
    HV_GCU(g, cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(g->ev_fork, g->stream);
    if (e != cudaSuccess) {
      cudaGraph_t dead = nullptr;
      cudaStreamEndCapture(g->stream, &dead);
      if (dead) cudaGraphDestroy(dead);
      return gfail(g, HV_ERR_CUDA, std::string("fork event: ") + cudaGetErrorString(e));
    }
  }
  // 3. every member's copies and kernels, each on its own stream (one graph branch)
  uint64_t launches_before = 0;
  for (auto* h : g->hs) launches_before += h->st.kernel_launches;
  hv_status s = HV_OK;
  for (uint32_t i = 0; i < n && s == HV_OK; ++i) {
    hv_handle* h = g->hs[i];
    if (graph) {
      cudaError_t e = cudaStreamWaitEvent(h->stream, g->ev_fork, 0);
      if (e != cudaSuccess) {
        s = cuda_fail(h, e, "join member stream");
        break;
      }
    }
    const uint32_t nf = n_frames ? n_frames[i] : 0;
    if (nf) s = enqueue_push_device(h, frames[i], nf);
    if (s != HV_OK) break;
    const uint32_t nw = outs[i] ? windows_ready(h, out_capacity_floats[i]) : 0;
    if (nw) s = enqueue_windows(h, outs[i], nw, graph);
    if (s != HV_OK) break;
    n_windows[i] = nw;
    cudaError_t e = cudaEventRecord(g->ev_join[i], h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->stream, g->ev_join[i], 0);
    if (e != cudaSuccess) s = cuda_fail(h, e, "join event");
  }
  uint64_t launches_after = 0;
  for (auto* h : g->hs) launches_after += h->st.kernel_launches;
  g->st.kernel_launches += launches_after - launches_before;
  if (graph) {
    cudaGraph_t gr = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(g->stream, &gr);
    if (s != HV_OK || ec != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      if (s == HV_OK) return gfail(g, HV_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(ec));
      for (auto* h : g->hs)
        if (!h->err.empty()) return gfail(g, s, h->err);
      return gfail(g, s, "capture failed");
    }
    if (g->exec) {
      cudaGraphExecUpdateResultInfo info{};
      if (cudaGraphExecUpdate(g->exec, gr, &info) == cudaSuccess) {
        ++g->st.graph_updates;
      } else {
        cudaGetLastError();  // clear the update's error; the graph is rebuilt below
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
      }
    }
    if (!g->exec) {
      const cudaError_t ei = cudaGraphInstantiate(&g->exec, gr, 0);
      if (ei != cudaSuccess) {
        cudaGraphDestroy(gr);
        g->exec = nullptr;
        return gfail(g, HV_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
      }
      ++g->st.graph_instantiations;
    }
    cudaGraphDestroy(gr);
    g->st.capture_us_last = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    HV_GCU(g, cudaGraphLaunch(g->exec, g->stream));
    ++g->st.graph_launches;
  } else if (s != HV_OK) {
    for (auto* h : g->hs)
      if (!h->err.empty()) return gfail(g, s, h->err);
    return gfail(g, s, "enqueue failed");
  }
  // 4. members' later work (pushes, renders) follows the batch
  HV_GCU(g, cudaEventRecord(g->ev_done, g->stream));
  for (auto* h : g->hs) {
    HV_GCU(g, cudaStreamWaitEvent(h->stream, g->ev_done, 0));
    if (graph) {
      HV_GCU(g, cudaEventRecord(h->ev_consumed, h->stream));
      if (note_consumed(h) != HV_OK) return gfail(g, HV_ERR_CUDA, h->err);
    }
  }
  ++g->st.steps;
  return HV_OK;
}

hv_status hv_group_get_stats(const hv_group* g, hv_group_stats* s) {
  if (!g || !s) return HV_ERR_ARG;
  *s = g->st;
  return HV_OK;
}

const char* hv_group_last_error(const hv_group* g) { return g ? g->err.c_str() : ""; }

const char* hv_last_error(const hv_handle* h) { return h ? h->err.c_str() : g_open_err.c_str(); }

const char* hv_version(void) { return "hv-gb300 0.1 (sm_103a)"; }

}  // extern "C"
