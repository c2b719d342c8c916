// hv_internal.h -- launchers shared between the C-ABI runtime and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hv {

// Frames live in rings: frame f of the stream sits in slot (f mod capacity).
// A launch covers n consecutive frames starting at ring slot `slot0`.
struct RingRef {
  void* base;        // ring storage
  uint32_t cap;      // capacity in frames
  uint32_t slot0;    // slot of the first frame of the launch
};

// Input element kinds of the first spatial pass.
enum InKind { IN_U8 = 0, IN_U16 = 1 };

// Spatial transform of n frames (Sec. III-B.1), raw ring -> time-queue ring.
struct SpatialArgs {
  int spatial;          // HV_SPATIAL_*
  int in_kind;          // IN_U8 / IN_U16
  uint32_t W, H;
  uint32_t n;           // frames in this launch
  RingRef raw;          // uint8/uint16 frames
  RingRef tq;           // complex64 frames
  float2* scratch1;     // n * W * H complex64 (transposed intermediate)
  float2* scratch2;     // n * W * H complex64 (ASP only)
  const float2* tw_w;   // twiddle table of length W
  const float2* tw_h;   // twiddle table of length H
  const float2* asp_ht; // ASP transfer function, transposed [kx][ky], includes 1/(W H)
  const float2* asp_h;  // the same, row-major [ky][kx] (NULL where not built)
  const float2* chirp_x;// Fresnel chirp factors along x (length W), fftshift folded in
  const float2* chirp_y;// along y (length H)
  int use_cluster;      // 1: whole-frame cluster kernel when the size allows it
  int use_pp;           // 1: persistent prefetching multi-pass kernels when the size allows
  double* tam_acc;      // focus sweep: frame i adds (sum |u|, sum |u|^2) at tam_acc + i * tam_stride
  uint32_t tam_stride;
  int discard_inputs;   // persistent passes: scratch1/scratch2 are read once, drop their L2 lines after staging
  float* cells;         // PASS_ROW_CELLS output [n][H/2][W/2]
  unsigned* err;        // device flags (bit 3: a row pass's wait for its staged strip gave up;
                        // bit 4: a fused-transform wait for another CTA's pass gave up); may be NULL
  // fused transform (one persistent launch for every pass of every frame, 256 x 256):
  // scratch1 / scratch2 are rings of `ring` frames each, fused_ctr holds
  // 1 + kFusedPasses ring counters (ticket, then per-slot completed items of each pass)
  int use_fused;
  uint32_t ring;
  unsigned* fused_ctr;
  int stall;            // fault injection (tests): the fused row items wait on a condition nothing sets
};
cudaError_t launch_spatial(const SpatialArgs& a, cudaStream_t s, int* launches);
bool spatial_cluster_supported(const SpatialArgs& a);
bool spatial_pp_supported(const SpatialArgs& a);
cudaError_t launch_spatial_pp(const SpatialArgs& a, cudaStream_t s, int* launches);
cudaError_t launch_spatial_cluster(const SpatialArgs& a, cudaStream_t s, int* launches);
// Fused transform: frames of 256 x 256, ASP or Fresnel; needs ring >= kFusedRing
// frames in scratch1 (and scratch2 for ASP), fused_ctr and err.
constexpr uint32_t kFusedRing = 96;
constexpr uint32_t kFusedPasses = 4;  // counter sets: ASP takes four passes, Fresnel two
bool spatial_fused_supported(const SpatialArgs& a);
cudaError_t launch_spatial_fused(const SpatialArgs& a, cudaStream_t s, int* launches);

// Single passes of the persistent multi-pass transform (sides 64..512):
//   PASS_COL_FFT   raw -> column FFT (chirped when spatial is Fresnel) -> scratch1 [ky][x]
//   PASS_ROW_ASP   scratch1 -> row FFT, x asp_ht, row IFFT -> scratch2 [x][ky]
//   PASS_COL_IFFT  scratch2 -> column IFFT -> tq ring [y][x]
//   PASS_ROW_FFT   scratch1 -> row FFT -> tq ring [ky][kx]
//   PASS_COL_IFFT_TAMURA  scratch2 -> column IFFT -> (sum |u|, sum |u|^2) per frame
//   PASS_ROW_CELLS scratch1 -> row FFT -> network-input cells (sides 64..256): the
//                  centred spectrum's 2 x 2 blocks as log1p(mean |F|) (DC bin as 0)
//                  into cells [frame][H/2][W/2], and (sum v, sum v^2) per frame
//                  into tam_acc + frame * tam_stride
enum { PASS_COL_FFT = 0, PASS_ROW_ASP = 1, PASS_COL_IFFT = 2, PASS_ROW_FFT = 3, PASS_COL_IFFT_TAMURA = 4,
       PASS_ROW_CELLS = 5 };
cudaError_t launch_pp_pass(const SpatialArgs& a, int pass, cudaStream_t s);

// STFT band moments of nwin windows (Sec. III-B.1), time-queue ring -> images.
struct StftArgs {
  uint32_t W, H, T, S;
  uint32_t nwin;
  RingRef tq;           // complex64 frames; slot0 = slot of window 0's first frame
  const float2* tw_t;   // twiddle table of length T
  uint32_t klo, khi;    // inclusive band
  float fscale;         // kHz per bin: fs / T / 1000
  uint32_t mask;        // HV_MOM_* bits
  uint32_t nout;        // popcount(mask)
  float* out;           // [nwin][nout][H*W]
  unsigned* err;        // device flags: bit 1 set when a wait for staged frames gave up
  int tma;              // set by the launcher: staged frames through a TMA tensor map
  int kernel;           // STFT_AUTO: windows that do not overlap (S >= T) one CTA per
                        // (window, pixel tile); STFT_WIDE: the same with twice the pixels
                        // per CTA; STFT_PIPE: persistent CTAs over the (window, tile)
                        // items, the next item's frames loaded while the current one is
                        // transformed; STFT_WALK: CTAs walk all windows of their pixels
  // post-processing without convolution, fused into the epilogue: when post_ring is
  // set, the images of window w go to ring slot (post_count + w) mod post_R (layout
  // [R][nout][H*W]) instead of out, and when post_sums is set each image's sum is
  // added (float64 atomics) into post_sums [slot][image][kPostSub], zeroed beforehand
  float* post_ring;
  uint32_t post_R;
  uint64_t post_count;
  double* post_sums;
};
// float64 sums of a post-processed image are kept as kPostSub partial sums, so that
// the CTAs that produce it add into different words
constexpr uint32_t kPostSub = 32;
enum { STFT_AUTO = 0, STFT_WALK = 1, STFT_WIDE = 2, STFT_PIPE = 3, STFT_TMA = 4, STFT_TMA_PIPE = 5 };
cudaError_t launch_stft(const StftArgs& a, cudaStream_t s, int* launches);

// Encodes a 2-D tiled TMA tensor map (map: a CUtensorMap, 64-byte aligned) over
// 8-byte elements: {inner, outer} elements, rows pitch_bytes apart, box
// {box_inner, box_outer}, 64-byte swizzle or none. False when the driver entry
// point is missing or the encoder rejects the shape.
bool encode_map_2d_u64(void* map, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch_bytes,
                       uint32_t box_inner, uint32_t box_outer, bool swizzle64);
// The same for 1-, 2-, 4- or 8-byte elements, no swizzle.
bool encode_map_2d(void* map, const void* base, int elem_bytes, uint64_t inner, uint64_t outer,
                   uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_outer);

// PCA of one window (Sec. III-B.1), time-queue ring -> energy image.
struct PcaArgs {
  uint32_t W, H, T;
  RingRef tq;           // slot0 = slot of the first window's first frame
  uint32_t nwin;        // windows in this launch (batched only for T <= 64, else 1)
  uint32_t wstride;     // frames between window starts (S)
  uint32_t chunk;       // pixels per covariance CTA
  uint32_t nchunks;
  uint32_t lo, M, Mpad; // sub-basis: ranks lo .. lo+M-1 (1-based), padded to 64
  int max_sweeps;
  double tol, tol_abs;  // Jacobi skip thresholds (relative, and x largest diagonal)
  double stop_rel;      // > 0: a float64 sweep whose off-diagonal entries are all below
                        // stop_rel x trace ends the iteration (refinement after float32)
  float2* partials;     // nwin x nchunks x upper tiles x TS x TS
  double2* C;           // nwin x T x T
  double2* C2;          // T x T second copy (large-T path: the rounds alternate between C and C2)
  float2* Cf;           // T x T float32 copies and rotations of the large-T path's first phase
  float2* Cf2;
  float2* Vf;
  double2* V;           // T x T (large-T path)
  double* rot;          // T/2 rotations (4 doubles each); after the eigensolver, the
                        // Rayleigh quotients and inverse norms of the columns of V
  unsigned* counters;   // 4 counters followed by one double (largest diagonal)
  double* cmax;         // = (double*)(counters + 4)
  double* lam;          // nwin x T eigenvalues, descending
  float2* Vs;           // nwin x T x Mpad sub-basis
  // tensor-core covariance (precision BF16 / split-BF16)
  int precision;        // HV_PREC_*
  float* tc_partials;   // nchunks x ntiles x 128 x 256 float
  uint32_t tc_chunk, tc_nchunks, tc_ntiles;
  // the window as BF16 operands, hi part then (split-BF16) lo part, each
  // [64-pixel step][2T/8 row blocks][8 k blocks][8 rows][8 pixels]: every step's
  // rows form the MMA's no-swizzle K-major core-matrix layout, contiguous
  uint16_t* tc_stage;
  size_t tc_stage_part;  // bf16 elements per part: steps x 2T x 64
  uint8_t tc_tile_i[32], tc_tile_j[32];
  unsigned* err;        // device error flag (bounded waits that gave up)
};
size_t pca_partials_floats2(uint32_t T, uint32_t nchunks);
size_t cov_tc_partials_floats(uint32_t ntiles, uint32_t nchunks);
uint32_t cov_tc_tiles(uint32_t T, uint8_t* ti, uint8_t* tj);
cudaError_t launch_cov_tc(PcaArgs& a, cudaStream_t s, int* launches);
// ev (optional, 6 events): start and end of the covariance, of the eigensolver and of
// the projection
cudaError_t launch_pca(PcaArgs& a, float* out, cudaStream_t s, int* launches, cudaEvent_t* ev);
// Adds the float32 and refinement sweep counts of the last window (counters[1],
// counters[2]) to total[0], total[1] (one thread; stage profiling).
cudaError_t launch_pca_sweeps_add(const unsigned* counters, unsigned long long* total, cudaStream_t s);
// The three stages of launch_pca, for callers that run them on different streams:
// covariance into a.C (and the counters cleared), eigensolver (a.C, the shared
// eigensolver scratch -> a.lam, a.Vs), projection (a.Vs, the window's frames -> out).
cudaError_t launch_pca_cov(PcaArgs& a, cudaStream_t s, int* launches);
cudaError_t launch_pca_eig(PcaArgs& a, cudaStream_t s, int* launches);
cudaError_t launch_pca_proj(PcaArgs& a, float* out, cudaStream_t s, int* launches);

// Autofocus: Tamura coefficients from per-(frame, distance) amplitude sums, and the
// network input (2 x 2 binned log-magnitude spectrum, standardised, bfloat16)
// from n unshifted spectra [ky][kx].
cudaError_t launch_tamura_finish(const double* acc, uint32_t count, uint32_t pixels, float* metric, cudaStream_t s);
cudaError_t launch_af_features(const float2* spec, uint32_t n, uint32_t W, uint32_t H, void* out_bf16,
                               cudaStream_t s);
// The network input from the cells and per-frame sums of PASS_ROW_CELLS:
// (v - mean) / deviation per frame, rounded to bfloat16.
cudaError_t launch_af_standardize(const float* cells, const double* sums, uint32_t sum_stride, uint32_t n,
                                  uint32_t ncell, void* out_bf16, cudaStream_t s);

// Post-processing of rendered images [window][nout][H][W] (Sec. III-B): periodic
// K x K convolution into ring slot (count + window) mod R, per-image float64 sums
// when re-normalising (added by the kernel that writes the slot), then each image
// replaced in place by the mean of its last min(A, count + window + 1) ring slots.
// H, W multiples of 16.
struct PostArgs {
  uint32_t W, H, nout;
  int K;                // 0 (no convolution) or odd
  const float* kern;    // device K * K weights
  int renorm;
  uint32_t A, R;
  uint64_t count;       // images of each output already in the ring
  float* ring;          // [R][nout][H][W]
  double* sums;         // [R][nout][kPostSub] partial sums
  int fused;            // the STFT epilogue already wrote the ring slots and their sums
};
// Zeroes the partial sums of the ring slots the next nwin windows write.
cudaError_t launch_post_zero(const PostArgs& a, uint32_t nwin, cudaStream_t s);
// Unfused: zeroes the slots' sums, convolves (or copies) the images into the ring
// adding the sums, then averages; fused: averages only. `images` is the output.
cudaError_t launch_post(float* images, uint32_t nwin, const PostArgs& a, cudaStream_t s, int* launches);

// Copy propagated frames out as interleaved complex images.
cudaError_t launch_copy_frames(const RingRef& tq, uint32_t n, uint32_t hw, float* out,
                               cudaStream_t s, int* launches);

}  // namespace hv
