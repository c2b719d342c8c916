/*
 * hv.h -- C ABI of the GB300 hologram-rendering hot path.
 *
 * The library turns a stream of raw camera interferograms into rendered images
 * (the paper's computation pipeline, Sec. III-B and Fig. 1):
 *
 *   raw frames --convert--> complex --spatial--> time-transformation queue
 *              --temporal (STFT moments | PCA energy)--> images
 *
 * All types in the signatures are plain C. Pointers are either host pointers
 * or CUDA device pointers, as each argument says. Every call returns an
 * hv_status; nothing throws across the ABI. Calls on one handle must be
 * serialised by the caller; separate handles are independent.
 *
 * Device work runs on the handle's stream (the cudaStream_t given at open, or
 * one the library creates). Results written to device memory are ready when
 * that stream reaches them; results written to host memory are ready when the
 * call returns.
 */
#ifndef HV_H
#define HV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hv_handle hv_handle; /* opaque; created by hv_open, owned by the library */

typedef enum {
  HV_OK = 0,
  HV_ERR_ARG = -1,         /* invalid argument (NULL, size, unsupported value)   */
  HV_ERR_STATE = -2,       /* call not valid in the handle's state (no params)    */
  HV_ERR_QUEUE_FULL = -3,  /* input queue cannot take the frames; nothing copied  */
  HV_ERR_NOMEM = -4,       /* device or host allocation failed                    */
  HV_ERR_CUDA = -5,        /* a CUDA runtime call failed; see hv_last_error       */
  HV_ERR_TIMEOUT = -6,     /* a bounded device wait gave up                       */
  HV_ERR_UNSUPPORTED = -7  /* valid request this build does not implement         */
} hv_status;

/* Memory kinds of the buffers a call reads or writes. HV_MEM_HOST_ASYNC is host
 * memory (page-locked for full speed) whose copy is only queued: the call
 * returns before it has run, as the paper's pipeline runs asynchronously to its
 * input and output streams (Sec. III). */
enum { HV_MEM_HOST = 0, HV_MEM_DEVICE = 1, HV_MEM_HOST_ASYNC = 2, HV_MEM_DEVICE_ASYNC = 3 };

/* Spatial demodulation (Sec. III-B.1; benchmarks Sec. VI-B). */
enum { HV_SPATIAL_NONE = 0, HV_SPATIAL_ASP = 1, HV_SPATIAL_FRESNEL = 2 };

/* Temporal analysis (Sec. III-B.1). HV_TEMPORAL_NONE renders every propagated
 * frame as a complex image (2 floats per pixel, re then im). */
enum { HV_TEMPORAL_STFT = 0, HV_TEMPORAL_PCA = 1, HV_TEMPORAL_NONE = 2 };

/* STFT outputs, rendered in this order for the bits set. */
enum {
  HV_MOM_M0 = 1,   /* sum over band of |S_k|^2                         */
  HV_MOM_M1 = 2,   /* sum over band of f_k |S_k|^2, f_k in kHz         */
  HV_MOM_M2 = 4,   /* sum over band of f_k^2 |S_k|^2                   */
  HV_MOM_M1N = 8,  /* M1 / M0 (kHz), computed in FP64, 0 where M0 = 0  */
  HV_MOM_M2N = 16  /* sqrt(M2 / M0) (kHz), FP64, 0 where M0 = 0        */
};

/* Arithmetic of the PCA covariance. */
enum { HV_PREC_FP32 = 0, HV_PREC_BF16 = 1, HV_PREC_SPLIT_BF16 = 2 };

typedef struct {
  uint32_t struct_size;       /* sizeof(hv_open_desc)                                 */
  int32_t device;             /* CUDA device ordinal                                   */
  uint32_t max_width;         /* largest frame width this handle will accept           */
  uint32_t max_height;        /* largest frame height                                  */
  uint32_t pixel_bits;        /* 8 (uint8 frames) or 16 (uint16 frames, e.g. 12-bit)   */
  uint32_t queue_capacity_frames; /* raw input ring capacity in frames (>= 1)          */
  uint32_t time_queue_frames; /* propagated-frame ring capacity (0 = automatic)        */
  uint32_t reserved;
  void* stream;               /* cudaStream_t for all device work; NULL = own stream   */
} hv_open_desc;

typedef struct {
  uint32_t struct_size;       /* sizeof(hv_params)                                     */
  uint32_t width, height;     /* frame size; powers of two in [16, 1024]               */
  int32_t spatial;            /* HV_SPATIAL_*                                          */
  int32_t fftshift;           /* Fresnel only: 1 = centre the zero frequency           */
  double z_m;                 /* propagation distance [m] (ASP, Fresnel)               */
  double lambda_m;            /* wavelength [m]                                        */
  double pitch_x_m, pitch_y_m;/* sensor pixel pitch [m]                                */
  int32_t temporal;           /* HV_TEMPORAL_*                                         */
  uint32_t T;                 /* window length in frames (power of two, 8..1024)       */
  uint32_t stride;            /* time stride S in frames (>= 1)                        */
  uint32_t moments_mask;      /* STFT: OR of HV_MOM_*                                  */
  double fs_hz;               /* camera frame rate [Hz]                                */
  uint32_t band_lo_bin;       /* STFT band, inclusive bin indices, used when           */
  uint32_t band_hi_bin;       /*   band_lo_hz and band_hi_hz are both <= 0             */
  double band_lo_hz;          /* STFT band in Hz (> 0 to use): bins ceil(lo T/fs) ..   */
  double band_hi_hz;          /*   floor(hi T/fs)                                      */
  uint32_t pca_lo, pca_hi;    /* PCA: eigenvectors ranked pca_lo..pca_hi (1-based,
                                 inclusive, descending eigenvalue)                     */
  int32_t precision;          /* PCA covariance arithmetic, HV_PREC_*                  */
  int32_t tuned;              /* 1 = tuned form (spatial kernels chosen by timing)    */
  uint32_t spatial_chunk;     /* frames per spatial launch (0 = automatic)             */
  uint32_t spatial_kernel;    /* HV_SK_*: which spatial kernels (default automatic):
                                 multi-pass (one strip per CTA), persistent multi-pass
                                 (CTAs loop over strips, prefetching the next), the
                                 whole-frame cluster kernel, or the fused transform
                                 (256 x 256 frames: every pass of every frame in one
                                 persistent launch, intermediates in L2-resident rings) */
  double highpass_cpp;        /* ASP only: high-pass spatial filter applied after the
                                 propagation (Sec. VI-B.1): spatial frequencies whose
                                 radius sqrt((m/W)^2 + (n/H)^2) in cycles per pixel is
                                 below this cutoff are zeroed; 0 = off. Folded into
                                 the transfer function. */
  int32_t stft_kernel;        /* STFT kernel for windows that do not overlap (S >= T):
                                 0 = automatic (the autotuner's choice when tuned = 1,
                                 else the walking kernel launched once per window),
                                 HV_STFT_WALK, HV_STFT_WINDOW, HV_STFT_WINDOW_WIDE,
                                 HV_STFT_WINDOW_PIPELINED (persistent CTAs that load
                                 their next window tile while transforming one),
                                 HV_STFT_WINDOW_TMA or HV_STFT_WINDOW_TMA_PIPELINED
                                 (T = 512: a window tile brought in by TMA tensor
                                 loads and transformed in place; the second
                                 persistent and double-buffered; at other T, and
                                 where a window's queue slots wrap, the
                                 HV_STFT_WINDOW kernel runs instead)              */
  uint32_t reserved;
} hv_params;

/* Spatial kernel selection: automatic = the autotuner's choice when tuned = 1,
 * the multi-pass kernels otherwise. */
enum { HV_SK_AUTO = 0, HV_SK_MULTIPASS = 1, HV_SK_CLUSTER = 2, HV_SK_PERSISTENT = 3, HV_SK_FUSED = 4 };

typedef struct {
  uint64_t frames_pushed;     /* frames accepted by hv_push_frames                     */
  uint64_t frames_rejected;   /* frames refused with HV_ERR_QUEUE_FULL                 */
  uint64_t frames_dropped;    /* frames lost after acceptance (always 0)               */
  uint64_t frames_propagated; /* frames through the spatial transform                 */
  uint64_t windows_rendered;  /* windows through the temporal transform               */
  uint64_t kernel_launches;   /* kernels launched by this handle                       */
} hv_stats;

/* Open a handle on a device: allocates the raw input ring (capacity x max frame
 * size) and creates or adopts the stream. Nothing is rendered until
 * hv_set_params. *out receives the handle (NULL on failure).
 * Errors: HV_ERR_ARG (bad descriptor), HV_ERR_NOMEM, HV_ERR_CUDA. */
hv_status hv_open(const hv_open_desc* desc, hv_handle** out);

/* Set the compute settings. Validated now; applied at the next window boundary,
 * i.e. at the start of the next hv_render (the paper's "delayed" settings,
 * Sec. IV-B). On application the time-transformation queue is flushed and the
 * next window starts at the first frame that the previous window sequence had
 * not yet consumed; the device workspace (time queue, tables) is (re)allocated
 * when sizes change. Errors: HV_ERR_ARG (invalid or unsupported combination).
 * The previous settings stay in force when an error is returned. */
hv_status hv_set_params(hv_handle* h, const hv_params* p);

/* Read back the settings last accepted by hv_set_params. */
hv_status hv_get_params(const hv_handle* h, hv_params* p);

/* Enqueue n raw frames (width x height of the current settings, or of max size
 * when none are set) into the input ring (Sec. III-A): `frames` is a host
 * pointer (mem_kind HV_MEM_HOST; copied before return, the caller may reuse it)
 * or a device pointer (HV_MEM_DEVICE; copied on the handle's stream, so the
 * frames must be completely written before that stream reaches the copy -- work
 * of another stream that produces them must be ordered before it, e.g. by
 * giving the handle the producer's stream in hv_open or by synchronising -- and
 * must stay valid until the stream passes it) or a host pointer whose copy is
 * only queued (HV_MEM_HOST_ASYNC: on the handle's copy stream, after the ring
 * slots it overwrites have been consumed; the buffer must stay unchanged until
 * hv_synchronize returns or until an hv_render with HV_MEM_HOST output that
 * renders windows using these frames returns), or a device pointer whose frames
 * the library reads in place (HV_MEM_DEVICE_ASYNC: they must be completely
 * written when the call is made -- no stream is ordered before their use -- and
 * stay valid and unchanged until every window that contains them has been
 * rendered and hv_synchronize has returned; the spatial stage reads them straight
 * from `frames`, nothing is copied; a pointer that is not 16-byte aligned is
 * copied instead, on the copy stream after the ring slots it overwrites have been
 * consumed; only hv_push_frames takes it). Frames are uint8 or uint16
 * by pixel_bits, row-major, frames contiguous. All-or-nothing: if the ring
 * cannot take all n frames, nothing is copied and HV_ERR_QUEUE_FULL is returned
 * (backpressure; frames are never dropped). */
hv_status hv_push_frames(hv_handle* h, const void* frames, uint32_t n, int mem_kind);

/* Render every complete window in the queue (at most as many as fit in `out`).
 * Images are written window-major: STFT -> one float image per selected moment
 * (order M0, M1, M2, M1N, M2N); PCA -> one float image E; TEMPORAL_NONE -> one
 * complex image per frame (2 floats per pixel). out_capacity_floats bounds the
 * write; *n_windows receives the number of windows rendered (0 is not an
 * error). out_mem_kind says whether `out` is host or device memory; with
 * HV_MEM_HOST_ASYNC the device-to-host copy is queued on the handle's stream and
 * the images are in `out` once hv_synchronize returns.
 * Errors: HV_ERR_STATE (no params), HV_ERR_ARG, HV_ERR_CUDA. */
hv_status hv_render(hv_handle* h, float* out, size_t out_capacity_floats, int out_mem_kind,
                    uint32_t* n_windows);

/* Number of floats one rendered window occupies with the current settings. */
hv_status hv_window_floats(const hv_handle* h, size_t* floats_per_window);

/* Eigenvalues (descending, FP64) of the last PCA window rendered; n <= T. */
hv_status hv_pca_eigenvalues(const hv_handle* h, double* out, uint32_t n);

/* Choices of the tuned form (hv_params.tuned = 1), made when the settings are
 * applied by timing each candidate on the handle's own buffers. */
typedef struct {
  int32_t tuned;                    /* 1 once the autotuner has run                   */
  int32_t spatial_kernel;           /* HV_SK_MULTIPASS, _CLUSTER, _PERSISTENT or _FUSED */
  uint32_t spatial_chunk;           /* frames per multi-pass launch                   */
  int32_t stft_kernel;              /* HV_STFT_WALK, _WINDOW, _WINDOW_WIDE,
                                       _WINDOW_PIPELINED, _WINDOW_TMA or
                                       _WINDOW_TMA_PIPELINED                          */
  float candidate_us_per_frame[12]; /* measured us per frame: multi-pass with 16, 32, 64,
                                       128, 256 frames per launch; persistent
                                       multi-pass with 64, 128, 256, 512; the cluster
                                       kernel; the fused transform (0 where not
                                       applicable)                                    */
  float stft_us_per_window[6];      /* measured us per window of the STFT kernels:
                                       walking (CTAs walk every window of their
                                       pixels), one CTA per (window, pixel tile), the
                                       same with twice the pixels per CTA, persistent
                                       double-buffered CTAs over the (window, tile)
                                       items, the TMA-fed kernel, the same persistent
                                       and double-buffered; 0 where not applicable
                                       (all but the first need S >= T, the last two
                                       T = 512)                                       */
} hv_tuning;

/* STFT kernels the autotuner chooses between (windows that do not overlap). */
enum { HV_STFT_WALK = 1, HV_STFT_WINDOW = 2, HV_STFT_WINDOW_WIDE = 3, HV_STFT_WINDOW_PIPELINED = 4,
       HV_STFT_WINDOW_TMA = 5, HV_STFT_WINDOW_TMA_PIPELINED = 6 };

/* The autotuner's choices for the applied settings. Errors: HV_ERR_STATE. */
hv_status hv_get_tuning(const hv_handle* h, hv_tuning* t);

/* Counters of the handle. */
hv_status hv_get_stats(const hv_handle* h, hv_stats* s);

/* Per-stage device timing (CUDA events on the handle's stream around the
 * spatial and the temporal launches of every hv_render). */
typedef struct {
  double spatial_ms;          /* summed device time of the spatial stage           */
  double temporal_ms;         /* summed device time of the temporal stage          */
  uint64_t renders;           /* hv_render calls recorded                          */
  uint64_t frames;            /* frames propagated while recording                 */
  uint64_t windows;           /* windows rendered while recording                  */
  double pca_cov_ms;          /* PCA: covariance (partials and reduction)           */
  double pca_eig_ms;          /* PCA: Jacobi eigendecomposition and selection       */
  double pca_proj_ms;         /* PCA: projection and energy                         */
  uint64_t pca_sweeps;        /* PCA: refinement sweeps (float64 diagonal and eigenvectors,
                                 float32 off-diagonal) summed over recorded windows */
  uint64_t pca_sweeps_f32;    /* PCA: float32 Jacobi sweeps (first phase) summed likewise */
} hv_profile;

/* Start (on = 1, counters reset) or stop (on = 0) recording stage times. */
hv_status hv_profile_enable(hv_handle* h, int on);

/* Stage times recorded so far; waits for the handle's stream. */
hv_status hv_profile_read(hv_handle* h, hv_profile* out);

/* Wait for all device work of the handle (its stream and its copy stream).
 * Returns HV_ERR_CUDA if a kernel of the handle gave up a bounded wait (for
 * staged frames or for tensor-core work, about two seconds): the flag is sticky
 * and the images of that launch are not valid. */
hv_status hv_synchronize(hv_handle* h);

/* Fault injection for tests of that failure path (no part of the method; the
 * paper's own guard is backpressure, Sec. III). what = HV_INJECT_FUSED_STALL:
 * the next launch of the fused 256 x 256 spatial transform of this handle makes
 * its row items wait on a condition that nothing sets, as if another CTA's pass
 * never finished. The producers' bounded waits give up (about 2^31 SM clocks, a
 * second), every CTA returns, the launch ends, and the next hv_synchronize
 * returns HV_ERR_CUDA; the device flags stay set, so the handle is to be closed.
 * Nothing faults, traps or hangs. The injection waits for the next fused launch
 * (the autotuner's timing launches included); HV_INJECT_NONE cancels it.
 * HV_ERR_ARG for another value of `what`. */
#define HV_INJECT_NONE 0
#define HV_INJECT_FUSED_STALL 1
hv_status hv_debug_inject(hv_handle* h, int what);

/* Free every resource of the handle. NULL is accepted (no-op). */
hv_status hv_close(hv_handle* h);

/* ------------------------------------------------------------------------
 * Post-processing of rendered images (Sec. III-B, "post processing and image
 * accumulation"): each rendered image (every moment of STFT, the energy of
 * PCA) is, in this order,
 *   1. convolved with a K x K kernel, the image taken as periodic:
 *      out[y][x] = sum_{a,b} k[a][b] img[(y + a - K/2) mod H][(x + b - K/2) mod W]
 *      (the kernel applied as written, not flipped);
 *   2. re-normalised: divided by its spatial mean (0 where the mean is 0);
 *   3. accumulated: replaced by the mean of the last A images of the same
 *      output (the same moment of the previous windows), fewer while fewer
 *      exist.
 * Not applicable to HV_TEMPORAL_NONE.
 * ------------------------------------------------------------------------ */
#define HV_POST_MAX_KERNEL 31u
#define HV_POST_MAX_ACCUMULATE 64u

typedef struct {
  uint32_t struct_size;  /* sizeof(hv_post)                                               */
  uint32_t kernel_size;  /* K: 0 (no convolution) or odd, 1 .. HV_POST_MAX_KERNEL          */
  const float* kernel;   /* host, K * K row-major weights (copied by the call); NULL: the
                            Gaussian exp(-(dx^2 + dy^2) / (2 sigma^2)) normalised to sum 1 */
  float gauss_sigma;     /* sigma of that Gaussian (> 0 when kernel is NULL and K > 0)     */
  int32_t renormalize;   /* 1: step 2 on; 0: off                                          */
  uint32_t accumulate;   /* A, 1 .. HV_POST_MAX_ACCUMULATE (1: no accumulation)            */
  uint32_t reserved;
} hv_post;

/* Post-processing settings: validated now, applied at the start of the next
 * hv_render (like hv_set_params); applying them, or new settings, restarts
 * the accumulation history. K = 0, renormalize = 0 and A = 1 turn it off.
 * Errors: HV_ERR_ARG (bad fields); HV_ERR_UNSUPPORTED from hv_render when the
 * temporal analysis is HV_TEMPORAL_NONE and post-processing is on. */
hv_status hv_set_postprocess(hv_handle* h, const hv_post* p);

/* ------------------------------------------------------------------------
 * .holo files (the paper's "Holofile system" section): a 64-byte header, the
 * frames as one binary stream, and an optional JSON footer with the rendering
 * settings used while recording. Header fields, at byte offsets:
 *   0 "HOLO" magic (4 bytes), 4 version (uint16, 7), 6 bits per pixel (uint16,
 *   a multiple of 8), 8 width (uint32), 12 height (uint32), 16 number of images
 *   (uint32), 20 total data size in bytes (uint64), 28 endianness of the data
 *   (uint8: 0 little, 1 big), 29 data type (uint8: 0 raw, 1 processed), 30..63
 *   zero padding. Header integers are little-endian.
 * These calls are host code: they need no GPU unless a destination is device
 * memory. Paths are NUL-terminated file names.
 * ------------------------------------------------------------------------ */
typedef struct {
  uint16_t version;        /* 7                                     */
  uint16_t bits_per_pixel; /* 8, 16, 32, ...                        */
  uint32_t width, height;
  uint32_t n_images;
  uint64_t data_bytes;     /* n_images * width * height * bits / 8  */
  uint8_t endianness;      /* 0 little, 1 big                       */
  uint8_t data_type;       /* 0 raw, 1 processed                    */
  uint8_t reserved[6];
} hv_holo_header;

/* Parses and checks the header: magic, version 7, bits a multiple of 8,
 * data_bytes equal to the frames' size and within the file. Errors:
 * HV_ERR_ARG (NULL, unreadable or malformed file), HV_ERR_UNSUPPORTED (another
 * version). */
hv_status hv_holo_read_header(const char* path, hv_holo_header* hdr);

/* Reads frames first .. first + n - 1 into dst: host memory (mem_kind
 * HV_MEM_HOST) or device memory (HV_MEM_DEVICE, copied through a pinned buffer
 * on `stream`, a cudaStream_t or NULL; the call returns after the copies
 * complete). Big-endian pixels are byte-swapped to the host's order. Errors:
 * HV_ERR_ARG (range past the last frame, short file, NULL), HV_ERR_CUDA. */
hv_status hv_holo_read_frames(const char* path, uint64_t first, uint32_t n, void* dst, int mem_kind,
                              void* stream);

/* The footer (the bytes after the frames, JSON text) into buf with a NUL
 * terminator; *len = its length (0 when there is none). buf may be NULL to
 * query the length. Errors: HV_ERR_ARG (file, or cap <= *len with buf). */
hv_status hv_holo_read_footer(const char* path, char* buf, size_t cap, size_t* len);

/* Writes a .holo file: the header from hdr (version, data_bytes and padding are
 * filled in; endianness must be 0, data written as given), n_images frames from
 * host memory, and footer_json (may be NULL) after them. Errors: HV_ERR_ARG. */
hv_status hv_holo_write(const char* path, const hv_holo_header* hdr, const void* frames, const char* footer_json);

/* ------------------------------------------------------------------------
 * Autofocus. The paper propagates to a distance the user sets (Sec. III-B.1);
 * these calls give the plain focus search (a sweep of distances scored by a
 * focus metric) and the input of the small network that replaces it
 * (include/hv_af.h). Both use the handle's frame size, pixel depth,
 * wavelength and pitches (its current settings) and its scratch buffers;
 * sides must be powers of two in [64, 512]. Frames are raw device frames
 * [n][height][width] (uint8 or uint16 by pixel_bits). Work is queued on the
 * handle's stream.
 * ------------------------------------------------------------------------ */

/* Plain z-sweep: for each of the nz distances z[j] (host array, metres), the
 * angular-spectrum propagation of the hologram with its mean removed (the
 * transfer function's DC bin set to zero), then the Tamura coefficient
 * sqrt(sigma / mu) of the amplitude |U| over the frame (population sigma; 0
 * when mu = 0). metric: device float array [n][nz]. The distances' transfer
 * functions are built on the host in float64 and cached until the distances or
 * the optics change. Errors: HV_ERR_ARG (NULL, n = 0, nz not in [1, 1024]),
 * HV_ERR_STATE (no settings), HV_ERR_UNSUPPORTED (frame size), HV_ERR_NOMEM,
 * HV_ERR_CUDA. */
hv_status hv_focus_sweep(hv_handle* h, const void* frames, uint32_t n, const double* z, uint32_t nz, float* metric);

/* Network input of each frame: the magnitude of the centred 2-D spectrum of
 * the mean-removed hologram, averaged over 2 x 2 bins, log(1 + .), standardised
 * to zero mean and unit population deviation over the frame. out: device array
 * [n][height/2][width/2] of bfloat16 (raw 16-bit patterns, rounded to nearest,
 * ties to even). Errors as hv_focus_sweep. */
hv_status hv_af_features(hv_handle* h, const void* frames, uint32_t n, void* out_bf16);

/* ------------------------------------------------------------------------
 * Groups: several handles (streams of uneven frame sizes, window lengths and
 * transforms) stepped together. The paper runs one camera stream through the
 * pipeline of Sec. III-B (ingest, spatial demodulation, time queue, temporal
 * analysis); a group runs that pipeline for every member in one launch.
 *
 * With use_graph = 1, each hv_render_group call captures the whole batch
 * into one CUDA graph: every member's frame copies and kernels on its own
 * branch, the branches running concurrently. The graph is then launched once
 * on the group's stream. The executable graph is kept and updated in place
 * while the batch keeps its shape; a batch of another shape re-instantiates
 * it. With use_graph = 0, the same work is issued directly on each member's
 * stream (the plain form).
 * ------------------------------------------------------------------------ */
typedef struct hv_group hv_group;

/* Counters of a group. */
typedef struct {
  uint64_t steps;                /* hv_render_group calls that launched work     */
  uint64_t graph_launches;       /* graph launches (use_graph = 1)               */
  uint64_t graph_instantiations; /* executable graphs built from scratch         */
  uint64_t graph_updates;        /* executable graphs updated in place           */
  uint64_t kernel_launches;      /* kernels enqueued by the members, all steps   */
  double capture_us_last;        /* host time of the last capture + update       */
} hv_group_stats;

/* Creates a group over n >= 1 open handles (all on the same device, each with
 * settings, each appearing once). `stream` (cudaStream_t or NULL) is the
 * group's stream: graphs launch on it, and it is ordered after the members'
 * earlier work. The group does not own the handles; close it before them.
 * Errors: HV_ERR_ARG (NULL, n = 0, a repeated handle, another device),
 * HV_ERR_CUDA. */
hv_status hv_group_open(hv_handle* const* handles, uint32_t n, void* stream, int use_graph, hv_group** out);

/* One batch for every member i: copies n_frames[i] raw frames from the
 * device pointer frames[i] (NULL when n_frames[i] = 0) into the member's
 * input queue, then renders every complete window of member i into the
 * device buffer outs[i] (capacity out_capacity_floats[i] floats), as
 * hv_push_frames + hv_render would. n_windows[i] receives the windows
 * rendered. Work is asynchronous: it completes on the group's stream, which
 * every member's stream then waits for.
 *
 * Pending settings are applied first (this may synchronise and autotune). A
 * member with profiling on, with PCA over T > 64 frames (its cooperative
 * eigensolver launch), or whose copies would overflow its input queue,
 * makes the call fail before any work is issued.
 * Errors: HV_ERR_ARG, HV_ERR_STATE, HV_ERR_QUEUE_FULL, HV_ERR_UNSUPPORTED,
 * HV_ERR_CUDA (the text is on hv_group_last_error). */
hv_status hv_render_group(hv_group* g, const void* const* frames, const uint32_t* n_frames, float* const* outs,
                          const size_t* out_capacity_floats, uint32_t* n_windows);

/* Counters of the group. */
hv_status hv_group_get_stats(const hv_group* g, hv_group_stats* s);

/* Text of the group's last error. */
const char* hv_group_last_error(const hv_group* g);

/* Waits for the group's work, frees the graph and the group (NULL: no-op). */
hv_status hv_group_close(hv_group* g);

/* Maximum n * width * height of one hv_spatial_static call (12 frames of
 * 256 x 256, or 3 of 512 x 512). */
#define HV_STATIC_MAX_PIXELS 786432u

/* Spatial transform of n frames that allocates nothing -- for callers that may
 * not call cudaMalloc/cudaFree where they run (allocator or memory-pool
 * callbacks, plugins inside a host framework that owns all device memory,
 * real-time loops that must never enter the allocator). The paper has no
 * counterpart; it is the same transform as HV_TEMPORAL_NONE rendering.
 *
 * `frames`: device pointer to n raw frames (uint8 or uint16 by pixel_bits),
 * p->width x p->height, row-major, contiguous; 2-byte aligned for 16-bit
 * pixels. `out`: device pointer to n * width * height complex values (2 floats
 * each, re then im), 8-byte aligned. Only the spatial fields of `p` are read
 * (width, height, spatial, z_m, lambda_m, pitch_x_m, pitch_y_m, fftshift,
 * highpass_cpp). Work is queued on `stream` (NULL = the default stream); the
 * caller keeps ownership of both buffers.
 *
 * Scratch (tables and the intermediates of the 2-D FFT passes, about 14 MiB)
 * is a file-scope __device__ array that every GPU loading the library holds
 * until exit. The first call on a device -- and the first call after the
 * current driver context changed, e.g. after cudaDeviceReset -- resolves that
 * array's device address (cudaGetSymbolAddress, with the device current);
 * make that call before any stream capture. Every call shares the array and
 * leaves its contents behind; nothing in it needs to start at zero. Calls
 * whose GPU work may overlap race on it, so order them on one stream or with
 * events.
 *
 * Errors: HV_ERR_ARG for NULL pointers, misaligned pointers, n = 0, width or
 * height not a power of two in [16, 512], n * width * height >
 * HV_STATIC_MAX_PIXELS, invalid optics, or a high-pass cutoff with a transform
 * other than ASP; HV_ERR_CUDA if a CUDA call fails, or if a CUDA error was
 * already pending on the calling thread when the call began (it is left
 * pending for the caller). No error text is recorded. */
hv_status hv_spatial_static(const void* frames, uint32_t pixel_bits, uint32_t n, const hv_params* p,
                            float* out, void* stream);

/* Text of the handle's last error (or of the last failed hv_open when h is
 * NULL). Valid until the next call on the handle. */
const char* hv_last_error(const hv_handle* h);

/* Measured arithmetic peaks of a device: FP32 and FP64 fused multiply-add
 * throughput (2 flop per FMA) of kernels that do nothing else, timed with CUDA
 * events on `stream` (NULL: the legacy default stream; best of five launches,
 * about 60 ms, synchronous).
 * They serve as the roofline denominators of ALU-bound kernels.
 * Errors: HV_ERR_ARG, HV_ERR_NOMEM, HV_ERR_CUDA. */
typedef struct {
  double fp32_tflops;
  double fp64_tflops;
  int sm_count;
  int sm_clock_khz; /* maximum SM clock the device reports */
} hv_peaks;
hv_status hv_probe_peaks(int device, void* stream, hv_peaks* out);

/* Version string of the library. */
const char* hv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HV_H */
