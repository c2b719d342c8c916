/* hv_af.h -- the learned autofocus network: a small CNN that proposes the
 * propagation distance z of a hologram from its log-spectrum, trained on the
 * GPU by the library's own forward and backward kernels.
 *
 * The paper propagates to a distance the user sets (Sec. III-B.1) and has no
 * autofocus. The network replaces a plain z-sweep (hv_focus_sweep in hv.h:
 * angular-spectrum propagation to 64 distances, Tamura coefficient of each
 * image, the best distance as label), which also generates its training labels
 * and measures its error.
 *
 * Input: the network input of hv_af_features (hv.h), bfloat16 [n][1][128][128]
 * (raw 16-bit patterns), in device memory.
 * Network: four 3 x 3 convolutions with stride 2 and zero padding 1 (channels
 * 1 -> 16 -> 32 -> 64 -> 64), each with ReLU; global average pool; dense
 * 64 -> 32 with ReLU; dense 32 -> 1. The output y is the normalised distance:
 * z = 0.35 + 0.25 y metres. Loss: the batch mean of (y - (z_target - 0.35) /
 * 0.25)^2.
 * Arithmetic: activations and convolution weights in bfloat16 (the weights are
 * a rounded copy of the float32 parameters), products accumulated in float32;
 * dense layers, gradients and Adam in float32.
 * Parameters: HV_AF_NPARAMS float32 values, in this order: w1 [16][1][3][3],
 * b1 [16], w2 [32][16][3][3], b2 [32], w3 [64][32][3][3], b3 [64],
 * w4 [64][64][3][3], b4 [64], f1w [32][64], f1b [32], f2w [1][32], f2b [1].
 *
 * Every call returns an hv_status (hv.h); work is queued on the network's
 * stream and the device pointers must stay valid until it completes. */
#ifndef HV_AF_H
#define HV_AF_H

#include <stddef.h>
#include <stdint.h>

#include "hv.h"

#ifdef __cplusplus
extern "C" {
#endif

#define HV_AF_NPARAMS 62337u
#define HV_AF_SIDE 128u

typedef struct hv_af hv_af;

typedef struct {
  uint32_t struct_size; /* sizeof(hv_af_desc)                                        */
  int device;           /* CUDA device ordinal                                       */
  uint32_t max_batch;   /* largest n of any call (1 .. 4096)                          */
  uint32_t reserved;
  void* stream;         /* cudaStream_t to use, or NULL for a stream of its own       */
} hv_af_desc;

typedef struct {
  float lr;    /* step size                        */
  float beta1; /* first-moment decay (e.g. 0.9)    */
  float beta2; /* second-moment decay (e.g. 0.999) */
  float eps;   /* denominator floor (e.g. 1e-8)    */
} hv_af_adam;

/* Allocates the network's buffers for max_batch images (about 0.7 MB per image)
 * with zero parameters. Errors: HV_ERR_ARG, HV_ERR_NOMEM, HV_ERR_CUDA. */
hv_status hv_af_open(const hv_af_desc* desc, hv_af** out);

/* Sets the float32 parameters from host memory (n must be HV_AF_NPARAMS) and
 * resets the Adam state (moments zero, step count zero). Errors: HV_ERR_ARG,
 * HV_ERR_CUDA. */
hv_status hv_af_set_params(hv_af* af, const float* params, size_t n);

/* Copies the float32 parameters to host memory (waits for the stream). */
hv_status hv_af_get_params(hv_af* af, float* params, size_t n);

/* Inference: z_out[i] (device float array, metres) for the n inputs x.
 * Errors: HV_ERR_ARG (NULL, n = 0 or n > max_batch), HV_ERR_CUDA. */
hv_status hv_af_forward(hv_af* af, const void* x_bf16, uint32_t n, float* z_out);

/* Loss of the n inputs against the target distances z_target (device floats,
 * metres) into *loss (device float), and its gradient with respect to the
 * parameters into grad (device, HV_AF_NPARAMS floats; NULL to skip the copy).
 * The parameters do not change. Errors as hv_af_forward. */
hv_status hv_af_loss_grad(hv_af* af, const void* x_bf16, const float* z_target, uint32_t n, float* loss,
                          float* grad);

/* One training step: forward, backward, and one Adam update of every parameter
 * (bias-corrected with the network's step count, which this call advances).
 * *loss (device float, optional) receives the loss before the update.
 * Errors as hv_af_forward. */
hv_status hv_af_train_step(hv_af* af, const void* x_bf16, const float* z_target, uint32_t n,
                           const hv_af_adam* adam, float* loss);

/* Waits for the network's work on its stream. Returns HV_ERR_CUDA if a
 * tensor-core convolution gave up a bounded wait (about two seconds; the flag is
 * sticky and the outputs of that call are not valid). */
hv_status hv_af_synchronize(hv_af* af);

/* Text of the network's last error. */
const char* hv_af_last_error(const hv_af* af);

/* Waits for the network's work and frees it (NULL: no-op). */
hv_status hv_af_close(hv_af* af);

#ifdef __cplusplus
}
#endif
#endif /* HV_AF_H */
