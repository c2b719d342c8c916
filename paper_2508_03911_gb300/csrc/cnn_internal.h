// cnn_internal.h -- the autofocus network's device state and launchers (k_cnn.cu),
// shared with the C ABI (af_api.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hv {
namespace cnn {

// Offsets of the tensors in the flat parameter vector (float32).
constexpr int OFF_W1 = 0, OFF_B1 = 144, OFF_W2 = 160, OFF_B2 = 4768, OFF_W3 = 4800, OFF_B3 = 23232,
              OFF_W4 = 23296, OFF_B4 = 60160, OFF_F1W = 60224, OFF_F1B = 62272, OFF_F2W = 62304,
              OFF_F2B = 62336, NPARAMS = 62337;
constexpr int IN_SIDE = 128;

// Device buffers of one network (sizes for max_batch images).
struct Net {
  float* prm;               // NPARAMS float32 parameters
  __nv_bfloat16* prm_bf;    // bfloat16 mirror (the convolutions read their weights here)
  float* grad;              // NPARAMS gradient of the last backward pass
  float* m;                 // Adam first moment
  float* v;                 // Adam second moment
  __nv_bfloat16* a1;        // [n][16][64][64]
  __nv_bfloat16* a2;        // [n][32][32][32]
  __nv_bfloat16* a3;        // [n][64][16][16]
  __nv_bfloat16* a4;        // [n][64][8][8]
  float* dbuf0;             // [n][32][32][32] floats (dZ4, then dZ2)
  float* dbuf1;             // [n][16][64][64] floats (dZ3, then dZ1)
  float* head;              // [n][130] head scratch
  float* part;              // weight-gradient partials, dw_part_floats(dw_chunks)
  float* partb;             // [dw_chunks][64] bias-gradient partials
  uint32_t dw_chunks;       // pixel chunks of the weight-gradient reduction
  unsigned* err;            // device flags: bit 2 set when a tensor-core convolution gave up a bounded wait
};

// y = relu(conv3x3_stride2(x, w) + b) for [n][CI][HI][HI] bfloat16 inputs on the
// tensor cores (k_conv_tc.cu); instantiated for the network's layers 2-4.
template <int CI, int CO, int HI>
cudaError_t conv_tc(const __nv_bfloat16* x, const __nv_bfloat16* w, const float* bias, __nv_bfloat16* y,
                    uint32_t n, unsigned* err, cudaStream_t s);

// Forward pass of n inputs x (bfloat16 [n][1][128][128]). zout (optional):
// predicted distances in metres. ztarget (optional, metres): also computes the
// loss terms and the gradient at the pooled layer (dZ4), ready for net_backward.
cudaError_t net_forward(const Net& t, const void* x, uint32_t n, const float* ztarget, float* zout, cudaStream_t s);
// Backward pass after net_forward with targets: gradient of the batch-mean loss
// into t.grad, the loss into *loss (device, optional).
cudaError_t net_backward(const Net& t, const void* x, uint32_t n, float* loss, cudaStream_t s);
// One Adam update from t.grad; c1 = 1 / (1 - b1^step), c2 = 1 / (1 - b2^step).
cudaError_t net_adam(const Net& t, float lr, float b1, float b2, float eps, float c1, float c2, cudaStream_t s);
// Refresh the bfloat16 mirror from the float32 parameters.
cudaError_t net_sync_bf16(const Net& t, cudaStream_t s);
size_t dw_part_floats(uint32_t nchunks);

}  // namespace cnn
}  // namespace hv
