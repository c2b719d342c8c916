// af_api.cu -- the C ABI of the autofocus network (include/hv_af.h): device
// buffers, parameter upload, inference, gradients and the Adam training step.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/hv_af.h"
#include "cnn_internal.h"

using namespace hv::cnn;

struct hv_af {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint32_t max_batch = 0;
  Net t{};
  void* mem = nullptr;
  uint64_t step = 0;
  std::string err;
};

namespace {

hv_status af_fail(hv_af* a, hv_status s, const std::string& m) {
  if (a) a->err = m;
  return s;
}

#define AF_CU(a, call)                                                                                   \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) return af_fail(a, HV_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

hv_status check_batch(hv_af* a, const void* x, uint32_t n) {
  if (!x) return af_fail(a, HV_ERR_ARG, "input is NULL");
  if (n == 0 || n > a->max_batch) return af_fail(a, HV_ERR_ARG, "n must be in [1, max_batch]");
  return HV_OK;
}

}  // namespace

extern "C" {

hv_status hv_af_close(hv_af* a) {
  if (!a) return HV_OK;
  cudaSetDevice(a->device);
  if (a->stream) cudaStreamSynchronize(a->stream);
  if (a->mem) cudaFree(a->mem);
  if (a->own_stream && a->stream) cudaStreamDestroy(a->stream);
  delete a;
  return HV_OK;
}

hv_status hv_af_open(const hv_af_desc* d, hv_af** out) {
  if (!out) return HV_ERR_ARG;
  *out = nullptr;
  if (!d || d->struct_size != sizeof(hv_af_desc) || d->max_batch < 1 || d->max_batch > 4096) return HV_ERR_ARG;
  hv_af* a = new hv_af();
  a->device = d->device;
  a->max_batch = d->max_batch;
  auto bail = [&](hv_status s) {
    hv_af_close(a);
    return s;
  };
  if (cudaSetDevice(a->device) != cudaSuccess) return bail(HV_ERR_CUDA);
  if (d->stream) {
    a->stream = static_cast<cudaStream_t>(d->stream);
  } else {
    if (cudaStreamCreateWithFlags(&a->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(HV_ERR_CUDA);
    a->own_stream = true;
  }
  const size_t B = d->max_batch;
  Net& t = a->t;
  t.dw_chunks = 256;
  // one allocation, carved in 256-byte aligned pieces
  struct Piece {
    void** p;
    size_t bytes;
  } pieces[] = {
      {reinterpret_cast<void**>(&t.prm), NPARAMS * 4},
      {reinterpret_cast<void**>(&t.prm_bf), NPARAMS * 2},
      {reinterpret_cast<void**>(&t.grad), NPARAMS * 4},
      {reinterpret_cast<void**>(&t.m), NPARAMS * 4},
      {reinterpret_cast<void**>(&t.v), NPARAMS * 4},
      {reinterpret_cast<void**>(&t.a1), B * 16 * 64 * 64 * 2},
      {reinterpret_cast<void**>(&t.a2), B * 32 * 32 * 32 * 2},
      {reinterpret_cast<void**>(&t.a3), B * 64 * 16 * 16 * 2},
      {reinterpret_cast<void**>(&t.a4), B * 64 * 8 * 8 * 2},
      {reinterpret_cast<void**>(&t.dbuf0), B * 32 * 32 * 32 * 4},
      {reinterpret_cast<void**>(&t.dbuf1), B * 16 * 64 * 64 * 4},
      {reinterpret_cast<void**>(&t.head), B * 130 * 4},
      {reinterpret_cast<void**>(&t.part), dw_part_floats(t.dw_chunks) * 4},
      {reinterpret_cast<void**>(&t.partb), size_t(t.dw_chunks) * 64 * 4},
      {reinterpret_cast<void**>(&t.err), 16},
  };
  size_t total = 0;
  for (auto& p : pieces) total += (p.bytes + 255) / 256 * 256;
  if (cudaMalloc(&a->mem, total) != cudaSuccess) return bail(HV_ERR_NOMEM);
  char* c = static_cast<char*>(a->mem);
  for (auto& p : pieces) {
    *p.p = c;
    c += (p.bytes + 255) / 256 * 256;
  }
  if (cudaMemsetAsync(a->mem, 0, total, a->stream) != cudaSuccess) return bail(HV_ERR_CUDA);
  *out = a;
  return HV_OK;
}

hv_status hv_af_set_params(hv_af* a, const float* params, size_t n) {
  if (!a) return HV_ERR_ARG;
  if (!params || n != NPARAMS) return af_fail(a, HV_ERR_ARG, "expected HV_AF_NPARAMS host floats");
  AF_CU(a, cudaSetDevice(a->device));
  AF_CU(a, cudaMemcpyAsync(a->t.prm, params, NPARAMS * 4, cudaMemcpyHostToDevice, a->stream));
  AF_CU(a, cudaMemsetAsync(a->t.m, 0, NPARAMS * 4, a->stream));
  AF_CU(a, cudaMemsetAsync(a->t.v, 0, NPARAMS * 4, a->stream));
  AF_CU(a, net_sync_bf16(a->t, a->stream));
  AF_CU(a, cudaStreamSynchronize(a->stream));  // the host array may be reused on return
  a->step = 0;
  return HV_OK;
}

hv_status hv_af_get_params(hv_af* a, float* params, size_t n) {
  if (!a) return HV_ERR_ARG;
  if (!params || n != NPARAMS) return af_fail(a, HV_ERR_ARG, "expected HV_AF_NPARAMS host floats");
  AF_CU(a, cudaSetDevice(a->device));
  AF_CU(a, cudaMemcpyAsync(params, a->t.prm, NPARAMS * 4, cudaMemcpyDeviceToHost, a->stream));
  AF_CU(a, cudaStreamSynchronize(a->stream));
  return HV_OK;
}

hv_status hv_af_forward(hv_af* a, const void* x, uint32_t n, float* z_out) {
  if (!a) return HV_ERR_ARG;
  hv_status s = check_batch(a, x, n);
  if (s != HV_OK) return s;
  if (!z_out) return af_fail(a, HV_ERR_ARG, "z_out is NULL");
  AF_CU(a, cudaSetDevice(a->device));
  AF_CU(a, net_forward(a->t, x, n, nullptr, z_out, a->stream));
  return HV_OK;
}

hv_status hv_af_loss_grad(hv_af* a, const void* x, const float* z_target, uint32_t n, float* loss, float* grad) {
  if (!a) return HV_ERR_ARG;
  hv_status s = check_batch(a, x, n);
  if (s != HV_OK) return s;
  if (!z_target) return af_fail(a, HV_ERR_ARG, "z_target is NULL");
  AF_CU(a, cudaSetDevice(a->device));
  AF_CU(a, net_forward(a->t, x, n, z_target, nullptr, a->stream));
  AF_CU(a, net_backward(a->t, x, n, loss, a->stream));
  if (grad) AF_CU(a, cudaMemcpyAsync(grad, a->t.grad, NPARAMS * 4, cudaMemcpyDeviceToDevice, a->stream));
  return HV_OK;
}

hv_status hv_af_train_step(hv_af* a, const void* x, const float* z_target, uint32_t n, const hv_af_adam* adam,
                           float* loss) {
  if (!a) return HV_ERR_ARG;
  if (!adam) return af_fail(a, HV_ERR_ARG, "adam is NULL");
  hv_status s = hv_af_loss_grad(a, x, z_target, n, loss, nullptr);
  if (s != HV_OK) return s;
  ++a->step;
  const double c1 = 1.0 / (1.0 - std::pow(double(adam->beta1), double(a->step)));
  const double c2 = 1.0 / (1.0 - std::pow(double(adam->beta2), double(a->step)));
  AF_CU(a, net_adam(a->t, adam->lr, adam->beta1, adam->beta2, adam->eps, float(c1), float(c2), a->stream));
  return HV_OK;
}

hv_status hv_af_synchronize(hv_af* a) {
  if (!a) return HV_ERR_ARG;
  AF_CU(a, cudaSetDevice(a->device));
  AF_CU(a, cudaStreamSynchronize(a->stream));
  unsigned flags = 0;
  AF_CU(a, cudaMemcpy(&flags, a->t.err, sizeof(flags), cudaMemcpyDeviceToHost));
  if (flags != 0)
    return af_fail(a, HV_ERR_CUDA, "a tensor-core convolution gave up a bounded wait (flags " + std::to_string(flags) + ")");
  return HV_OK;
}

const char* hv_af_last_error(const hv_af* a) { return a ? a->err.c_str() : ""; }

}  // extern "C"
