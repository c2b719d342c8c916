// k_probe.cu -- measured arithmetic peaks of the device: fused multiply-add
// throughput in FP32 and FP64 from kernels that do nothing else (8 independent
// accumulator chains per thread, 8 CTAs of 256 threads per SM), the best of five
// launches timed with CUDA events. They are the roofline denominators of the ALU-bound kernels (the FFTs,
// the Jacobi sweeps), where no library routine gives the figure.
#include <cuda_runtime.h>

#include "../../include/hv.h"

namespace {

template <typename F>
__global__ void __launch_bounds__(256) k_fma(F* out, int iters, F m, F c) {
  F a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = F(threadIdx.x) * F(1e-6) + F(k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = a[k] * m + c;  // contracted to one FMA
  }
  F s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == F(-1)) out[blockIdx.x] = s;  // never true; keeps the chains live
}

// Best of five timed launches (after one warm-up launch): the burst rate.
template <typename F>
cudaError_t time_fma(cudaStream_t st, int nsm, int iters, F* buf, double* tflops) {
  const int blocks = nsm * 8;
  cudaEvent_t ev[6] = {};
  cudaError_t e = cudaSuccess;
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  if (e == cudaSuccess) k_fma<F><<<blocks, 256, 0, st>>>(buf, iters / 4, F(0.999999), F(1e-7));  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
  for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
    k_fma<F><<<blocks, 256, 0, st>>>(buf, iters, F(0.999999), F(1e-7));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev[r + 1], st);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[5]);
  float best = 0.f;
  for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ev[r], ev[r + 1]);
    if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) *tflops = 2.0 * 8.0 * double(iters) * blocks * 256 / (double(best) * 1e-3) / 1e12;
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  return e;
}

}  // namespace

extern "C" hv_status hv_probe_peaks(int device, void* stream, hv_peaks* out) {
  if (!out) return HV_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return HV_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int nsm = 0, clk = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device) != cudaSuccess)
    return HV_ERR_CUDA;
  void* buf = nullptr;
  if (cudaMalloc(&buf, size_t(nsm) * 8 * sizeof(double)) != cudaSuccess) return HV_ERR_NOMEM;
  hv_peaks p{};
  p.sm_count = nsm;
  p.sm_clock_khz = clk;
  cudaError_t e = time_fma<float>(st, nsm, 1 << 15, static_cast<float*>(buf), &p.fp32_tflops);
  if (e == cudaSuccess) e = time_fma<double>(st, nsm, 1 << 10, static_cast<double*>(buf), &p.fp64_tflops);
  cudaFree(buf);
  if (e != cudaSuccess) return HV_ERR_CUDA;
  *out = p;
  return HV_OK;
}
