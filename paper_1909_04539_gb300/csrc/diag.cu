// Measurement aid: the device's sustained FP64 fused-multiply-add rate, the
// ceiling of the sweeps that run in native FP64 arithmetic.
#include "internal.h"

namespace bs {

constexpr int kDiagChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma_rate(double* sink, int iters, double s) {
  double a[kDiagChains];
#pragma unroll
  for (int c = 0; c < kDiagChains; c++) a[c] = threadIdx.x * 1e-3 + c;
  for (int k = 0; k < iters; k++)
#pragma unroll
    for (int c = 0; c < kDiagChains; c++) a[c] = fma(a[c], s, 0.5);
  double t = 0.0;
#pragma unroll
  for (int c = 0; c < kDiagChains; c++) t += a[c];
  if (t == 12345.678) sink[0] = t;  // keeps the chains live; never true for these inputs
}

}  // namespace bs

extern "C" bs_status bs_measure_fp64_rate(double* fma_per_s, bs_stream stream) {
  using namespace bs;
  if (!fma_per_s) return set_error(BS_EINVAL, "bs_measure_fp64_rate: null output");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const DeviceInfo& d = device_info();
  const int blocks = d.sms * 8, threads = 256, iters = 2048;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  if (e == cudaSuccess) {
    k_fp64_fma_rate<<<blocks, threads, 0, st>>>(sink, iters / 4, 0.999);  // warm-up
    cudaEventRecord(e0, st);
    k_fp64_fma_rate<<<blocks, threads, 0, st>>>(sink, iters, 0.999);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return cuda_error(e, "bs_measure_fp64_rate");
  *fma_per_s = (double)blocks * threads * iters * kDiagChains / (ms * 1e-3);
  return BS_OK;
}
