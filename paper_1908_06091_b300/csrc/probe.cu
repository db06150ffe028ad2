// probe.cu -- the FP64 rate that the FP64 operator path is measured against.
//
// On B300 the FP64 operators are bound by the FP64 units, not by HBM, so
// their roofline is the device's FP64 FMA rate.  It is measured here on the
// same GPU: every thread runs kChains independent FMA chains in registers
// (enough independent work to hide the FMA latency) for `iters` steps, two
// flops per FMA, on a grid of four CTAs per SM.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"
#include "kernels_common.cuh"

namespace nb {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) fp64_fma_chains(int64_t iters, double a, double b,
                                                                 double *sink) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (sink != nullptr && s == -1.0) sink[0] = s;  // never true (sink is NULL); keeps the chains live
}

}  // namespace nb

extern "C" int nb_probe_fp64_rate(int64_t iters, void *stream, double *tflops, double *ms) {
  if (!tflops || !ms || iters < 1 || iters > (int64_t)1 << 30) {
    nb::set_error("nb_probe_fp64_rate: NULL output or iters outside [1, 2^30]");
    return NB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  NB_CUDA(cudaGetDevice(&dev));
  NB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = 4 * sms;
  // x -> x a + b with a slightly below 1 keeps every chain bounded
  const double a = 0.999999, b = 1e-6;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  NB_CUDA(cudaEventCreate(&e0));
  NB_CUDA(cudaEventCreate(&e1));
  nb::fp64_fma_chains<<<grid, nb::kProbeThreads, 0, st>>>(iters / 8 + 1, a, b, nullptr);  // warm-up
  nb::count_launch(1);
  cudaEventRecord(e0, st);
  nb::fp64_fma_chains<<<grid, nb::kProbeThreads, 0, st>>>(iters, a, b, nullptr);
  nb::count_launch(1);
  cudaEventRecord(e1, st);
  const cudaError_t err = cudaEventSynchronize(e1);
  float t = 0.f;
  if (err == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  NB_CUDA(err);
  NB_CUDA(cudaGetLastError());
  const double fmas = (double)grid * nb::kProbeThreads * nb::kChains * (double)iters;
  *ms = t;
  *tflops = t > 0 ? 2.0 * fmas / (t * 1e-3) / 1e12 : 0.0;
  return NB_OK;
}
