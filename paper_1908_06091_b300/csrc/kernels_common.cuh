// kernels_common.cuh -- device helpers shared by the library's kernel files.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace nb {

int cuda_fail(cudaError_t e, const char *what);
void count_launch(int n);

#define NB_CUDA(call)                                       \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return ::nb::cuda_fail(_e, #call); \
  } while (0)

// Compensated (Kahan) accumulation.  add_prod forms the product w * d and
// subtracts the running correction in one FMA, so each term costs one FFMA
// and three FADD; the final value is s - c.
struct KahanAcc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_prod(float w, float d) {
    const float y = __fmaf_rn(w, d, -c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ void add(float y0) {
    const float y = __fsub_rn(y0, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ float value() const { return __fsub_rn(s, c); }
};

// Plain FP32 FMA chain (comparison mode).
struct PlainAcc {
  float s = 0.f;
  __device__ __forceinline__ void add_prod(float w, float d) { s = __fmaf_rn(w, d, s); }
  __device__ __forceinline__ void add(float y) { s = __fadd_rn(s, y); }
  __device__ __forceinline__ float value() const { return s; }
};

int launch_direct(const nb_method *m, int op, const nb_field *in, const nb_field *out,
                  cudaStream_t st);

}  // namespace nb
