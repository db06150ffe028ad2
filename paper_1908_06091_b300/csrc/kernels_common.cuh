// kernels_common.cuh -- device helpers shared by the library's kernel files.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace nb {

int cuda_fail(cudaError_t e, const char *what);
void count_launch(int n);
// device address of the status word on the current device (tiled.cu)
int status_word(int **out);

#define NB_CUDA(call)                                       \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return ::nb::cuda_fail(_e, #call); \
  } while (0)

// Index checks of the bounds-checked build (-DNB_BOUNDS_CHECK): an index
// outside [lo, hi) records NB_EINVAL in the device status word and is
// replaced by lo, so that no access leaves its buffer; the host sees the
// error after synchronising (nb_device_status).  Other builds compile the
// check away.
#ifdef NB_BOUNDS_CHECK
__device__ __forceinline__ int64_t nb_checked_index(int64_t x, int64_t lo, int64_t hi, int *status) {
  if (x >= lo && x < hi) return x;
  if (status) atomicCAS(status, 0, (int)NB_EINVAL);
  return lo;
}
#define NB_IDX(x, lo, hi, status) nb_checked_index((x), (lo), (hi), (status))
#else
#define NB_IDX(x, lo, hi, status) (x)
#endif

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

// Load LPT consecutive values of a scalar column starting at level l0;
// values at levels >= nlev are returned as 0 and never read past the row.
template <int LPT>
__device__ __forceinline__ void load_scalar_f32(const float *col, int l0, int nlev, float (&v)[LPT]) {
  if constexpr (LPT == 4) {
    if (l0 < nlev) {
      const float4 x = __ldg(reinterpret_cast<const float4 *>(col + l0));
      v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
      v[0] = v[1] = v[2] = v[3] = 0.f;
    }
  } else {
#pragma unroll
    for (int k = 0; k < LPT; ++k) v[k] = (l0 + k < nlev) ? __ldg(col + l0 + k) : 0.f;
  }
}
// Load LPT levels of a (u, v) column.
template <int LPT>
__device__ __forceinline__ void load_vector_f32(const float *col, int l0, int nlev, float (&u)[LPT],
                                                float (&v)[LPT]) {
  if constexpr (LPT == 4) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (l0 + 2 * h < nlev) {
        const float4 x = __ldg(reinterpret_cast<const float4 *>(col + 2 * (l0 + 2 * h)));
        u[2 * h] = x.x; v[2 * h] = x.y; u[2 * h + 1] = x.z; v[2 * h + 1] = x.w;
      } else {
        u[2 * h] = v[2 * h] = u[2 * h + 1] = v[2 * h + 1] = 0.f;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      if (l0 + k < nlev) {
        u[k] = __ldg(col + 2 * (l0 + k));
        v[k] = __ldg(col + 2 * (l0 + k) + 1);
      } else {
        u[k] = v[k] = 0.f;
      }
    }
  }
}

int launch_direct(const nb_method *m, int op, const nb_field *in, const nb_field *out,
                  cudaStream_t st, const void *q = nullptr, int64_t q_stride = 0);
int launch_edge(nb_method *m, int op, const nb_field *in, const nb_field *out, cudaStream_t st);

}  // namespace nb
