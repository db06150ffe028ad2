// reduce.cu -- NodeColumns reductions over the nodes of a field (Sec. 4.5:
// global minimum, maximum and mean values), per level and component, plus
// the dual-volume (area) weighted mean and root mean square used as error
// norms.  Two deterministic passes: CTA b reduces a fixed node range into
// partials[b][k] (k = level * nvar + component) in FP64, then one thread per
// k combines the partials in CTA order.  Nothing depends on scheduling, so
// repeated calls give identical results.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <string>

#include "internal.h"
#include "kernels_common.cuh"

namespace nb {

constexpr int kReduceThreads = 256;
constexpr int kReduceBlocks = 296;  // two CTAs per SM on 148 SMs

// kind: NB_REDUCE_* ; w: dual volumes (area kinds) or nullptr.  Thread t of
// CTA b walks nodes b, b + B, ... for value slot k = t, t + 256, ... < nk.
template <class T>
__global__ void __launch_bounds__(kReduceThreads) reduce_partial_kernel(
    const T *__restrict__ x, int64_t V, int64_t node_stride, int nlev, int nvar, int kind,
    const double *__restrict__ vol, double *__restrict__ partial) {
  const int nk = nlev * nvar;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    const int l = k / nvar, c = k - l * nvar;
    double acc = kind == NB_REDUCE_MIN ? DBL_MAX : kind == NB_REDUCE_MAX ? -DBL_MAX : 0.0;
    for (int64_t i = blockIdx.x; i < V; i += gridDim.x) {
      const double v = (double)x[i * node_stride + (int64_t)l * nvar + c];
      switch (kind) {
        case NB_REDUCE_MIN: acc = fmin(acc, v); break;
        case NB_REDUCE_MAX: acc = fmax(acc, v); break;
        case NB_REDUCE_SUM: acc += v; break;
        case NB_REDUCE_AREA_MEAN: acc = fma(vol[i], v, acc); break;
        default: acc = fma(vol[i] * v, v, acc); break;  // NB_REDUCE_AREA_RMS
      }
    }
    partial[(int64_t)blockIdx.x * nk + k] = acc;
  }
}

__global__ void reduce_final_kernel(const double *__restrict__ partial, int nblocks, int nk, int kind,
                                    double norm, double *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  double acc = kind == NB_REDUCE_MIN ? DBL_MAX : kind == NB_REDUCE_MAX ? -DBL_MAX : 0.0;
  for (int b = 0; b < nblocks; ++b) {
    const double v = partial[(int64_t)b * nk + k];
    if (kind == NB_REDUCE_MIN) acc = fmin(acc, v);
    else if (kind == NB_REDUCE_MAX) acc = fmax(acc, v);
    else acc += v;
  }
  if (kind == NB_REDUCE_AREA_MEAN) acc /= norm;
  if (kind == NB_REDUCE_AREA_RMS) acc = sqrt(acc / norm);
  out[k] = acc;
}

}  // namespace nb

extern "C" int nb_field_reduce(const nb_method *m, const nb_field *f, int kind, double *host_out,
                               void *stream) {
  using namespace nb;
  if (!m || !f || !host_out) {
    set_error("nb_field_reduce: NULL argument");
    return NB_EINVAL;
  }
  if (kind < NB_REDUCE_MIN || kind > NB_REDUCE_AREA_RMS) {
    set_error("nb_field_reduce: unknown reduction");
    return NB_EINVAL;
  }
  if (f->dtype != NB_F32 && f->dtype != NB_F64) {
    set_error("nb_field_reduce: unknown dtype");
    return NB_EDTYPE;
  }
  if (f->nnodes != m->mesh->V || f->nlev < 1 || (f->nvar != 1 && f->nvar != 2) || f->lev_stride != f->nvar ||
      f->node_stride < (int64_t)f->nlev * f->nvar || !f->data) {
    set_error("nb_field_reduce: field shape does not match the method's mesh");
    return NB_ESHAPE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nk = f->nlev * f->nvar;
  const DevAlloc alloc = current_allocator();
  void *partial = nullptr, *dout = nullptr;
  const size_t pbytes = (size_t)kReduceBlocks * nk * sizeof(double), obytes = (size_t)nk * sizeof(double);
  int rc = dev_alloc_async(alloc, &partial, pbytes, stream, "nb_field_reduce partials");
  if (rc != NB_OK) return rc;
  rc = dev_alloc_async(alloc, &dout, obytes, stream, "nb_field_reduce result");
  if (rc != NB_OK) {
    dev_free_async(alloc, partial, pbytes, stream);
    return rc;
  }
  double norm = m->area;  // total area
  const bool area = kind == NB_REDUCE_AREA_MEAN || kind == NB_REDUCE_AREA_RMS;
  const double *vol = area ? m->d_vol : nullptr;
  if (kind == NB_REDUCE_SUM) norm = 1.0;
  if (f->dtype == NB_F64)
    reduce_partial_kernel<double><<<kReduceBlocks, kReduceThreads, 0, st>>>(
        static_cast<const double *>(f->data), f->nnodes, f->node_stride, f->nlev, f->nvar, kind, vol,
        static_cast<double *>(partial));
  else
    reduce_partial_kernel<float><<<kReduceBlocks, kReduceThreads, 0, st>>>(
        static_cast<const float *>(f->data), f->nnodes, f->node_stride, f->nlev, f->nvar, kind, vol,
        static_cast<double *>(partial));
  reduce_final_kernel<<<(nk + 255) / 256, 256, 0, st>>>(static_cast<const double *>(partial), kReduceBlocks, nk,
                                                         kind, norm, static_cast<double *>(dout));
  count_launch(2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, dout, obytes, cudaMemcpyDeviceToHost, st);
  dev_free_async(alloc, partial, pbytes, stream);
  dev_free_async(alloc, dout, obytes, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "nb_field_reduce");
  return NB_OK;
}
