// noalloc.cu -- Laplacian entry point that allocates no memory.
//
// Some callers cannot allocate device memory once they are running: a
// component embedded in a larger model that owns a fixed device-memory
// budget set at start-up, or a latency-critical loop in which cudaMalloc /
// cudaFree (which may synchronise the whole device) are not allowed.  The
// Laplacian needs an intermediate gradient field, so for these callers it
// is kept in a fixed-size array that is part of the library image.  Under
// the CUDA runtime's default lazy module loading, a device takes the array's
// NB_NOALLOC_SCRATCH_BYTES when the first call runs on it (the address
// lookup below loads the module); it keeps them until the process exits.
// Callers make that first call at start-up, inside their memory budget.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels_common.cuh"

namespace nb {

int validate_op(const nb_method *m, int op, const nb_field *in, const nb_field *out,
                const nb_field *scratch);

// The intermediate gradient of nb_nabla_laplacian_noalloc.  Device code may
// name it directly; host code must not pass its name to a kernel (on the host
// it is only a stand-in, not a device address) and uses the address looked
// up below instead.
static __device__ __align__(256) unsigned char g_lap_scratch[NB_NOALLOC_SCRATCH_BYTES];

// Device address of g_lap_scratch, looked up once per device with that
// device current.
static int scratch_address(void **out) {
  static std::mutex mu;
  static void *addr[64] = {};
  int dev = 0;
  NB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("nb_nabla_laplacian_noalloc: device index out of range");
    return NB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    NB_CUDA(cudaGetSymbolAddress(&p, g_lap_scratch));
    addr[dev] = p;
  }
  *out = addr[dev];
  return NB_OK;
}

}  // namespace nb

extern "C" int nb_nabla_laplacian_noalloc(const nb_method *m, const nb_field *f,
                                          const nb_field *lap, void *stream) {
  int st = nb::validate_op(m, NB_OP_LAP, f, lap, nullptr);
  if (st != NB_OK) return st;
  // intermediate gradient: [V][Lq][2] with Lq = nlev rounded up to a multiple
  // of 4 (FP32) or 2 (FP64), the padded stride a functionspace reports
  const int64_t elem = f->dtype == NB_F64 ? 8 : 4;
  const int q = f->dtype == NB_F64 ? 2 : 4;
  const int64_t stride = 2 * (int64_t)((f->nlev + q - 1) / q) * q;
  const int64_t need = stride * f->nnodes * elem;
  if (need > (int64_t)NB_NOALLOC_SCRATCH_BYTES) {
    nb::set_error("nb_nabla_laplacian_noalloc: the intermediate gradient needs " +
                  std::to_string(need) + " bytes, more than the fixed " +
                  std::to_string((long long)NB_NOALLOC_SCRATCH_BYTES) +
                  "-byte scratch; use nb_nabla_laplacian with a caller scratch field");
    return NB_ESHAPE;
  }
  void *base = nullptr;
  if ((st = nb::scratch_address(&base)) != NB_OK) return st;
  nb_field tmp = *f;
  tmp.data = base;
  tmp.nvar = 2;
  tmp.node_stride = stride;
  tmp.lev_stride = 2;
  // The gradient pass writes every value the divergence pass reads, so
  // nothing in the scratch has to start at zero.  Direct kernels only: they
  // allocate nothing (the staged kernels build their tile plans on first use).
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (m->mesh->V == 0) return NB_OK;
  st = nb::launch_direct(m, NB_OP_GRAD, f, &tmp, s);
  if (st == NB_OK) st = nb::launch_direct(m, NB_OP_DIV, &tmp, lap, s);
  return st;
}
