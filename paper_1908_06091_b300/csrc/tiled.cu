// tiled.cu -- shared-memory staged variant of the nabla kernels (placeholder
// dispatcher until the staged kernels land: every call falls through to the
// direct kernels).
#include "kernels_common.cuh"

namespace nb {

int launch_tiled(nb_method *, int, const nb_field *, const nb_field *, cudaStream_t,
                 bool *handled) {
  *handled = false;
  return NB_OK;
}

}  // namespace nb
