// Backward pass (placeholder until the adjoint kernels land).
#include "hdf_internal.cuh"

namespace hdf {

cudaError_t launch_backward(hdf_handle*, const float*, const void*, const float*, float*, double*,
                            cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace hdf
