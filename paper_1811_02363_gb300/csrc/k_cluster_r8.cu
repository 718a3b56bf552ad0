// Clustering kernel instantiated for guides of up to 8 dimensions.
#include "cluster_kernel.cuh"

namespace hdf {

cudaError_t launch_cluster_r8(const clus::ClArgs& a, int G, cudaStream_t st) {
  return clus::launch_cl<8>(a, G, st);
}

}  // namespace hdf
