// Clustering kernel instantiated for guides of up to 64 dimensions.
#include "cluster_kernel.cuh"

namespace hdf {

cudaError_t launch_cluster_r64(const clus::ClArgs& a, int G, cudaStream_t st) {
  return clus::launch_cl<64>(a, G, st);
}

}  // namespace hdf
