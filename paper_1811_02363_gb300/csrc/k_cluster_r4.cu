// Clustering kernel instantiated for guides of up to 4 dimensions.
#include "cluster_kernel.cuh"

namespace hdf {

cudaError_t launch_cluster_r4(const clus::ClArgs& a, int G, cudaStream_t st) {
  return clus::launch_cl<4>(a, G, st);
}

}  // namespace hdf
