// Clustering kernel instantiated for guides of up to 4 dimensions.
#define HDF_CL_THREADS 512   // threads per block of this instantiation
#include "cluster_kernel.cuh"

namespace hdf {

cudaError_t launch_cluster_r4(const clus::ClArgs* table, const int4* groups, int ngroups,
                              const int* order, const void* p_override, int rho_max, int grid,
                              unsigned long long wait_ns, cudaStream_t st) {
  return clus::launch_cl<4>(table, groups, ngroups, order, p_override, rho_max, grid, wait_ns, st);
}

}  // namespace hdf
