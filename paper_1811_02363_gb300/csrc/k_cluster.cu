// Bisecting K-means (placeholder until the clustering kernel lands).
#include "hdf_internal.cuh"

namespace hdf {

size_t cluster_workspace_bytes(int N, int rho, int K) { return 256; }

cudaError_t launch_cluster(hdf_handle*, const void*, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace hdf
