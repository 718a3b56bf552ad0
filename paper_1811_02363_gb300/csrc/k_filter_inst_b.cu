// Instantiations of the fused tile kernel for window half-width 15.
#include "filter_tile.cuh"

namespace hdf {

cudaError_t launch_filter_group_b(int SB, int P, const FilterArgs& a, const Taps& t,
                                  cudaStream_t st) {
  if (SB == 15) {
    if (P == 4) return launch_filter_tile<15, 4, 64>(a, t, st);
    return launch_filter_tile<15, 2, 64>(a, t, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace hdf
