// Instantiations of the fused tile kernel for window half-widths 3, 6, 9, 12.
#include "filter_tile.cuh"

namespace hdf {

cudaError_t launch_filter_group_a(int SB, int P, const FilterArgs& a, const Taps& t,
                                  cudaStream_t st) {
  if (P == 4) {
    switch (SB) {
      case 3: return launch_filter_tile<3, 4, 64>(a, t, st);
      case 6: return launch_filter_tile<6, 4, 64>(a, t, st);
      case 9: return launch_filter_tile<9, 4, 64>(a, t, st);
      case 12: return launch_filter_tile<12, 4, 64>(a, t, st);
    }
  } else {
    switch (SB) {
      case 3: return launch_filter_tile<3, 2, 64>(a, t, st);
      case 6: return launch_filter_tile<6, 2, 64>(a, t, st);
      case 9: return launch_filter_tile<9, 2, 64>(a, t, st);
      case 12: return launch_filter_tile<12, 2, 64>(a, t, st);
    }
  }
  return cudaErrorNotSupported;
}

}  // namespace hdf
