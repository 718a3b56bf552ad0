// Backward tile kernels for window half-widths 3, 6, 9, 12.
#include "bwd_tile.cuh"

namespace hdf {

cudaError_t launch_bwd_group_a(int SB, int mode, const BwdArgs& a, const Taps& t1, const Taps& t2,
                               cudaStream_t st) {
  if (mode == MODE_GAMMA) {
    switch (SB) {
      case 3: return launch_bwd_tile<3, MODE_GAMMA, 64>(a, t1, t2, st);
      case 6: return launch_bwd_tile<6, MODE_GAMMA, 64>(a, t1, t2, st);
      case 9: return launch_bwd_tile<9, MODE_GAMMA, 64>(a, t1, t2, st);
      case 12: return launch_bwd_tile<12, MODE_GAMMA, 64>(a, t1, t2, st);
    }
  } else {
    switch (SB) {
      case 3: return launch_bwd_tile<3, MODE_ADJ, 64>(a, t1, t2, st);
      case 6: return launch_bwd_tile<6, MODE_ADJ, 64>(a, t1, t2, st);
      case 9: return launch_bwd_tile<9, MODE_ADJ, 64>(a, t1, t2, st);
      case 12: return launch_bwd_tile<12, MODE_ADJ, 64>(a, t1, t2, st);
    }
  }
  return cudaErrorNotSupported;
}

}  // namespace hdf
