// Backward tile kernels for window half-widths 15, 18, 24, 32 (tile height 64;
// 32 for the widest bucket, where the two row-pass outputs of a 64-row tile
// would not fit in shared memory).
#include "bwd_tile.cuh"

namespace hdf {

cudaError_t launch_bwd_group_a(int, int, const BwdArgs&, const Taps&, const Taps&, cudaStream_t);

cudaError_t launch_bwd_sb(int SB, int mode, const BwdArgs& a, const Taps& t1, const Taps& t2,
                          cudaStream_t st) {
  if (SB <= 12) return launch_bwd_group_a(SB, mode, a, t1, t2, st);
  if (mode == MODE_GAMMA) {
    switch (SB) {
      case 15: return launch_bwd_tile<15, MODE_GAMMA, 64>(a, t1, t2, st);
      case 18: return launch_bwd_tile<18, MODE_GAMMA, 64>(a, t1, t2, st);
      case 24: return launch_bwd_tile<24, MODE_GAMMA, 64>(a, t1, t2, st);
      case 32: return launch_bwd_tile<32, MODE_GAMMA, 32>(a, t1, t2, st);
    }
  } else {
    switch (SB) {
      case 15: return launch_bwd_tile<15, MODE_ADJ, 64>(a, t1, t2, st);
      case 18: return launch_bwd_tile<18, MODE_ADJ, 64>(a, t1, t2, st);
      case 24: return launch_bwd_tile<24, MODE_ADJ, 64>(a, t1, t2, st);
      case 32: return launch_bwd_tile<32, MODE_ADJ, 32>(a, t1, t2, st);
    }
  }
  return cudaErrorNotSupported;
}

}  // namespace hdf
