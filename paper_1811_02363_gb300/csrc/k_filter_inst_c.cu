// Instantiations of the fused tile kernel for window half-widths 18, 24, 32
// (two planes per chunk so that the staged halo fits in shared memory).
#include "filter_tile.cuh"

namespace hdf {

cudaError_t launch_filter_group_c(int SB, int P, const FilterArgs& a, const Taps& t,
                                  cudaStream_t st) {
  (void)P;
  switch (SB) {
    case 18: return launch_filter_tile<18, 2, 64>(a, t, st);
    case 24: return launch_filter_tile<24, 2, 64>(a, t, st);
    case 32: return launch_filter_tile<32, 2, 32>(a, t, st);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_filter_group_a(int, int, const FilterArgs&, const Taps&, cudaStream_t);
cudaError_t launch_filter_group_b(int, int, const FilterArgs&, const Taps&, cudaStream_t);

cudaError_t launch_filter_sb(int SB, int P, const FilterArgs& a, const Taps& t, cudaStream_t st) {
  if (SB <= 12) return launch_filter_group_a(SB, P, a, t, st);
  if (SB == 15) return launch_filter_group_b(SB, P, a, t, st);
  return launch_filter_group_c(SB, P, a, t, st);
}

}  // namespace hdf
