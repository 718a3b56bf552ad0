// Instantiations of the register-blocked brute-force tile kernel
// (brute_tile.cuh) for guides and images of up to 8 channels, every window bucket.
#include "brute_tile.cuh"

namespace hdf {

namespace {

template <int MAXC, int SB>
cudaError_t launch_bt(const BruteTileArgs& a, const Taps& t, cudaStream_t st) {
  using Cfg = BruteTileCfg<MAXC, SB>;
  const int planes = a.alias ? a.rho : a.rho + a.n;
  const size_t smem = sizeof(float) * Cfg::smem_floats(planes, a.rho);
  if (smem > 227 * 1024) return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(brute_tile_kernel<MAXC, SB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 block(16, Cfg::TY);
  dim3 grid((a.W + Cfg::TX - 1) / Cfg::TX, (a.H + Cfg::TY - 1) / Cfg::TY);
  brute_tile_kernel<MAXC, SB><<<grid, block, smem, st>>>(a, t);
  return cudaGetLastError();
}

template <int MAXC>
cudaError_t launch_bt_sb(int SB, const BruteTileArgs& a, const Taps& t, cudaStream_t st) {
  switch (SB) {
    case 3: return launch_bt<MAXC, 3>(a, t, st);
    case 6: return launch_bt<MAXC, 6>(a, t, st);
    case 9: return launch_bt<MAXC, 9>(a, t, st);
    case 12: return launch_bt<MAXC, 12>(a, t, st);
    case 15: return launch_bt<MAXC, 15>(a, t, st);
    case 18: return launch_bt<MAXC, 18>(a, t, st);
    case 24: return launch_bt<MAXC, 24>(a, t, st);
    case 32: return launch_bt<MAXC, 32>(a, t, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace

cudaError_t launch_brute_tile_a(int maxc, int SB, const BruteTileArgs& a, const Taps& t,
                                   cudaStream_t st) {
  if (maxc == 4) return launch_bt_sb<4>(SB, a, t, st);
  if (maxc == 8) return launch_bt_sb<8>(SB, a, t, st);
  return cudaErrorNotSupported;
}

}  // namespace hdf
