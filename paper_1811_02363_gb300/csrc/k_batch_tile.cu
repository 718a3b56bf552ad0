// The persistent batch tile kernel: one launch works through the item list of
// a whole batch (batch_tile.cuh), dispatching each item to the body compiled
// for its window bucket.
#include "batch_tile.cuh"

namespace hdf {
namespace {

__global__ void __launch_bounds__(BT_THREADS, 1)
batch_tile_kernel(const BatchImg* __restrict__ imgs, const int4* __restrict__ items, int nitems,
                  int* __restrict__ counter) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_item;
  while (true) {
    __syncthreads();   // the previous item is finished with shared memory
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const int4 w = items[it];   // (image, tile x, tile y, plane chunk)
    const BatchImg* im = imgs + w.x;
    const int x0 = w.y * BT_TX, y0 = w.z * im->TY;
    switch (im->SB) {
      case 3: batch_tile_item<3>(im, x0, y0, w.w, sm); break;
      case 6: batch_tile_item<6>(im, x0, y0, w.w, sm); break;
      case 9: batch_tile_item<9>(im, x0, y0, w.w, sm); break;
      case 12: batch_tile_item<12>(im, x0, y0, w.w, sm); break;
      case 15: batch_tile_item<15>(im, x0, y0, w.w, sm); break;
      case 18: batch_tile_item<18>(im, x0, y0, w.w, sm); break;
      case 24: batch_tile_item<24>(im, x0, y0, w.w, sm); break;
      case 32: batch_tile_item<32>(im, x0, y0, w.w, sm); break;
      default: break;
    }
  }
}

}  // namespace

int batch_tile_max_blocks_per_sm(size_t smem) {
  if (cudaFuncSetAttribute(batch_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_tile_kernel, BT_THREADS, smem) !=
      cudaSuccess)
    return 0;
  return occ;
}

cudaError_t launch_batch_tile(const BatchImg* imgs, const int4* items, int nitems, int* counter,
                              size_t smem, int grid, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(batch_tile_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  batch_tile_kernel<<<grid, BT_THREADS, smem, st>>>(imgs, items, nitems, counter);
  return cudaGetLastError();
}

}  // namespace hdf
