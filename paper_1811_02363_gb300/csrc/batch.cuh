// Device tables of a batch (hdf_batch.cu builds them; k_batch.cu,
// k_batch_tile.cu and k_fit.cu read them).
#pragma once

#include "batch_tile.cuh"
#include "cluster_args.cuh"
#include "hdf_internal.cuh"

namespace hdf {

// One image's guide converted to bfloat16 storage.
struct GuideJob {
  const float* src;
  __nv_bfloat16* dst;
  size_t count;
};

// Range maps and coefficients of one image.
struct RmJob {
  const void* p;        // guide (rho, H, W)
  int p_bf16;           // guide stored as bfloat16
  int N, rho, coef;
  float inv2sr2;
  const float* mu;      // K x rho
  const float* pinv;    // K x K float32
  const int* ctrl;
  float* B;
  float* C;
  uint8_t* s;
};

// Launchers (k_batch.cu).
int batch_blocks_for(size_t count, int per_thread);
cudaError_t launch_batch_prep(const BatchImg* imgs, int nimg, const clus::ClArgs* cl,
                              const int* cl_list, int ncl, int* counter, cudaStream_t st);
cudaError_t launch_batch_to_bf16(const GuideJob* jobs, const int* block0, int njobs, int nblocks,
                                 cudaStream_t st);
cudaError_t launch_batch_rangemap(const RmJob* jobs, const int* block0, int njobs, int nblocks,
                                  int Kmax, int smem_floats, cudaStream_t st);
cudaError_t launch_batch_normalise(const BatchImg* imgs, const int* block0, int nimg, int nblocks,
                                   cudaStream_t st);

}  // namespace hdf
