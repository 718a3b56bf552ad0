// Batch kernels around the persistent tile kernel (k_batch_tile.cu): per-run
// reset of the control words, guide conversion to bfloat16 storage, range
// maps and coefficients of every image (Algorithm 1 loops "for1"/"for2"),
// and the normalisation with guard and indicator fix-up (Eq. (15)-(18)).
// Each kernel covers all images of a batch in one launch; a block finds its
// image from a table of first-block indices.
#include "batch.cuh"
#include "cluster_args.cuh"
#include "combine.cuh"

namespace hdf {
namespace {

constexpr int BK_THREADS = 256;

// Image of block b: the last j with block0[j] <= b (block0 ascending).
__device__ __forceinline__ int job_of_block(const int* __restrict__ block0, int njobs, int b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(block0 + mid) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void batch_prep_kernel(const BatchImg* __restrict__ imgs, int nimg,
                                  const clus::ClArgs* __restrict__ cl, const int* __restrict__ cl_list,
                                  int ncl, int* __restrict__ counter) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) *counter = 0;
  if (t < nimg) {
    int* c = imgs[t].ctrl;
    c[CTRL_FALLBACK] = 0;
    c[CTRL_BARRIER] = 0;
    c[CTRL_BARRIER_GEN] = 0;
  }
  if (t < ncl) cl[cl_list[t]].trace[0] = 0;
}

// Guide storage in bfloat16 (round to nearest even) of the images that use it.
__global__ void batch_to_bf16_kernel(const GuideJob* __restrict__ jobs, const int* __restrict__ block0,
                                     int njobs) {
  const int j = job_of_block(block0, njobs, blockIdx.x);
  const GuideJob g = jobs[j];
  const size_t base = (size_t)(blockIdx.x - block0[j]) * BK_THREADS * 4;
  for (int u = 0; u < 4; ++u) {
    const size_t i = base + (size_t)u * BK_THREADS + threadIdx.x;
    if (i < g.count) g.dst[i] = __float2bfloat16_rn(__ldg(g.src + i));
  }
}

template <int KMAX>
__global__ void __launch_bounds__(BK_THREADS)
batch_rangemap_kernel(const RmJob* __restrict__ jobs, const int* __restrict__ block0, int njobs) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_j;
  if (threadIdx.x == 0) s_j = job_of_block(block0, njobs, blockIdx.x);
  __syncthreads();
  const RmJob& jb = jobs[s_j];
  const int K = jb.ctrl[CTRL_K_EFF];
  const int rho = jb.rho;
  rangemap_stage(jb.mu, jb.pinv, K, rho, sm);
  __syncthreads();
  const int pix = (blockIdx.x - block0[s_j]) * BK_THREADS + threadIdx.x;
  if (pix >= jb.N) return;
  if (jb.p_bf16)
    rangemap_pixel<KMAX>((const __nv_bfloat16*)jb.p, (size_t)jb.N, (size_t)pix, rho, K, sm,
                         jb.inv2sr2, jb.coef, jb.B, jb.C, jb.s);
  else
    rangemap_pixel<KMAX>((const float*)jb.p, (size_t)jb.N, (size_t)pix, rho, K, sm,
                         jb.inv2sr2, jb.coef, jb.B, jb.C, jb.s);
}

__global__ void __launch_bounds__(BK_THREADS)
batch_divide_kernel(const BatchImg* __restrict__ imgs, const int* __restrict__ block0, int nimg) {
  const int j = job_of_block(block0, nimg, blockIdx.x);
  const BatchImg& im = imgs[j];
  const int N = im.H * im.W;
  const int base = (blockIdx.x - block0[j]) * BK_THREADS * 4;
  for (int u = 0; u < 4; ++u) {
    const int pix = base + u * BK_THREADS + threadIdx.x;
    if (pix < N) divide_pixel(im.g, im.den, im.rmax, im.ctrl, im.fix_list, N, im.n, pix);
  }
}

// blockIdx.y = image; the guarded pixels of that image (usually none).
__global__ void batch_fixup_kernel(const BatchImg* __restrict__ imgs) {
  const BatchImg& im = imgs[blockIdx.y];
  const int N = im.H * im.W;
  int count = im.ctrl[CTRL_FALLBACK];
  if (count > N) count = N;
  const long long total = (long long)count * im.n;
  const int SB = im.SB;
  const float* taps = im.taps;
  for (long long item = blockIdx.x * (long long)blockDim.x + threadIdx.x; item < total;
       item += (long long)gridDim.x * blockDim.x) {
    const int idx = (int)(item / im.n), ch = (int)(item % im.n);
    const int pix = im.fix_list[idx];
    im.g[(size_t)ch * N + pix] = fixup_value(im.f, im.B, im.s, im.H, im.W, im.S,
                                             [&](int jj) { return taps[SB + jj]; }, pix, ch);
  }
}

}  // namespace

int batch_blocks_for(size_t count, int per_thread) {
  const size_t per_block = (size_t)BK_THREADS * per_thread;
  return (int)((count + per_block - 1) / per_block);
}

cudaError_t launch_batch_prep(const BatchImg* imgs, int nimg, const clus::ClArgs* cl,
                              const int* cl_list, int ncl, int* counter, cudaStream_t st) {
  const int n = nimg > ncl ? nimg : ncl;
  const int blocks = n > 0 ? (n + BK_THREADS - 1) / BK_THREADS : 1;
  batch_prep_kernel<<<blocks, BK_THREADS, 0, st>>>(imgs, nimg, cl, cl_list, ncl, counter);
  return cudaGetLastError();
}

cudaError_t launch_batch_to_bf16(const GuideJob* jobs, const int* block0, int njobs, int nblocks,
                                 cudaStream_t st) {
  if (njobs < 1 || nblocks < 1) return cudaSuccess;
  batch_to_bf16_kernel<<<nblocks, BK_THREADS, 0, st>>>(jobs, block0, njobs);
  return cudaGetLastError();
}

cudaError_t launch_batch_rangemap(const RmJob* jobs, const int* block0, int njobs, int nblocks,
                                  int Kmax, int smem_floats, cudaStream_t st) {
  if (njobs < 1 || nblocks < 1) return cudaSuccess;
  const size_t smem = sizeof(float) * (size_t)smem_floats;
  if (Kmax <= 8)
    batch_rangemap_kernel<8><<<nblocks, BK_THREADS, smem, st>>>(jobs, block0, njobs);
  else if (Kmax <= 16)
    batch_rangemap_kernel<16><<<nblocks, BK_THREADS, smem, st>>>(jobs, block0, njobs);
  else if (Kmax <= 32)
    batch_rangemap_kernel<32><<<nblocks, BK_THREADS, smem, st>>>(jobs, block0, njobs);
  else
    batch_rangemap_kernel<64><<<nblocks, BK_THREADS, smem, st>>>(jobs, block0, njobs);
  return cudaGetLastError();
}

cudaError_t launch_batch_normalise(const BatchImg* imgs, const int* block0, int nimg, int nblocks,
                                   cudaStream_t st) {
  if (nimg < 1) return cudaSuccess;
  batch_divide_kernel<<<nblocks, BK_THREADS, 0, st>>>(imgs, block0, nimg);
  batch_fixup_kernel<<<dim3(8, nimg), BK_THREADS, 0, st>>>(imgs);
  return cudaGetLastError();
}

}  // namespace hdf
