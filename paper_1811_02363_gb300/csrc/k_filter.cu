// Algorithm 1 loops "for1" and "for2" (range maps b_k and coefficients c),
// the guard fix-up, and the dispatch of the fused convolution/combine tile
// kernel (filter_tile.cuh) for hdf_apply.
#include <math.h>
#include <stdint.h>

#include "combine.cuh"
#include "filter_tile.cuh"
#include "hdf_internal.cuh"

namespace hdf {
namespace {

constexpr int RM_THREADS = 256;

// Range maps and coefficients of every pixel (combine.cuh).
template <int KMAX, typename GT>
__global__ void __launch_bounds__(RM_THREADS)
rangemap_kernel(const GT* __restrict__ p, int N, int rho, const float* __restrict__ mu,
                const float* __restrict__ pinv, const int* __restrict__ ctrl, float inv2sr2,
                int coef, float* __restrict__ B, float* __restrict__ C,
                uint8_t* __restrict__ s_out) {
  extern __shared__ __align__(16) float sm[];
  const int K = ctrl[CTRL_K_EFF];
  rangemap_stage(mu, pinv, K, rho, sm);
  __syncthreads();
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= N) return;
  rangemap_pixel<KMAX>(p, (size_t)N, (size_t)pix, rho, K, sm, inv2sr2, coef, B, C, s_out);
}

template <int KMAX>
cudaError_t launch_rm(hdf_handle* h, const void* p, cudaStream_t st) {
  const hdf_desc& d = h->d;
  const size_t smem = sizeof(float) * (size_t)rm_smem_floats(d.K, d.rho);   // K_eff <= K
  const float inv2sr2 = (float)(1.0 / (2.0 * d.sigma_r * d.sigma_r));
  const int grid = (h->N + RM_THREADS - 1) / RM_THREADS;
  if (d.guide_dtype == HDF_GUIDE_BF16)
    rangemap_kernel<KMAX, __nv_bfloat16><<<grid, RM_THREADS, smem, st>>>(
        (const __nv_bfloat16*)p, h->N, d.rho, h->mu, h->pinv32, h->ctrl, inv2sr2, d.coef, h->B,
        h->C, h->s);
  else
    rangemap_kernel<KMAX, float><<<grid, RM_THREADS, smem, st>>>(
        (const float*)p, h->N, d.rho, h->mu, h->pinv32, h->ctrl, inv2sr2, d.coef, h->B, h->C,
        h->s);
  return cudaGetLastError();
}

// Pixels where the denominator guard fired take the indicator value of
// Eq. (18) (combine.cuh).
__global__ void fixup_kernel(const float* __restrict__ f, const float* __restrict__ B,
                             const uint8_t* __restrict__ s, const int* __restrict__ fix_list,
                             const int* __restrict__ ctrl, int H, int W, int n, int S,
                             const Taps taps, float* __restrict__ g) {
  const size_t N = (size_t)H * W;
  int count = ctrl[CTRL_FALLBACK];
  if (count > (int)N) count = (int)N;
  const long long total = (long long)count * n;
  for (long long item = blockIdx.x * (long long)blockDim.x + threadIdx.x; item < total;
       item += (long long)gridDim.x * blockDim.x) {
    const int idx = (int)(item / n), ch = (int)(item % n);
    const int pix = fix_list[idx];
    g[(size_t)ch * N + pix] =
        fixup_value(f, B, s, H, W, S, [&](int j) { return taps.w[j + S]; }, pix, ch);
  }
}

// Eq. (15)-(16) normalisation with the denominator guard (combine.cuh).
__global__ void divide_kernel(float* __restrict__ g, const float* __restrict__ den,
                              const float* __restrict__ rmax, const float* __restrict__ dabs,
                              int* __restrict__ ctrl, int* __restrict__ fix_list, int N, int n) {
  for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < N; pix += gridDim.x * blockDim.x)
    divide_pixel(g, den, rmax, ctrl, fix_list, N, n, pix, dabs);
}

}  // namespace

cudaError_t launch_rangemap(hdf_handle* h, const void* p, cudaStream_t st) {
  const int K = h->d.K;
  if (K <= 8) return launch_rm<8>(h, p, st);
  if (K <= 16) return launch_rm<16>(h, p, st);
  if (K <= 32) return launch_rm<32>(h, p, st);
  return launch_rm<64>(h, p, st);
}

// Compiled half-widths of the tile kernel; a call's S runs on the smallest
// bucket >= S with zero weights beyond S.
static const int kBuckets[] = {3, 6, 9, 12, 15, 18, 24, 32};

int filter_bucket(int S) {
  for (int b : kBuckets)
    if (S <= b) return b;
  return -1;
}

cudaError_t launch_filter(hdf_handle* h, const float* f, const void* p, float* g, cudaStream_t st,
                          int rescue) {
  const hdf_desc& d = h->d;
  if (d.spatial == HDF_SPATIAL_YOUNG) return launch_young(h, f, g, st);
  const int SB = filter_bucket(d.S);
  if (SB < 0) return cudaErrorInvalidValue;
  const int P = (d.n == 1 || SB > 16) ? 2 : 4;
  // Taps centred in the bucket: w[SB + j] = omega_1(j) for |j| <= S, 0 beyond.
  Taps exact = make_taps(d.sigma_s, d.S, d.spatial);
  Taps taps;
  for (int t = 0; t < 2 * HDF_MAX_S + 1; ++t) taps.w[t] = 0.0f;
  for (int j = -d.S; j <= d.S; ++j) taps.w[SB + j] = exact.w[d.S + j];
  cudaError_t e = cudaMemsetAsync(h->ctrl + CTRL_FALLBACK, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(h->ctrl + CTRL_RESCUED, 0, 2 * sizeof(int), st);   // and CTRL_FALLBACK64
  if (e != cudaSuccess) return e;
  float* dabs = rescue ? h->dabs : nullptr;
  FilterArgs a{f, h->B, h->C, g, h->den, h->rmax, dabs, h->ctrl, d.H, d.W, d.n,
               d.spatial == HDF_SPATIAL_BOX ? 1 : 0, d.S,
               (d.W % 4 == 0 && reinterpret_cast<uintptr_t>(f) % 16 == 0) ? 1 : 0};
  e = launch_filter_sb(SB, P, a, taps, st);
  if (e != cudaSuccess) return e;
  if (h->timing && rescue && (e = cudaEventRecord(h->tev[2], st)) != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  divide_kernel<<<sms * 4, 256, 0, st>>>(g, h->den, h->rmax, dabs, h->ctrl, h->fix_list, h->N, d.n);
  fixup_kernel<<<sms, 256, 0, st>>>(f, h->B, h->s, h->fix_list, h->ctrl, d.H, d.W, d.n, d.S,
                                    exact, g);
  e = cudaGetLastError();
  if (e != cudaSuccess || !rescue) return e;
  return launch_rescue(h, f, p, g, h->fix_list, st);   // ill-conditioned pixels, in FP64
}

}  // namespace hdf
