// Algorithm 1 "for3" with the Gaussian convolutions by Young and van Vliet's
// recursive filter (the O(1) convolution Sec. II-C names), for hdf_apply with
// HDF_SPATIAL_YOUNG.  Per centre k, for every plane q (q = 0: b_k, q = 1 + c:
// b_k f_c):
//   rows kernel:    causal then anticausal third-order recursion along each
//                   row (zero states at both ends), written to the scratch T
//                   (all centres in one launch, K (n + 1) planes);
//   columns kernel: the same along each column of T, in place (all centres);
//   combine kernel: per pixel, sum_k c_k v_k and sum_k c_k r_k (Eq. (15)-(16))
//                   in a fixed order, max_k r_k, the division, and the guard
//                   with the indicator value v_s / r_s of the nearest centre s
//                   (Eq. (18)) read from the filtered planes.
// Recursion: w[t] = B x[t] + a1 w[t-1] + a2 w[t-2] + a3 w[t-3], then
// y[t] = B w[t] + a1 y[t+1] + a2 y[t+2] + a3 y[t+3], in FP32.
#include <math.h>

#include "combine.cuh"
#include "hdf_internal.cuh"

namespace hdf {
namespace {

struct YoungCoef {
  float B, a1, a2, a3;
};

constexpr int YR_WARPS = 2;   // warps (32 rows each) per block of the rows kernel
constexpr int YC_THREADS = 128;

// Rows: a warp owns 32 consecutive rows of one plane.  Tiles of 32 x 32 are
// loaded and stored coalesced through shared memory (stride 33: the row-wise
// walk of a lane and the column-wise copy are both free of bank conflicts);
// lane r walks row r of the tile, carrying the recursion state across tiles.
__global__ void __launch_bounds__(32 * YR_WARPS)
young_rows_kernel(const float* __restrict__ f, const float* __restrict__ B, float* __restrict__ T,
                  int n, int H, int W, YoungCoef cf, const int* __restrict__ ctrl) {
  const int k = blockIdx.z;   // every centre in one launch: T holds K (n + 1) planes
  if (k >= ctrl[CTRL_K_EFF]) return;
  __shared__ float tile[YR_WARPS][32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = blockIdx.y;
  const int y0 = (blockIdx.x * YR_WARPS + warp) * 32;
  if (y0 >= H) return;   // whole warp
  const size_t N = (size_t)H * W;
  const float* Bk = B + (size_t)k * N;
  const float* fq = q > 0 ? f + (size_t)(q - 1) * N : nullptr;
  float* Tq = T + ((size_t)k * (n + 1) + q) * N;
  float (*tl)[33] = tile[warp];
  const int nr = min(32, H - y0);      // rows of the warp inside the image
  // causal pass, left to right
  float w1 = 0.0f, w2 = 0.0f, w3 = 0.0f;
  for (int x0 = 0; x0 < W; x0 += 32) {
    const int x = x0 + lane;
    const int nc = min(32, W - x0);
    for (int r = 0; r < nr; ++r) {
      float v = 0.0f;
      if (x < W) {
        const size_t i = (size_t)(y0 + r) * W + x;
        v = __ldg(Bk + i);
        if (fq) v *= __ldg(fq + i);
      }
      tl[r][lane] = v;
    }
    __syncwarp();
    if (lane < nr) {
      for (int c = 0; c < nc; ++c) {
        const float w = fmaf(cf.B, tl[lane][c], fmaf(cf.a1, w1, fmaf(cf.a2, w2, cf.a3 * w3)));
        w3 = w2;
        w2 = w1;
        w1 = w;
        tl[lane][c] = w;
      }
    }
    __syncwarp();
    if (x < W)
      for (int r = 0; r < nr; ++r) Tq[(size_t)(y0 + r) * W + x] = tl[r][lane];
    __syncwarp();
  }
  // anticausal pass, right to left, in place
  float v1 = 0.0f, v2 = 0.0f, v3 = 0.0f;
  for (int x0 = ((W - 1) / 32) * 32; x0 >= 0; x0 -= 32) {
    const int x = x0 + lane;
    const int nc = min(32, W - x0);
    if (x < W)
      for (int r = 0; r < nr; ++r) tl[r][lane] = Tq[(size_t)(y0 + r) * W + x];
    __syncwarp();
    if (lane < nr) {
      for (int c = nc - 1; c >= 0; --c) {
        const float v = fmaf(cf.B, tl[lane][c], fmaf(cf.a1, v1, fmaf(cf.a2, v2, cf.a3 * v3)));
        v3 = v2;
        v2 = v1;
        v1 = v;
        tl[lane][c] = v;
      }
    }
    __syncwarp();
    if (x < W)
      for (int r = 0; r < nr; ++r) Tq[(size_t)(y0 + r) * W + x] = tl[r][lane];
    __syncwarp();
  }
}

// Columns: a thread owns one column of one plane of one centre (the accesses
// of a warp are 32 consecutive pixels of a row): causal pass down, then the
// anticausal pass up, both in place; rows go in blocks of YB whose loads are
// issued together.
constexpr int YB = 16;

__global__ void __launch_bounds__(YC_THREADS)
young_cols_kernel(float* __restrict__ T, int n, int H, int W, YoungCoef cf,
                  const int* __restrict__ ctrl) {
  const int k = blockIdx.z;
  if (k >= ctrl[CTRL_K_EFF]) return;
  const int x = blockIdx.x * YC_THREADS + threadIdx.x;
  const int q = blockIdx.y;
  if (x >= W) return;
  const size_t N = (size_t)H * W;
  float* Tq = T + ((size_t)k * (n + 1) + q) * N + x;
  float w1 = 0.0f, w2 = 0.0f, w3 = 0.0f;
  for (int y0 = 0; y0 < H; y0 += YB) {
    const int nb = min(YB, H - y0);
    float t[YB];
#pragma unroll
    for (int j = 0; j < YB; ++j) t[j] = j < nb ? Tq[(size_t)(y0 + j) * W] : 0.0f;
#pragma unroll
    for (int j = 0; j < YB; ++j) {
      const float w = fmaf(cf.B, t[j], fmaf(cf.a1, w1, fmaf(cf.a2, w2, cf.a3 * w3)));
      w3 = w2;
      w2 = w1;
      w1 = w;
      t[j] = w;
    }
#pragma unroll
    for (int j = 0; j < YB; ++j)
      if (j < nb) Tq[(size_t)(y0 + j) * W] = t[j];
  }
  float v1 = 0.0f, v2 = 0.0f, v3 = 0.0f;
  for (int ye = H; ye > 0; ye -= YB) {   // rows ye - nb .. ye - 1, upwards
    const int nb = min(YB, ye);
    const int yb = ye - nb;
    float t[YB];
#pragma unroll
    for (int j = 0; j < YB; ++j) t[j] = j < nb ? Tq[(size_t)(yb + j) * W] : 0.0f;
#pragma unroll
    for (int j = YB - 1; j >= 0; --j) {
      if (j < nb) {
        const float v = fmaf(cf.B, t[j], fmaf(cf.a1, v1, fmaf(cf.a2, v2, cf.a3 * v3)));
        v3 = v2;
        v2 = v1;
        v1 = v;
        t[j] = v;
      }
    }
#pragma unroll
    for (int j = 0; j < YB; ++j)
      if (j < nb) Tq[(size_t)(yb + j) * W] = t[j];
  }
}

// Combine and normalise per pixel (Eq. (15)-(16)) from the filtered planes
// v_k (planes 1..n of centre k) and r_k (plane 0), summed over k in a fixed
// order; the guard (sum_k c_k r_k <= 1e-6 max_k r_k) takes the indicator value
// v_s / r_s of the nearest centre s (Eq. (18)), f where r_s = 0.
__global__ void young_combine_kernel(const float* __restrict__ T, const float* __restrict__ C,
                                     const uint8_t* __restrict__ s, const float* __restrict__ f,
                                     int n, int N, int* __restrict__ ctrl, float* __restrict__ g) {
  const int K = ctrl[CTRL_K_EFF];
  const size_t P = (size_t)(n + 1) * N;   // planes of one centre
  for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < N; pix += gridDim.x * blockDim.x) {
    float den = 0.0f, rmax = 0.0f;
    for (int k = 0; k < K; ++k) {
      const float r = T[(size_t)k * P + pix];
      den = fmaf(__ldg(C + (size_t)k * N + pix), r, den);
      rmax = fmaxf(rmax, r);
    }
    if (!(den > kGuardRel * rmax)) {   // the guard of divide_pixel
      atomicAdd(ctrl + CTRL_FALLBACK, 1);
      const size_t so = (size_t)s[pix] * P;
      const float rs = T[so + pix];
      for (int c = 0; c < n; ++c)
        g[(size_t)c * N + pix] = rs > 0.0f ? T[so + (size_t)(c + 1) * N + pix] / rs
                                           : f[(size_t)c * N + pix];
      continue;
    }
    const float inv = 1.0f / den;
    for (int c = 0; c < n; ++c) {
      float num = 0.0f;
      for (int k = 0; k < K; ++k)
        num = fmaf(__ldg(C + (size_t)k * N + pix), T[(size_t)k * P + (size_t)(c + 1) * N + pix], num);
      g[(size_t)c * N + pix] = num * inv;
    }
  }
}

}  // namespace

// Coefficients of the recursion (the published formulas for sigma >= 0.5):
// q from sigma, b0..b3, a_i = b_i / b0 and B = 1 - (a1 + a2 + a3).  The a_i
// are rounded to float first and B is formed from the rounded values, so the
// float recursion keeps unit gain exactly: its error, amplified by about 1/B
// (the recursion's gain for its own rounding, 150 at sigma = 8), then comes
// from the per-step rounding only (about 3-4 times less than with every
// coefficient rounded separately).
static YoungCoef young_coef(double sigma) {
  const double q = sigma >= 2.5 ? 0.98711 * sigma - 0.96330
                                : 3.97156 - 4.14554 * sqrt(1.0 - 0.26891 * sigma);
  const double b0 = 1.57825 + 2.44413 * q + 1.4281 * q * q + 0.422205 * q * q * q;
  const double b1 = 2.44413 * q + 2.85619 * q * q + 1.26661 * q * q * q;
  const double b2 = -(1.4281 * q * q + 1.26661 * q * q * q);
  const double b3 = 0.422205 * q * q * q;
  YoungCoef c;
  c.a1 = (float)(b1 / b0);
  c.a2 = (float)(b2 / b0);
  c.a3 = (float)(b3 / b0);
  c.B = (float)(1.0 - ((double)c.a1 + (double)c.a2 + (double)c.a3));
  return c;
}

cudaError_t launch_young(hdf_handle* h, const float* f, float* g, cudaStream_t st) {
  const hdf_desc& d = h->d;
  if (!h->young_T) return cudaErrorInvalidValue;
  const int n = d.n, H = d.H, W = d.W;
  const YoungCoef cf = young_coef(d.sigma_s);
  cudaError_t e = cudaMemsetAsync(h->ctrl + CTRL_FALLBACK, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  float* T = h->young_T;   // K (n + 1) planes: b_k f rows-filtered, then fully filtered
  const dim3 grid_r((H + 32 * YR_WARPS - 1) / (32 * YR_WARPS), n + 1, d.K);   // blocks of centres
  const dim3 grid_c((W + YC_THREADS - 1) / YC_THREADS, n + 1, d.K);           // beyond K_eff return
  young_rows_kernel<<<grid_r, 32 * YR_WARPS, 0, st>>>(f, h->B, T, n, H, W, cf, h->ctrl);
  young_cols_kernel<<<grid_c, YC_THREADS, 0, st>>>(T, n, H, W, cf, h->ctrl);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  young_combine_kernel<<<sms * 8, 256, 0, st>>>(T, h->C, h->s, f, n, h->N, h->ctrl, g);
  return cudaGetLastError();
}

}  // namespace hdf
