// Per-pixel pieces of Algorithm 1 shared by the single-image kernels
// (k_filter.cu) and the batch kernels (k_batch.cu): the range maps and
// coefficients (loops "for1"/"for2"), the normalisation of Eq. (15)-(16) with
// the denominator guard, and the indicator fix-up of Eq. (18) for guarded
// pixels.
#pragma once

#include <math.h>

#include "hdf_internal.cuh"

namespace hdf {

constexpr float kGuardRel = 1e-6f;   // guard: sum_k c_k r_k <= 1e-6 max_k r_k

// b_k(i) = phi(mu_k - p(i)) (Eq. (12)) from direct differences in FP32;
// c(i) = A^+ b(i) (Eq. (11)) or e_s (Eq. (17)); s(i) = nearest centre (ties
// -> lowest k).  smu (K x rho) and spi (K x K) are in shared memory.
template <int KMAX, typename GT>
__device__ __forceinline__ void rangemap_pixel(const GT* __restrict__ p, size_t N, size_t pix,
                                               int rho, int K, const float* smu,
                                               const float* spi, float inv2sr2, int coef,
                                               float* __restrict__ B, float* __restrict__ C,
                                               uint8_t* __restrict__ s_out) {
  float d2[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) d2[k] = 0.0f;
  for (int d = 0; d < rho; ++d) {
    const float x = guide_load(p, (size_t)d * N + pix);
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      if (k < K) {
        const float t = x - smu[k * rho + d];
        d2[k] = fmaf(t, t, d2[k]);
      }
    }
  }
  int s = 0;
  float best = d2[0];
#pragma unroll
  for (int k = 1; k < KMAX; ++k)
    if (k < K && d2[k] < best) { best = d2[k]; s = k; }
  float b[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) b[k] = (k < K) ? expf(-d2[k] * inv2sr2) : 0.0f;
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
    if (k < K) B[(size_t)k * N + pix] = b[k];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    if (k < K) {
      float c;
      if (coef == HDF_COEF_OPT) {
        c = 0.0f;
#pragma unroll
        for (int l = 0; l < KMAX; ++l)
          if (l < K) c = fmaf(spi[k * K + l], b[l], c);
      } else {
        c = (k == s) ? 1.0f : 0.0f;
      }
      C[(size_t)k * N + pix] = c;
    }
  }
  s_out[pix] = (uint8_t)s;
}

// Eq. (15)-(16): g_hat = (sum_k c_k v_k) / (sum_k c_k r_k) at one pixel, the
// numerators already in g.  A pixel failing the guard is appended to
// fix_list (count in ctrl[CTRL_FALLBACK]) for the indicator fix-up.
__device__ __forceinline__ void divide_pixel(float* __restrict__ g, const float* __restrict__ den,
                                             const float* __restrict__ rmax, int* ctrl,
                                             int* __restrict__ fix_list, int N, int n, int pix) {
  const float D = den[pix];
  if (!(D > kGuardRel * rmax[pix])) {
    const int pos = atomicAdd(ctrl + CTRL_FALLBACK, 1);
    if (pos < N) fix_list[pos] = pix;
    return;
  }
  const float inv = 1.0f / D;
  for (int c = 0; c < n; ++c) g[(size_t)c * N + pix] *= inv;
}

// Indicator value v_s(i) / r_s(i) of Eq. (18) for channel ch of a guarded
// pixel (s = nearest centre), by direct sums over the window from the stored
// b_s plane; f(i) if r_s(i) = 0.  w(j) returns omega_1(j) for |j| <= S.
template <class TapF>
__device__ __forceinline__ float fixup_value(const float* __restrict__ f,
                                             const float* __restrict__ B,
                                             const uint8_t* __restrict__ s, int H, int W, int S,
                                             TapF w, int pix, int ch) {
  const size_t N = (size_t)H * W;
  const int y = pix / W, x = pix % W;
  const float* Bs = B + (size_t)s[pix] * N;
  const float* fc = f + (size_t)ch * N;
  float r = 0.0f, v = 0.0f;
  for (int j1 = -S; j1 <= S; ++j1) {
    const int yy = y - j1;
    if (yy < 0 || yy >= H) continue;
    for (int j2 = -S; j2 <= S; ++j2) {
      const int xx = x - j2;
      if (xx < 0 || xx >= W) continue;
      const float wt = w(j1) * w(j2) * Bs[(size_t)yy * W + xx];
      r += wt;
      v = fmaf(wt, fc[(size_t)yy * W + xx], v);
    }
  }
  return (r > 0.0f) ? v / r : fc[pix];
}

}  // namespace hdf
