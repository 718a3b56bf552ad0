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
// The float32 denominator sum_k c_k r_k carries a rounding of a few units of
// 2^-24 times sum_k |c_k| r_k.  Where that sum exceeds kIllCond times
// |sum_k c_k r_k| (cancellation: the float32 value of g_hat may be off by more
// than 1e-4), or the guard's threshold lies within kNearBand times it (the
// float32 decision may go either way), the pixel is recomputed in FP64.
constexpr float kIllCond = 64.0f;
constexpr float kNearBand = 1.0f / 262144.0f;   // 2^-18

// Shared-memory tables of the range-map kernels: the centres transposed,
// smu[d][k], and A^+ by rows, spi[k][l], both with rows of KP = K rounded up
// to 4 floats (zero padding), so that a 16-byte load brings 4 centres.
__host__ __device__ constexpr int rm_pitch(int K) { return (K + 3) & ~3; }
__host__ __device__ constexpr int rm_smem_floats(int K, int rho) { return rm_pitch(K) * (rho + K); }

__device__ __forceinline__ void rangemap_stage(const float* __restrict__ mu,
                                               const float* __restrict__ pinv, int K, int rho,
                                               float* sm) {
  const int KP = rm_pitch(K);
  float* smu = sm;
  float* spi = sm + rho * KP;
  for (int i = threadIdx.x; i < rho * KP; i += blockDim.x) {
    const int d = i / KP, k = i - d * KP;
    smu[i] = k < K ? mu[k * rho + d] : 0.0f;
  }
  for (int i = threadIdx.x; i < K * KP; i += blockDim.x) {
    const int k = i / KP, l = i - k * KP;
    spi[i] = l < K ? pinv[k * K + l] : 0.0f;
  }
}

// b_k(i) = phi(mu_k - p(i)) (Eq. (12)) from direct differences in FP32;
// c(i) = A^+ b(i) (Eq. (11)) or e_s (Eq. (17)); s(i) = nearest centre (ties
// -> lowest k).  sm holds the tables of rangemap_stage.  The guide values
// are loaded RB at a time (independent loads in flight); every sum runs in
// ascending d or l.
template <int KMAX, typename GT>
__device__ __forceinline__ void rangemap_pixel(const GT* __restrict__ p, size_t N, size_t pix,
                                               int rho, int K, const float* sm, float inv2sr2,
                                               int coef, float* __restrict__ B,
                                               float* __restrict__ C,
                                               uint8_t* __restrict__ s_out) {
  constexpr int RB = 8;
  constexpr int K4 = KMAX / 4;
  const int KP = rm_pitch(K);
  const float* smu = sm;
  const float* spi = sm + rho * KP;
  float d2[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) d2[k] = 0.0f;
  for (int d0 = 0; d0 < rho; d0 += RB) {
    float x[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) x[u] = (d0 + u < rho) ? guide_load(p, (size_t)(d0 + u) * N + pix) : 0.0f;
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      if (d0 + u >= rho) break;
      const float4* m4 = reinterpret_cast<const float4*>(smu + (d0 + u) * KP);
#pragma unroll
      for (int q = 0; q < K4; ++q) {
        if (4 * q < K) {
          const float4 m = m4[q];
          const float t0 = x[u] - m.x, t1 = x[u] - m.y, t2 = x[u] - m.z, t3 = x[u] - m.w;
          d2[4 * q] = fmaf(t0, t0, d2[4 * q]);
          d2[4 * q + 1] = fmaf(t1, t1, d2[4 * q + 1]);
          d2[4 * q + 2] = fmaf(t2, t2, d2[4 * q + 2]);
          d2[4 * q + 3] = fmaf(t3, t3, d2[4 * q + 3]);
        }
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
        const float4* r4 = reinterpret_cast<const float4*>(spi + k * KP);
#pragma unroll
        for (int q = 0; q < K4; ++q) {
          if (4 * q < K) {   // padded entries are 0 and b beyond K is 0
            const float4 a = r4[q];
            c = fmaf(a.x, b[4 * q], c);
            c = fmaf(a.y, b[4 * q + 1], c);
            c = fmaf(a.z, b[4 * q + 2], c);
            c = fmaf(a.w, b[4 * q + 3], c);
          }
        }
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
// fix_list (count in ctrl[CTRL_FALLBACK]) for the indicator fix-up.  With
// dabs (sum_k |c_k| r_k per pixel) given, a pixel whose float32 denominator
// is ill-conditioned or within rounding of the guard's threshold is instead
// appended, from the end, to the same list (count in ctrl[CTRL_RESCUED]) for
// the FP64 recomputation; a pixel is in at most one of the two parts.
__device__ __forceinline__ void divide_pixel(float* __restrict__ g, const float* __restrict__ den,
                                             const float* __restrict__ rmax, int* ctrl,
                                             int* __restrict__ fix_list, int N, int n, int pix,
                                             const float* __restrict__ dabs = nullptr) {
  const float D = den[pix];
  const float thr = kGuardRel * rmax[pix];
  if (dabs) {
    const float Ab = dabs[pix];
    if (!(Ab <= kIllCond * fabsf(D)) || fabsf(D - thr) <= kNearBand * Ab) {
      const int pos = atomicAdd(ctrl + CTRL_RESCUED, 1);
      if (pos < N) fix_list[N - 1 - pos] = pix;
      return;
    }
  }
  if (!(D > thr)) {
    const int pos = atomicAdd(ctrl + CTRL_FALLBACK, 1);
    if (pos < N) fix_list[pos] = pix;
    return;
  }
  const float inv = 1.0f / D;
  constexpr int CB = 8;   // channels whose loads are issued together
  for (int c0 = 0; c0 < n; c0 += CB) {
    float v[CB];
#pragma unroll
    for (int u = 0; u < CB; ++u)
      if (c0 + u < n) v[u] = g[(size_t)(c0 + u) * N + pix];
#pragma unroll
    for (int u = 0; u < CB; ++u)
      if (c0 + u < n) g[(size_t)(c0 + u) * N + pix] = v[u] * inv;
  }
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
