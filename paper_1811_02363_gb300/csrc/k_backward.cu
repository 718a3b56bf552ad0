// hdf_backward: gradients of L(g_hat) with respect to the image f, log sigma_s
// and log sigma_r, with the centres mu and the window half-width S fixed.
// The paper has no backward pass; this differentiates Eq. (15)-(16) with
// c(i) = A^{-1} b(i) (Eq. (11) for a full-rank A).
//
// Steps (all on `stream`, no allocation, no host synchronisation):
//   1. forward recompute: range maps, filter -> g_hat, denominator D (skipped
//      by hdf_backward_after_apply, which takes them from the last apply);
//   2. pixels where the denominator guard fired use the indicator form
//      (c = e_s, D = r_s): their coefficient columns become one-hot and they
//      are flagged (no gradient through c there);
//   3. lambda planes: lambda_D = -<G, g_hat>/D, lambda_N = G/D;
//   4. MODE_GAMMA tile pass: gamma_k = <lambda_N, v_k> + lambda_D r_k and the
//      log sigma_s derivative sum_k <c_k lambda, omega' * u_k>;
//   5. MODE_ADJ tile pass: dL/df (direct) = sum_k b_k (omega * (c_k lambda_N)),
//      beta_k = omega * (c_k lambda_D) + <omega * (c_k lambda_N), f>;
//   6. per pixel: eta = A^{-1} gamma, dL/db_k = beta_k + eta_k; if the guide is
//      the image, dL/df += sum_k dL/db_k b_k (mu_k - f)/sigma_r^2; the
//      log sigma_r derivative sum_k dL/db_k b_k |p - mu_k|^2/sigma_r^2
//      - eta . (dA c) with dA_kl = A_kl |mu_k - mu_l|^2 / sigma_r^2;
//   7. FP64 sums of the per-block scalar partials.
#include <math.h>
#include <stdint.h>

#include "bwd_tile.cuh"
#include "hdf_internal.cuh"

namespace hdf {

int filter_bucket(int S);   // k_filter.cu

namespace {

constexpr int BW_THREADS = 256;
constexpr int PART_SIGMA_S = 0;        // offsets into h->grad_scratch (doubles)
constexpr int PART_SIGMA_R = 1 << 15;

// Guarded pixels: D := r_s (window sum of b_s), c := e_s, flag.
__global__ void bwd_fallback_kernel(const float* __restrict__ B, const uint8_t* __restrict__ s,
                                    const int* __restrict__ fix_list, const int* __restrict__ ctrl,
                                    int H, int W, int K, int S, const Taps taps, float* __restrict__ den,
                                    float* __restrict__ C, uint8_t* __restrict__ flag) {
  const size_t N = (size_t)H * W;
  int count = ctrl[CTRL_FALLBACK];
  if (count > (int)N) count = (int)N;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += gridDim.x * blockDim.x) {
    const int pix = fix_list[idx];
    const int y = pix / W, x = pix % W, k0 = s[pix];
    const float* Bs = B + (size_t)k0 * N;
    float r = 0.0f;
    for (int j1 = -S; j1 <= S; ++j1) {
      const int yy = y - j1;
      if (yy < 0 || yy >= H) continue;
      for (int j2 = -S; j2 <= S; ++j2) {
        const int xx = x - j2;
        if (xx >= 0 && xx < W) r += taps.w[j1 + S] * taps.w[j2 + S] * Bs[(size_t)yy * W + xx];
      }
    }
    den[pix] = r > 0.0f ? r : 1.0f;
    for (int k = 0; k < K; ++k) C[(size_t)k * N + pix] = (k == k0) ? 1.0f : 0.0f;
    flag[pix] = 1;
  }
}

__global__ void bwd_lambda_kernel(const float* __restrict__ G, const float* __restrict__ g,
                                  const float* __restrict__ den, int N, int n,
                                  float* __restrict__ lam) {
  for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < N; pix += gridDim.x * blockDim.x) {
    const float inv = 1.0f / den[pix];
    float dot = 0.0f;
    for (int c = 0; c < n; ++c) {
      const float gc = G[(size_t)c * N + pix];
      dot = fmaf(gc, g[(size_t)c * N + pix], dot);
      lam[(size_t)(1 + c) * N + pix] = gc * inv;
    }
    lam[pix] = -dot * inv;
  }
}

template <int KMAX, int RMAX, typename GT>
__global__ void __launch_bounds__(BW_THREADS)
bwd_final_kernel(const float* __restrict__ f, const GT* __restrict__ p, int guide_is_image,
                 const float* __restrict__ B, const float* __restrict__ C,
                 const float* __restrict__ gam, const float* __restrict__ bet,
                 const uint8_t* __restrict__ flag, const float* __restrict__ mu,
                 const float* __restrict__ pinv, int* ctrl, int N, int n, int rho, float inv_sr2,
                 float* __restrict__ grad_f, double* __restrict__ part) {
  extern __shared__ float dsm[];
  __shared__ double red[BW_THREADS / 32];
  const int K = ctrl[CTRL_K_EFF];
  const int KP = (K + 3) & ~3;            // row pitch of A^{-1} and dA: 16-byte rows, zero padded
  float* spi = dsm;                       // K x KP
  float* sdA = spi + K * KP;              // K x KP
  float* smu = sdA + K * KP;              // K x rho
  for (int i = threadIdx.x; i < K * rho; i += blockDim.x) smu[i] = mu[i];
  for (int i = threadIdx.x; i < K * KP; i += blockDim.x) {
    const int k = i / KP, l = i % KP;
    spi[i] = l < K ? pinv[k * K + l] : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < K * KP; i += blockDim.x) {
    const int k = i / KP, l = i % KP;
    float v = 0.0f;
    if (l < K) {
      float d2 = 0.0f;
      for (int d = 0; d < rho; ++d) {
        const float t = smu[k * rho + d] - smu[l * rho + d];
        d2 = fmaf(t, t, d2);
      }
      v = expf(-0.5f * d2 * inv_sr2) * d2 * inv_sr2;     // dA_kl / dlog sigma_r
    }
    sdA[i] = v;
  }
  if (threadIdx.x == 0 && blockIdx.x == 0 && ctrl[CTRL_RANKDEF]) record_error(ctrl, HDF_EDOMAIN);
  __syncthreads();
  double acc = 0.0;
  for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < N; pix += gridDim.x * blockDim.x) {
    const bool fb = flag[pix] != 0;
    float gv[KMAX], cv[KMAX], x[RMAX], gacc[RMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      gv[k] = (k < K) ? gam[(size_t)k * N + pix] : 0.0f;
      cv[k] = (k < K) ? C[(size_t)k * N + pix] : 0.0f;
    }
#pragma unroll
    for (int d = 0; d < RMAX; ++d) {
      x[d] = (d < rho) ? guide_load(p, (size_t)d * N + pix) : 0.0f;
      gacc[d] = 0.0f;
    }
    float t = 0.0f;
    // centres in groups of KC: their b_k and beta_k loaded together first
    // (up to 16 centres; beyond, the registers this takes cost more
    // occupancy than the loads in flight gain)
    constexpr int KC = KMAX <= 16 ? 8 : 1;
#pragma unroll 1
    for (int k0 = 0; k0 < K; k0 += KC) {
      float bkv[KC], btv[KC];
#pragma unroll
      for (int j = 0; j < KC; ++j) {
        const int k = k0 + j;
        bkv[j] = k < K ? B[(size_t)k * N + pix] : 0.0f;
        btv[j] = k < K ? bet[(size_t)k * N + pix] : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < KC; ++j) {
        const int k = k0 + j;
        if (k >= K) break;
        float eta = 0.0f, dAc = 0.0f;
        if (!fb) {
          const float4* pr = reinterpret_cast<const float4*>(spi + k * KP);
          const float4* dr = reinterpret_cast<const float4*>(sdA + k * KP);
#pragma unroll
          for (int q = 0; q < KMAX / 4; ++q) {
            if (4 * q < K) {   // padded entries are 0, and gv, cv are 0 beyond K
              const float4 pa = pr[q], da = dr[q];
              eta = fmaf(pa.x, gv[4 * q], eta);
              eta = fmaf(pa.y, gv[4 * q + 1], eta);
              eta = fmaf(pa.z, gv[4 * q + 2], eta);
              eta = fmaf(pa.w, gv[4 * q + 3], eta);
              dAc = fmaf(da.x, cv[4 * q], dAc);
              dAc = fmaf(da.y, cv[4 * q + 1], dAc);
              dAc = fmaf(da.z, cv[4 * q + 2], dAc);
              dAc = fmaf(da.w, cv[4 * q + 3], dAc);
            }
          }
        }
        const float beta = btv[j] + eta;                              // dL/db_k
        const float coef = beta * bkv[j] * inv_sr2;
        float d2 = 0.0f;
#pragma unroll
        for (int d = 0; d < RMAX; ++d) {
          if (d < rho) {
            const float dd = smu[k * rho + d] - x[d];
            d2 = fmaf(dd, dd, d2);
            gacc[d] = fmaf(coef, dd, gacc[d]);                       // b_k (mu_k - p) / sigma_r^2
          }
        }
        t += coef * d2 - eta * dAc;
      }
    }
    acc += (double)t;
    if (guide_is_image) {
#pragma unroll
      for (int d = 0; d < RMAX; ++d)
        if (d < rho) grad_f[(size_t)d * N + pix] += gacc[d];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < BW_THREADS / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

__global__ void bwd_sum_kernel(const double* __restrict__ ps, int ns, const double* __restrict__ pr,
                               int nr, double* __restrict__ out) {
  __shared__ double red[2][BW_THREADS];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) a += ps[i];
  for (int i = threadIdx.x; i < nr; i += blockDim.x) b += pr[i];
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[0][0];
    out[1] = red[1][0];
  }
}

template <int KMAX, int RMAX>
cudaError_t launch_final(hdf_handle* h, const float* f, const void* p, int gi, float* grad_f,
                         int blocks, cudaStream_t st) {
  const hdf_desc& d = h->d;
  const float inv_sr2 = (float)(1.0 / (d.sigma_r * d.sigma_r));
  const size_t smem = sizeof(float) * ((size_t)d.K * d.rho + 2 * (size_t)d.K * ((d.K + 3) & ~3));
  if (d.guide_dtype == HDF_GUIDE_BF16)
    bwd_final_kernel<KMAX, RMAX, __nv_bfloat16><<<blocks, BW_THREADS, smem, st>>>(
        f, (const __nv_bfloat16*)p, gi, h->B, h->C, h->bw_gam, h->bw_bet, h->bw_flag, h->mu,
        h->pinv32, h->ctrl, h->N, d.n, d.rho, inv_sr2, grad_f, h->grad_scratch + PART_SIGMA_R);
  else
    bwd_final_kernel<KMAX, RMAX, float><<<blocks, BW_THREADS, smem, st>>>(
        f, (const float*)p, gi, h->B, h->C, h->bw_gam, h->bw_bet, h->bw_flag, h->mu, h->pinv32,
        h->ctrl, h->N, d.n, d.rho, inv_sr2, grad_f, h->grad_scratch + PART_SIGMA_R);
  return cudaGetLastError();
}

template <int KMAX>
cudaError_t launch_final_r(hdf_handle* h, const float* f, const void* p, int gi, float* grad_f,
                           int blocks, cudaStream_t st) {
  const int rho = h->d.rho;
  if (rho <= 4) return launch_final<KMAX, 4>(h, f, p, gi, grad_f, blocks, st);
  if (rho <= 8) return launch_final<KMAX, 8>(h, f, p, gi, grad_f, blocks, st);
  if (rho <= 32) return launch_final<KMAX, 32>(h, f, p, gi, grad_f, blocks, st);
  return launch_final<KMAX, 64>(h, f, p, gi, grad_f, blocks, st);
}

}  // namespace

cudaError_t launch_backward(hdf_handle* h, const float* f, const void* p, const float* G,
                            float* grad_f, double* grad_ls, cudaStream_t st, const float* g_fwd) {
  const hdf_desc& d = h->d;
  const int SB = filter_bucket(d.S);
  if (SB < 0) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  const int ty = SB > 24 ? 32 : 64;            // tile height of the backward tile kernels
  const int ntiles = ((d.W + 31) / 32) * ((d.H + ty - 1) / ty);
  if (ntiles > PART_SIGMA_R) return cudaErrorInvalidValue;   // per-tile partials must fit
  // 1. forward recompute (g_hat into scratch, D, guard list), unless the
  //    handle still holds the state of the apply that produced g_fwd
  const float* ghat = g_fwd;
  if (!ghat) {
    if ((e = launch_rangemap(h, p, st)) != cudaSuccess) return e;
    if ((e = launch_filter(h, f, p, h->bw_g, st, 0)) != cudaSuccess) return e;
    ghat = h->bw_g;
  }
  // 2. guarded pixels
  if ((e = cudaMemsetAsync(h->bw_flag, 0, h->N, st)) != cudaSuccess) return e;
  const Taps exact = make_taps(d.sigma_s, d.S, d.spatial);
  bwd_fallback_kernel<<<sms, 256, 0, st>>>(h->B, h->s, h->fix_list, h->ctrl, d.H, d.W, d.K, d.S,
                                           exact, h->den, h->C, h->bw_flag);
  // 3. lambda planes
  bwd_lambda_kernel<<<sms * 4, 256, 0, st>>>(G, ghat, h->den, h->N, d.n, h->bw_lam);
  // 4./5. tile passes; omega_1 and omega_1' = omega_1 t^2 / sigma_s^2 centred in the bucket
  Taps t1, t2;
  for (int t = 0; t < 2 * HDF_MAX_S + 1; ++t) t1.w[t] = t2.w[t] = 0.0f;
  for (int j = -d.S; j <= d.S; ++j) {
    t1.w[SB + j] = exact.w[d.S + j];
    t2.w[SB + j] = (float)((double)exact.w[d.S + j] * j * j / (d.sigma_s * d.sigma_s));
  }
  BwdArgs a{f, h->bw_lam, h->B, h->C, h->bw_gam, h->bw_bet, grad_f,
            h->grad_scratch + PART_SIGMA_S, h->ctrl, d.H, d.W, d.n,
            (d.W % 4 == 0 && reinterpret_cast<uintptr_t>(f) % 16 == 0) ? 1 : 0};
  if ((e = launch_bwd_sb(SB, MODE_GAMMA, a, t1, t2, st)) != cudaSuccess) return e;
  if ((e = launch_bwd_sb(SB, MODE_ADJ, a, t1, t2, st)) != cudaSuccess) return e;
  // 6. per-pixel closing terms
  const int gi = (p == (const void*)f && d.rho == d.n && d.guide_dtype == HDF_GUIDE_F32) ? 1 : 0;
  const int blocks = sms * 4;
  const int K = d.K;
  if (K <= 8) e = launch_final_r<8>(h, f, p, gi, grad_f, blocks, st);
  else if (K <= 16) e = launch_final_r<16>(h, f, p, gi, grad_f, blocks, st);
  else if (K <= 32) e = launch_final_r<32>(h, f, p, gi, grad_f, blocks, st);
  else e = launch_final_r<64>(h, f, p, gi, grad_f, blocks, st);
  if (e != cudaSuccess) return e;
  // 7. scalar sums
  bwd_sum_kernel<<<1, BW_THREADS, 0, st>>>(h->grad_scratch + PART_SIGMA_S, ntiles,
                                           h->grad_scratch + PART_SIGMA_R, blocks, grad_ls);
  return cudaGetLastError();
}

}  // namespace hdf
