// FP64 recomputation of the pixels whose float32 combine cannot be trusted
// (hdf_apply): the divide kernel lists, from the end of the guard list, the
// pixels where sum_k |c_k| r_k exceeds 64 |sum_k c_k r_k| (the float32
// numerator and denominator lose more than 1e-4 to cancellation) or where the
// guard's threshold lies within the denominator's rounding.  For each listed
// pixel i one block evaluates Eq. (13)-(16) from their definitions in FP64:
//   b_k(i) = phi(mu_k - p(i)), c(i) = A^+ b(i) (Eq. (11)) or e_s (Eq. (17)),
//   beta(j) = sum_k c_k(i) phi(mu_k - p(i - j)),
//   r = sum_j omega(j) beta(j),  v = sum_j omega(j) beta(j) f(i - j),
//   r_k = sum_j omega(j) phi(mu_k - p(i - j))   (max_k r_k for the guard),
// then decides the guard in FP64 (r <= 1e-6 max_k r_k takes v_s / r_s, s the
// nearest centre, Eq. (18); f(i) if r_s = 0) and writes g_hat(i).  Window
// positions outside the image are left out (zero extension).  Every sum runs
// over the window in a fixed order (a fixed thread per position, xor trees in
// the warps, warps in ascending order), so the result is deterministic.
#include <math.h>

#include "combine.cuh"
#include "hdf_internal.cuh"

namespace hdf {
namespace {

constexpr int RS_THREADS = 128;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_CB = 8;   // channels summed together
constexpr int EXP_INT = 746;   // exp(-a), a = 0 .. 745 (beyond, exp(-x) underflows to 0)
constexpr int EXP_FRAC = 64;   // exp(-b / 64), b = 0 .. 63

// exp(-x) for x >= 0 in FP64 from two tables and a short polynomial:
// x = a + b / 64 + r with integers a, b and 0 <= r < 1/64, so that
// exp(-x) = exp(-a) exp(-b / 64) exp(-r), the last by its Taylor polynomial
// of degree 7 (truncation below (1/64)^8 / 8! < 2e-19).  The tables hold
// values of CUDA's exp computed once per block; the products carry a few
// units of 2^-53.  About half the FP64 operations of a general exp.
__device__ __forceinline__ double exp_neg(double x, const double* e_int, const double* e_frac) {
  if (!(x < (double)EXP_INT)) return 0.0;
  const double x64 = x * 64.0;
  const int k = (int)x64;                 // floor for x >= 0
  const int a = k >> 6, b = k & 63;
  const double r = (x64 - (double)k) * (1.0 / 64.0);   // exact: x64 - k < 1, then a power of 2
  double q = -1.0 / 5040.0;               // Horner for sum_{i<=7} (-r)^i / i!
  q = fma(q, r, 1.0 / 720.0);
  q = fma(q, r, -1.0 / 120.0);
  q = fma(q, r, 1.0 / 24.0);
  q = fma(q, r, -1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, -1.0);
  q = fma(q, r, 1.0);
  return e_int[a] * e_frac[b] * q;
}

struct RescueArgs {
  const float* f;        // (n, H, W)
  const void* p;         // (rho, H, W) guide
  int p_bf16;
  const float* mu;       // K x rho centres (float32, as the filter uses them)
  const double* pinv;    // K x K A^+ (FP64)
  int* ctrl;
  const int* list;       // the rescued pixels at list[N - 1 - e]
  float* g;              // (n, H, W) output
  int H, W, n, rho, S, box, coef;
  double sigma_s, inv2sr2;
};

__device__ __forceinline__ double guide_d(const RescueArgs& a, size_t i) {
  return a.p_bf16 ? (double)__bfloat162float(((const __nv_bfloat16*)a.p)[i])
                  : (double)__ldg((const float*)a.p + i);
}

// Sums over the block of nv <= NV per-thread values, fixed order: an xor tree
// within each warp, then the warps in ascending order.  red: RS_WARPS * NV
// shared doubles; out: nv shared doubles.  Ends with a block barrier.
template <int NV>
__device__ void block_sum_fixed(double (&v)[NV], int nv, double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < nv; ++k) {
    double t = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[warp * NV + k] = t;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nv; k += RS_THREADS) {
    double t = red[k];
    for (int w = 1; w < RS_WARPS; ++w) t += red[w * NV + k];
    out[k] = t;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(RS_THREADS)
rescue_kernel(const RescueArgs a) {
  extern __shared__ double dsm[];
  const int WS = 2 * a.S + 1, NWIN = WS * WS;
  const int rho = a.rho;
  const size_t N = (size_t)a.H * a.W;
  const int K = min(a.ctrl[CTRL_K_EFF], HDF_MAX_K);
  double* sWB = dsm;                 // [NWIN] omega(j) beta(j)
  double* sWS = sWB + NWIN;          // [NWIN] omega(j) phi_s(j)
  double* smu = sWS + NWIN;          // [K * rho] centres
  __shared__ double s_x[HDF_MAX_RHO], s_b[HDF_MAX_K], s_c[HDF_MAX_K], s_d2[HDF_MAX_K];
  __shared__ double s_w1[2 * HDF_MAX_S + 1];
  __shared__ double s_red[RS_WARPS * (HDF_MAX_K + 1)];
  __shared__ double s_sum[HDF_MAX_K + 1];
  __shared__ int s_s, s_guard;
  __shared__ double s_den, s_rs;
  __shared__ double e_int[EXP_INT], e_frac[EXP_FRAC];
  const int tid = threadIdx.x;
  int count = a.ctrl[CTRL_RESCUED];
  if (count > (int)N) count = (int)N;
  if (count <= (int)blockIdx.x) return;
  for (int t = tid; t < WS; t += RS_THREADS) {
    const double j = (double)(t - a.S);
    s_w1[t] = a.box ? 1.0 : exp(-(j * j) / (2.0 * a.sigma_s * a.sigma_s));
  }
  for (int i = tid; i < K * rho; i += RS_THREADS) smu[i] = (double)a.mu[i];
  for (int i = tid; i < EXP_INT; i += RS_THREADS) e_int[i] = exp(-(double)i);
  for (int i = tid; i < EXP_FRAC; i += RS_THREADS) e_frac[i] = exp(-(double)i / 64.0);
  for (int e = blockIdx.x; e < count; e += gridDim.x) {
    const int pix = a.list[N - 1 - e];
    if (pix < 0 || (size_t)pix >= N) {   // inconsistent list: record, write nothing
      if (tid == 0) record_error(a.ctrl, HDF_EDOMAIN);
      continue;
    }
    const int y = pix / a.W, x = pix - y * a.W;
    __syncthreads();   // the previous pixel's shared values are no longer read
    for (int d = tid; d < rho; d += RS_THREADS) s_x[d] = guide_d(a, (size_t)d * N + pix);
    __syncthreads();
    for (int k = tid; k < K; k += RS_THREADS) {
      double d2 = 0.0;
      for (int d = 0; d < rho; ++d) {
        const double t = s_x[d] - smu[k * rho + d];
        d2 = fma(t, t, d2);
      }
      s_d2[k] = d2;
      s_b[k] = exp_neg(d2 * a.inv2sr2, e_int, e_frac);
    }
    __syncthreads();
    if (tid == 0) {   // nearest centre, ties -> lowest k
      int s = 0;
      for (int k = 1; k < K; ++k)
        if (s_d2[k] < s_d2[s]) s = k;
      s_s = s;
    }
    __syncthreads();
    const int s = s_s;
    for (int k = tid; k < K; k += RS_THREADS) {
      double c = 0.0;
      if (a.coef == HDF_COEF_OPT) {
        for (int l = 0; l < K; ++l) c = fma(a.pinv[k * K + l], s_b[l], c);
      } else {
        c = (k == s) ? 1.0 : 0.0;
      }
      s_c[k] = c;
    }
    __syncthreads();
    // window pass: omega beta and omega phi_s per position, r_k and r partials
    double part[HDF_MAX_K + 1];
    for (int k = 0; k <= K; ++k) part[k] = 0.0;   // [0, K): r_k, [K]: r
    for (int q = tid; q < NWIN; q += RS_THREADS) {
      const int j1 = q / WS - a.S, j2 = q % WS - a.S;
      const int yy = y - j1, xx = x - j2;
      double wb = 0.0, wsv = 0.0;
      if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
        const size_t qi = (size_t)yy * a.W + xx;
        const double wt = s_w1[j1 + a.S] * s_w1[j2 + a.S];
        double xq[HDF_MAX_RHO];
        for (int d = 0; d < rho; ++d) xq[d] = guide_d(a, (size_t)d * N + qi);
        double beta = 0.0, phs = 0.0;
        for (int k = 0; k < K; ++k) {
          double d2 = 0.0;
          for (int d = 0; d < rho; ++d) {
            const double t = xq[d] - smu[k * rho + d];
            d2 = fma(t, t, d2);
          }
          const double ph = exp_neg(d2 * a.inv2sr2, e_int, e_frac);
          part[k] = fma(wt, ph, part[k]);
          beta = fma(s_c[k], ph, beta);
          if (k == s) phs = ph;
        }
        wb = wt * beta;
        wsv = wt * phs;
        part[K] += wb;
      }
      sWB[q] = wb;
      sWS[q] = wsv;
    }
    block_sum_fixed<HDF_MAX_K + 1>(part, K + 1, s_red, s_sum);
    if (tid == 0) {
      double rmax = 0.0;
      for (int k = 0; k < K; ++k) rmax = fmax(rmax, s_sum[k]);
      s_den = s_sum[K];
      s_rs = s_sum[s];
      s_guard = !(s_sum[K] > 1e-6 * rmax) ? 1 : 0;   // the guard, decided in FP64
      if (s_guard) atomicAdd(a.ctrl + CTRL_FALLBACK64, 1);
    }
    __syncthreads();
    const int guard = s_guard;
    const double den = s_den, rs = s_rs;
    const double* wgt = guard ? sWS : sWB;
    for (int c0 = 0; c0 < a.n; c0 += RS_CB) {
      const int nc = min(RS_CB, a.n - c0);
      double acc[RS_CB];
#pragma unroll
      for (int u = 0; u < RS_CB; ++u) acc[u] = 0.0;
      for (int q = tid; q < NWIN; q += RS_THREADS) {
        const int j1 = q / WS - a.S, j2 = q % WS - a.S;
        const int yy = y - j1, xx = x - j2;
        if (yy < 0 || yy >= a.H || xx < 0 || xx >= a.W) continue;
        const size_t qi = (size_t)yy * a.W + xx;
        const double w = wgt[q];
#pragma unroll
        for (int u = 0; u < RS_CB; ++u)
          if (u < nc) acc[u] = fma(w, (double)__ldg(a.f + (size_t)(c0 + u) * N + qi), acc[u]);
      }
      block_sum_fixed<RS_CB>(acc, nc, s_red, s_sum);
      for (int u = tid; u < nc; u += RS_THREADS) {
        const size_t o = (size_t)(c0 + u) * N + pix;
        double val;
        if (!guard) val = s_sum[u] / den;
        else val = rs > 0.0 ? s_sum[u] / rs : (double)a.f[o];
        a.g[o] = (float)val;
      }
    }
  }
}

}  // namespace

cudaError_t launch_rescue(hdf_handle* h, const float* f, const void* p, float* g, int* list,
                          cudaStream_t st) {
  const hdf_desc& d = h->d;
  RescueArgs a;
  a.f = f;
  a.p = p;
  a.p_bf16 = d.guide_dtype == HDF_GUIDE_BF16 ? 1 : 0;
  a.mu = h->mu;
  a.pinv = h->pinv64;
  a.ctrl = h->ctrl;
  a.list = list;
  a.g = g;
  a.H = d.H;
  a.W = d.W;
  a.n = d.n;
  a.rho = d.rho;
  a.S = d.S;
  a.box = d.spatial == HDF_SPATIAL_BOX ? 1 : 0;
  a.coef = d.coef;
  a.sigma_s = d.sigma_s;
  a.inv2sr2 = 1.0 / (2.0 * d.sigma_r * d.sigma_r);
  const int WS = 2 * d.S + 1;
  const size_t smem = sizeof(double) * (2 * (size_t)WS * WS + (size_t)d.K * d.rho);
  cudaError_t e = cudaFuncSetAttribute(rescue_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  rescue_kernel<<<(sms > 0 ? sms : 1) * 8, RS_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hdf
