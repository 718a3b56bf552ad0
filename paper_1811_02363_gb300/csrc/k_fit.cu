// Algorithm 1 "pinv": the kernel matrix A_kl = phi(mu_k - mu_l) (Eq. (12))
// and its Moore-Penrose pseudo-inverse in FP64 (Sec. II-C uses MATLAB pinv),
// computed by one CTA on the device so that no host round trip is needed
// between clustering and filtering.
//
// Two routes, same result up to rounding:
//  * A = L D L^T (unit lower L, square-root free Cholesky) and
//    A^{-1} = L^{-T} D^{-1} L^{-1}, taken when every pivot is positive and
//    the Frobenius bound ||A||_F ||A^{-1}||_F K 2^-52 < 1/2 certifies that
//    every eigenvalue of A exceeds MATLAB's default tolerance K eps(||A||_2)
//    -- then pinv(A) is the inverse.  This is the common case (distinct
//    centres make the Gaussian Gram matrix positive definite) and costs
//    O(K^3/2) FP64 FMAs.
//  * otherwise cyclic Jacobi A = Q diag(lam) Q^T (Golub & Van Loan, symmetric
//    Schur rotations) and A^+ = sum over |lam| > K eps(max|lam|) of
//    q q^T / lam, the MATLAB rule.
#include <math.h>

#include "hdf_internal.cuh"

namespace hdf {
namespace {

constexpr int FIT_THREADS = 256;

__device__ double matlab_tol(double norm2, int K) {
  // eps(x) for a double x > 0: 2^(floor(log2 x) - 52).
  if (!(norm2 > 0.0)) return 0.0;
  int e;
  frexp(norm2, &e);  // norm2 = m 2^e, m in [0.5, 1)
  return (double)K * ldexp(1.0, e - 53);
}

// Pair p (0 <= p < K (K - 1) / 2) of the strict upper triangle in row-major
// order -> (k, l), k < l.  Row r starts at r (2K - r - 1) / 2.
__device__ __forceinline__ void pair_of(int p, int K, int& k, int& l) {
  const float b = 2.0f * K - 1.0f;
  int r = (int)floorf((b - sqrtf(b * b - 8.0f * (float)p)) * 0.5f);
  r = max(0, min(r, K - 2));
  while (r + 1 <= K - 2 && (r + 1) * (2 * K - r - 2) / 2 <= p) ++r;
  while (r > 0 && r * (2 * K - r - 1) / 2 > p) --r;
  k = r;
  l = p - r * (2 * K - r - 1) / 2 + r + 1;
}

// Entry t of a lower triangle (b <= a) in row-major order -> (a, b).
__device__ __forceinline__ void tri_of(int t, int& a, int& b) {
  int r = (int)floorf((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  r = max(r, 0);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  a = r;
  b = t - r * (r + 1) / 2;
}

// FP64 on this part issues at a small fraction of the FP32 rate, so the
// routes below keep the dependent FP64 steps few: every elimination step is
// one block-wide phase (one barrier), and the one reciprocal a step needs is
// taken by the thread that produced the next pivot in the previous phase.
__device__ void fit_run(const float* __restrict__ mu, int rho, int* ctrl, double inv2sr2,
                        double* __restrict__ pinv64, float* __restrict__ pinv32, double* sm) {
  const int K = ctrl[CTRL_K_EFF];
  const int tid = threadIdx.x, nt = blockDim.x;
  double* A = sm;              // K x K (kept for the eigen route)
  double* L = A + K * K;       // K x K: L D L^T in place, then Jacobi eigenvectors
  double* X = L + K * K;       // K x K: L^{-1}, then the working matrix of Jacobi
  __shared__ int s_flag;
  __shared__ double s_red[FIT_THREADS];
  __shared__ double s_cs[2];
  __shared__ double s_rd[HDF_MAX_K];   // 1 / d_j

  // A_kl = phi(mu_k - mu_l) for k < l (symmetric; phi(0) = 1 on the diagonal)
  for (int p = tid; p < K * (K - 1) / 2; p += nt) {
    int k, l;
    pair_of(p, K, k, l);
    double d2 = 0.0;
    for (int d = 0; d < rho; ++d) {
      const double t = (double)mu[k * rho + d] - (double)mu[l * rho + d];
      d2 += t * t;
    }
    const double v = exp(-d2 * inv2sr2);
    A[k * K + l] = v;
    A[l * K + k] = v;
    L[l * K + k] = v;   // the lower triangle is the factorisation's copy
  }
  for (int k = tid; k < K; k += nt) {
    A[k * K + k] = 1.0;
    L[k * K + k] = 1.0;
  }
  for (int idx = tid; idx < K * K; idx += nt) X[idx] = (idx / K == idx % K) ? 1.0 : 0.0;
  if (tid == 0) {
    s_flag = 1;
    s_rd[0] = 1.0;   // d_0 = A_00 = 1
  }
  __syncthreads();

  // ---- L D L^T, right-looking: in step j the lower trailing entries
  // (i >= l > j) take L_il -= L_ij L_lj / d_j with column j still unscaled
  // (L_ij = A'_ij); the thread of entry (j+1, j+1) then holds d_{j+1} and
  // takes its reciprocal.  Columns are scaled by 1 / d_j afterwards.
  for (int j = 0; j + 1 < K; ++j) {
    const double rdj = s_rd[j];
    const int m = K - 1 - j;
    for (int t = tid; t < m * (m + 1) / 2; t += nt) {
      int ai, bl;
      tri_of(t, ai, bl);
      const int i = j + 1 + ai, l = j + 1 + bl;
      const double v = L[i * K + l] - L[i * K + j] * (L[l * K + j] * rdj);
      L[i * K + l] = v;
      if (t == 0) {   // (j+1, j+1): the next pivot
        if (!(v > 0.0)) s_flag = 0;
        s_rd[j + 1] = v > 0.0 ? __drcp_rn(v) : 0.0;
      }
    }
    __syncthreads();
    if (s_rd[j + 1] == 0.0) break;   // written in this step only: a uniform exit
  }
  bool full_rank = false;
  if (tid == 0) ctrl[CTRL_RANKDEF] = 0;
  if (s_flag) {
    for (int t = tid; t < K * (K - 1) / 2; t += nt) {   // L_ij = A'_ij / d_j, i > j
      int ai, bj;
      tri_of(t, ai, bj);
      L[(ai + 1) * K + bj] *= s_rd[bj];
    }
    __syncthreads();
    // X = L^{-1} (unit lower), right-looking: in step m the rows i > m take
    // X_ic -= L_im X_mc for c <= m (row m is final after step m - 1).
    for (int m = 0; m + 1 < K; ++m) {
      const int w = m + 1;
      for (int t = tid; t < (K - 1 - m) * w; t += nt) {
        const int i = m + 1 + t / w, c = t % w;
        X[i * K + c] -= L[i * K + m] * X[m * K + c];
      }
      __syncthreads();
    }
    // A^{-1}_kl = sum_{m >= max(k, l)} X_mk X_ml / d_m: Y = D^{-1} X into L
    // (the factor is no longer needed), then one pass per entry k <= l.
    for (int idx = tid; idx < K * K; idx += nt) L[idx] = X[idx] * s_rd[idx / K];
    __syncthreads();
    double fx = 0.0, fa = 0.0;
    for (int idx = tid; idx < K * K; idx += nt) {
      const int k = idx % K, l = idx / K;   // a warp shares l: equal trip counts
      fa += A[idx] * A[idx];
      if (k > l) continue;
      double s = 0.0;
      for (int m = l; m < K; ++m) s = fma(L[m * K + k], X[m * K + l], s);
      pinv64[k * K + l] = s;
      pinv64[l * K + k] = s;
      fx += (k == l ? 1.0 : 2.0) * s * s;
    }
    s_red[tid] = fx;
    __syncthreads();
    for (int o = nt / 2; o > 0; o >>= 1) {
      if (tid < o) s_red[tid] += s_red[tid + o];
      __syncthreads();
    }
    const double nx = sqrt(s_red[0]);
    __syncthreads();
    s_red[tid] = fa;
    __syncthreads();
    for (int o = nt / 2; o > 0; o >>= 1) {
      if (tid < o) s_red[tid] += s_red[tid + o];
      __syncthreads();
    }
    const double na = sqrt(s_red[0]);
    full_rank = isfinite(nx) && nx * na * (double)K * ldexp(1.0, -52) < 0.5;
    __syncthreads();
  }
  if (!full_rank) {
    // ---- Cyclic Jacobi on X = A, eigenvectors accumulated in L.
    for (int idx = tid; idx < K * K; idx += nt) {
      X[idx] = A[idx];
      L[idx] = (idx / K == idx % K) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 60; ++sweep) {
      double off = 0.0, dia = 0.0;
      for (int idx = tid; idx < K * K; idx += nt) {
        const double v = X[idx] * X[idx];
        if (idx / K == idx % K) dia += v; else off += v;
      }
      s_red[tid] = off;
      __syncthreads();
      for (int o = nt / 2; o > 0; o >>= 1) {
        if (tid < o) s_red[tid] += s_red[tid + o];
        __syncthreads();
      }
      const double off_all = s_red[0];
      __syncthreads();
      s_red[tid] = dia;
      __syncthreads();
      for (int o = nt / 2; o > 0; o >>= 1) {
        if (tid < o) s_red[tid] += s_red[tid + o];
        __syncthreads();
      }
      const double dia_all = s_red[0];
      __syncthreads();
      if (off_all <= 1e-34 * dia_all || off_all == 0.0) break;
      for (int p = 0; p < K - 1; ++p) {
        for (int q = p + 1; q < K; ++q) {
          if (tid == 0) {
            const double apq = X[p * K + q];
            double c = 1.0, s = 0.0;
            if (apq != 0.0) {
              const double tau = (X[q * K + q] - X[p * K + p]) / (2.0 * apq);
              const double t = tau >= 0.0 ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                          : -1.0 / (-tau + sqrt(1.0 + tau * tau));
              c = 1.0 / sqrt(1.0 + t * t);
              s = t * c;
            }
            s_cs[0] = c;
            s_cs[1] = s;
          }
          __syncthreads();
          const double c = s_cs[0], s = s_cs[1];
          if (s != 0.0) {
            for (int k = tid; k < K; k += nt) {  // columns p, q of X J
              const double xp = X[k * K + p], xq = X[k * K + q];
              X[k * K + p] = c * xp - s * xq;
              X[k * K + q] = s * xp + c * xq;
            }
            __syncthreads();
            for (int k = tid; k < K; k += nt) {  // rows p, q of J^T (X J)
              const double xp = X[p * K + k], xq = X[q * K + k];
              X[p * K + k] = c * xp - s * xq;
              X[q * K + k] = s * xp + c * xq;
              const double vp = L[k * K + p], vq = L[k * K + q];
              L[k * K + p] = c * vp - s * vq;
              L[k * K + q] = s * vp + c * vq;
            }
          }
          __syncthreads();
        }
      }
    }
    // Eigenvalues X_mm, eigenvectors L[:, m]; MATLAB tolerance on max |lam|.
    double lmax = 0.0;
    for (int m = 0; m < K; ++m) lmax = fmax(lmax, fabs(X[m * K + m]));
    const double tol = matlab_tol(lmax, K);
    if (tid == 0) {
      int dropped = 0;
      for (int m = 0; m < K; ++m) dropped += !(fabs(X[m * K + m]) > tol);
      ctrl[CTRL_RANKDEF] = dropped > 0;
    }
    for (int idx = tid; idx < K * K; idx += nt) {
      const int k = idx / K, l = idx % K;
      double s = 0.0;
      for (int m = 0; m < K; ++m) {
        const double lam = X[m * K + m];
        if (fabs(lam) > tol) s += L[k * K + m] * L[l * K + m] / lam;
      }
      pinv64[idx] = s;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < K * K; idx += nt) pinv32[idx] = (float)pinv64[idx];
}

__global__ void __launch_bounds__(FIT_THREADS)
fit_kernel(const float* __restrict__ mu, int rho, int* ctrl, double inv2sr2,
           double* __restrict__ pinv64, float* __restrict__ pinv32) {
  extern __shared__ double sm[];
  fit_run(mu, rho, ctrl, inv2sr2, pinv64, pinv32, sm);
}

// One block per entry of a batch table.
__global__ void __launch_bounds__(FIT_THREADS)
fit_batch_kernel(const FitJob* __restrict__ jobs) {
  extern __shared__ double sm[];
  const FitJob j = jobs[blockIdx.x];
  fit_run(j.mu, j.rho, j.ctrl, j.inv2sr2, j.pinv64, j.pinv32, sm);
}

__global__ void set_int_kernel(int* p, int v) { *p = v; }

}  // namespace

cudaError_t launch_fit(hdf_handle* h, cudaStream_t st) {
  const int K = h->d.K;
  const size_t smem = 3 * (size_t)K * K * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const double inv2sr2 = 1.0 / (2.0 * h->d.sigma_r * h->d.sigma_r);
  fit_kernel<<<1, FIT_THREADS, smem, st>>>(h->mu, h->d.rho, h->ctrl, inv2sr2, h->pinv64,
                                           h->pinv32);
  return cudaGetLastError();
}

cudaError_t launch_fit_batch(const FitJob* jobs, int njobs, int Kmax, cudaStream_t st) {
  if (njobs < 1) return cudaSuccess;
  const size_t smem = 3 * (size_t)Kmax * Kmax * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fit_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  fit_batch_kernel<<<njobs, FIT_THREADS, smem, st>>>(jobs);
  return cudaGetLastError();
}

cudaError_t launch_set_int(int* p, int v, cudaStream_t st) {
  set_int_kernel<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}

}  // namespace hdf
