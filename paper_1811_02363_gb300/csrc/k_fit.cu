// Algorithm 1 "pinv": the kernel matrix A_kl = phi(mu_k - mu_l) (Eq. (12))
// and its Moore-Penrose pseudo-inverse in FP64 (Sec. II-C uses MATLAB pinv),
// computed by one CTA on the device so that no host round trip is needed
// between clustering and filtering.
//
// Two routes, same result up to rounding:
//  * Cholesky A = L L^T and A^{-1} = L^{-T} L^{-1}, taken when the Frobenius
//    bound ||A||_F ||A^{-1}||_F K 2^-52 < 1/2 certifies that every eigenvalue
//    of A exceeds MATLAB's default tolerance K eps(||A||_2) -- then pinv(A)
//    is the inverse.  This is the common case (distinct centres make the
//    Gaussian Gram matrix positive definite) and costs O(K^3/3) FP64 FMAs.
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

__device__ void fit_run(const float* __restrict__ mu, int rho, int* ctrl, double inv2sr2,
                        double* __restrict__ pinv64, float* __restrict__ pinv32, double* sm) {
  const int K = ctrl[CTRL_K_EFF];
  const int tid = threadIdx.x, nt = blockDim.x;
  double* A = sm;              // K x K
  double* L = A + K * K;       // K x K (Cholesky factor, then Jacobi eigenvectors)
  double* X = L + K * K;       // K x K (inverse / working matrix)
  __shared__ int s_flag;
  __shared__ double s_red[FIT_THREADS];
  __shared__ double s_cs[2];

  for (int idx = tid; idx < K * K; idx += nt) {
    const int k = idx / K, l = idx % K;
    double d2 = 0.0;
    for (int d = 0; d < rho; ++d) {
      const double t = (double)mu[k * rho + d] - (double)mu[l * rho + d];
      d2 += t * t;
    }
    A[idx] = exp(-d2 * inv2sr2);
    L[idx] = 0.0;
  }
  if (tid == 0) s_flag = 1;
  __syncthreads();

  // ---- Cholesky, column by column.
  for (int j = 0; j < K; ++j) {
    if (tid == 0) {
      double s = A[j * K + j];
      for (int m = 0; m < j; ++m) s -= L[j * K + m] * L[j * K + m];
      if (!(s > 0.0)) s_flag = 0;
      L[j * K + j] = s > 0.0 ? sqrt(s) : 1.0;
    }
    __syncthreads();
    if (!s_flag) break;
    const double djj = L[j * K + j];
    for (int i = j + 1 + tid; i < K; i += nt) {
      double s = A[i * K + j];
      for (int m = 0; m < j; ++m) s -= L[i * K + m] * L[j * K + m];
      L[i * K + j] = s / djj;
    }
    __syncthreads();
  }
  bool full_rank = false;
  if (tid == 0) ctrl[CTRL_RANKDEF] = 0;
  if (s_flag) {
    // Column c of L^{-1} by forward substitution (one thread per column),
    // stored transposed: X[c*K + i] = (L^{-1})_{i c}.
    for (int c = tid; c < K; c += nt) {
      for (int i = 0; i < K; ++i) {
        double s = (i == c) ? 1.0 : 0.0;
        for (int m = c; m < i; ++m) s -= L[i * K + m] * X[c * K + m];
        X[c * K + i] = (i < c) ? 0.0 : s / L[i * K + i];
      }
    }
    __syncthreads();
    // A^{-1}_{kl} = sum_m (L^{-1})_{m k} (L^{-1})_{m l}; written to pinv64.
    double fx = 0.0, fa = 0.0;
    for (int idx = tid; idx < K * K; idx += nt) {
      const int k = idx / K, l = idx % K;
      double s = 0.0;
      for (int m = (k > l ? k : l); m < K; ++m) s += X[k * K + m] * X[l * K + m];
      pinv64[idx] = s;
      fx += s * s;
      fa += A[idx] * A[idx];
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
