// Brute-force high-dimensional bilateral / NLM filter, Eq. (1)-(2):
//   g(i) = sum_{j in W} omega(j) phi(p(i-j) - p(i)) f(i-j) / eta(i).
// Float32 guides of up to 32 dimensions take the register-blocked tile kernel
// (brute_tile.cuh); the others (bfloat16 guides, more dimensions, the widest
// bucket at 32 dimensions) take the kernel below: one thread per output pixel,
// the window's guide (and image, unless it aliases the guide) staged in shared
// memory per tile when it fits, read through the cache otherwise.  Neighbours
// outside the image are left out.
#include <math.h>

#include "brute_tile.cuh"
#include "hdf_internal.cuh"

namespace hdf {

cudaError_t launch_brute_tile_a(int maxc, int SB, const BruteTileArgs& a, const Taps& t,
                                cudaStream_t st);
cudaError_t launch_brute_tile_b(int maxc, int SB, const BruteTileArgs& a, const Taps& t,
                                cudaStream_t st);

namespace {

struct BruteArgs {
  const float* f;
  const void* p;
  float* g;
  int H, W, n, rho, S;
  int alias;          // guide is the image (p == f, rho == n, float32)
  float inv2sr2;
};

template <int MAXC, typename GT, bool STAGED>
__global__ void __launch_bounds__(256)
brute_kernel(const BruteArgs a, const Taps taps) {
  extern __shared__ float sm[];
  const int TXb = blockDim.x, TYb = blockDim.y;
  const int H = a.H, W = a.W, n = a.n, rho = a.rho, S = a.S;
  const size_t N = (size_t)H * W;
  const int x = blockIdx.x * TXb + threadIdx.x;
  const int y = blockIdx.y * TYb + threadIdx.y;
  const int HRb = TYb + 2 * S, HCb = TXb + 2 * S;
  const int ox = blockIdx.x * TXb - S, oy = blockIdx.y * TYb - S;
  const GT* p = (const GT*)a.p;
  float* sP = sm;                                   // [rho][HRb][HCb]
  float* sF = a.alias ? sm : sm + (size_t)rho * HRb * HCb;   // [n][HRb][HCb]
  if (STAGED) {
    const int tid = threadIdx.y * TXb + threadIdx.x, nt = TXb * TYb;
    const int planes = a.alias ? rho : rho + n;
    for (int idx = tid; idx < planes * HRb * HCb; idx += nt) {
      const int q = idx / (HRb * HCb);
      const int r = (idx / HCb) % HRb, c = idx % HCb;
      const int yy = oy + r, xx = ox + c;
      float v = 0.0f;
      if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
        const size_t off = (size_t)yy * W + xx;
        v = (q < rho) ? guide_load(p, (size_t)q * N + off) : __ldg(a.f + (size_t)(q - rho) * N + off);
      }
      sm[idx] = v;
    }
    __syncthreads();
  }
  if (x >= W || y >= H) return;
  float pi[MAXC], num[MAXC];
#pragma unroll
  for (int d = 0; d < MAXC; ++d) {
    pi[d] = (d < rho) ? guide_load(p, (size_t)d * N + (size_t)y * W + x) : 0.0f;
    num[d] = 0.0f;
  }
  float den = 0.0f;
  for (int j1 = -S; j1 <= S; ++j1) {
    const int yy = y - j1;
    if (yy < 0 || yy >= H) continue;
    const float wy = taps.w[j1 + S];
    for (int j2 = -S; j2 <= S; ++j2) {
      const int xx = x - j2;
      if (xx < 0 || xx >= W) continue;
      float d2 = 0.0f;
      if (STAGED) {
        const int off = (yy - oy) * HCb + (xx - ox);
#pragma unroll
        for (int d = 0; d < MAXC; ++d)
          if (d < rho) {
            const float t = sP[(size_t)d * HRb * HCb + off] - pi[d];
            d2 = fmaf(t, t, d2);
          }
        const float wt = wy * taps.w[j2 + S] * expf(-d2 * a.inv2sr2);
        den += wt;
#pragma unroll
        for (int c = 0; c < MAXC; ++c)
          if (c < n) num[c] = fmaf(wt, sF[(size_t)c * HRb * HCb + off], num[c]);
      } else {
        const size_t off = (size_t)yy * W + xx;
#pragma unroll
        for (int d = 0; d < MAXC; ++d)
          if (d < rho) {
            const float t = guide_load(p, (size_t)d * N + off) - pi[d];
            d2 = fmaf(t, t, d2);
          }
        const float wt = wy * taps.w[j2 + S] * expf(-d2 * a.inv2sr2);
        den += wt;
#pragma unroll
        for (int c = 0; c < MAXC; ++c)
          if (c < n) num[c] = fmaf(wt, __ldg(a.f + (size_t)c * N + off), num[c]);
      }
    }
  }
  const float inv = 1.0f / den;
#pragma unroll
  for (int c = 0; c < MAXC; ++c)
    if (c < n) a.g[(size_t)c * N + (size_t)y * W + x] = num[c] * inv;
}

template <int MAXC, typename GT>
cudaError_t launch_brute_t(const BruteArgs& a, const Taps& taps, cudaStream_t st) {
  const int planes = a.alias ? a.rho : a.rho + a.n;
  const size_t limit = 227 * 1024;
  int TXb = 16, TYb = 16;
  size_t smem = sizeof(float) * planes * (size_t)(TYb + 2 * a.S) * (TXb + 2 * a.S);
  if (smem > limit) {
    TYb = 8;
    smem = sizeof(float) * planes * (size_t)(TYb + 2 * a.S) * (TXb + 2 * a.S);
  }
  dim3 block(TXb, TYb);
  dim3 grid((a.W + TXb - 1) / TXb, (a.H + TYb - 1) / TYb);
  if (smem <= limit) {
    cudaError_t e = cudaFuncSetAttribute(brute_kernel<MAXC, GT, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    brute_kernel<MAXC, GT, true><<<grid, block, smem, st>>>(a, taps);
  } else {
    brute_kernel<MAXC, GT, false><<<grid, block, 0, st>>>(a, taps);
  }
  return cudaGetLastError();
}

template <typename GT>
cudaError_t launch_brute_c(const BruteArgs& a, const Taps& taps, cudaStream_t st) {
  const int c = a.n > a.rho ? a.n : a.rho;
  if (c <= 4) return launch_brute_t<4, GT>(a, taps, st);
  if (c <= 8) return launch_brute_t<8, GT>(a, taps, st);
  if (c <= 16) return launch_brute_t<16, GT>(a, taps, st);
  if (c <= 32) return launch_brute_t<32, GT>(a, taps, st);
  if (c <= 64) return launch_brute_t<64, GT>(a, taps, st);
  return cudaErrorNotSupported;
}

}  // namespace

cudaError_t launch_bruteforce(const hdf_desc& d, const float* f, const void* p, float* g,
                              cudaStream_t st) {
  BruteArgs a{f, p, g, d.H, d.W, d.n, d.rho, d.S,
              (p == (const void*)f && d.rho == d.n && d.guide_dtype == HDF_GUIDE_F32) ? 1 : 0,
              (float)(1.0 / (2.0 * d.sigma_r * d.sigma_r))};
  const Taps taps = make_taps(d.sigma_s, d.S, d.spatial);
  if (d.guide_dtype == HDF_GUIDE_BF16) return launch_brute_c<__nv_bfloat16>(a, taps, st);
  const int SB = filter_bucket(d.S);
  const int c = d.n > d.rho ? d.n : d.rho;
  const int maxc = c <= 4 ? 4 : c <= 8 ? 8 : c <= 16 ? 16 : c <= 32 ? 32 : 0;
  if (SB > 0 && maxc > 0) {
    // taps centred in the bucket: w[SB + j] = omega_1(j) for |j| <= S, 0 beyond
    Taps tb;
    for (int t = 0; t < 2 * HDF_MAX_S + 1; ++t) tb.w[t] = 0.0f;
    for (int j = -d.S; j <= d.S; ++j) tb.w[SB + j] = taps.w[d.S + j];
    BruteTileArgs bt{f, (const float*)p, g, d.H, d.W, d.n, d.rho, a.alias, a.inv2sr2};
    const cudaError_t e = maxc <= 8 ? launch_brute_tile_a(maxc, SB, bt, tb, st)
                                    : launch_brute_tile_b(maxc, SB, bt, tb, st);
    if (e != cudaErrorNotSupported) return e;
  }
  return launch_brute_c<float>(a, taps, st);
}

}  // namespace hdf
