// Guide for nonlocal means: every pixel's patch (patch x patch pixels of each
// channel around it; Sec. I-A), reduced by PCA to rho features (PCA-NLM,
// Sec. III-C): subtract the mean patch, take the eigenvectors of the patch
// covariance with the rho largest eigenvalues, project.  Borders are mirrored
// without repeating the edge pixel.
//
// Kernels: per-channel means (shift against cancellation), per-block sums of
// shifted patch vectors and their products (FP32 within a block, FP64 across
// blocks), one CTA for the covariance and its eigendecomposition (cyclic
// Jacobi in round-robin order, D/2 disjoint rotations per step, in float32),
// and the projection.
#include <math.h>

#include "hdf_internal.cuh"

namespace hdf {
namespace {

constexpr int NL_THREADS = 256;
constexpr int NL_TILE = 16;          // pixels per tile side in the covariance pass
constexpr int NL_MAXD = 96;          // patch dimension n * patch^2 handled by the FP64 eigen step
constexpr int EIG_THREADS = 1024;    // the one-CTA eigendecomposition: short row loops per round

__device__ __forceinline__ int mirror(int i, int n) {
  // reflect without repeating the edge: -1 -> 1, n -> n - 2 (n >= 2)
  if (i < 0) i = -i;
  if (i >= n) i = 2 * (n - 1) - i;
  return i;
}

// Patch coordinate a = (channel, dy, dx) in channel-major order, as in the oracle.
__device__ __forceinline__ float patch_val(const float* f, int H, int W, int m, int a, int y, int x) {
  const int h = m / 2;
  const int c = a / (m * m), r = a % (m * m);
  const int yy = mirror(y + r / m - h, H), xx = mirror(x + r % m - h, W);
  return __ldg(f + (size_t)c * H * W + (size_t)yy * W + xx);
}

__global__ void nlm_mean_kernel(const float* __restrict__ f, int n, int N, double* part) {
  __shared__ double red[NL_THREADS];
  for (int c = 0; c < n; ++c) {
    float s = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
      s += __ldg(f + (size_t)c * N + i);
    red[threadIdx.x] = (double)s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * n + c] = red[0];
    __syncthreads();
  }
}

// Per-block sums of the shifted patch vectors and of their pairwise products
// over the block's tiles of NL_TILE x NL_TILE pixels (s = per-channel mean):
// part[blk] = [sum_i (x_a - s)(x_b - s) for a <= b in row-major pair order,
// then sum_i (x_a - s)].  The patch values of a tile are staged pixel-major
// (odd pitch); each thread accumulates a 4 x 4 block of the covariance over
// one parity class of the tile's pixels (8 shared loads per 16 FMAs), and the
// parity classes are added in a fixed order at the end.
__global__ void __launch_bounds__(NL_THREADS)
nlm_cov_kernel(const float* __restrict__ f, int n, int H, int W, int m, const double* mean_part,
               int nblk_mean, float* __restrict__ part) {
  extern __shared__ float sm[];
  const int D = n * m * m;
  const int NP = D * (D + 1) / 2;
  const int DP = (D + 3) & ~3;                      // padded to whole 4 x 4 blocks (zeros)
  const int LDX = DP | 1;                           // odd pitch: a warp's reads hit distinct banks
  const int NBR = DP / 4;                           // block rows
  const int NB = NBR * (NBR + 1) / 2;               // blocks bi <= bj
  const int NPAR = NB <= NL_THREADS ? NL_THREADS / NB : 1;   // pixel parity classes
  float* sX = sm;                                   // [NL_TILE*NL_TILE][LDX] shifted patch values
  float* sAcc = sm + NL_TILE * NL_TILE * LDX;       // [NPAR][NB][16] the classes' block sums
  __shared__ float shift[4];
  const int tid = threadIdx.x;
  if (tid < n) {
    double t = 0.0;
    for (int b = 0; b < nblk_mean; ++b) t += mean_part[(size_t)b * n + tid];
    shift[tid] = (float)(t / ((double)H * W));
  }
  __syncthreads();
  const int first = NB <= NL_THREADS ? tid % NB : tid;   // this thread's first block
  const int par = NB <= NL_THREADS ? tid / NB : 0;       // and its pixel class
  float acc1 = 0.0f;
  const int tiles_x = (W + NL_TILE - 1) / NL_TILE, tiles = tiles_x * ((H + NL_TILE - 1) / NL_TILE);
  // blocks b = first, first + 256, ... (a single one while NB <= 256); every
  // thread runs the same number of block passes so that the barriers match
  const int npass = (NB + NL_THREADS - 1) / NL_THREADS;
  for (int ps = 0; ps < npass; ++ps) {
    const int b0 = first + ps * NL_THREADS;
    const bool active = par < NPAR && b0 < NB;
    int bi = 0, rem = active ? b0 : 0;              // b0 -> (bi, bj), bi <= bj, row-major
    while (rem >= NBR - bi) { rem -= NBR - bi; ++bi; }
    const int bj = bi + rem;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.0f;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      const int y0 = (t / tiles_x) * NL_TILE, x0 = (t % tiles_x) * NL_TILE;
      __syncthreads();
      for (int idx = tid; idx < DP * NL_TILE * NL_TILE; idx += NL_THREADS) {
        const int a = idx / (NL_TILE * NL_TILE), pix = idx % (NL_TILE * NL_TILE);
        const int y = y0 + pix / NL_TILE, x = x0 + pix % NL_TILE;
        float v = 0.0f;
        if (a < D && y < H && x < W) v = patch_val(f, H, W, m, a, y, x) - shift[a / (m * m)];
        sX[pix * LDX + a] = v;                      // 0 outside the image and beyond D
      }
      __syncthreads();
      if (active) {
        for (int pix = par; pix < NL_TILE * NL_TILE; pix += NPAR) {
          const float* xr = sX + pix * LDX;
          float xa[4], xb[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            xa[r] = xr[4 * bi + r];
            xb[r] = xr[4 * bj + r];
          }
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(xa[r], xb[c], acc[r][c]);
        }
      }
      if (ps == 0 && tid < D)
        for (int pix = 0; pix < NL_TILE * NL_TILE; ++pix) acc1 += sX[pix * LDX + tid];
    }
    if (active) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) sAcc[((size_t)par * NB + b0) * 16 + 4 * r + c] = acc[r][c];
    }
  }
  __syncthreads();
  // combine the parity classes in order and write the upper triangle
  float* out = part + (size_t)blockIdx.x * (NP + D);
  for (int v = tid; v < NB * 16; v += NL_THREADS) {
    const int b0 = v / 16, rc = v % 16, r = rc / 4, c = rc % 4;
    int bi = 0, rem = b0;
    while (rem >= NBR - bi) { rem -= NBR - bi; ++bi; }
    const int bj = bi + rem;
    const int a = 4 * bi + r, bb = 4 * bj + c;
    if (a >= D || bb >= D || a > bb) continue;
    float t = sAcc[(size_t)b0 * 16 + rc];
    for (int q = 1; q < NPAR; ++q) t += sAcc[((size_t)q * NB + b0) * 16 + rc];
    out[a * D - a * (a - 1) / 2 + (bb - a)] = t;
  }
  if (tid < D) out[NP + tid] = acc1;
}

// The same per-block partials on the tensor cores (patch dimension D <= 64):
// the block's pixels are taken in tiles of up to TC_KC pixels of one image
// row; the tile's input rows (mirrored at the borders) are staged in shared
// memory, loaded into registers during the previous tile; the tile's shifted
// patch values x are split into a TF32 head and tail, x = h + l (h = x rounded to
// TF32, l = x - h), and staged as a 128 x TC_KC operand whose rows 0..63 hold
// h_a and rows 64..127 hold l_a (rows D..63 and 64 + D..127 zero).  One
// tcgen05.mma chain per tile (kind::tf32, M = 128, N = 64, K = 8 pixels per
// instruction) accumulates in tensor memory
//   rows 0..63:   H_ab = sum_i h_a h_b,   rows 64..127: L_ab = sum_i l_a h_b,
// and sum_i x_a x_b = H_ab + (L_ab + L_ba) up to the dropped sum_i l_a l_b
// (relative 2^-22).  Operands in the no-swizzle K-major layout: 8-row x
// 16-byte core matrices, K-adjacent ones 128 bytes apart, row-group-adjacent
// ones TC_KC / 4 * 128 bytes apart.  Two operand buffers: the next tile is
// staged while the tensor cores work on the current one.  Every wait is
// bounded (the device status records HDF_ETIMEOUT).
constexpr int TC_KC = 128;           // pixels per tile
constexpr int TC_THREADS = 512;
constexpr int TC_ROWS = 128;
constexpr size_t TC_BUF_FLOATS = (size_t)TC_ROWS * TC_KC;

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  constexpr uint32_t LBO = 128, SBO = (TC_KC / 4) * 128;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ bool tc_wait(unsigned long long* mbar, unsigned parity,
                                        unsigned long long limit_ns) {
  const uint32_t m = (uint32_t)__cvta_generic_to_shared(mbar);
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(m), "r"(parity) : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

constexpr int TC_HALO = 2048;        // staged input floats per tile: n m (TC_KC + m - 1)
constexpr int TC_HPT = TC_HALO / TC_THREADS;

__global__ void __launch_bounds__(TC_THREADS, 1)
nlm_cov_tc_kernel(const float* __restrict__ f, int n, int H, int W, int m, const double* mean_part,
                  int nblk_mean, float* __restrict__ part, int* ctrl) {
  extern __shared__ __align__(128) float tsm[];     // 2 operand buffers (then the epilogue), input rows
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ float shift[4];
  __shared__ float fsum[TC_THREADS / 32][64];
  __shared__ int roff[64];   // feature r -> offset of its (channel, dy, dx) in the staged rows
  __shared__ int rch[64];    //            -> its channel
  __shared__ int stop;
  float* halo = tsm + 2 * TC_BUF_FLOATS;
  const int D = n * m * m;
  const int NP = D * (D + 1) / 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int hm = m / 2;
  const int LDH = TC_KC + m - 1;                     // staged columns per input row
  const int nhalo = n * m * LDH;                     // <= TC_HALO (checked by the launcher)
  const int tpr = (W + TC_KC - 1) / TC_KC;           // tiles per image row
  const int ntiles = H * tpr;
  constexpr unsigned long long LIMIT = 2000000000ull;   // 2 s
  if (tid < n) {
    double t = 0.0;
    for (int b = 0; b < nblk_mean; ++b) t += mean_part[(size_t)b * n + tid];
    shift[tid] = (float)(t / ((double)H * W));
  }
  if (tid < 64) {
    const int r = tid < D ? tid : 0;
    const int c = r / (m * m), rr = r % (m * m);
    roff[tid] = (c * m + rr / m) * LDH + rr % m;
    rch[tid] = c;
  }
  for (size_t i = tid; i < 2 * TC_BUF_FLOATS; i += TC_THREADS) tsm[i] = 0.0f;
  if (warp == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(dst) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    stop = 0;
    for (int b = 0; b < 2; ++b) {
      const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar[b]);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  // the input rows of tile t: value v = (channel, dy, column j) of the
  // rows y - hm .. y + hm and columns x0 - hm .. x0 + TC_KC - 1 + hm, mirrored
  auto load_halo = [&](int t, float (&hv)[TC_HPT]) {
    const int y = t / tpr, x0 = (t % tpr) * TC_KC;
#pragma unroll
    for (int u = 0; u < TC_HPT; ++u) {
      const int v = u * TC_THREADS + tid;
      hv[u] = 0.0f;
      if (t < ntiles && v < nhalo) {
        const int j = v % LDH, cd = v / LDH, dy = cd % m, c = cd / m;
        const int yy = mirror(y + dy - hm, H), xx = mirror(min(x0 + j - hm, W - 1 + hm), W);
        hv[u] = __ldg(f + (size_t)c * H * W + (size_t)yy * W + xx);
      }
    }
  };
  // staging map: lane -> (row r & 7, column k & 3); a warp covers one
  // 8 x 4 core matrix per step (conflict-free stores)
  const int r8 = lane >> 2, k4 = lane & 3;
  const int ngroups = (D + 7) / 8;
  float fs[8];
#pragma unroll
  for (int g = 0; g < 8; ++g) fs[g] = 0.0f;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (8u << 17) | (8u << 24);
  float hv[TC_HPT];
  load_halo(blockIdx.x, hv);
  int i = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
    const int b = i & 1;
    float* buf = tsm + (size_t)b * TC_BUF_FLOATS;
    const int cnt = min(TC_KC, W - (t % tpr) * TC_KC);   // pixels of this tile
#pragma unroll
    for (int u = 0; u < TC_HPT; ++u) {
      const int v = u * TC_THREADS + tid;
      if (v < nhalo) halo[v] = hv[u];
    }
    load_halo(t + gridDim.x, hv);   // the next tile's rows, in flight while this one is built
    if (i >= 2) {   // the MMAs of tile i - 2 read this buffer
      if (!tc_wait(&mbar[b], ((i - 2) >> 1) & 1, LIMIT) && tid == 0) stop = 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    __syncthreads();   // halo staged
    // row group g (rows 8g + r8) of the operand: a warp fills the core
    // matrices kq = warp, warp + 8, ... of each group
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      if (g >= ngroups) break;
      const int r = 8 * g + r8;
      const bool live = r < D;
      const float* src = halo + (live ? roff[r] : 0);
      const float sh = live ? shift[rch[r]] : 0.0f;
      // float index of (row r, column k) of the operand:
      // ((r / 8) (TC_KC / 4) + k / 4) 32 + (r % 8) 4 + k % 4
      const int hi0 = ((g * (TC_KC / 4)) << 5) + (r8 << 2) + k4;         // (r, 4 kq + k4) - 32 kq
      const int lo0 = (((8 + g) * (TC_KC / 4)) << 5) + (r8 << 2) + k4;   // the same for row 64 + r
      float acc = 0.0f;
#pragma unroll
      for (int kq = warp; kq < TC_KC / 4; kq += TC_THREADS / 32) {
        const int k = 4 * kq + k4;
        const float x = (live && k < cnt) ? src[k] - sh : 0.0f;
        acc += x;
        const float h = to_tf32(x);
        buf[hi0 + (kq << 5)] = h;
        buf[lo0 + (kq << 5)] = x - h;
      }
      fs[g] += acc;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (stop) break;   // uniform
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
      for (int j = 0; j < TC_KC / 8; ++j) {
        const uint64_t d = tc_desc(base + j * 256);   // 8 pixels = two core matrices along K
        const uint32_t acc = (i > 0 || j > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                     ::"r"(tmem), "l"(d), "l"(d), "r"(idesc), "r"(acc) : "memory");
      }
      const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar[b]);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(mb) : "memory");
    }
  }
  const int nmine = i;
  // the last commit covers every MMA issued before it
  bool ok = !stop;
  if (nmine > 0) {
    const int L = nmine - 1;
    if (!tc_wait(&mbar[L & 1], (L >> 1) & 1, LIMIT)) ok = false;
    if (!ok) tc_wait(&mbar[L & 1], (L >> 1) & 1, LIMIT);   // let the MMAs land before leaving
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (__syncthreads_or(!ok)) {
    if (tid == 0) record_error(ctrl, HDF_ETIMEOUT);
  } else {
    // feature sums: lanes with the same row (r8) and group, then warps, in a fixed order
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      float v = fs[g];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      if (k4 == 0) fsum[warp][8 * g + r8] = v;
    }
    float* ep = tsm;   // [128][65] accumulator rows
    if (warp < 4) {
      for (int half = 0; half < 2; ++half) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(half * 32);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                     "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                       "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                       "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                       "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                     : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int row = warp * 32 + lane;
#pragma unroll
        for (int c = 0; c < 32; ++c) ep[row * 65 + half * 32 + c] = nmine > 0 ? __uint_as_float(v[c]) : 0.0f;
      }
    }
    __syncthreads();
    float* out = part + (size_t)blockIdx.x * (NP + D);
    for (int v = tid; v < D * D; v += TC_THREADS) {
      const int a = v / D, bb = v % D;
      if (a > bb) continue;
      out[a * D - a * (a - 1) / 2 + (bb - a)] = ep[a * 65 + bb] + (ep[(64 + a) * 65 + bb] + ep[(64 + bb) * 65 + a]);
    }
    if (tid < D) {
      float t = 0.0f;
      for (int w = 0; w < TC_THREADS / 32; ++w) t += fsum[w][tid];
      out[NP + tid] = t;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

// FP64 sums over the blocks of their partials, one thread per entry (pair
// sums and feature sums), the blocks in ascending order.
__global__ void __launch_bounds__(128)
nlm_sum_kernel(const float* __restrict__ part, int nblk, int len, double* __restrict__ sum) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= len) return;
  double t = 0.0;
  int b = 0;
  for (; b + 8 <= nblk; b += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldg(part + (size_t)(b + u) * len + q);
#pragma unroll
    for (int u = 0; u < 8; ++u) t += (double)v[u];
  }
  for (; b < nblk; ++b) t += (double)__ldg(part + (size_t)b * len + q);
  sum[q] = t;
}

// One CTA: the covariance in FP64 (from the FP64 sums of the blocks' float32
// partials), its eigendecomposition by cyclic Jacobi in float32, the top-rho
// basis.  The
// blocks' partial sums are float32 sums over some 7000 pixels each, so the
// covariance carries a relative rounding of order 1e-6; float32 rotations
// (1e-7) add nothing of consequence, and on this GPU they run at the FP32
// rate instead of the much lower FP64 one.  Threshold rule: a pair (p, q) is
// rotated only while |a_pq| exceeds 2^-23 sqrt(|a_pp a_qq|) (below that the
// rotation is a no-op in float32); the sweeps stop after one without
// rotations, at the float32 rounding level of the off-diagonal norm, or when
// a sweep no longer halves that norm (Jacobi converges quadratically until
// rounding noise is all that is left).
__global__ void __launch_bounds__(EIG_THREADS)
nlm_eig_kernel(const double* __restrict__ csum, int n, int m, int N, int rho,
               const double* mean_part, int nblk_mean, float* __restrict__ basis,
               float* __restrict__ pmean, int* ctrl) {
  extern __shared__ double dm[];
  const int D = n * m * m, NP = D * (D + 1) / 2;
  const int DE = D + (D & 1);                       // even size for the round-robin schedule
  double* mu = dm;                                  // D  mean of the shifted patch vectors
  float* A = (float*)(mu + D + (D & 1));            // DE x DE
  float* V = A + DE * DE;                           // DE x DE eigenvectors (columns)
  __shared__ float cs[NL_MAXD / 2 + 1][2];
  __shared__ int pp[NL_MAXD / 2 + 1], qq[NL_MAXD / 2 + 1];
  __shared__ double shift[4];
  __shared__ int rotated;
  const int tid = threadIdx.x;
  if (tid == 0 && ctrl) ctrl[CTRL_NLM_SWEEPS] = 0;
  if (tid < n) {
    double t = 0.0;
    for (int b = 0; b < nblk_mean; ++b) t += mean_part[(size_t)b * n + tid];
    shift[tid] = (double)(float)(t / (double)N);    // the float shift the covariance pass used
  }
  for (int a = tid; a < D; a += EIG_THREADS) mu[a] = csum[NP + a] / (double)N;
  __syncthreads();
  for (int idx = tid; idx < DE * DE; idx += EIG_THREADS) {
    const int i = idx / DE, j = idx % DE;
    double v = 0.0;
    if (i < D && j < D) {
      const int a = i < j ? i : j, b = i < j ? j : i;
      const int q = a * D - a * (a - 1) / 2 + (b - a);  // pair index of (a, b)
      v = csum[q] / (double)N - mu[a] * mu[b];
    }
    A[idx] = (float)v;
    V[idx] = (i == j) ? 1.0f : 0.0f;
  }
  __syncthreads();
  const int half = DE / 2;
  __shared__ float red[EIG_THREADS];
  __shared__ float off_prev;
  for (int sweep = 0; sweep < 40; ++sweep) {
    // off-diagonal and diagonal squared norms: stop at float32 rounding level
    // (off <= 2^-23 dia), or once a sweep no longer halves off (stagnation:
    // the rotations would only move rounding noise around)
    float off = 0.0f, dia = 0.0f;
    for (int idx = tid; idx < DE * DE; idx += EIG_THREADS) {
      const float v = A[idx] * A[idx];
      if (idx / DE == idx % DE) dia += v; else off += v;
    }
    red[tid] = off;
    __syncthreads();
    for (int o = EIG_THREADS / 2; o > 0; o >>= 1) {
      if (tid < o) red[tid] += red[tid + o];
      __syncthreads();
    }
    const float off_all = red[0];
    __syncthreads();
    red[tid] = dia;
    __syncthreads();
    for (int o = EIG_THREADS / 2; o > 0; o >>= 1) {
      if (tid < o) red[tid] += red[tid + o];
      __syncthreads();
    }
    const float dia_all = red[0];
    const bool stop = off_all <= 1.42e-14f * dia_all ||          // (2^-23)^2
                      (sweep >= 3 && off_all > 0.25f * off_prev);  // norm not halved
    __syncthreads();
    if (tid == 0) { off_prev = off_all; rotated = 0; }
    if (stop) break;
    __syncthreads();
    for (int r = 0; r < DE - 1; ++r) {
      if (tid < half) {   // round-robin pairs: position 0 fixed, the others rotate
        const int j = tid;
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + ((pos - 1 + r) % (DE - 1)); };
        int p = player(j), q = player(DE - 1 - j);
        if (p > q) { const int t = p; p = q; q = t; }
        pp[j] = p;
        qq[j] = q;
        float c = 1.0f, sn = 0.0f;
        const float apq = A[p * DE + q];
        const float app = A[p * DE + p], aqq = A[q * DE + q];
        // |a_pq| > 2^-23 sqrt(|a_pp a_qq|), squared; then the smaller root t
        // of t^2 + 2 theta t - 1 = 0, theta = (a_qq - a_pp) / (2 a_pq), as
        // sgn(d) e / (|d| + sqrt(d^2 + e^2)) with d = a_qq - a_pp, e = 2 a_pq
        // (one square root and one division on the round's serial path)
        if (apq * apq > 1.4210855e-14f * fabsf(app * aqq) && apq != 0.0f) {
          const float d = aqq - app, e = 2.0f * apq;
          const float t = (d >= 0.0f ? e : -e) / (fabsf(d) + sqrtf(d * d + e * e));
          c = 1.0f / sqrtf(1.0f + t * t);
          sn = t * c;
          rotated = 1;
        }
        cs[j][0] = c;
        cs[j][1] = sn;
      }
      __syncthreads();
      // a lane per rotation (pair j), the block's warps over the rows k
      constexpr int NG = EIG_THREADS / 32;
      const int lane = tid & 31, grp = tid >> 5;
      for (int j = lane; j < half; j += 32) {   // columns p, q of A J and V J
        const float c = cs[j][0], sn = cs[j][1];
        if (sn == 0.0f) continue;
        const int p = pp[j], q = qq[j];
        for (int k = grp; k < DE; k += NG) {
          const float ap = A[k * DE + p], aq = A[k * DE + q];
          A[k * DE + p] = c * ap - sn * aq;
          A[k * DE + q] = sn * ap + c * aq;
          const float vp = V[k * DE + p], vq = V[k * DE + q];
          V[k * DE + p] = c * vp - sn * vq;
          V[k * DE + q] = sn * vp + c * vq;
        }
      }
      __syncthreads();
      for (int j = lane; j < half; j += 32) {   // rows p, q of J^T (A J)
        const float c = cs[j][0], sn = cs[j][1];
        if (sn == 0.0f) continue;
        const int p = pp[j], q = qq[j];
        for (int k = grp; k < DE; k += NG) {
          const float ap = A[p * DE + k], aq = A[q * DE + k];
          A[p * DE + k] = c * ap - sn * aq;
          A[q * DE + k] = sn * ap + c * aq;
        }
      }
      __syncthreads();
    }
    const int any = rotated;   // read after the barrier that ended the sweep's last step
    __syncthreads();           // everyone has read it before thread 0 resets it
    if (tid == 0 && ctrl) ctrl[CTRL_NLM_SWEEPS] = sweep + 1;
    if (!any) break;
  }
  // the rho largest eigenvalues (ties -> lower index); basis[d][a], mean patch
  if (tid == 0) {
    bool used[NL_MAXD];
    for (int i = 0; i < D; ++i) used[i] = false;
    for (int d = 0; d < rho; ++d) {
      int best = -1;
      for (int i = 0; i < D; ++i)
        if (!used[i] && (best < 0 || A[i * DE + i] > A[best * DE + best])) best = i;
      used[best] = true;
      pp[d] = best;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < rho * D; idx += EIG_THREADS) {
    const int d = idx / D, a = idx % D;
    basis[idx] = V[a * DE + pp[d]];
  }
  for (int a = tid; a < D; a += EIG_THREADS) pmean[a] = (float)(mu[a] + shift[a / (m * m)]);
}

// Projection of every pixel's shifted patch on the rho leading eigenvectors.
// Per patch coordinate a the block keeps its offset from the pixel (for
// pixels at least m / 2 from every border, one load per coordinate) and its
// (channel, dy, dx) for the mirrored border pixels.
template <int RMAX>
__global__ void __launch_bounds__(NL_THREADS)
nlm_project_kernel(const float* __restrict__ f, int n, int H, int W, int m, int rho,
                   const float* __restrict__ basis, const float* __restrict__ pmean,
                   float* __restrict__ p) {
  extern __shared__ float sb[];
  const int D = n * m * m, hm = m / 2;
  const size_t N = (size_t)H * W;
  float* sbasis = sb;                // rho x D
  float* smean = sb + rho * D;       // D
  long long* soff = reinterpret_cast<long long*>(smean + D + ((rho * D + D) & 1));   // D
  int* sdy = reinterpret_cast<int*>(soff + D);                                        // D
  int* sdx = sdy + D;
  int* sch = sdx + D;
  float* sbt = reinterpret_cast<float*>(sch + D + (((size_t)(sch + D) & 15) ? (16 - ((size_t)(sch + D) & 15)) / 4 : 0));   // D x 8
  for (int i = threadIdx.x; i < rho * D; i += blockDim.x) sbasis[i] = basis[i];
  if (RMAX <= 8)
    for (int i = threadIdx.x; i < 8 * D; i += blockDim.x) {
      const int a = i / 8, d = i % 8;
      sbt[i] = d < rho ? basis[d * D + a] : 0.0f;
    }
  for (int a = threadIdx.x; a < D; a += blockDim.x) {
    smean[a] = pmean[a];
    const int c = a / (m * m), r = a % (m * m);
    sdy[a] = r / m - hm;
    sdx[a] = r % m - hm;
    sch[a] = c;
    soff[a] = (long long)c * (long long)N + (long long)sdy[a] * W + sdx[a];
  }
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)N; i += gridDim.x * blockDim.x) {
    const int y = i / W, x = i % W;
    float acc[RMAX];
#pragma unroll
    for (int d = 0; d < RMAX; ++d) acc[d] = 0.0f;
    if (RMAX <= 8 && y >= hm && y < H - hm && x >= hm && x < W - hm) {
      // basis rows of coordinate a as two 16-byte words (coordinate-major copy)
      const float4* bt = reinterpret_cast<const float4*>(sbt);
      const float* fp = f + i;
#pragma unroll 7
      for (int a = 0; a < D; ++a) {
        const float v = __ldg(fp + soff[a]) - smean[a];
        const float4 b0 = bt[2 * a], b1 = bt[2 * a + 1];
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int d = 0; d < (RMAX < 8 ? RMAX : 8); ++d) acc[d] = fmaf(bv[d], v, acc[d]);
      }
    } else {
      for (int a = 0; a < D; ++a) {
        const int yy = mirror(y + sdy[a], H), xx = mirror(x + sdx[a], W);
        const float v = __ldg(f + (size_t)sch[a] * N + (size_t)yy * W + xx) - smean[a];
#pragma unroll
        for (int d = 0; d < RMAX; ++d)
          if (d < rho) acc[d] = fmaf(sbasis[d * D + a], v, acc[d]);
      }
    }
#pragma unroll
    for (int d = 0; d < RMAX; ++d)
      if (d < rho) p[(size_t)d * N + i] = acc[d];
  }
}

}  // namespace

size_t nlm_workspace_bytes(int G) {
  const int D = NL_MAXD;
  return sizeof(float) * (size_t)G * (D * (D + 1) / 2 + D) + sizeof(double) * (size_t)G * 4 +
         sizeof(float) * (D * HDF_MAX_RHO + D) + sizeof(double) * (D * (D + 1) / 2 + D) + 1024;
}

cudaError_t launch_nlm_guide(const float* f, int n, int H, int W, int m, int rho, float* p,
                             void* ws, size_t ws_bytes, int* ctrl, cudaStream_t st) {
  const int D = n * m * m;
  if (D > NL_MAXD || n > 4 || rho > HDF_MAX_RHO || rho > D || (m & 1) == 0 || H < m / 2 + 1 ||
      W < m / 2 + 1)
    return cudaErrorInvalidValue;
  const int NP = D * (D + 1) / 2;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int G = sms;
  if (nlm_workspace_bytes(G) > ws_bytes) return cudaErrorInvalidValue;
  unsigned char* w = (unsigned char*)ws;
  float* cov_part = (float*)w;
  double* mean_part = (double*)(w + sizeof(float) * (size_t)G * (NP + D) + 64 - ((sizeof(float) * (size_t)G * (NP + D)) & 63));
  double* cov_sum = mean_part + (size_t)G * 4;       // NP + D
  float* basis = (float*)(cov_sum + NP + D);
  float* pmean = basis + rho * D;
  const int N = H * W;
  nlm_mean_kernel<<<G, NL_THREADS, 0, st>>>(f, n, N, mean_part);
  cudaError_t e;
  if (D <= 64 && n * m * (TC_KC + m - 1) <= TC_HALO) {   // tensor cores
    const size_t smem_tc = sizeof(float) * (2 * TC_BUF_FLOATS + TC_HALO);
    e = cudaFuncSetAttribute(nlm_cov_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_tc);
    if (e != cudaSuccess) return e;
    nlm_cov_tc_kernel<<<G, TC_THREADS, smem_tc, st>>>(f, n, H, W, m, mean_part, G, cov_part, ctrl);
  } else {
    const int DP = (D + 3) & ~3, NBR = DP / 4, NB = NBR * (NBR + 1) / 2;
    const int NPAR = NB <= NL_THREADS ? NL_THREADS / NB : 1;
    const size_t smem_cov =
        sizeof(float) * ((size_t)(DP | 1) * NL_TILE * NL_TILE + (size_t)NPAR * NB * 16);
    e = cudaFuncSetAttribute(nlm_cov_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_cov);
    if (e != cudaSuccess) return e;
    nlm_cov_kernel<<<G, NL_THREADS, smem_cov, st>>>(f, n, H, W, m, mean_part, G, cov_part);
  }
  const int DE = D + (D & 1);
  const size_t smem_eig = sizeof(double) * (size_t)(D + (D & 1)) + sizeof(float) * 2 * (size_t)DE * DE;
  e = cudaFuncSetAttribute(nlm_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_eig);
  if (e != cudaSuccess) return e;
  nlm_sum_kernel<<<(NP + D + 127) / 128, 128, 0, st>>>(cov_part, G, NP + D, cov_sum);
  nlm_eig_kernel<<<1, EIG_THREADS, smem_eig, st>>>(cov_sum, n, m, N, rho, mean_part, G, basis,
                                                  pmean, ctrl);
  const size_t smem_p = sizeof(float) * ((size_t)rho * D + D + 1) + (sizeof(long long) + 3 * sizeof(int)) * (size_t)D +
                        16 + sizeof(float) * 8 * (size_t)D;
  if (rho <= 8)
    nlm_project_kernel<8><<<G * 4, NL_THREADS, smem_p, st>>>(f, n, H, W, m, rho, basis, pmean, p);
  else
    nlm_project_kernel<64><<<G * 4, NL_THREADS, smem_p, st>>>(f, n, H, W, m, rho, basis, pmean, p);
  return cudaGetLastError();
}

}  // namespace hdf
