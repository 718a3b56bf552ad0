// Register-blocked brute-force filter, Eq. (1)-(2):
//   g(i) = sum_{j in W} omega(j) phi(p(i-j) - p(i)) f(i-j) / eta(i),
//   eta(i) = sum_{j in W} omega(j) phi(p(i-j) - p(i)),
// neighbours outside the image left out of both sums.
//
// A block computes a tile of TY x TX outputs (TY = 8 rows, a thread per row
// and RX consecutive columns, 16 threads per row).  The window is walked one
// row offset j1 at a time; the halo rows the tile needs for that offset (TY
// rows of TX + 2 SB columns of every guide / image plane) sit in a ring of
// TY + 1 row slots in shared memory, and each step brings in the next row by
// cp.async while the current one is used, so every staged value is read from
// global memory once.  Per guide dimension a thread loads each of the
// RX + 2 SB staged values of its row once and updates the squared distances
// of all its RX outputs to every column offset they cover (RX (2 SB + 1)
// accumulators in registers); the weights omega(j) phi(.) then replace the
// distances in place and the numerator reuses the same staged rows channel by
// channel.  SB is the compiled window bucket: the taps are omega_1 centred in
// it, zero beyond the call's S, so offsets beyond S weigh nothing.
#pragma once

#include <math.h>

#include "hdf_internal.cuh"

namespace hdf {

struct BruteTileArgs {
  const float* f;       // (n, H, W)
  const float* p;       // (rho, H, W) float32 guide (may be f)
  float* g;             // (n, H, W)
  int H, W, n, rho;
  int alias;            // p == f and rho == n: the guide planes are the image planes
  float inv2sr2;        // 1 / (2 sigma_r^2)
};

template <int MAXC, int SB>
struct BruteTileCfg {
  static constexpr int RX = (SB <= 12 && MAXC <= 16) ? 4 : 2;   // outputs per thread
  static constexpr int TXT = 16;                                 // threads per tile row
  static constexpr int TY = 8;                                   // tile rows
  static constexpr int NT = TXT * TY;
  static constexpr int TX = TXT * RX;                            // tile columns
  static constexpr int NC = TX + 2 * SB;                         // staged columns
  static constexpr int LD = NC | 1;                              // odd row pitch
  static constexpr int NSLOT = TY + 1;                           // ring of row slots
  static constexpr int NTAP = 2 * SB + 1;
  static constexpr int PLD = TX + 1;                             // pitch of the tile's own guide
  // shared floats for `planes` staged planes and rho guide planes of the tile
  static constexpr size_t smem_floats(int planes, int rho) {
    return (size_t)NSLOT * planes * LD + (size_t)rho * TY * PLD;
  }
};

__device__ __forceinline__ void brute_cp4(float* smem, const float* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int bytes = valid ? 4 : 0;   // 0 bytes read: zero-filled
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}

template <int MAXC, int SB>
__global__ void __launch_bounds__(128, 2)
brute_tile_kernel(const BruteTileArgs a, const Taps taps) {
  using Cfg = BruteTileCfg<MAXC, SB>;
  constexpr int RX = Cfg::RX, TY = Cfg::TY, TX = Cfg::TX, NC = Cfg::NC, LD = Cfg::LD;
  constexpr int NSLOT = Cfg::NSLOT, NTAP = Cfg::NTAP, PLD = Cfg::PLD, NT = Cfg::NT;
  extern __shared__ __align__(16) float sm[];
  const int H = a.H, W = a.W, n = a.n, rho = a.rho;
  const size_t N = (size_t)H * W;
  const int planes = a.alias ? rho : rho + n;
  float* ring = sm;                                           // [NSLOT][planes][LD]
  float* pin = sm + (size_t)NSLOT * planes * LD;              // [rho][TY][PLD]
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int xb = x0 + RX * tx;        // first output column of this thread
  const int y = y0 + ty;              // output row

  // halo row k (image row y0 - SB + k, k = 0 .. TY + 2 SB - 1) into its slot
  auto stage_row = [&](int k) {
    float* dst = ring + (size_t)(k % NSLOT) * planes * LD;
    const int yy = y0 - SB + k;
    const bool rok = yy >= 0 && yy < H;
    for (int i = tid; i < planes * NC; i += NT) {
      const int q = i / NC, c = i - q * NC;
      const int xx = x0 - SB + c;
      const bool ok = rok && xx >= 0 && xx < W;
      const float* src = q < rho ? a.p + (size_t)q * N : a.f + (size_t)(q - rho) * N;
      brute_cp4(dst + (size_t)q * LD + c, ok ? src + (size_t)yy * W + xx : a.f, ok);
    }
  };
  for (int i = tid; i < rho * TY * TX; i += NT) {   // the tile's own guide values
    const int d = i / (TY * TX), r = (i / TX) % TY, c = i % TX;
    const int yy = y0 + r, xx = x0 + c;
    pin[(d * TY + r) * PLD + c] = (yy < H && xx < W) ? __ldg(a.p + (size_t)d * N + (size_t)yy * W + xx)
                                                     : 0.0f;
  }
  for (int k = 0; k < TY; ++k) stage_row(k);
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();

  float num[RX][MAXC], den[RX];
#pragma unroll
  for (int o = 0; o < RX; ++o) {
    den[o] = 0.0f;
#pragma unroll
    for (int c = 0; c < MAXC; ++c) num[o][c] = 0.0f;
  }
  // columns of this thread's window are inside the image for every output?
  const bool cols_inside = xb - SB >= 0 && xb + RX - 1 + SB < W;

  for (int m = 0; m <= 2 * SB; ++m) {      // row offset j1 = SB - m
    if (m + TY <= TY + 2 * SB - 1) stage_row(m + TY);   // the next row, into the free slot
    asm volatile("cp.async.commit_group;\n" ::);
    const float wy = taps.w[2 * SB - m];   // omega_1(j1) centred in the bucket
    const int yy = y - (SB - m);
    if (wy != 0.0f && yy >= 0 && yy < H) {
      const float* row = ring + (size_t)((ty + m) % NSLOT) * planes * LD + RX * tx;
      float acc[RX][NTAP];                 // squared distances, then weights
#pragma unroll
      for (int o = 0; o < RX; ++o)
#pragma unroll
        for (int t = 0; t < NTAP; ++t) acc[o][t] = 0.0f;
      for (int d = 0; d < rho; ++d) {
        const float* rd = row + (size_t)d * LD;
        float pi[RX];
#pragma unroll
        for (int o = 0; o < RX; ++o) pi[o] = pin[(d * TY + ty) * PLD + RX * tx + o];
#pragma unroll
        for (int kk = 0; kk < RX + 2 * SB; ++kk) {
          const float v = rd[kk];
#pragma unroll
          for (int o = 0; o < RX; ++o) {
            const int t = o + 2 * SB - kk;   // column offset j2 = t - SB
            if (t >= 0 && t < NTAP) {
              const float df = pi[o] - v;
              acc[o][t] = fmaf(df, df, acc[o][t]);
            }
          }
        }
      }
#pragma unroll
      for (int o = 0; o < RX; ++o) {
#pragma unroll
        for (int t = 0; t < NTAP; ++t) {
          const int xx = xb + o - (t - SB);
          float w = wy * taps.w[t] * __expf(-acc[o][t] * a.inv2sr2);
          if (!cols_inside && (xx < 0 || xx >= W)) w = 0.0f;   // outside the image: left out
          acc[o][t] = w;
          den[o] += w;
        }
      }
#pragma unroll
      for (int c = 0; c < MAXC; ++c) {
        if (c < n) {
          const float* rc = row + (size_t)(a.alias ? c : rho + c) * LD;
#pragma unroll
          for (int kk = 0; kk < RX + 2 * SB; ++kk) {
            const float v = rc[kk];
#pragma unroll
            for (int o = 0; o < RX; ++o) {
              const int t = o + 2 * SB - kk;
              if (t >= 0 && t < NTAP) num[o][c] = fmaf(acc[o][t], v, num[o][c]);
            }
          }
        }
      }
    }
    asm volatile("cp.async.wait_all;\n" ::);
    __syncthreads();   // the next row has landed; this step's slot may be refilled
  }
  if (y < H) {
#pragma unroll
    for (int o = 0; o < RX; ++o) {
      const int x = xb + o;
      if (x < W) {
        const float inv = 1.0f / den[o];
#pragma unroll
        for (int c = 0; c < MAXC; ++c)
          if (c < n) a.g[(size_t)c * N + (size_t)y * W + x] = num[o][c] * inv;
      }
    }
  }
}

}  // namespace hdf
