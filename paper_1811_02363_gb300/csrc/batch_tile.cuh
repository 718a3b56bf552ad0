// Persistent form of the fused convolution + combine tile kernel
// (filter_tile.cuh) for a batch of images of different sizes, channel counts,
// centre counts and spatial sigmas, all in ONE launch.
//
// Work items (image, tile column, tile row, plane chunk) sit in a list sorted
// by estimated cost, largest first; each CTA takes the next item from a global
// counter until the list is exhausted, so images of very different sizes
// share the GPU without a tail per image.  Each item runs Algorithm 1 loop
// "for3" on its tile: per centre k, the row and column FIRs of the plane
// chunk (plane 0 = omega * b_k, plane 1 + c = omega * (b_k f_c)) and the
// c_k-weighted accumulation of Eq. (15)-(16)'s sums; normalisation follows in
// a separate pass.
//
// The window half-width SB is a compile-time bucket (the image's S <= SB,
// taps beyond S are zero), selected per item by a switch; YV (outputs per
// thread of the column pass) is fixed per bucket, and the tile shape --
// P planes per item and tile height TY with P * TY = 16 YV -- is a run-time
// choice per image, so the autotuner can pick it without recompiling.
// Tile width 32, 512 threads, one CTA per SM.
#pragma once

#include "filter_tile.cuh"
#include "hdf_internal.cuh"

namespace hdf {

constexpr int BT_THREADS = 512;
constexpr int BT_TX = 32;

// Per-image record of the device table.
struct BatchImg {
  const float* f;       // (n, H, W) image
  const float* B;       // (K, H, W) range maps
  const float* C;       // (K, H, W) coefficients
  float* g;             // (n, H, W) output
  float* den;           // (H, W) sum_k c_k r_k
  float* rmax;          // (H, W) max_k r_k
  int* ctrl;            // control words of the image
  int* fix_list;        // (H * W) guarded pixels
  const uint8_t* s;     // (H * W) nearest centre
  int H, W, n, S;
  int SB, P, TY, pad;
  float taps[2 * HDF_MAX_S + 1];   // omega_1 centred in the bucket: taps[SB + j], |j| <= S
};

// Outputs per thread of the column pass for each compiled bucket.
__host__ __device__ constexpr int batch_yv(int SB) { return SB <= 15 ? 16 : (SB <= 24 ? 8 : 4); }

__host__ __device__ constexpr int batch_ld(int SB) {
  return round_ld(16 + 4 * ((16 + 2 * SB + 3) / 4));
}

// Shared memory (bytes) of an item of bucket SB with shape (P, TY).
__host__ __device__ constexpr size_t batch_smem(int SB, int P, int TY) {
  return sizeof(float) * ((size_t)(P + 2) * (TY + 2 * SB) * batch_ld(SB) +
                          (size_t)P * (TY + 2 * SB) * round_ld(BT_TX) + (size_t)TY * BT_TX);
}

template <int SB>
__device__ __forceinline__ void batch_tile_item(const BatchImg* __restrict__ imp, int x0, int y0,
                                                int chunk, float* sm) {
  constexpr int YV = batch_yv(SB);
  constexpr int TX = BT_TX, NT = BT_THREADS, XH = 16, NSEG = TX / XH;
  constexpr int LD = batch_ld(SB), LDH = round_ld(TX);
  constexpr int NTAP = 2 * SB + 1;
  const int P = imp->P, TY = imp->TY;
  const int H = imp->H, W = imp->W, n = imp->n;
  const int HR = TY + 2 * SB;
  const int SBF = HR * LD;
  float* sF = sm;                          // [P][HR][LD]
  float* sB0 = sF + P * SBF;               // [2][HR][LD]
  float* sH = sB0 + 2 * SBF;               // [P][HR][LDH]
  float* sR = sH + P * HR * LDH;           // [TY][TX]
  const float* f = imp->f;
  const float* Bp = imp->B;
  const float* Cp = imp->C;
  const size_t N = (size_t)H * W;
  const int K = imp->ctrl[CTRL_K_EFF];
  const int tid = threadIdx.x;
  const int runs = TY / YV;
  const int qv = tid / (TX * runs);
  const int xv = tid % TX;
  const int yv0 = ((tid / TX) % runs) * YV;
  const int gx = x0 + xv;
  const int qgv = chunk * P + qv;
  // omega_1 is even: taps[SB + j] = taps[SB - j], so SB + 1 registers hold them
  float wh[SB + 1];
#pragma unroll
  for (int t = 0; t <= SB; ++t) wh[t] = __ldg(imp->taps + t);

  // staging (cp.async, zero-filled outside the image): a warp copies whole
  // halo rows, lanes over the columns (column bounds fixed per lane)
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  constexpr int HC = TX + 2 * SB;
  constexpr int CPL = (HC + 31) / 32;
  unsigned col_ok = 0;
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int c = lane + 32 * j, xx = x0 - SB + c;
    if (c < HC && xx >= 0 && xx < W) col_ok |= 1u << j;
  }
  auto stage_rows = [&](const float* plane, float* dst) {
    for (int r = warp; r < HR; r += NW) {
      const int yy = y0 - SB + r;
      const bool rok = yy >= 0 && yy < H;
      const float* grow = plane + (ptrdiff_t)yy * W + (x0 - SB);
      float* srow = dst + r * LD;
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int c = lane + 32 * j;
        if (c < HC) {
          const bool ok = rok && ((col_ok >> j) & 1u);
          cp_async4(srow + c, ok ? grow + c : plane, ok);
        }
      }
    }
  };
  for (int q = 0; q < P; ++q) {
    const int ch = chunk * P + q - 1;
    if (ch >= 0 && ch < n) stage_rows(f + (size_t)ch * N, sF + q * SBF);
    else for (int i = tid; i < SBF; i += NT) sF[q * SBF + i] = 0.0f;
  }
  auto stage_b = [&](int k, float* dst) { stage_rows(Bp + (size_t)k * N, dst); };
  stage_b(0, sB0);
  cp_async_commit();
  for (int i = tid; i < TY * TX; i += NT) sR[i] = 0.0f;

  float acc[YV];
#pragma unroll
  for (int o = 0; o < YV; ++o) acc[o] = 0.0f;
  for (int k = 0; k < K; ++k) {
    float* sB = sB0 + (k & 1) * SBF;
    if (k + 1 < K) stage_b(k + 1, sB0 + ((k + 1) & 1) * SBF);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    // c_k at this thread's outputs; the loads complete during the row pass
    float ccur[YV];
#pragma unroll
    for (int o = 0; o < YV; ++o) {
      const int gy = y0 + yv0 + o;
      ccur[o] = (qgv <= n && gy < H && gx < W) ? __ldg(Cp + (size_t)k * N + (size_t)gy * W + gx)
                                                : 0.0f;
    }
    // row pass over every halo row of every plane of the chunk; the rounds
    // that do not fill the block run tasks of XH / 2 outputs, unless all
    // tasks fit in one round (then they stay whole)
    {
      const int T = P * HR * NSEG;
      const int FULL = T <= NT ? T : (T / NT) * NT;
      auto tap = [&](int t) { return wh[t <= SB ? t : 2 * SB - t]; };
      auto task_rows = [&](int task, int& q, int& r, int& seg) {
        q = task / (HR * NSEG);
        const int rem = task - q * (HR * NSEG);
        r = rem / NSEG;
        seg = rem - r * NSEG;
      };
      for (int task = tid; task < FULL; task += NT) {
        int q, r, seg;
        task_rows(task, q, r, seg);
        const int qg = chunk * P + q;
        if (qg > n) continue;
        fir_row<SB, XH>(sB + r * LD + seg * XH, sF + (q * HR + r) * LD + seg * XH, qg == 0, tap,
                        sH + (q * HR + r) * LDH + seg * XH);
      }
      for (int hk = tid; hk < 2 * (T - FULL); hk += NT) {
        int q, r, seg;
        task_rows(FULL + (hk >> 1), q, r, seg);
        const int qg = chunk * P + q;
        if (qg > n) continue;
        const int x = seg * XH + (hk & 1) * (XH / 2);
        fir_row<SB, XH / 2>(sB + r * LD + x, sF + (q * HR + r) * LD + x, qg == 0, tap,
                            sH + (q * HR + r) * LDH + x);
      }
    }
    __syncthreads();
    // column pass at the tile's pixels, accumulate c_k V
    if (qgv <= n) {
      float in[YV + 2 * SB];
      const float* ph = sH + (qv * HR + yv0) * LDH + xv;
#pragma unroll
      for (int t = 0; t < YV + 2 * SB; ++t) in[t] = ph[t * LDH];
      float v[YV];
#pragma unroll
      for (int o = 0; o < YV; ++o) v[o] = 0.0f;
#pragma unroll
      for (int t = 0; t < NTAP; ++t) {
#pragma unroll
        for (int o = 0; o < YV; ++o) v[o] = fmaf(wh[t <= SB ? t : 2 * SB - t], in[o + t], v[o]);
      }
#pragma unroll
      for (int o = 0; o < YV; ++o) acc[o] = fmaf(ccur[o], v[o], acc[o]);
      if (qgv == 0) {
#pragma unroll
        for (int o = 0; o < YV; ++o) {
          float* pr = sR + (yv0 + o) * TX + xv;
          *pr = fmaxf(*pr, v[o]);
        }
      }
    }
  }
  if (qgv <= n) {
#pragma unroll
    for (int o = 0; o < YV; ++o) {
      const int gy = y0 + yv0 + o;
      if (gy < H && gx < W) {
        const size_t pix = (size_t)gy * W + gx;
        if (qgv == 0) {
          imp->den[pix] = acc[o];
          imp->rmax[pix] = sR[(yv0 + o) * TX + xv];
        } else {
          imp->g[(size_t)(qgv - 1) * N + pix] = acc[o];
        }
      }
    }
  }
}

// Host side (k_batch_tile.cu).
cudaError_t launch_batch_tile(const BatchImg* imgs, const int4* items, int nitems, int* counter,
                              size_t smem, int grid, cudaStream_t st);
int batch_tile_max_blocks_per_sm(size_t smem);

}  // namespace hdf
