// Fused convolution + combine of Algorithm 1 (loop "for3" and the final
// division, Eq. (15)-(16)) for one output tile per CTA.
//
// For each chunk of P "planes" (plane 0 is the denominator plane b_k, plane
// 1 + c is channel c of u_k = b_k f) and each centre k:
//   1. stage the halo tile of b_k (from the range-map planes) in shared memory;
//   2. row pass: H = omega_1 (*) U on every halo row, U = b_k * f formed on the
//      fly from the staged image tile (kept for all k of the chunk);
//   3. column pass: V = omega_1 (*) H at the tile's pixels, and accumulate
//      c_k(i) V(i) in registers (sum_k c_k v_k and sum_k c_k r_k of Eq. (15)-(16)).
// The window W = [-S, S]^2 factorises, omega(j) = omega_1(j_1) omega_1(j_2),
// so the two 1-D passes give exactly the 2-D sum over W (Sec. II-B); pixels
// outside the image contribute nothing (zero extension).
//
// Template parameters: SB = compiled half-width (taps beyond the call's S are
// zero weights), P = planes per chunk, TY = tile height.  The tile is 32
// pixels wide; 256 threads; each thread owns YV consecutive rows of one
// column of one plane across the whole k loop.
#pragma once

#include "hdf_internal.cuh"

namespace hdf {

constexpr float kGuardRel = 1e-6f;

struct FilterArgs {
  const float* f;       // (n, H, W)
  const float* B;       // (K, H, W) range maps b_k
  const float* C;       // (K, H, W) coefficients c_k
  float* g;             // (n, H, W)
  int* ctrl;
  int* fix_list;
  int H, W, n;
};

template <int SB, int P, int TY>
struct TileCfg {
  static constexpr int TX = 32;
  static constexpr int NT = 256;
  static constexpr int YV = TX * TY * P / NT;         // column-pass outputs per thread
  static constexpr int XH = (P == 4) ? 16 : 8;         // row-pass outputs per task
  static constexpr int NSEG = TX / XH;
  static constexpr int HR = TY + 2 * SB;               // halo rows
  static constexpr int HC = TX + 2 * SB;               // halo columns
  static constexpr int LD = HC + 1;                    // odd stride: conflict-free row reads
  static constexpr int LDH = TX + 1;
  static constexpr int SF = P * HR * LD;               // floats
  static constexpr int SBF = HR * LD;
  static constexpr int SH = P * HR * LDH;
  static constexpr int SD = TY * TX;
  static constexpr size_t SMEM = sizeof(float) * (size_t)(SF + SBF + SH + 2 * SD);
  static_assert(TY % YV == 0, "tile height must be a multiple of the per-thread run");
  static_assert(TX * (TY / YV) * P == NT, "one column run per thread");
};

template <int SB, int P, int TY>
__global__ void __launch_bounds__(256, 1)
filter_tile_kernel(const FilterArgs a, const Taps taps) {
  using Cfg = TileCfg<SB, P, TY>;
  constexpr int TX = Cfg::TX, NT = Cfg::NT, YV = Cfg::YV, XH = Cfg::XH, NSEG = Cfg::NSEG;
  constexpr int HR = Cfg::HR, HC = Cfg::HC, LD = Cfg::LD, LDH = Cfg::LDH;
  constexpr int NTAP = 2 * SB + 1;
  extern __shared__ float sm[];
  float* sF = sm;                        // [P][HR][LD] image channels of the chunk
  float* sB = sF + Cfg::SF;              // [HR][LD]    b_k
  float* sH = sB + Cfg::SBF;             // [P][HR][LDH] row-pass results
  float* sD = sH + Cfg::SH;              // [TY][TX] denominator sum_k c_k r_k
  float* sR = sD + Cfg::SD;              // [TY][TX] max_k r_k (guard)

  const int tid = threadIdx.x;
  const int H = a.H, W = a.W, n = a.n;
  const size_t N = (size_t)H * W;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int K = a.ctrl[CTRL_K_EFF];
  const int nchunks = (n + 1 + P - 1) / P;

  // column-pass ownership: plane qv, column xv, rows yv0 .. yv0 + YV - 1
  const int qv = tid / (TX * (TY / YV));
  const int xv = tid % TX;
  const int yv0 = ((tid / TX) % (TY / YV)) * YV;
  const int gx = x0 + xv;

  for (int i = tid; i < Cfg::SD; i += NT) sR[i] = 0.0f;

  for (int chunk = 0; chunk < nchunks; ++chunk) {
    // ---- stage the image channels of this chunk (halo included, zero outside)
    for (int idx = tid; idx < P * HR * HC; idx += NT) {
      const int q = idx / (HR * HC);
      const int r = (idx / HC) % HR;
      const int c = idx % HC;
      const int ch = chunk * P + q - 1;
      const int yy = y0 - SB + r, xx = x0 - SB + c;
      float v = 0.0f;
      if (ch >= 0 && ch < n && yy >= 0 && yy < H && xx >= 0 && xx < W)
        v = __ldg(a.f + (size_t)ch * N + (size_t)yy * W + xx);
      sF[(q * HR + r) * LD + c] = v;
    }
    float acc[YV];
#pragma unroll
    for (int o = 0; o < YV; ++o) acc[o] = 0.0f;
    const int qgv = chunk * P + qv;      // global plane of this thread's column run

    for (int k = 0; k < K; ++k) {
      __syncthreads();
      const float* Bk = a.B + (size_t)k * N;
      for (int idx = tid; idx < HR * HC; idx += NT) {
        const int r = idx / HC, c = idx % HC;
        const int yy = y0 - SB + r, xx = x0 - SB + c;
        float v = 0.0f;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = __ldg(Bk + (size_t)yy * W + xx);
        sB[r * LD + c] = v;
      }
      __syncthreads();
      // ---- row pass over every halo row: H = omega_1 (*) (b_k f)
      for (int task = tid; task < P * HR * NSEG; task += NT) {
        const int q = task / (HR * NSEG);
        const int rem = task % (HR * NSEG);
        const int r = rem / NSEG, seg = rem % NSEG;
        const int qg = chunk * P + q;
        if (qg > n) continue;
        const float* pb = sB + r * LD + seg * XH;
        const float* pf = sF + (q * HR + r) * LD + seg * XH;
        float in[XH + 2 * SB];
        if (qg == 0) {
#pragma unroll
          for (int t = 0; t < XH + 2 * SB; ++t) in[t] = pb[t];
        } else {
#pragma unroll
          for (int t = 0; t < XH + 2 * SB; ++t) in[t] = pb[t] * pf[t];
        }
        float* ph = sH + (q * HR + r) * LDH + seg * XH;
#pragma unroll
        for (int o = 0; o < XH; ++o) {
          float h = 0.0f;
#pragma unroll
          for (int t = 0; t < NTAP; ++t) h = fmaf(taps.w[t], in[o + t], h);
          ph[o] = h;
        }
      }
      __syncthreads();
      // ---- column pass at the tile's pixels, accumulate c_k V
      if (qgv <= n) {
        float in[YV + 2 * SB];
        const float* ph = sH + (qv * HR + yv0) * LDH + xv;
#pragma unroll
        for (int t = 0; t < YV + 2 * SB; ++t) in[t] = ph[t * LDH];
        const float* Ck = a.C + (size_t)k * N;
#pragma unroll
        for (int o = 0; o < YV; ++o) {
          float v = 0.0f;
#pragma unroll
          for (int t = 0; t < NTAP; ++t) v = fmaf(taps.w[t], in[o + t], v);
          const int gy = y0 + yv0 + o;
          if (gy < H && gx < W) {
            acc[o] = fmaf(__ldg(Ck + (size_t)gy * W + gx), v, acc[o]);
            if (qgv == 0) {
              float* pr = sR + (yv0 + o) * TX + xv;
              *pr = fmaxf(*pr, v);
            }
          }
        }
      }
    }
    // ---- end of the k loop for this chunk
    if (chunk == 0 && qgv == 0) {
#pragma unroll
      for (int o = 0; o < YV; ++o) {
        const int gy = y0 + yv0 + o;
        float D = acc[o];
        if (gy < H && gx < W) {
          const float rmax = sR[(yv0 + o) * TX + xv];
          if (!(D > kGuardRel * rmax)) {       // guard: take the indicator value later
            const int pos = atomicAdd(a.ctrl + CTRL_FALLBACK, 1);
            if (pos < (int)N) a.fix_list[pos] = gy * W + gx;
            D = 1.0f;
          }
        }
        sD[(yv0 + o) * TX + xv] = D;
      }
    }
    __syncthreads();
    if (qgv >= 1 && qgv <= n) {
      float* gc = a.g + (size_t)(qgv - 1) * N;
#pragma unroll
      for (int o = 0; o < YV; ++o) {
        const int gy = y0 + yv0 + o;
        if (gy < H && gx < W) gc[(size_t)gy * W + gx] = acc[o] / sD[(yv0 + o) * TX + xv];
      }
    }
  }
}

// Launch one instantiation; returns cudaErrorInvalidValue if it cannot hold
// the call's window.
template <int SB, int P, int TY>
cudaError_t launch_filter_tile(const FilterArgs& a, const Taps& taps, cudaStream_t st) {
  using Cfg = TileCfg<SB, P, TY>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(filter_tile_kernel<SB, P, TY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  dim3 grid((a.W + Cfg::TX - 1) / Cfg::TX, (a.H + TY - 1) / TY);
  filter_tile_kernel<SB, P, TY><<<grid, Cfg::NT, Cfg::SMEM, st>>>(a, taps);
  return cudaGetLastError();
}

// Dispatch entry points, one per translation unit (compiled in parallel).
cudaError_t launch_filter_sb(int SB, int P, const FilterArgs& a, const Taps& taps,
                             cudaStream_t st);

}  // namespace hdf
