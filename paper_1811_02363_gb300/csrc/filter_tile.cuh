// Fused convolution + combine of Algorithm 1 (loop "for3", the sums of
// Eq. (15)-(16) before the division) for one output tile and one chunk of
// P "planes" per CTA.  Plane 0 is the denominator plane (omega * b_k, summed
// with weights c_k into sum_k c_k r_k); plane 1 + c is channel c of
// u_k = b_k f (summed into sum_k c_k v_k).
//
// Per centre k, with the halo tile of b_k double-buffered in shared memory by
// cp.async (zero-filled outside the image = the zero extension of the sums):
//   row pass:    H = omega_1 (*) (b_k f) on every halo row (b_k f formed on
//                the fly from the image tile, staged once per CTA);
//   column pass: V = omega_1 (*) H at the tile's pixels, acc += c_k(i) V(i).
// The window W = [-S, S]^2 factorises, omega(j) = omega_1(j_1) omega_1(j_2),
// so the two 1-D passes give exactly the 2-D sum over W (Sec. II-B).
//
// Template parameters: SB = compiled half-width (taps beyond the call's S
// are zero weights), P = planes per CTA, TY = tile height.  Tile width 32,
// 512 threads; each thread owns YV consecutive rows of one column of one
// plane for the whole k loop.  Outputs: the numerator planes (unnormalised)
// into g, and for the chunk holding plane 0 the denominator and max_k r_k
// into per-pixel scratch, normalised afterwards by the divide kernel; also
// sum_k |c_k| r_k, the scale of the denominator's rounding (the divide kernel
// hands pixels whose denominator is ill-conditioned to an FP64 recomputation).
#pragma once

#include "hdf_internal.cuh"

namespace hdf {

struct FilterArgs {
  const float* f;       // (n, H, W)
  const float* B;       // (K, H, W) range maps b_k
  const float* C;       // (K, H, W) coefficients c_k
  float* g;             // (n, H, W) numerator sum_k c_k v_k (normalised later)
  float* den;           // (H, W) sum_k c_k r_k
  float* rmax;          // (H, W) max_k r_k
  float* dabs;          // (H, W) sum_k |c_k| r_k, the rounding scale of the denominator (may be null)
  const int* ctrl;
  int H, W, n;
  int box, S;           // box spatial kernel (omega = 1 on W) of half-width S <= SB
  int vec;              // W % 4 == 0 and f 16-byte aligned: halo rows staged in 16-byte copies
};

__device__ __forceinline__ void cp_async16(float* smem, const float* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int bytes = valid ? 16 : 0;   // 0 bytes read: the 4 words are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int bytes = valid ? 4 : 0;   // 0 bytes read: the word is zero-filled
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

constexpr int round_ld(int need) {  // smallest stride >= need with stride % 32 == 4
  return ((need + 27) / 32) * 32 + 4;
}

template <int SB, int P, int TY>
struct TileCfg {
  static constexpr int TX = 32;
  static constexpr int NT = 512;
  static constexpr int YV = TX * TY * P / NT;          // column-pass outputs per thread
  static constexpr int XH = 16;                         // row-pass outputs per task
  static constexpr int NSEG = TX / XH;
  static constexpr int SA = (SB + 3) & ~3;              // staged half-width (16-byte aligned)
  static constexpr int OFF = SA - SB;                   // first used column of a staged row
  static constexpr int NIN = XH + 2 * SB + OFF;         // row-pass inputs per task (from the aligned start)
  static constexpr int NIN4 = (NIN + 3) / 4;            // 128-bit loads per task
  static constexpr int HR = TY + 2 * SB;                // halo rows
  static constexpr int HC = TX + 2 * SA;                // staged columns x0 - SA .. x0 + TX + SA - 1
  static constexpr int LD = round_ld((NSEG - 1) * XH + 4 * NIN4 > HC ? (NSEG - 1) * XH + 4 * NIN4 : HC);
  static constexpr int LDH = round_ld(TX);
  static constexpr int SF = P * HR * LD;                // floats
  static constexpr int SBF = HR * LD;
  static constexpr int SH = P * HR * LDH;
  static constexpr int SR = TY * TX;
  static constexpr size_t SMEM = sizeof(float) * (size_t)(SF + 2 * SBF + SH + 2 * SR);
  static_assert(TY % YV == 0 && YV >= 1, "tile height must be a multiple of the per-thread run");
  static_assert(TX * (TY / YV) * P == NT, "one column run per thread");
  static_assert(LD >= HC, "row stride must hold the halo");
  static_assert(SMEM <= 232448, "shared memory per block");
};

// XW outputs of the row FIR omega_1 (*) u on one halo row, u = b (plane 0)
// or b f (the other planes), from 16-byte-aligned shared rows; results to out.
// tap(t) is the weight of tap t (0 <= t <= 2 SB).
// The inputs of XW row outputs: XW + 2 SB values starting OFF words after the
// 16-byte-aligned row pointers (b, or b f off plane 0), loaded as float4.
template <int SB, int XW, int OFF>
__device__ __forceinline__ void row_inputs(const float* __restrict__ brow,
                                           const float* __restrict__ frow, bool plane0,
                                           float (&in)[XW + 2 * SB]) {
  constexpr int NIN4 = (XW + 2 * SB + OFF + 3) / 4;
  const float4* pb = reinterpret_cast<const float4*>(brow);
  const float4* pf = reinterpret_cast<const float4*>(frow);
  float raw[4 * NIN4];
#pragma unroll
  for (int t = 0; t < NIN4; ++t) {
    const float4 b = pb[t];
    if (plane0) {
      raw[4 * t] = b.x; raw[4 * t + 1] = b.y; raw[4 * t + 2] = b.z; raw[4 * t + 3] = b.w;
    } else {
      const float4 v = pf[t];
      raw[4 * t] = b.x * v.x; raw[4 * t + 1] = b.y * v.y;
      raw[4 * t + 2] = b.z * v.z; raw[4 * t + 3] = b.w * v.w;
    }
  }
#pragma unroll
  for (int i = 0; i < XW + 2 * SB; ++i) in[i] = raw[i + OFF];
}

template <int SB, int XW, class Wt, int OFF = 0>
__device__ __forceinline__ void fir_row(const float* __restrict__ brow, const float* __restrict__ frow,
                                        bool plane0, const Wt& tap, float* __restrict__ out) {
  constexpr int NTAP = 2 * SB + 1;
  float in[XW + 2 * SB];
  row_inputs<SB, XW, OFF>(brow, frow, plane0, in);
  float h[XW];
#pragma unroll
  for (int o = 0; o < XW; ++o) h[o] = 0.0f;
#pragma unroll
  for (int t = 0; t < NTAP; ++t) {
#pragma unroll
    for (int o = 0; o < XW; ++o) h[o] = fmaf(tap(t), in[o + t], h[o]);
  }
  float4* ph = reinterpret_cast<float4*>(out);
#pragma unroll
  for (int o = 0; o < XW / 4; ++o) ph[o] = make_float4(h[4 * o], h[4 * o + 1], h[4 * o + 2], h[4 * o + 3]);
}

// Largest D = SB - S of a call whose half-width S falls in bucket SB (the
// buckets are 3, 6, 9, 12, 15, 18, 24, 32).
__host__ __device__ constexpr int box_dmax(int SB) { return SB <= 18 ? 2 : (SB <= 24 ? 5 : 7); }

// Box window sums over a register array: out[o] = sum of in[o + t] for
// t = d .. 2 SB - d (the box kernel of half-width S = SB - d), o < NO, with d
// in 0 .. box_dmax(SB) known only at run time.  Prefix sums P[m] = in[0] +
// ... + in[m - 1] make every window one difference, P[o + 2 SB + 1 - d] -
// P[o + d]; the candidates for each d have compile-time indices and the
// uniform d selects one, so nothing is indexed at run time.  O(1) per output;
// the differences of prefix sums carry about as much rounding as a FIR.
template <int SB, int NO, int NI>
__device__ __forceinline__ void box_sums(int d, const float (&in)[NI], float (&out)[NO]) {
  constexpr int DM = box_dmax(SB);
  constexpr int NP = NO + 2 * SB + 1;   // prefix sums needed: P[0 .. NO + 2 SB]
  static_assert(NP - 1 <= NI, "window inputs");
  float P[NP];
  P[0] = 0.0f;
#pragma unroll
  for (int m = 1; m < NP; ++m) P[m] = P[m - 1] + in[m - 1];
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    float r = P[o + 2 * SB + 1] - P[o];
#pragma unroll
    for (int D = 1; D <= DM; ++D)
      if (d == D) r = P[o + 2 * SB + 1 - D] - P[o + D];
    out[o] = r;
  }
}

// The box kernel's row pass (omega_1 = 1 on [-S, S]): the inputs are loaded
// as in fir_row, the XW outputs are running window sums.
template <int SB, int XW, int OFF>
__device__ __forceinline__ void box_row(const float* __restrict__ brow, const float* __restrict__ frow,
                                        bool plane0, int S, float* __restrict__ out) {
  float in[XW + 2 * SB];
  row_inputs<SB, XW, OFF>(brow, frow, plane0, in);
  float h[XW];
  box_sums<SB, XW, XW + 2 * SB>(SB - S, in, h);
  float4* ph = reinterpret_cast<float4*>(out);
#pragma unroll
  for (int o = 0; o < XW / 4; ++o) ph[o] = make_float4(h[4 * o], h[4 * o + 1], h[4 * o + 2], h[4 * o + 3]);
}

template <int SB, int P, int TY, bool BOX>
__global__ void __launch_bounds__(512, 1)
filter_tile_kernel(const FilterArgs a, const Taps taps) {
  using Cfg = TileCfg<SB, P, TY>;
  constexpr int TX = Cfg::TX, NT = Cfg::NT, YV = Cfg::YV, XH = Cfg::XH, NSEG = Cfg::NSEG;
  constexpr int HR = Cfg::HR, HC = Cfg::HC, LD = Cfg::LD, LDH = Cfg::LDH;
  constexpr int NTAP = 2 * SB + 1;
  extern __shared__ __align__(16) float sm[];
  float* sF = sm;                        // [P][HR][LD] image channels of the chunk
  float* sB0 = sF + Cfg::SF;             // [2][HR][LD] b_k, double-buffered
  float* sH = sB0 + 2 * Cfg::SBF;        // [P][HR][LDH] row-pass results
  float* sR = sH + Cfg::SH;              // [TY][TX] max_k r_k (plane 0 only)
  float* sA = sR + Cfg::SR;              // [TY][TX] sum_k |c_k| r_k (plane 0 only)

  const int tid = threadIdx.x;
  const int H = a.H, W = a.W, n = a.n;
  const size_t N = (size_t)H * W;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int chunk = blockIdx.z;
  const int K = a.ctrl[CTRL_K_EFF];

  // column-pass ownership: plane qv, column xv, rows yv0 .. yv0 + YV - 1
  const int qv = tid / (TX * (TY / YV));
  const int xv = tid % TX;
  const int yv0 = ((tid / TX) % (TY / YV)) * YV;
  const int gx = x0 + xv;
  const int qgv = chunk * P + qv;        // global plane of this thread's column run

  // ---- staging (cp.async, zero-filled outside the image) of the columns
  // x0 - SA .. x0 + TX + SA - 1 (a 16-byte-aligned start; the row pass reads
  // from column OFF = SA - SB on).  With W % 4 == 0 and aligned planes a
  // 16-byte chunk is either inside the image or outside it, and a warp copies
  // CPR chunks of each of its rows; otherwise single words, a warp per row,
  // lanes over the columns.
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  constexpr int SA = Cfg::SA, OFF = Cfg::OFF;
  constexpr int CPR = HC / 4;           // 16-byte chunks per staged row
  constexpr int RPW = (HR + NW - 1) / NW;   // rows per warp
  constexpr int CPL = (HC + 31) / 32;   // columns per lane (word path)
  unsigned col_ok = 0;                  // bit j: column lane + 32 j inside the image
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int c = lane + 32 * j, xx = x0 - SA + c;
    if (c < HC && xx >= 0 && xx < W) col_ok |= 1u << j;
  }
  const bool vec = a.vec != 0;
  auto stage_rows = [&](const float* plane, float* dst, int r0, int nrows) {
    if (vec) {
      for (int i = lane; i < RPW * CPR; i += 32) {
        const int rl = i / CPR, ch = i - rl * CPR;
        const int r = r0 + rl * NW;
        if (r >= nrows) continue;
        const int yy = y0 - SB + r, xx = x0 - SA + 4 * ch;
        const bool ok = yy >= 0 && yy < H && xx >= 0 && xx + 4 <= W;
        cp_async16(dst + r * LD + 4 * ch, ok ? plane + (size_t)yy * W + xx : plane, ok);
      }
      return;
    }
    for (int r = r0; r < nrows; r += NW) {
      const int yy = y0 - SB + r;
      const bool rok = yy >= 0 && yy < H;
      const float* grow = plane + (ptrdiff_t)yy * W + (x0 - SA);
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
    if (ch >= 0 && ch < n) {
      stage_rows(a.f + (size_t)ch * N, sF + q * HR * LD, warp, HR);
    } else {
      for (int i = tid; i < HR * LD; i += NT) sF[q * HR * LD + i] = 0.0f;
    }
  }
  auto stage_b = [&](int k, float* dst) { stage_rows(a.B + (size_t)k * N, dst, warp, HR); };
  stage_b(0, sB0);
  cp_async_commit();
  for (int i = tid; i < 2 * Cfg::SR; i += NT) sR[i] = 0.0f;   // sR and sA

  float acc[YV], cnext[YV];
  // c_k at this thread's pixels: rows yv0 .. yv0 + YV - 1 of column gx
  const bool colin = gx < W;
  const int nrow_in = colin ? max(0, min(YV, H - (y0 + yv0))) : 0;
  const float* cptr = a.C + (size_t)(y0 + yv0) * W + gx;   // dereferenced for rows < nrow_in only
#pragma unroll
  for (int o = 0; o < YV; ++o) {
    acc[o] = 0.0f;
    cnext[o] = (o < nrow_in) ? __ldg(cptr + (size_t)o * W) : 0.0f;
  }

  for (int k = 0; k < K; ++k) {
    float* sB = sB0 + (k & 1) * Cfg::SBF;
    if (k + 1 < K) stage_b(k + 1, sB0 + ((k + 1) & 1) * Cfg::SBF);
    cp_async_commit();
    cp_async_wait<1>();                  // everything but b_{k+1} has landed
    __syncthreads();
    float ccur[YV];
    cptr += N;
    const int nnext = (k + 1 < K) ? nrow_in : 0;
#pragma unroll
    for (int o = 0; o < YV; ++o) {
      ccur[o] = cnext[o];
      cnext[o] = (o < nnext) ? __ldg(cptr + (size_t)o * W) : 0.0f;
    }
    // ---- row pass over every halo row: H = omega_1 (*) (b_k f).  Tasks of
    // XH outputs fill whole rounds of the block; the remainder is split into
    // tasks of XH / 2 outputs, so that the last round keeps every thread busy.
    // When all tasks fit in one round they stay whole (halves would take two
    // rounds and load each input window twice as often per output).
    {
      constexpr int T = P * HR * NSEG;
      constexpr int FULL = T <= NT ? T : (T / NT) * NT;
      auto task_rows = [&](int task, int& q, int& r, int& seg) {
        q = task / (HR * NSEG);
        const int rem = task - q * (HR * NSEG);
        r = rem / NSEG;
        seg = rem - r * NSEG;
      };
      auto tap = [&](int t) { return taps.w[t]; };
      for (int task = tid; task < FULL; task += NT) {
        int q, r, seg;
        task_rows(task, q, r, seg);
        const int qg = chunk * P + q;
        if (qg > n) continue;
        if constexpr (BOX)
          box_row<SB, XH, OFF>(sB + r * LD + seg * XH, sF + (q * HR + r) * LD + seg * XH, qg == 0,
                               a.S, sH + (q * HR + r) * LDH + seg * XH);
        else
          fir_row<SB, XH, decltype(tap), OFF>(sB + r * LD + seg * XH,
                                              sF + (q * HR + r) * LD + seg * XH, qg == 0, tap,
                                              sH + (q * HR + r) * LDH + seg * XH);
      }
      for (int hk = tid; hk < 2 * (T - FULL); hk += NT) {
        int q, r, seg;
        task_rows(FULL + (hk >> 1), q, r, seg);
        const int qg = chunk * P + q;
        if (qg > n) continue;
        const int x = seg * XH + (hk & 1) * (XH / 2);
        if constexpr (BOX)
          box_row<SB, XH / 2, OFF>(sB + r * LD + x, sF + (q * HR + r) * LD + x, qg == 0, a.S,
                                   sH + (q * HR + r) * LDH + x);
        else
          fir_row<SB, XH / 2, decltype(tap), OFF>(sB + r * LD + x, sF + (q * HR + r) * LD + x,
                                                  qg == 0, tap, sH + (q * HR + r) * LDH + x);
      }
    }
    __syncthreads();
    // ---- column pass at the tile's pixels, accumulate c_k V
    if (qgv <= n) {
      const float* ph = sH + (qv * HR + yv0) * LDH + xv;
      float v[YV];
      float in[YV + 2 * SB];
#pragma unroll
      for (int t = 0; t < YV + 2 * SB; ++t) in[t] = ph[t * LDH];
      if constexpr (BOX) {   // column window sums of the box kernel
        box_sums<SB, YV, YV + 2 * SB>(SB - a.S, in, v);
      } else {
#pragma unroll
        for (int o = 0; o < YV; ++o) v[o] = 0.0f;
#pragma unroll
        for (int t = 0; t < NTAP; ++t) {
#pragma unroll
          for (int o = 0; o < YV; ++o) v[o] = fmaf(taps.w[t], in[o + t], v[o]);
        }
      }
#pragma unroll
      for (int o = 0; o < YV; ++o) acc[o] = fmaf(ccur[o], v[o], acc[o]);
      if (qgv == 0) {
#pragma unroll
        for (int o = 0; o < YV; ++o) {
          float* pr = sR + (yv0 + o) * TX + xv;
          *pr = fmaxf(*pr, v[o]);
          float* pa = sA + (yv0 + o) * TX + xv;
          *pa = fmaf(fabsf(ccur[o]), v[o], *pa);
        }
      }
    }
  }
  // ---- write the sums of this chunk's planes
  if (qgv <= n) {
#pragma unroll
    for (int o = 0; o < YV; ++o) {
      const int gy = y0 + yv0 + o;
      if (gy < H && gx < W) {
        const size_t pix = (size_t)gy * W + gx;
        if (qgv == 0) {
          a.den[pix] = acc[o];
          a.rmax[pix] = sR[(yv0 + o) * TX + xv];
          if (a.dabs) a.dabs[pix] = sA[(yv0 + o) * TX + xv];
        } else {
          a.g[(size_t)(qgv - 1) * N + pix] = acc[o];
        }
      }
    }
  }
}

template <int SB, int P, int TY, bool BOX>
cudaError_t launch_filter_tile_k(const FilterArgs& a, const Taps& taps, cudaStream_t st) {
  using Cfg = TileCfg<SB, P, TY>;
  cudaError_t e = cudaFuncSetAttribute(filter_tile_kernel<SB, P, TY, BOX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Cfg::SMEM);
  if (e != cudaSuccess) return e;
  const int nchunks = (a.n + 1 + P - 1) / P;
  dim3 grid((a.W + Cfg::TX - 1) / Cfg::TX, (a.H + TY - 1) / TY, nchunks);
  filter_tile_kernel<SB, P, TY, BOX><<<grid, Cfg::NT, Cfg::SMEM, st>>>(a, taps);
  return cudaGetLastError();
}

// The Gaussian (taps) or the box (running sums) instantiation.
template <int SB, int P, int TY>
cudaError_t launch_filter_tile(const FilterArgs& a, const Taps& taps, cudaStream_t st) {
  return a.box ? launch_filter_tile_k<SB, P, TY, true>(a, taps, st)
               : launch_filter_tile_k<SB, P, TY, false>(a, taps, st);
}

// Dispatch entry point over the compiled (SB, P, TY) instantiations.
cudaError_t launch_filter_sb(int SB, int P, const FilterArgs& a, const Taps& taps,
                             cudaStream_t st);

}  // namespace hdf
