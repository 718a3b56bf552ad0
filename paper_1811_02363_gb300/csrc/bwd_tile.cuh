// Backward pass of the fast filter (gradients of Eq. (15)-(16) with the
// centres and S fixed; the paper has no backward pass).  With
//   lambda_N = G / D,   lambda_D = -<G, g_hat> / D          (per pixel)
// the chain rule through N = sum_k c_k v_k, D = sum_k c_k r_k gives
//   dL/dv_k = c_k lambda_N,  dL/dr_k = c_k lambda_D,
//   dL/dc_k = gamma_k = <lambda_N, v_k> + lambda_D r_k,
// and, because omega is even, the adjoint of v_k = omega * u_k (zero
// extension) is the same convolution: dL/du_k = omega * (c_k lambda_N).
//
// Two tile kernels share the structure of the forward tile kernel:
//   MODE_GAMMA  recomputes V = omega * U and V' = omega' * U for the planes
//               U = b_k f_q (plane 0: b_k) and contracts them at each pixel:
//               gamma_k += lambda_q V, and the log sigma_s term
//               sum c_k lambda_q V' with omega' = omega |j|^2 / sigma_s^2
//               = omega_1' (x) omega_1 + omega_1 (x) omega_1', omega_1'(t) =
//               omega_1(t) t^2 / sigma_s^2;
//   MODE_ADJ    convolves the planes w = c_k lambda_q and contracts:
//               dL/df_q += b_k (omega * w),  beta_k += (omega * w_0) +
//               sum_q (omega * w_q) f_q   (the direct part of dL/db_k).
// One CTA = a 32 x 64 tile, all planes (2 per chunk, chunk loop inside the
// CTA), so per-pixel sums over planes stay in the CTA and are deterministic.
#pragma once

#include "filter_tile.cuh"
#include "hdf_internal.cuh"

namespace hdf {

enum { MODE_GAMMA = 0, MODE_ADJ = 1 };

struct BwdArgs {
  const float* f;        // (n, H, W)
  const float* lam;      // (n + 1, H, W): plane 0 lambda_D, plane 1 + c lambda_N,c
  const float* B;        // (K, H, W)
  const float* C;        // (K, H, W)
  float* gam;            // MODE_GAMMA out: (K, H, W)
  float* bet;            // MODE_ADJ out:   (K, H, W) direct part of dL/db_k
  float* grad_f;         // MODE_ADJ out:   (n, H, W) direct part of dL/df
  double* part;          // MODE_GAMMA out: per-CTA log sigma_s partial
  const int* ctrl;
  int H, W, n;
  int vec;               // W % 4 == 0 and f 16-byte aligned: 16-byte halo staging
};

template <int SB, int MODE, int TY_>
struct BwdCfg {
  static constexpr int TX = 32, TY = TY_, P = 2, NT = 512;
  static constexpr int YV = TX * TY * P / NT;          // 8 (TY 64) or 4 (TY 32)
  static constexpr int XH = 16, NSEG = TX / XH;
  static constexpr int SA = (SB + 3) & ~3, OFF = SA - SB;   // aligned staging start x0 - SA
  static constexpr int NIN = XH + 2 * SB + OFF, NIN4 = (NIN + 3) / 4;
  static constexpr int HR = TY + 2 * SB, HC = TX + 2 * SA;
  // row stride: >= the staged columns and the row pass's 16-byte loads, and
  // = 4 (mod 8) words, so that the 16-byte loads of 8 consecutive tasks (rows
  // r .. r + 3, two segments each) fall in distinct bank quads
  static constexpr int NEED = (NSEG - 1) * XH + 4 * NIN4 > HC ? (NSEG - 1) * XH + 4 * NIN4 : HC;
  static constexpr int LD = ((NEED + 3) / 8) * 8 + 4;
  static constexpr int LDH = round_ld(TX);
  static constexpr int NH = MODE == MODE_GAMMA ? 2 : 1;  // row-pass outputs per plane
  static constexpr int SF = P * HR * LD, SBF = HR * LD, SH = NH * P * HR * LDH, SRED = P * TY * TX;
  static constexpr size_t SMEM = sizeof(float) * (size_t)(SF + 2 * SBF + SH + SRED);
  static_assert(TX * (TY / YV) * P == NT, "one column run per thread");
  static_assert(LD >= HC, "row stride must hold the staged columns");
  static_assert(SMEM <= 232448, "shared memory per block");
};

template <int SB, int MODE, int TY_>
__global__ void __launch_bounds__(512, 1)
bwd_tile_kernel(const BwdArgs a, const Taps taps, const Taps taps2) {
  using Cfg = BwdCfg<SB, MODE, TY_>;
  constexpr int TX = Cfg::TX, TY = Cfg::TY, P = Cfg::P, NT = Cfg::NT, YV = Cfg::YV;
  constexpr int XH = Cfg::XH, NSEG = Cfg::NSEG, HR = Cfg::HR, HC = Cfg::HC, LD = Cfg::LD;
  constexpr int LDH = Cfg::LDH, NIN4 = Cfg::NIN4, NTAP = 2 * SB + 1;
  constexpr int SA = Cfg::SA, OFF = Cfg::OFF, CPR = HC / 4;
  extern __shared__ __align__(16) float sm[];
  float* sF = sm;                              // [P][HR][LD] f (GAMMA) or lambda (ADJ)
  float* sB0 = sF + Cfg::SF;                   // [2][HR][LD] b_k (GAMMA) or c_k (ADJ)
  float* sH = sB0 + 2 * Cfg::SBF;              // [NH][P][HR][LDH]
  float* sRed = sH + Cfg::SH;                  // [P][TY][TX] per-plane contributions

  const int tid = threadIdx.x;
  const int H = a.H, W = a.W, n = a.n;
  const size_t N = (size_t)H * W;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int K = a.ctrl[CTRL_K_EFF];
  const int nchunks = (n + 1 + P - 1) / P;
  const int qv = tid / (TX * (TY / YV));
  const int xv = tid % TX;
  const int yv0 = ((tid / TX) % (TY / YV)) * YV;
  const int gx = x0 + xv;
  const float* S1 = MODE == MODE_GAMMA ? a.B : a.C;   // the per-k plane multiplying sF
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int CPL = (HC + 31) / 32;   // halo columns per lane
  unsigned col_ok = 0;                  // bit j: column lane + 32 j inside the image
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int c = lane + 32 * j, xx = x0 - SA + c;
    if (c < HC && xx >= 0 && xx < W) col_ok |= 1u << j;
  }
  const bool vec = a.vec != 0;
  double sig = 0.0;                                   // GAMMA: log sigma_s partial

  for (int chunk = 0; chunk < nchunks; ++chunk) {
    const int qgv = chunk * P + qv;
    // ---- stage the chunk's planes (image channels, or lambda planes) and the
    // per-k plane, columns x0 - SA .. x0 + TX + SA - 1: 16-byte copies when
    // the image allows (a chunk is then wholly inside or outside it), else a
    // warp per halo row, lanes over the columns; the row pass reads from
    // column OFF = SA - SB on
    auto stage_rows = [&](const float* plane, float* dst) {
      if (vec) {
        constexpr int RPW = (HR + NT / 32 - 1) / (NT / 32);
        for (int i = lane; i < RPW * CPR; i += 32) {
          const int rl = i / CPR, ch = i - rl * CPR;
          const int r = warp + rl * (NT / 32);
          if (r >= HR) continue;
          const int yy = y0 - SB + r, xx = x0 - SA + 4 * ch;
          const bool ok = yy >= 0 && yy < H && xx >= 0 && xx + 4 <= W;
          cp_async16(dst + r * LD + 4 * ch, ok ? plane + (size_t)yy * W + xx : plane, ok);
        }
        return;
      }
      for (int r = warp; r < HR; r += NT / 32) {
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
      const int qg = chunk * P + q;
      const bool have = MODE == MODE_GAMMA ? (qg >= 1 && qg <= n) : qg <= n;
      if (have) {
        stage_rows(MODE == MODE_GAMMA ? a.f + (size_t)(qg - 1) * N : a.lam + (size_t)qg * N,
                   sF + q * HR * LD);
      } else {
        for (int i = tid; i < HR * LD; i += NT) sF[q * HR * LD + i] = 0.0f;
      }
    }
    auto stage = [&](int k, float* dst) { stage_rows(S1 + (size_t)k * N, dst); };
    stage(0, sB0);
    cp_async_commit();
    // own-pixel values of this thread's plane
    float own[YV], gf[YV];
#pragma unroll
    for (int o = 0; o < YV; ++o) {
      const int gy = y0 + yv0 + o;
      const bool in = gy < H && gx < W && qgv <= n;
      const size_t pix = (size_t)gy * W + gx;
      if (MODE == MODE_GAMMA) own[o] = in ? __ldg(a.lam + (size_t)qgv * N + pix) : 0.0f;   // lambda_q
      else own[o] = (in && qgv >= 1) ? __ldg(a.f + (size_t)(qgv - 1) * N + pix) : 0.0f;   // f_q
      gf[o] = 0.0f;
    }
    for (int k = 0; k < K; ++k) {
      float* sB = sB0 + (k & 1) * Cfg::SBF;
      if (k + 1 < K) stage(k + 1, sB0 + ((k + 1) & 1) * Cfg::SBF);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      // per-pixel factor at this thread's pixels: c_k (GAMMA) or b_k (ADJ)
      float pk[YV];
      const float* PK = (MODE == MODE_GAMMA ? a.C : a.B) + (size_t)k * N;
#pragma unroll
      for (int o = 0; o < YV; ++o) {
        const int gy = y0 + yv0 + o;
        pk[o] = (gy < H && gx < W) ? __ldg(PK + (size_t)gy * W + gx) : 0.0f;
      }
      // ---- row pass over the halo rows
      for (int task = tid; task < P * HR * NSEG; task += NT) {
        const int q = task / (HR * NSEG);
        const int rem = task % (HR * NSEG);
        const int r = rem / NSEG, seg = rem % NSEG;
        const int qg = chunk * P + q;
        if (qg > n) continue;
        const float4* pb = reinterpret_cast<const float4*>(sB + r * LD + seg * XH);
        const float4* pf = reinterpret_cast<const float4*>(sF + (q * HR + r) * LD + seg * XH);
        const bool plain = (MODE == MODE_GAMMA && qg == 0);   // U_0 = b_k
        float raw[4 * NIN4];
#pragma unroll
        for (int t = 0; t < NIN4; ++t) {
          const float4 b = pb[t];
          if (plain) {
            raw[4 * t] = b.x; raw[4 * t + 1] = b.y; raw[4 * t + 2] = b.z; raw[4 * t + 3] = b.w;
          } else {
            const float4 v = pf[t];
            raw[4 * t] = b.x * v.x; raw[4 * t + 1] = b.y * v.y;
            raw[4 * t + 2] = b.z * v.z; raw[4 * t + 3] = b.w * v.w;
          }
        }
        float in[XH + 2 * SB];
#pragma unroll
        for (int i = 0; i < XH + 2 * SB; ++i) in[i] = raw[i + OFF];
        float h[XH];
#pragma unroll
        for (int o = 0; o < XH; ++o) h[o] = 0.0f;
#pragma unroll
        for (int t = 0; t < NTAP; ++t) {
#pragma unroll
          for (int o = 0; o < XH; ++o) h[o] = fmaf(taps.w[t], in[o + t], h[o]);
        }
        float4* ph = reinterpret_cast<float4*>(sH + (q * HR + r) * LDH + seg * XH);
#pragma unroll
        for (int o = 0; o < XH / 4; ++o) ph[o] = make_float4(h[4 * o], h[4 * o + 1], h[4 * o + 2], h[4 * o + 3]);
        if (MODE == MODE_GAMMA) {
#pragma unroll
          for (int o = 0; o < XH; ++o) h[o] = 0.0f;
#pragma unroll
          for (int t = 0; t < NTAP; ++t) {
#pragma unroll
            for (int o = 0; o < XH; ++o) h[o] = fmaf(taps2.w[t], in[o + t], h[o]);
          }
          float4* ph2 = reinterpret_cast<float4*>(sH + ((P + q) * HR + r) * LDH + seg * XH);
#pragma unroll
          for (int o = 0; o < XH / 4; ++o) ph2[o] = make_float4(h[4 * o], h[4 * o + 1], h[4 * o + 2], h[4 * o + 3]);
        }
      }
      __syncthreads();
      // ---- column pass and the per-pixel contributions
      {
        float ctr[YV];
#pragma unroll
        for (int o = 0; o < YV; ++o) ctr[o] = 0.0f;
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
            for (int o = 0; o < YV; ++o) v[o] = fmaf(taps.w[t], in[o + t], v[o]);
          }
          if (MODE == MODE_GAMMA) {
            // V' = omega_1' (column) on H + omega_1 (column) on H'
            float v2[YV];
#pragma unroll
            for (int o = 0; o < YV; ++o) v2[o] = 0.0f;
#pragma unroll
            for (int t = 0; t < NTAP; ++t) {
#pragma unroll
              for (int o = 0; o < YV; ++o) v2[o] = fmaf(taps2.w[t], in[o + t], v2[o]);
            }
            const float* ph2 = sH + ((P + qv) * HR + yv0) * LDH + xv;
#pragma unroll
            for (int t = 0; t < YV + 2 * SB; ++t) in[t] = ph2[t * LDH];
#pragma unroll
            for (int t = 0; t < NTAP; ++t) {
#pragma unroll
              for (int o = 0; o < YV; ++o) v2[o] = fmaf(taps.w[t], in[o + t], v2[o]);
            }
            float sk = 0.0f;
#pragma unroll
            for (int o = 0; o < YV; ++o) {
              ctr[o] = own[o] * v[o];                       // lambda_q V
              sk = fmaf(pk[o] * own[o], v2[o], sk);         // c_k lambda_q V'
            }
            sig += (double)sk;
          } else {
#pragma unroll
            for (int o = 0; o < YV; ++o) {
              if (qgv >= 1) {
                gf[o] = fmaf(pk[o], v[o], gf[o]);           // b_k (omega * w_q)
                ctr[o] = v[o] * own[o];                      // (omega * w_q) f_q
              } else {
                ctr[o] = v[o];                               // omega * w_0
              }
            }
          }
        }
#pragma unroll
        for (int o = 0; o < YV; ++o) sRed[(qv * TY + yv0 + o) * TX + xv] = ctr[o];
      }
      __syncthreads();
      // ---- sum over the chunk's planes, accumulate over chunks (this CTA owns the pixels)
      float* out = (MODE == MODE_GAMMA ? a.gam : a.bet) + (size_t)k * N;
      for (int i = tid; i < TY * TX; i += NT) {
        const int ty = i / TX, tx = i % TX;
        const int gy = y0 + ty, gxx = x0 + tx;
        if (gy >= H || gxx >= W) continue;
        float t = 0.0f;
#pragma unroll
        for (int q = 0; q < P; ++q) t += sRed[(q * TY + ty) * TX + tx];
        float* po = out + (size_t)gy * W + gxx;
        *po = (chunk == 0) ? t : *po + t;
      }
    }
    if (MODE == MODE_ADJ && qgv >= 1 && qgv <= n) {
#pragma unroll
      for (int o = 0; o < YV; ++o) {
        const int gy = y0 + yv0 + o;
        if (gy < H && gx < W) a.grad_f[(size_t)(qgv - 1) * N + (size_t)gy * W + gx] = gf[o];
      }
    }
    __syncthreads();
  }
  if (MODE == MODE_GAMMA) {
    // block sum of the log sigma_s partial (fixed order)
    __shared__ double red[NT / 32];
    double x = sig;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((tid & 31) == 0) red[tid >> 5] = x;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += red[w];
      a.part[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
  }
}

template <int SB, int MODE, int TY_>
cudaError_t launch_bwd_tile(const BwdArgs& a, const Taps& t1, const Taps& t2, cudaStream_t st) {
  using Cfg = BwdCfg<SB, MODE, TY_>;
  cudaError_t e = cudaFuncSetAttribute(bwd_tile_kernel<SB, MODE, TY_>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid((a.W + Cfg::TX - 1) / Cfg::TX, (a.H + Cfg::TY - 1) / Cfg::TY);
  bwd_tile_kernel<SB, MODE, TY_><<<grid, Cfg::NT, Cfg::SMEM, st>>>(a, t1, t2);
  return cudaGetLastError();
}

cudaError_t launch_bwd_sb(int SB, int mode, const BwdArgs& a, const Taps& t1, const Taps& t2,
                          cudaStream_t st);

}  // namespace hdf
