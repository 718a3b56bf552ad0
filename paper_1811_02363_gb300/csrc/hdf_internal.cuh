// Internal declarations shared by the translation units of libhdfilter.
// Nothing here is part of the C ABI (include/hdfilter.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hdfilter.h"

namespace hdf {

// Device control words of one handle (int32 unless noted).
enum CtrlSlot {
  CTRL_K_EFF = 0,        // centres in use
  CTRL_ERROR = 1,        // first hdf_status recorded on the device
  CTRL_FALLBACK = 2,     // pixels that took the denominator guard in the last apply
  CTRL_LLOYD_MAX = 3,    // largest 2-means iteration count of the last clustering
  CTRL_ROUNDS = 4,       // split rounds of the last clustering
  CTRL_RANKDEF = 5,      // 1 if the last fit dropped eigenvalues of A (truncated pseudo-inverse)
  CTRL_RESCUED = 6,      // pixels of the last apply recomputed in FP64 (ill-conditioned denominator)
  CTRL_FALLBACK64 = 7,   // of those, pixels that took the denominator guard
  CTRL_BARRIER = 8,      // grid barrier: arrival counter
  CTRL_BARRIER_GEN = 9,  // reserved (zeroed with the barrier counter)
  CTRL_NLM_SWEEPS = 10,  // Jacobi sweeps of the last NLM guide
  CTRL_WORDS = 16
};

// Default limit of every device-side wait (grid barriers, split finishers,
// tensor-core completion) before the kernel records HDF_ETIMEOUT and returns.
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;

// Record `code` as the device error unless one is already recorded.
__device__ __forceinline__ void record_error(int* ctrl, int code) {
  atomicCAS(ctrl + CTRL_ERROR, 0, code);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Guide element as float for either storage type.
__device__ __forceinline__ float guide_load(const float* p, size_t i) { return __ldg(p + i); }
__device__ __forceinline__ float guide_load(const __nv_bfloat16* p, size_t i) {
  return __bfloat162float(p[i]);
}

// Spatial weights of one filter call: omega_1(t) for t = -S..S stored at
// [t + S]; passed by value so that the taps sit in the constant bank.
struct Taps {
  float w[2 * HDF_MAX_S + 1];
};

}  // namespace hdf

// The handle.  Device buffers sized for desc.K, desc.rho, H*W at create time.
struct hdf_handle {
  hdf_desc d;
  int N;              // H * W
  int device;         // CUDA device the buffers live on
  int* ctrl;          // CTRL_WORDS control words
  unsigned long long wait_ns;   // limit of each device-side wait of the clustering
  float* mu;          // K x rho centres (float32, what the filter uses)
  double* mu64;       // K x rho centres before rounding (clustering means)
  double* pinv64;     // K x K A^+ (float64)
  float* pinv32;      // K x K A^+ rounded to float32
  double* ek;         // E_K of the last clustering
  float* B;           // K x N range maps b_k(i)
  float* C;           // K x N coefficients c_k(i)
  uint8_t* s;         // N nearest centre (Voronoi cell) per pixel
  float* den;         // N denominator sum_k c_k r_k of the last apply
  float* rmax;        // N max_k r_k of the last apply (guard)
  float* dabs;        // N sum_k |c_k| r_k of the last apply (rounding scale of the denominator)
  int* fix_list;      // N pixels that take the denominator guard
  double* grad_scratch;  // backward partial sums
  // clustering workspace (allocated in hdf_create, sized by N)
  void* cl_ws;
  size_t cl_ws_bytes;
  int32_t* labels;    // N labels of the last clustering
  // backward scratch
  float* bw_g;        // n x N recomputed g_hat
  float* bw_lam;      // (n+1) x N lambda planes
  float* bw_gam;      // K x N gamma_k
  float* bw_bet;      // K x N direct part of dL/db_k
  uint8_t* bw_flag;   // N pixels that took the denominator guard
  float* young_T;     // K x (n+1) x N row-filtered planes (recursive Gaussian only)
  void* nlm_ws;       // NLM guide workspace
  size_t nlm_ws_bytes;
  // stage timing of hdf_apply (hdf_set_stage_timing): events before the range
  // maps, after them, after the convolution tile kernel, after the last stage
  int timing;
  cudaEvent_t tev[4];
  int has_centers;    // centres present (hdf_cluster / hdf_set_centers ran)
  int after_apply;    // B, C, s, den and the guard list are those of the last hdf_apply
};

namespace hdf {

// One fit (A and A^+ of one image's centres) of a batch.
struct FitJob {
  const float* mu;
  int rho;
  int* ctrl;
  double inv2sr2;
  double* pinv64;
  float* pinv32;
};

// Launchers (each returns cudaGetLastError() of its launch).
cudaError_t launch_fit(hdf_handle* h, cudaStream_t st);           // A, A^+ from h->mu
cudaError_t launch_fit_batch(const FitJob* jobs, int njobs, int Kmax, cudaStream_t st);
cudaError_t launch_set_int(int* p, int v, cudaStream_t st);
cudaError_t launch_rangemap(hdf_handle* h, const void* p, cudaStream_t st);
// rescue = 0: no FP64 recomputation of ill-conditioned pixels (the backward
// pass's forward recomputation keeps every pixel on the float32 path).
cudaError_t launch_filter(hdf_handle* h, const float* f, const void* p, float* g, cudaStream_t st,
                          int rescue = 1);
cudaError_t launch_young(hdf_handle* h, const float* f, float* g, cudaStream_t st);
cudaError_t launch_rescue(hdf_handle* h, const float* f, const void* p, float* g, int* list,
                          cudaStream_t st);   // FP64 recomputation of the listed pixels
cudaError_t launch_bruteforce(const hdf_desc& d, const float* f, const void* p, float* g,
                              cudaStream_t st);
cudaError_t cluster_init(hdf_handle* h);                          // one-entry table, at create
cudaError_t launch_cluster(hdf_handle* h, const void* p, cudaStream_t st);
size_t cluster_workspace_bytes(int N, int rho, int K);
size_t nlm_workspace_bytes(int G);
cudaError_t launch_nlm_guide(const float* f, int n, int H, int W, int m, int rho, float* p,
                             void* ws, size_t ws_bytes, int* ctrl, cudaStream_t st);
cudaError_t cluster_trace(hdf_handle* h, long long* host, int cap, int* count, cudaStream_t st);
// g_fwd: null = recompute the forward pass; else the output of the last apply
// (whose B, C, s, den and guard list are still in the handle).
cudaError_t launch_backward(hdf_handle* h, const float* f, const void* p, const float* G,
                            float* grad_f, double* grad_ls, cudaStream_t st,
                            const float* g_fwd = nullptr);

// Host helpers.
Taps make_taps(double sigma_s, int S, int spatial);   // omega_1 at [t + S], 0 beyond S
hdf_status cuda_fail(cudaError_t e, const char* where);   // records the text for hdf_last_cuda_error
hdf_status check_desc(hdf_desc* d);                       // validates, fills S = ceil(3 sigma_s) if 0
int filter_bucket(int S);                                 // compiled window bucket >= S, -1 if none

// NVTX range over the host side of one stage (what a timeline tool shows
// next to the kernels the stage enqueues).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace hdf

// Return HDF_ECUDA (with the error text recorded) if a CUDA call fails.
#define HDF_CUDA(call, where)                                  \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return hdf::cuda_fail(e_, where);   \
  } while (0)
