// Peak-rate probes of the FP32 and FP64 FMA pipes (hdf_probe_peaks): the
// denominators of the roofline fractions of the FIR and brute-force kernels,
// measured on the device instead of derived from unit counts.  Each thread
// runs 8 independent FMA chains (enough to cover the pipe latency at the
// chosen occupancy), the grid covers every SM several times, and the time of
// the launch is taken with CUDA events on the caller's stream.  Not part of
// the paper's method.
#include "hdf_internal.cuh"

namespace hdf {
namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS)
fma_probe_kernel(int iters, T m, T c, int sink_flag, T* sink) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = fma(x[i], m, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) s += x[i];
  if (sink_flag == 0x5eed) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never at run time
}

template <typename T>
cudaError_t time_probe(int blocks, int iters, cudaStream_t st, double* flops_per_s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first launch warms up
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      fma_probe_kernel<T><<<blocks, PROBE_THREADS, 0, st>>>(iters, (T)0.999999, (T)1e-7, 0, nullptr);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * PROBE_CHAINS * 16.0 * (double)iters * blocks * PROBE_THREADS;
  *flops_per_s = best > 0.0f ? flops / (best * 1e-3) : 0.0;
  return cudaSuccess;
}

}  // namespace
}  // namespace hdf

extern "C" hdf_status hdf_probe_peaks(double* fp32_tflops, double* fp64_tflops, void* stream) {
  if (!fp32_tflops || !fp64_tflops) return HDF_EINVAL;
  int dev = 0, sms = 0;
  HDF_CUDA(cudaGetDevice(&dev), "probe cudaGetDevice");
  HDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "probe SM count");
  if (sms < 1) return HDF_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  hdf::NvtxRange r("hdf probe peaks");
  double f32 = 0.0, f64 = 0.0;
  // FP32: 8 blocks of 256 threads per SM (64 warps), ~20 ms per launch
  HDF_CUDA(hdf::time_probe<float>(sms * 8, 8192, st, &f32), "probe fp32");
  // FP64 runs at a small fraction of the FP32 rate: fewer iterations
  HDF_CUDA(hdf::time_probe<double>(sms * 8, 256, st, &f64), "probe fp64");
  *fp32_tflops = f32 * 1e-12;
  *fp64_tflops = f64 * 1e-12;
  return HDF_OK;
}
