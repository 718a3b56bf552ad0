// hdf_apply_static: the fast-filter apply (range maps, coefficients, the
// K(n+1) convolutions, combine and normalise) for callers that cannot
// allocate device memory.  Its scratch (coefficient fit, range maps b_k,
// coefficients c_k, nearest-centre map, denominator, guard list) lives in one
// file-scope static device array of fixed size instead of cudaMalloc'ed
// buffers; the caller passes only the inputs and the output.
//
// Who needs this: code that runs where an allocation is not allowed or not
// acceptable -- a framework or plug-in host that owns all device memory
// through its own pool and forbids foreign allocations, or a latency-critical
// path where a cudaMalloc/cudaFree pair (which can synchronise the device) is
// too slow.
//
// The array is part of the library's device image: every GPU on which the
// library's kernels are loaded holds it until the process exits.  Calls
// share it and it keeps the previous call's contents, so calls whose work
// overlaps on the GPU (concurrent streams, several host threads) race on
// it and must be serialised by the caller.  The call reports no device-side
// status (guard pixels, a truncated pseudo-inverse): there is no handle to
// read it from.
#include <math.h>
#include <string.h>

#include <mutex>

#include "hdf_internal.cuh"

namespace {

// Largest scratch one call may use: 32 MiB.  A call needs
//   K*K*12 + 64 + H*W*(8*K + 17) bytes (plus alignment),
// e.g. K = 32 at 256 x 256 pixels (17.9 MB) or K = 8 at 512 x 512 (21.2 MB).
constexpr size_t kStaticScratchBytes = 32u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device, looked up once per device
// with that device current (the host-side name of the array is not a device
// address).
void* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" hdf_status hdf_apply_static(const hdf_desc* desc, const float* d_mu, int K,
                                       const float* d_f, const void* d_p, float* d_g,
                                       void* stream) {
  if (!desc || !d_mu || !d_f || !d_p || !d_g) return HDF_EINVAL;
  if ((const void*)d_g == (const void*)d_f || (const void*)d_g == d_p) return HDF_EINVAL;
  hdf_desc d = *desc;
  d.K = K;
  hdf_status st = hdf::check_desc(&d);   // the same checks as hdf_create
  if (st != HDF_OK) return st;
  if (d.spatial == HDF_SPATIAL_YOUNG) return HDF_EUNSUPPORTED;   // needs per-plane scratch
  const size_t N = (size_t)d.H * d.W;

  // carve the scratch: control words, A^+ (f64, f32), B, C, s, den, rmax,
  // sum |c_k| r_k, guard list
  size_t off = 0, o_ctrl, o_p64, o_p32, o_B, o_C, o_s, o_den, o_rmax, o_dabs, o_fix;
  o_ctrl = off; off = align256(off + sizeof(int) * hdf::CTRL_WORDS);
  o_p64 = off;  off = align256(off + sizeof(double) * K * K);
  o_p32 = off;  off = align256(off + sizeof(float) * K * K);
  o_B = off;    off = align256(off + sizeof(float) * (size_t)K * N);
  o_C = off;    off = align256(off + sizeof(float) * (size_t)K * N);
  o_s = off;    off = align256(off + N);
  o_den = off;  off = align256(off + sizeof(float) * N);
  o_rmax = off; off = align256(off + sizeof(float) * N);
  o_dabs = off; off = align256(off + sizeof(float) * N);
  o_fix = off;  off = align256(off + sizeof(int) * N);
  if (off > kStaticScratchBytes) return HDF_EUNSUPPORTED;   // beyond the 32 MiB array

  int dev = 0;
  HDF_CUDA(cudaGetDevice(&dev), "apply_static cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return HDF_EUNSUPPORTED;
  void* base = nullptr;
  HDF_CUDA(scratch_address(dev, &base), "apply_static cudaGetSymbolAddress");
  unsigned char* w = (unsigned char*)base;
  cudaStream_t st_ = (cudaStream_t)stream;

  // A handle on the stack that points into the static scratch; the existing
  // launchers run unchanged on it.
  hdf_handle h;
  memset(&h, 0, sizeof(h));
  h.d = d;
  h.N = (int)N;
  h.device = dev;
  h.ctrl = (int*)(w + o_ctrl);
  h.mu = const_cast<float*>(d_mu);   // read only
  h.pinv64 = (double*)(w + o_p64);
  h.pinv32 = (float*)(w + o_p32);
  h.B = (float*)(w + o_B);
  h.C = (float*)(w + o_C);
  h.s = (uint8_t*)(w + o_s);
  h.den = (float*)(w + o_den);
  h.rmax = (float*)(w + o_rmax);
  h.dabs = (float*)(w + o_dabs);
  h.fix_list = (int*)(w + o_fix);

  // The previous call's contents stay in the array: clear the control words
  // (error, guard counter), then set K_eff.
  HDF_CUDA(cudaMemsetAsync(h.ctrl, 0, sizeof(int) * hdf::CTRL_WORDS, st_), "apply_static clear");
  HDF_CUDA(hdf::launch_set_int(h.ctrl + hdf::CTRL_K_EFF, K, st_), "apply_static K");
  HDF_CUDA(hdf::launch_fit(&h, st_), "apply_static fit");
  HDF_CUDA(hdf::launch_rangemap(&h, d_p, st_), "apply_static rangemap");
  HDF_CUDA(hdf::launch_filter(&h, d_f, d_p, d_g, st_), "apply_static filter");
  return HDF_OK;
}
