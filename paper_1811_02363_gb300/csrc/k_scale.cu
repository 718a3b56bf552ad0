// The guide in the units of an anisotropic range kernel (hdf_scale_guide):
// dimension d divided by sigma_{r,d}.  The anisotropic Gaussian of Sec. III-E,
// phi(x) = exp(-sum_d x_d^2 / (2 sigma_{r,d}^2)), is the isotropic Gaussian of
// unit width of the scaled guide, so every entry point of the library filters
// with it when given the scaled guide and sigma_r = 1 (the clustering then
// runs in the kernel's metric as well).
#include <math.h>

#include "hdf_internal.cuh"

namespace hdf {
namespace {

struct Scales {
  float s[HDF_MAX_RHO];   // sigma_{r,d}
};

template <typename GT>
__global__ void scale_guide_kernel(const GT* __restrict__ p, size_t N, int rho, const Scales sc,
                                   float* out) {
  const size_t total = N * (size_t)rho;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int d = (int)(i / N);
    out[i] = guide_load(p, i) / sc.s[d];
  }
}

}  // namespace
}  // namespace hdf

extern "C" hdf_status hdf_scale_guide(const void* d_p, int guide_dtype, int rho, int H, int W,
                                      const double* h_sigma_r, float* d_out, void* stream) {
  if (!d_p || !h_sigma_r || !d_out || rho < 1 || H < 1 || W < 1) return HDF_EINVAL;
  if (guide_dtype != HDF_GUIDE_F32 && guide_dtype != HDF_GUIDE_BF16) return HDF_EINVAL;
  if (guide_dtype == HDF_GUIDE_BF16 && (const void*)d_out == d_p) return HDF_EINVAL;
  if (rho > HDF_MAX_RHO || (long long)H * W >= (1LL << 31)) return HDF_EUNSUPPORTED;
  hdf::Scales sc;
  for (int d = 0; d < rho; ++d) {
    const double s = h_sigma_r[d];
    if (!(s > 0.0) || !isfinite(s)) return HDF_EINVAL;
    sc.s[d] = (float)s;
  }
  int dev = 0, sms = 0;
  HDF_CUDA(cudaGetDevice(&dev), "scale_guide cudaGetDevice");
  HDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "scale_guide SMs");
  const size_t N = (size_t)H * W;
  cudaStream_t st = (cudaStream_t)stream;
  hdf::NvtxRange r("hdf scale guide");
  if (guide_dtype == HDF_GUIDE_BF16)
    hdf::scale_guide_kernel<__nv_bfloat16><<<sms * 4, 256, 0, st>>>(
        (const __nv_bfloat16*)d_p, N, rho, sc, d_out);
  else
    hdf::scale_guide_kernel<float><<<sms * 4, 256, 0, st>>>((const float*)d_p, N, rho, sc, d_out);
  HDF_CUDA(cudaGetLastError(), "scale_guide");
  return HDF_OK;
}
