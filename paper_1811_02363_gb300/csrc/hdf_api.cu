// C ABI entry points of libhdfilter (declared in include/hdfilter.h):
// argument checking, workspace ownership and the order of the device stages
// of Algorithm 1.  The arithmetic lives in the k_*.cu kernels.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "hdf_internal.cuh"

namespace {
thread_local char g_cuda_err[256] = "";
}  // namespace

namespace hdf {

hdf_status cuda_fail(cudaError_t e, const char* where) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", where, cudaGetErrorString(e));
  return HDF_ECUDA;
}

hdf_status check_desc(hdf_desc* d) {
  if (!d) return HDF_EINVAL;
  if (d->H < 1 || d->W < 1 || d->n < 1 || d->rho < 1 || d->K < 1) return HDF_EINVAL;
  if (!(d->sigma_s > 0.0) || !(d->sigma_r > 0.0) || !isfinite(d->sigma_s) ||
      !isfinite(d->sigma_r))
    return HDF_EINVAL;
  if (d->S < 0) return HDF_EINVAL;
  if (d->S == 0) {
    // S = ceil(3 sigma_s), decided before the conversion to int so that a
    // huge sigma_s cannot overflow it
    if (3.0 * d->sigma_s > (double)HDF_MAX_S) return HDF_EUNSUPPORTED;
    d->S = (int)ceil(3.0 * d->sigma_s);
  }
  if (d->guide_dtype != HDF_GUIDE_F32 && d->guide_dtype != HDF_GUIDE_BF16) return HDF_EINVAL;
  if (d->coef != HDF_COEF_OPT && d->coef != HDF_COEF_INDICATOR) return HDF_EINVAL;
  if (d->spatial != HDF_SPATIAL_GAUSS && d->spatial != HDF_SPATIAL_BOX &&
      d->spatial != HDF_SPATIAL_YOUNG)
    return HDF_EINVAL;
  if (d->spatial == HDF_SPATIAL_YOUNG && !(d->sigma_s >= 0.5)) return HDF_EINVAL;
  if (d->K > HDF_MAX_K || d->rho > HDF_MAX_RHO || d->S > HDF_MAX_S || d->n > HDF_MAX_N)
    return HDF_EUNSUPPORTED;
  if ((long long)d->H * d->W >= (1LL << 31)) return HDF_EUNSUPPORTED;
  return HDF_OK;
}

}  // namespace hdf

namespace {

using hdf::check_desc;
using hdf::cuda_fail;

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, count * sizeof(T) + 16);
}

}  // namespace

namespace hdf {

Taps make_taps(double sigma_s, int S, int spatial) {
  Taps t;
  memset(&t, 0, sizeof(t));
  for (int j = -S; j <= S; ++j)
    t.w[j + S] = spatial == HDF_SPATIAL_BOX ? 1.0f
                                            : (float)exp(-(double)(j * j) / (2.0 * sigma_s * sigma_s));
  return t;
}

}  // namespace hdf

extern "C" {

const char* hdf_status_string(hdf_status s) {
  switch (s) {
    case HDF_OK: return "HDF_OK";
    case HDF_EINVAL: return "HDF_EINVAL: invalid argument";
    case HDF_ENOMEM: return "HDF_ENOMEM: device allocation failed";
    case HDF_ECUDA: return "HDF_ECUDA: CUDA runtime error";
    case HDF_ETIMEOUT: return "HDF_ETIMEOUT: bounded device wait gave up";
    case HDF_EDOMAIN: return "HDF_EDOMAIN: input outside the method's domain";
    case HDF_EUNSUPPORTED: return "HDF_EUNSUPPORTED: beyond the library's limits";
  }
  return "unknown hdf_status";
}

const char* hdf_last_cuda_error(void) { return g_cuda_err; }

hdf_status hdf_create(hdf_handle** out, const hdf_desc* desc) {
  if (!out || !desc) return HDF_EINVAL;
  *out = nullptr;
  hdf_desc d = *desc;
  hdf_status st = check_desc(&d);
  if (st != HDF_OK) return st;
  hdf_handle* h = new (std::nothrow) hdf_handle;
  if (!h) return HDF_ENOMEM;
  memset(h, 0, sizeof(*h));
  h->d = d;
  h->N = d.H * d.W;
  h->wait_ns = hdf::kDefaultWaitNs;
  HDF_CUDA(cudaGetDevice(&h->device), "cudaGetDevice");
  const size_t N = (size_t)h->N, K = (size_t)d.K, R = (size_t)d.rho;
  bool ok = true;
  // stop at the first allocation that fails (nothing more is attempted)
  auto take = [&](auto** p, size_t count) {
    if (ok) ok = dalloc(p, count) == cudaSuccess;
  };
  take(&h->ctrl, hdf::CTRL_WORDS);
  take(&h->mu, K * R);
  take(&h->mu64, K * R);
  take(&h->pinv64, K * K);
  take(&h->pinv32, K * K);
  take(&h->ek, 1);
  take(&h->B, K * N);
  take(&h->C, K * N);
  take(&h->s, N);
  take(&h->den, N);
  take(&h->rmax, N);
  take(&h->dabs, N);
  take(&h->fix_list, N);
  take(&h->grad_scratch, 1 << 16);
  take(&h->labels, N);
  take(&h->bw_g, (size_t)d.n * N);
  take(&h->bw_lam, (size_t)(d.n + 1) * N);
  take(&h->bw_gam, K * N);
  take(&h->bw_bet, K * N);
  take(&h->bw_flag, N);
  h->young_T = nullptr;
  if (d.spatial == HDF_SPATIAL_YOUNG) take(&h->young_T, K * (size_t)(d.n + 1) * N);
  {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    h->nlm_ws_bytes = hdf::nlm_workspace_bytes(sms > 0 ? sms : 1);
  }
  if (ok) ok = cudaMalloc(&h->nlm_ws, h->nlm_ws_bytes) == cudaSuccess;
  h->cl_ws_bytes = hdf::cluster_workspace_bytes(h->N, d.rho, d.K);
  if (ok) ok = cudaMalloc(&h->cl_ws, h->cl_ws_bytes) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    hdf_destroy(h);
    return HDF_ENOMEM;
  }
  if (cudaMemset(h->ctrl, 0, hdf::CTRL_WORDS * sizeof(int)) != cudaSuccess ||
      cudaMemset(h->mu, 0, K * R * sizeof(float)) != cudaSuccess ||
      cudaMemset(h->ek, 0, sizeof(double)) != cudaSuccess ||
      hdf::cluster_init(h) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    hdf_destroy(h);
    return cuda_fail(cudaGetLastError(), "hdf_create init");
  }
  *out = h;
  return HDF_OK;
}

void hdf_destroy(hdf_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (int i = 0; i < 4; ++i)
    if (h->tev[i]) cudaEventDestroy(h->tev[i]);
  cudaFree(h->ctrl);
  cudaFree(h->mu);
  cudaFree(h->mu64);
  cudaFree(h->pinv64);
  cudaFree(h->pinv32);
  cudaFree(h->ek);
  cudaFree(h->B);
  cudaFree(h->C);
  cudaFree(h->s);
  cudaFree(h->den);
  cudaFree(h->rmax);
  cudaFree(h->dabs);
  cudaFree(h->fix_list);
  cudaFree(h->grad_scratch);
  cudaFree(h->labels);
  cudaFree(h->bw_g);
  cudaFree(h->bw_lam);
  cudaFree(h->bw_gam);
  cudaFree(h->bw_bet);
  cudaFree(h->bw_flag);
  cudaFree(h->young_T);
  cudaFree(h->cl_ws);
  cudaFree(h->nlm_ws);
  delete h;
}

hdf_status hdf_set_stage_timing(hdf_handle* h, int on) {
  if (!h) return HDF_EINVAL;
  if (on && !h->tev[0]) {
    for (int i = 0; i < 4; ++i) HDF_CUDA(cudaEventCreate(&h->tev[i]), "timing events");
  }
  h->timing = on ? 1 : 0;
  return HDF_OK;
}

hdf_status hdf_get_stage_times(hdf_handle* h, float* h_ms, int cap, int* count) {
  if (!h || !h_ms || !count || cap < 0) return HDF_EINVAL;
  *count = 0;
  if (!h->tev[0]) return HDF_EINVAL;
  HDF_CUDA(cudaEventSynchronize(h->tev[3]), "timing sync");
  for (int i = 0; i < 3 && i < cap; ++i) {
    HDF_CUDA(cudaEventElapsedTime(h_ms + i, h->tev[i], h->tev[i + 1]), "timing elapsed");
    *count = i + 1;
  }
  return HDF_OK;
}

hdf_status hdf_set_wait_limit(hdf_handle* h, double seconds) {
  if (!h || !(seconds >= 0.0) || !(seconds <= 60.0)) return HDF_EINVAL;
  h->wait_ns = (unsigned long long)(seconds * 1e9);
  return HDF_OK;
}

hdf_status hdf_get_desc(const hdf_handle* h, hdf_desc* out) {
  if (!h || !out) return HDF_EINVAL;
  *out = h->d;
  return HDF_OK;
}

hdf_status hdf_cluster(hdf_handle* h, const void* d_p, void* stream) {
  if (!h || !d_p) return HDF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  {
    hdf::NvtxRange r("hdf cluster: bisecting K-means");
    HDF_CUDA(hdf::launch_cluster(h, d_p, st), "cluster");
  }
  hdf::NvtxRange r("hdf cluster: fit A, A^+");
  HDF_CUDA(hdf::launch_fit(h, st), "fit");
  h->has_centers = 1;
  h->after_apply = 0;
  return HDF_OK;
}

hdf_status hdf_set_sigmas(hdf_handle* h, double sigma_s, double sigma_r, void* stream) {
  if (!h || !(sigma_s > 0.0) || !(sigma_r > 0.0) || !isfinite(sigma_s) || !isfinite(sigma_r))
    return HDF_EINVAL;
  if (h->d.spatial == HDF_SPATIAL_YOUNG && !(sigma_s >= 0.5)) return HDF_EINVAL;
  h->d.sigma_s = sigma_s;
  h->d.sigma_r = sigma_r;
  h->after_apply = 0;
  if (h->has_centers) HDF_CUDA(hdf::launch_fit(h, (cudaStream_t)stream), "set_sigmas fit");
  return HDF_OK;
}

hdf_status hdf_set_centers(hdf_handle* h, const float* h_mu, int K, void* stream) {
  if (!h || !h_mu || K < 1 || K > h->d.K) return HDF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)K * h->d.rho * sizeof(float);
  HDF_CUDA(cudaMemcpyAsync(h->mu, h_mu, bytes, cudaMemcpyHostToDevice, st), "set_centers copy");
  HDF_CUDA(hdf::launch_set_int(h->ctrl + hdf::CTRL_K_EFF, K, st), "set_centers K");
  HDF_CUDA(hdf::launch_fit(h, st), "fit");
  h->has_centers = 1;
  h->after_apply = 0;
  return HDF_OK;
}

hdf_status hdf_get_centers(hdf_handle* h, float* h_mu, int* K_eff, void* stream) {
  if (!h || !h_mu || !K_eff) return HDF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int k = 0;
  HDF_CUDA(cudaMemcpyAsync(&k, h->ctrl + hdf::CTRL_K_EFF, sizeof(int), cudaMemcpyDeviceToHost, st),
           "get K");
  HDF_CUDA(cudaMemcpyAsync(h_mu, h->mu, (size_t)h->d.K * h->d.rho * sizeof(float),
                           cudaMemcpyDeviceToHost, st),
           "get centers");
  HDF_CUDA(cudaStreamSynchronize(st), "sync");
  *K_eff = k;
  return HDF_OK;
}

hdf_status hdf_get_pinv(hdf_handle* h, double* h_out, void* stream) {
  if (!h || !h_out) return HDF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  HDF_CUDA(cudaMemcpyAsync(h_out, h->pinv64, (size_t)h->d.K * h->d.K * sizeof(double),
                           cudaMemcpyDeviceToHost, st),
           "get pinv");
  HDF_CUDA(cudaStreamSynchronize(st), "sync");
  return HDF_OK;
}

hdf_status hdf_get_labels(hdf_handle* h, int32_t* d_labels, void* stream) {
  if (!h || !d_labels) return HDF_EINVAL;
  HDF_CUDA(cudaMemcpyAsync(d_labels, h->labels, (size_t)h->N * sizeof(int32_t),
                           cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
           "get labels");
  return HDF_OK;
}

hdf_status hdf_apply(hdf_handle* h, const float* d_f, const void* d_p, float* d_g, void* stream) {
  if (!h || !d_f || !d_p || !d_g) return HDF_EINVAL;
  if ((const void*)d_g == (const void*)d_f || (const void*)d_g == d_p) return HDF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  h->after_apply = 0;
  if (h->timing) HDF_CUDA(cudaEventRecord(h->tev[0], st), "timing event");
  {
    hdf::NvtxRange r("hdf apply: range maps");
    HDF_CUDA(hdf::launch_rangemap(h, d_p, st), "rangemap");
  }
  if (h->timing) {
    HDF_CUDA(cudaEventRecord(h->tev[1], st), "timing event");
    HDF_CUDA(cudaEventRecord(h->tev[2], st), "timing event");   // moved on by the tile kernel
  }
  hdf::NvtxRange r("hdf apply: convolutions + combine");
  HDF_CUDA(hdf::launch_filter(h, d_f, d_p, d_g, st), "filter");
  if (h->timing) HDF_CUDA(cudaEventRecord(h->tev[3], st), "timing event");
  h->after_apply = 1;
  return HDF_OK;
}

hdf_status hdf_backward(hdf_handle* h, const float* d_f, const void* d_p, const float* d_grad_g,
                        float* d_grad_f, double* d_grad_log_sigma, void* stream) {
  if (!h || !d_f || !d_p || !d_grad_g || !d_grad_f || !d_grad_log_sigma) return HDF_EINVAL;
  if (h->d.coef != HDF_COEF_OPT || h->d.spatial != HDF_SPATIAL_GAUSS) return HDF_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  hdf::NvtxRange r("hdf backward");
  h->after_apply = 0;   // the guard pixels' coefficient columns become one-hot
  HDF_CUDA(hdf::launch_backward(h, d_f, d_p, d_grad_g, d_grad_f, d_grad_log_sigma, st),
           "backward");
  return HDF_OK;
}

hdf_status hdf_backward_after_apply(hdf_handle* h, const float* d_f, const void* d_p,
                                    const float* d_g, const float* d_grad_g, float* d_grad_f,
                                    double* d_grad_log_sigma, void* stream) {
  if (!h || !d_f || !d_p || !d_g || !d_grad_g || !d_grad_f || !d_grad_log_sigma) return HDF_EINVAL;
  if (h->d.coef != HDF_COEF_OPT || h->d.spatial != HDF_SPATIAL_GAUSS) return HDF_EUNSUPPORTED;
  if (!h->after_apply) return HDF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  hdf::NvtxRange r("hdf backward after apply");
  h->after_apply = 0;
  HDF_CUDA(hdf::launch_backward(h, d_f, d_p, d_grad_g, d_grad_f, d_grad_log_sigma, st, d_g),
           "backward");
  return HDF_OK;
}

hdf_status hdf_nlm_guide(hdf_handle* h, const float* d_f, int patch, float* d_p, void* stream) {
  if (!h || !d_f || !d_p || patch < 1 || (patch & 1) == 0) return HDF_EINVAL;
  const hdf_desc& d = h->d;
  if (d.n * patch * patch > 96 || d.n > 4 || d.rho > d.n * patch * patch) return HDF_EUNSUPPORTED;
  if (d.H < patch / 2 + 1 || d.W < patch / 2 + 1) return HDF_EINVAL;
  hdf::NvtxRange r("hdf nlm guide");
  HDF_CUDA(hdf::launch_nlm_guide(d_f, d.n, d.H, d.W, patch, d.rho, d_p, h->nlm_ws, h->nlm_ws_bytes,
                                 h->ctrl, (cudaStream_t)stream),
           "nlm_guide");
  return HDF_OK;
}

hdf_status hdf_bruteforce(const hdf_desc* desc, const float* d_f, const void* d_p, float* d_g,
                          void* stream) {
  if (!desc || !d_f || !d_p || !d_g) return HDF_EINVAL;
  hdf_desc d = *desc;
  hdf_status s = check_desc(&d);
  if (s != HDF_OK) return s;
  hdf::NvtxRange r("hdf brute force");
  HDF_CUDA(hdf::launch_bruteforce(d, d_f, d_p, d_g, (cudaStream_t)stream), "bruteforce");
  return HDF_OK;
}

hdf_status hdf_get_trace(hdf_handle* h, int64_t* h_events, int cap, int* count, void* stream) {
  if (!h || !h_events || !count || cap < 0) return HDF_EINVAL;
  HDF_CUDA(hdf::cluster_trace(h, (long long*)h_events, cap, count, (cudaStream_t)stream), "trace");
  return HDF_OK;
}

hdf_status hdf_get_stats(hdf_handle* h, hdf_stats* out, void* stream) {
  if (!h || !out) return HDF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int c[hdf::CTRL_WORDS];
  double ek = 0.0;
  HDF_CUDA(cudaMemcpyAsync(c, h->ctrl, sizeof(c), cudaMemcpyDeviceToHost, st), "stats");
  HDF_CUDA(cudaMemcpyAsync(&ek, h->ek, sizeof(double), cudaMemcpyDeviceToHost, st), "stats");
  HDF_CUDA(cudaStreamSynchronize(st), "sync");
  out->K_eff = c[hdf::CTRL_K_EFF];
  out->device_error = c[hdf::CTRL_ERROR];
  out->fallback_pixels = c[hdf::CTRL_FALLBACK] + c[hdf::CTRL_FALLBACK64];
  out->rescued_pixels = c[hdf::CTRL_RESCUED];
  out->nlm_sweeps = c[hdf::CTRL_NLM_SWEEPS];
  out->lloyd_iters_max = c[hdf::CTRL_LLOYD_MAX];
  out->rounds = c[hdf::CTRL_ROUNDS];
  out->cluster_error = ek;
  return (hdf_status)c[hdf::CTRL_ERROR];
}

}  // extern "C"
