// Host side of the clustering stage (Algorithm 1 "cluster", Sec. II-C):
// workspace layout, grid size and dispatch to the per-dimension
// instantiations of the cooperative kernel (cluster_kernel.cuh), which are
// compiled in separate translation units.  One launch clusters a table of
// guides (one entry for a handle, one per image for a batch).
#include "cluster_args.cuh"

namespace hdf {

cudaError_t launch_cluster_r4(const clus::ClArgs*, const int4*, int, const int*, const void*, int,
                              int, unsigned long long,
                               cudaStream_t);
cudaError_t launch_cluster_r8(const clus::ClArgs*, const int4*, int, const int*, const void*, int,
                              int, unsigned long long,
                               cudaStream_t);
cudaError_t launch_cluster_r16(const clus::ClArgs*, const int4*, int, const int*, const void*,
                               int, int, unsigned long long,
                               cudaStream_t);
cudaError_t launch_cluster_r32(const clus::ClArgs*, const int4*, int, const int*, const void*,
                               int, int, unsigned long long,
                               cudaStream_t);
cudaError_t launch_cluster_r64(const clus::ClArgs*, const int4*, int, const int*, const void*,
                               int, int, unsigned long long,
                               cudaStream_t);

namespace clus {
namespace {

struct Layout {
  size_t perm, perm2, X, X2, side, marg, d32, nodes, node_sum, pf, pi, pd, pdd, px, chunk_cnt, trace, arrive, sout, gcen, gacc,
      tab, grp, ord, total;
};

Layout layout(int N, int rho, int G) {
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 255) & ~(size_t)255;
    return at;
  };
  const size_t maxchunks = (size_t)N / CH + MAXSEG + 2;
  L.perm = take(sizeof(uint32_t) * (size_t)N);
  L.perm2 = take(sizeof(uint32_t) * (size_t)N);
  L.X = take(sizeof(float) * (size_t)N * rho);
  L.X2 = take(sizeof(float) * (size_t)N * rho);
  L.side = take(2 * (size_t)N);
  L.marg = take(sizeof(float) * (size_t)N);
  L.d32 = take(sizeof(float) * (size_t)N);
  L.nodes = take(sizeof(NodeRec) * MAXNODES);
  L.node_sum = take(sizeof(double) * MAXNODES * (size_t)rho);
  L.pf = take(sizeof(float) * PF_REGIONS * (size_t)G * MAXSEG * record_floats(rho));
  L.pi = take(sizeof(int) * (size_t)G * MAXSEG * 2);
  L.pd = take(sizeof(float) * (size_t)G * MAXSEG);
  L.pdd = take(sizeof(double) * (size_t)G * MAXSEG);
  L.px = take(sizeof(int) * (size_t)G * MAXSEG);
  L.chunk_cnt = take(sizeof(int) * maxchunks);
  L.trace = take(sizeof(long long) * (1 + 2 * TRACE_CAP));
  L.arrive = take(sizeof(unsigned) * MAXACT);
  L.sout = take(sizeof(SlotOut) * MAXACT);
  L.gcen = take(sizeof(double) * MAXACT * 2 * (size_t)rho);
  L.gacc = take(sizeof(double) * MAXACT * (size_t)rho);
  L.tab = take(sizeof(ClArgs));
  L.grp = take(sizeof(int4));
  L.ord = take(sizeof(int));
  L.total = o;
  return L;
}

}  // namespace

int grid_blocks(int dev) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms > MAXG) sms = MAXG;
  return sms > 0 ? sms : 1;   // one block per SM (co-residency of a cooperative launch)
}

size_t ws_bytes(int N, int rho, int G) { return layout(N, rho, G).total; }

ClArgs make_args(void* ws, int N, int rho, int K, int G, int* ctrl, float* mu, double* mu64,
                 int32_t* labels, double* ek, const void* p, int p_bf16) {
  const Layout L = layout(N, rho, G);
  unsigned char* w = (unsigned char*)ws;
  ClArgs a;
  a.p = p;
  a.p_bf16 = p_bf16;
  a.N = N;
  a.rho = rho;
  a.K = K;
  a.G = G;
  a.bid = 0;
  a.ctrl = ctrl;
  a.mu = mu;
  a.mu64 = mu64;
  a.labels = labels;
  a.ek = ek;
  a.perm = (uint32_t*)(w + L.perm);
  a.perm2 = (uint32_t*)(w + L.perm2);
  a.X = (float*)(w + L.X);
  a.X2 = (float*)(w + L.X2);
  a.side = w + L.side;
  a.marg = (float*)(w + L.marg);
  a.d32 = (float*)(w + L.d32);
  a.nodes = (NodeRec*)(w + L.nodes);
  a.node_sum = (double*)(w + L.node_sum);
  a.pf = (float*)(w + L.pf);
  a.pi = (int*)(w + L.pi);
  a.pd = (float*)(w + L.pd);
  a.pdd = (double*)(w + L.pdd);
  a.px = (int*)(w + L.px);
  a.chunk_cnt = (int*)(w + L.chunk_cnt);
  a.trace = (long long*)(w + L.trace);
  a.arrive = (unsigned*)(w + L.arrive);
  a.sout = (SlotOut*)(w + L.sout);
  a.gcen = (double*)(w + L.gcen);
  a.gacc = (double*)(w + L.gacc);
  return a;
}

cudaError_t launch_table(int rho_max, const ClArgs* table, const int4* groups, int ngroups,
                         const int* order, const void* p_override, int grid,
                         unsigned long long wait_ns, cudaStream_t st) {
  if (rho_max <= 4)
    return launch_cluster_r4(table, groups, ngroups, order, p_override, rho_max, grid, wait_ns, st);
  if (rho_max <= 8)
    return launch_cluster_r8(table, groups, ngroups, order, p_override, rho_max, grid, wait_ns, st);
  if (rho_max <= 16)
    return launch_cluster_r16(table, groups, ngroups, order, p_override, rho_max, grid, wait_ns, st);
  if (rho_max <= 32)
    return launch_cluster_r32(table, groups, ngroups, order, p_override, rho_max, grid, wait_ns, st);
  return launch_cluster_r64(table, groups, ngroups, order, p_override, rho_max, grid, wait_ns, st);
}

}  // namespace clus

size_t cluster_workspace_bytes(int N, int rho, int K) {
  (void)K;
  int dev = 0;
  cudaGetDevice(&dev);
  return clus::ws_bytes(N, rho, clus::grid_blocks(dev));
}

// The one-entry table of a handle (all blocks in one group), written once at
// create time; the guide pointer is passed with every launch.
cudaError_t cluster_init(hdf_handle* h) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int G = clus::grid_blocks(dev);
  const clus::Layout L = clus::layout(h->N, h->d.rho, G);
  if (L.total > h->cl_ws_bytes) return cudaErrorInvalidValue;
  unsigned char* w = (unsigned char*)h->cl_ws;
  const clus::ClArgs a = clus::make_args(h->cl_ws, h->N, h->d.rho, h->d.K, G, h->ctrl, h->mu,
                                         h->mu64, h->labels, h->ek, nullptr,
                                         h->d.guide_dtype == HDF_GUIDE_BF16 ? 1 : 0);
  const int4 grp = make_int4(0, G, 0, 1);
  const int ord = 0;
  cudaError_t e = cudaMemcpy(w + L.tab, &a, sizeof(a), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(w + L.grp, &grp, sizeof(grp), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(w + L.ord, &ord, sizeof(ord), cudaMemcpyHostToDevice);
  return e;
}

cudaError_t launch_cluster(hdf_handle* h, const void* p, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int G = clus::grid_blocks(dev);
  const clus::Layout L = clus::layout(h->N, h->d.rho, G);
  if (L.total > h->cl_ws_bytes) return cudaErrorInvalidValue;
  unsigned char* w = (unsigned char*)h->cl_ws;
  // barrier words and the trace count start from zero for every launch
  cudaError_t e = cudaMemsetAsync(h->ctrl + CTRL_BARRIER, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w + L.trace, 0, sizeof(long long), st);
  if (e != cudaSuccess) return e;
  return clus::launch_table(h->d.rho, (const clus::ClArgs*)(w + L.tab),
                            (const int4*)(w + L.grp), 1, (const int*)(w + L.ord), p, G,
                            h->wait_ns, st);
}

cudaError_t cluster_trace(hdf_handle* h, long long* host, int cap, int* count, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  const clus::Layout L = clus::layout(h->N, h->d.rho, clus::grid_blocks(dev));
  const long long* t = (const long long*)((unsigned char*)h->cl_ws + L.trace);
  long long n = 0;
  cudaError_t e = cudaMemcpyAsync(&n, t, sizeof(n), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  if (n > clus::TRACE_CAP) n = clus::TRACE_CAP;
  if (n > cap) n = cap;
  if (n > 0) {
    e = cudaMemcpyAsync(host, t + 1, sizeof(long long) * 2 * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  *count = (int)n;
  return e;
}

}  // namespace hdf
