// Batches (include/hdfilter.h, hdf_batch_*): planning, device tables, the
// autotuner of tile shapes and CUDA-graph capture of a run.  Every stage of
// Algorithm 1 is one launch for all images of the batch:
//   reset -> bfloat16 guides -> clustering (one cooperative launch, one block
//   group per image) -> fit -> range maps -> persistent tiles -> normalise.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "batch.cuh"
#include "combine.cuh"

namespace hdf {
namespace {

constexpr int kStages = 7;   // reset, bf16, cluster, fit, rangemap, tiles, normalise

struct Img {
  hdf_desc d;
  int N = 0, SB = 0, planes = 0, P = 0, TY = 0;
  int user_centers = 0;      // centres installed by hdf_batch_set_centers: not clustered
  int bf16_own = 0;          // the run converts f into the batch's bfloat16 guide
  // device buffers (inside the arena)
  int* ctrl = nullptr;
  float* mu = nullptr;
  double* mu64 = nullptr;
  double* pinv64 = nullptr;
  float* pinv32 = nullptr;
  double* ek = nullptr;
  float* B = nullptr;
  float* C = nullptr;
  uint8_t* s = nullptr;
  float* den = nullptr;
  float* rmax = nullptr;
  int* fix_list = nullptr;
  int32_t* labels = nullptr;
  __nv_bfloat16* g16 = nullptr;
  void* cl_ws = nullptr;
  // bound buffers
  const float* f = nullptr;
  const void* p = nullptr;
  float* g = nullptr;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int smem_limit(int dev) {
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return optin - 1024;   // room for the kernel's static shared memory
}

// Compiled tile shapes of a bucket: P * TY = 16 * YV (512 threads, width 32).
std::vector<std::pair<int, int>> shape_candidates(int SB, int smem_max) {
  std::vector<std::pair<int, int>> out;
  const int yv = batch_yv(SB);
  const int pt = 16 * yv;
  for (int P = 1; P <= 8; P *= 2) {
    const int TY = pt / P;
    if (TY < yv || TY % yv != 0 || TY > 256) continue;
    if (batch_smem(SB, P, TY) > (size_t)smem_max) continue;
    out.push_back({P, TY});
  }
  return out;
}

// Default shape before tuning: the one the single-image kernel uses.
std::pair<int, int> default_shape(int SB, int planes, int smem_max) {
  const auto c = shape_candidates(SB, smem_max);
  auto has = [&](int P, int TY) {
    for (auto& x : c)
      if (x.first == P && x.second == TY) return true;
    return false;
  };
  if (SB <= 15) {
    if (planes <= 2 && has(2, 128)) return {2, 128};
    if (has(4, 64)) return {4, 64};
  } else if (SB <= 24) {
    if (has(2, 64)) return {2, 64};
  } else {
    if (has(2, 32)) return {2, 32};
  }
  return c.empty() ? std::pair<int, int>{0, 0} : c.front();
}

// Relative cost of one work item (FMA count of the two FIR passes).
double item_cost(const Img& m) {
  const int ntap = 2 * m.SB + 1;
  return (double)m.d.K * m.P * ntap * (2.0 * (m.TY + 2 * m.SB) + m.TY);
}

}  // namespace
}  // namespace hdf

struct hdf_batch {
  int count = 0;
  int device = 0;
  int sms = 1;
  int smem_max = 0;
  int Kmax = 1, rho_max = 1;
  std::vector<hdf::Img> im;
  bool bound = false;
  // device arena and tables
  void* arena = nullptr;
  size_t arena_bytes = 0;
  hdf::clus::ClArgs* d_cl = nullptr;
  int4* d_grp = nullptr;
  int* d_ord = nullptr;
  int* d_cl_list = nullptr;
  hdf::FitJob* d_fit = nullptr;      // fits of the clustered images (cl_list order)
  hdf::FitJob* d_fit1 = nullptr;     // one fit (hdf_batch_set_centers)
  hdf::RmJob* d_rm = nullptr;
  int* d_rm_block0 = nullptr;
  hdf::GuideJob* d_g16 = nullptr;
  int* d_g16_block0 = nullptr;
  hdf::BatchImg* d_img = nullptr;
  int* d_div_block0 = nullptr;
  int4* d_items = nullptr;
  int* d_counter = nullptr;
  size_t max_items = 0;
  // plans
  std::vector<int4> groups;
  std::vector<int> order, cl_list;
  int grid_cluster = 0, rho_max_cl = 1;
  int cl_groups = -1;       // clustering plan: -1 auto, 0 one group per image, M >= 1 M equal groups
  int rm_blocks = 0, div_blocks = 0, g16_blocks = 0, n_g16 = 0;
  int nitems = 0;
  size_t smem_tile = 0;
  int grid_tile = 0;
  // graph, timing, tuning
  cudaStream_t st_int = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t ev[hdf::kStages + 1] = {};
  bool timed_valid = false;
  cudaGraphExec_t exec = nullptr;
  int exec_flags = -1;
  int graph_state = 0;
  std::vector<hdf_tile_trial> trials;
};

namespace hdf {
namespace {

void drop_graph(hdf_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->exec_flags = -1;
}

// Clustering groups: the grid (one block per SM) is split among the images
// to cluster, each group sized so that the estimated times agree (a fixed
// latency per pass plus the image's points x dimensions over the group).
void plan_cluster(hdf_batch* b) {
  b->cl_list.clear();
  for (int i = 0; i < b->count; ++i)
    if (!b->im[i].user_centers) b->cl_list.push_back(i);
  b->groups.clear();
  b->order.clear();
  b->grid_cluster = 0;
  b->rho_max_cl = 1;
  const int L = (int)b->cl_list.size();
  if (L == 0) return;
  for (int i : b->cl_list) b->rho_max_cl = std::max(b->rho_max_cl, b->im[i].d.rho);
  const int G = b->sms;
  auto work = [&](int i) { return (double)b->im[i].N * b->im[i].d.rho * 4.0 / 30e9; };
  auto passes = [&](int i) { return 8.0 * (log2((double)b->im[i].d.K) + 1.0); };
  auto cost = [&](int i, int g) { return passes(i) * (4e-6 + 3e-8 * g + work(i) / g); };
  // auto: a group per image while each gets a sizeable share of the grid,
  // else four equal groups (the serving batch of 64 mixed images clustered
  // in 610 ms with a group per image, 245-260 ms with 2-8 groups)
  const int M = b->cl_groups >= 0 ? b->cl_groups : (L * 19 <= G ? 0 : 4);
  if (M >= 1 && M < L && M <= G) {
    // M groups of equal size, the images dealt longest first to the least
    // loaded group (each group clusters its images one after the other)
    const int gs = G / M;
    std::vector<int> idx(b->cl_list);
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return cost(x, gs) > cost(y, gs); });
    std::vector<std::vector<int>> lists(M);
    std::vector<double> load(M, 0.0);
    for (int i : idx) {
      const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lists[g].push_back(i);
      load[g] += cost(i, gs);
    }
    for (int g = 0; g < M; ++g) {
      const int z = (int)b->order.size();
      for (int i : lists[g]) b->order.push_back(i);
      b->groups.push_back(make_int4(g * gs, gs, z, (int)b->order.size()));
    }
    b->grid_cluster = M * gs;
  } else if (L <= G) {
    std::vector<int> gsz(L, 1);
    for (int extra = G - L; extra > 0; --extra) {
      int best = -1;
      double bc = -1.0;
      for (int t = 0; t < L; ++t) {
        const int i = b->cl_list[t];
        const double c = cost(i, gsz[t]);
        if (c > bc && cost(i, gsz[t] + 1) < c) { bc = c; best = t; }
      }
      if (best < 0) break;
      ++gsz[best];
    }
    int blk = 0;
    for (int t = 0; t < L; ++t) {
      b->groups.push_back(make_int4(blk, gsz[t], t, t + 1));
      b->order.push_back(b->cl_list[t]);
      blk += gsz[t];
    }
    b->grid_cluster = blk;
  } else {
    // more images than blocks: single-block groups, longest first to the least loaded
    std::vector<int> idx(b->cl_list);
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return cost(x, 1) > cost(y, 1); });
    std::vector<std::vector<int>> lists(G);
    std::vector<double> load(G, 0.0);
    for (int i : idx) {
      const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lists[g].push_back(i);
      load[g] += cost(i, 1);
    }
    for (int g = 0; g < G; ++g) {
      const int z = (int)b->order.size();
      for (int i : lists[g]) b->order.push_back(i);
      b->groups.push_back(make_int4(g, 1, z, (int)b->order.size()));
    }
    b->grid_cluster = G;
  }
}

// Work items of the persistent launch for the images in `sel`, largest first.
std::vector<int4> build_items(const hdf_batch* b, const std::vector<int>& sel) {
  struct It {
    double cost;
    int4 v;
  };
  std::vector<It> all;
  for (int i : sel) {
    const Img& m = b->im[i];
    const int tx = (m.d.W + BT_TX - 1) / BT_TX, ty = (m.d.H + m.TY - 1) / m.TY;
    const int chunks = (m.planes + m.P - 1) / m.P;
    const double c = item_cost(m);
    for (int ch = 0; ch < chunks; ++ch)
      for (int y = 0; y < ty; ++y)
        for (int x = 0; x < tx; ++x) all.push_back({c, make_int4(i, x, y, ch)});
  }
  std::stable_sort(all.begin(), all.end(), [](const It& a, const It& c) { return a.cost > c.cost; });
  std::vector<int4> out(all.size());
  for (size_t k = 0; k < all.size(); ++k) out[k] = all[k].v;
  return out;
}

BatchImg make_img(const Img& m) {
  BatchImg r;
  memset(&r, 0, sizeof(r));
  r.f = m.f;
  r.B = m.B;
  r.C = m.C;
  r.g = m.g;
  r.den = m.den;
  r.rmax = m.rmax;
  r.ctrl = m.ctrl;
  r.fix_list = m.fix_list;
  r.s = m.s;
  r.H = m.d.H;
  r.W = m.d.W;
  r.n = m.d.n;
  r.S = m.d.S;
  r.SB = m.SB;
  r.P = m.P;
  r.TY = m.TY;
  const Taps t = make_taps(m.d.sigma_s, m.d.S, m.d.spatial);
  for (int j = -m.d.S; j <= m.d.S; ++j) r.taps[m.SB + j] = t.w[m.d.S + j];
  return r;
}

const void* guide_of(const Img& m) { return m.bf16_own ? (const void*)m.g16 : m.p; }

// Device tables from the bound pointers and current plans (synchronous).
cudaError_t upload_tables(hdf_batch* b) {
  std::vector<clus::ClArgs> cl(b->count);
  std::vector<RmJob> rm(b->count);
  std::vector<int> rm_b0(b->count), div_b0(b->count);
  std::vector<BatchImg> img(b->count);
  std::vector<GuideJob> g16;
  std::vector<int> g16_b0;
  int rmb = 0, divb = 0, g16b = 0;
  b->smem_tile = 0;
  for (int i = 0; i < b->count; ++i) {
    Img& m = b->im[i];
    const void* p = guide_of(m);
    const int pbf = m.d.guide_dtype == HDF_GUIDE_BF16 ? 1 : 0;
    cl[i] = clus::make_args(m.cl_ws, m.N, m.d.rho, m.d.K, b->sms, m.ctrl, m.mu, m.mu64, m.labels,
                            m.ek, p, pbf);
    rm[i].p = p;
    rm[i].p_bf16 = pbf;
    rm[i].N = m.N;
    rm[i].rho = m.d.rho;
    rm[i].coef = m.d.coef;
    rm[i].inv2sr2 = (float)(1.0 / (2.0 * m.d.sigma_r * m.d.sigma_r));
    rm[i].mu = m.mu;
    rm[i].pinv = m.pinv32;
    rm[i].ctrl = m.ctrl;
    rm[i].B = m.B;
    rm[i].C = m.C;
    rm[i].s = m.s;
    rm_b0[i] = rmb;
    rmb += batch_blocks_for((size_t)m.N, 1);
    div_b0[i] = divb;
    divb += batch_blocks_for((size_t)m.N, 4);
    img[i] = make_img(m);
    b->smem_tile = std::max(b->smem_tile, batch_smem(m.SB, m.P, m.TY));
    if (m.bf16_own) {
      g16.push_back({m.f, m.g16, (size_t)m.N * m.d.n});
      g16_b0.push_back(g16b);
      g16b += batch_blocks_for((size_t)m.N * m.d.n, 4);
    }
  }
  // group sizes of the clustering plan
  for (auto& gr : b->groups)
    for (int t = gr.z; t < gr.w; ++t) cl[b->order[t]].G = gr.y;
  std::vector<FitJob> fit;
  for (int i : b->cl_list) {
    const Img& m = b->im[i];
    fit.push_back({m.mu, m.d.rho, m.ctrl, 1.0 / (2.0 * m.d.sigma_r * m.d.sigma_r), m.pinv64,
                   m.pinv32});
  }
  b->rm_blocks = rmb;
  b->div_blocks = divb;
  b->g16_blocks = g16b;
  b->n_g16 = (int)g16.size();
  cudaError_t e = cudaMemcpy(b->d_cl, cl.data(), sizeof(clus::ClArgs) * cl.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->groups.empty())
    e = cudaMemcpy(b->d_grp, b->groups.data(), sizeof(int4) * b->groups.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->order.empty())
    e = cudaMemcpy(b->d_ord, b->order.data(), sizeof(int) * b->order.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->cl_list.empty())
    e = cudaMemcpy(b->d_cl_list, b->cl_list.data(), sizeof(int) * b->cl_list.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !fit.empty())
    e = cudaMemcpy(b->d_fit, fit.data(), sizeof(FitJob) * fit.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_rm, rm.data(), sizeof(RmJob) * rm.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_rm_block0, rm_b0.data(), sizeof(int) * rm_b0.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_div_block0, div_b0.data(), sizeof(int) * div_b0.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_img, img.data(), sizeof(BatchImg) * img.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !g16.empty())
    e = cudaMemcpy(b->d_g16, g16.data(), sizeof(GuideJob) * g16.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !g16_b0.empty())
    e = cudaMemcpy(b->d_g16_block0, g16_b0.data(), sizeof(int) * g16_b0.size(), cudaMemcpyHostToDevice);
  return e;
}

cudaError_t upload_items(hdf_batch* b, const std::vector<int4>& items) {
  if (items.size() > b->max_items) return cudaErrorInvalidValue;
  b->nitems = (int)items.size();
  if (items.empty()) return cudaSuccess;
  return cudaMemcpy(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
}

std::vector<int> all_images(const hdf_batch* b) {
  std::vector<int> v(b->count);
  for (int i = 0; i < b->count; ++i) v[i] = i;
  return v;
}

cudaError_t tile_launch(hdf_batch* b, int nitems, size_t smem, cudaStream_t st) {
  const int occ = batch_tile_max_blocks_per_sm(smem);
  if (occ < 1) return cudaErrorInvalidConfiguration;
  b->grid_tile = b->sms * occ;
  return launch_batch_tile(b->d_img, b->d_items, nitems, b->d_counter, smem, b->grid_tile, st);
}

// All stages of one run on `st`; with `ev`, an event before each stage.
cudaError_t enqueue(hdf_batch* b, int flags, cudaStream_t st, cudaEvent_t* ev) {
  const bool cluster = !(flags & HDF_BATCH_SKIP_CLUSTER) && !b->cl_list.empty();
  const int ncl = cluster ? (int)b->cl_list.size() : 0;
  cudaError_t e = cudaSuccess;
  auto mark = [&](int k) {
    if (ev && e == cudaSuccess) e = cudaEventRecord(ev[k], st);
  };
  mark(0);
  if (e == cudaSuccess) e = launch_batch_prep(b->d_img, b->count, b->d_cl, b->d_cl_list, ncl, b->d_counter, st);
  mark(1);
  if (e == cudaSuccess && b->n_g16 > 0)
    e = launch_batch_to_bf16(b->d_g16, b->d_g16_block0, b->n_g16, b->g16_blocks, st);
  mark(2);
  if (e == cudaSuccess && cluster)
    e = clus::launch_table(b->rho_max_cl, b->d_cl, b->d_grp, (int)b->groups.size(), b->d_ord,
                           nullptr, b->grid_cluster, clus::DEFAULT_WAIT_NS, st);
  mark(3);
  if (e == cudaSuccess && cluster) e = launch_fit_batch(b->d_fit, ncl, b->Kmax, st);
  mark(4);
  if (e == cudaSuccess)
    e = launch_batch_rangemap(b->d_rm, b->d_rm_block0, b->count, b->rm_blocks, b->Kmax,
                              rm_smem_floats(b->Kmax, b->rho_max), st);
  mark(5);
  if (e == cudaSuccess) e = tile_launch(b, b->nitems, b->smem_tile, st);
  mark(6);
  if (e == cudaSuccess) e = launch_batch_normalise(b->d_img, b->d_div_block0, b->count, b->div_blocks, st);
  mark(7);
  return e;
}

int launches_per_run(const hdf_batch* b, int flags) {
  const bool cluster = !(flags & HDF_BATCH_SKIP_CLUSTER) && !b->cl_list.empty();
  return 1 + (b->n_g16 > 0 ? 1 : 0) + (cluster ? 2 : 0) + 1 + 1 + 2;
}

}  // namespace
}  // namespace hdf

using hdf::cuda_fail;

extern "C" {

hdf_status hdf_batch_create(hdf_batch** out, int count, const hdf_desc* descs) {
  if (!out || !descs || count < 1) return HDF_EINVAL;
  *out = nullptr;
  hdf_batch* b = new (std::nothrow) hdf_batch;
  if (!b) return HDF_ENOMEM;
  b->count = count;
  b->im.resize(count);
  for (int i = 0; i < count; ++i) {   // argument errors before any CUDA call
    hdf::Img& m = b->im[i];
    m.d = descs[i];
    hdf_status s = hdf::check_desc(&m.d);
    if (s != HDF_OK) { delete b; return s; }
    if (m.d.spatial == HDF_SPATIAL_YOUNG) { delete b; return HDF_EUNSUPPORTED; }   // FIR tiles only
    m.N = m.d.H * m.d.W;
    m.SB = hdf::filter_bucket(m.d.S);
    if (m.SB < 0) { delete b; return HDF_EUNSUPPORTED; }
    m.planes = m.d.n + 1;
    b->Kmax = std::max(b->Kmax, m.d.K);
    b->rho_max = std::max(b->rho_max, m.d.rho);
  }
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return cuda_fail(cudaGetLastError(), "cudaGetDevice");
  }
  b->sms = hdf::clus::grid_blocks(b->device);
  b->smem_max = hdf::smem_limit(b->device);
  for (auto& m : b->im) {
    const auto sh = hdf::default_shape(m.SB, m.planes, b->smem_max);
    if (sh.first == 0) { delete b; return HDF_EUNSUPPORTED; }
    m.P = sh.first;
    m.TY = sh.second;
  }
  // arena: per-image buffers, then the tables
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += hdf::align256(bytes + 16);
    return at;
  };
  std::vector<std::vector<size_t>> off(count);
  for (int i = 0; i < count; ++i) {
    const hdf::Img& m = b->im[i];
    const size_t N = (size_t)m.N, K = (size_t)m.d.K, R = (size_t)m.d.rho;
    std::vector<size_t>& v = off[i];
    v.push_back(take(sizeof(int) * hdf::CTRL_WORDS));
    v.push_back(take(sizeof(float) * K * R));
    v.push_back(take(sizeof(double) * K * R));
    v.push_back(take(sizeof(double) * K * K));
    v.push_back(take(sizeof(float) * K * K));
    v.push_back(take(sizeof(double)));
    v.push_back(take(sizeof(float) * K * N));
    v.push_back(take(sizeof(float) * K * N));
    v.push_back(take(N));
    v.push_back(take(sizeof(float) * N));
    v.push_back(take(sizeof(float) * N));
    v.push_back(take(sizeof(int) * N));
    v.push_back(take(sizeof(int32_t) * N));
    const bool g16 = m.d.guide_dtype == HDF_GUIDE_BF16 && m.d.rho == m.d.n;
    v.push_back(g16 ? take(sizeof(__nv_bfloat16) * N * R) : 0);
    v.push_back(take(hdf::clus::ws_bytes(m.N, m.d.rho, b->sms)));
  }
  // most items any compiled shape can produce
  size_t max_items = 0;
  for (int i = 0; i < count; ++i) {
    const hdf::Img& m = b->im[i];
    size_t best = 0;
    for (auto& c : hdf::shape_candidates(m.SB, b->smem_max)) {
      const size_t t = (size_t)((m.d.W + hdf::BT_TX - 1) / hdf::BT_TX) *
                       ((m.d.H + c.second - 1) / c.second) * ((m.planes + c.first - 1) / c.first);
      best = std::max(best, t);
    }
    max_items += best;
  }
  b->max_items = max_items;
  const size_t t_cl = take(sizeof(hdf::clus::ClArgs) * count);
  const size_t t_grp = take(sizeof(int4) * (size_t)b->sms);
  const size_t t_ord = take(sizeof(int) * count);
  const size_t t_cll = take(sizeof(int) * count);
  const size_t t_fit = take(sizeof(hdf::FitJob) * count);
  const size_t t_fit1 = take(sizeof(hdf::FitJob));
  const size_t t_rm = take(sizeof(hdf::RmJob) * count);
  const size_t t_rmb = take(sizeof(int) * count);
  const size_t t_g16 = take(sizeof(hdf::GuideJob) * count);
  const size_t t_g16b = take(sizeof(int) * count);
  const size_t t_img = take(sizeof(hdf::BatchImg) * count);
  const size_t t_divb = take(sizeof(int) * count);
  const size_t t_items = take(sizeof(int4) * (max_items + 1));
  const size_t t_cnt = take(sizeof(int));
  b->arena_bytes = o;
  if (cudaMalloc(&b->arena, o) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return HDF_ENOMEM;
  }
  unsigned char* a = (unsigned char*)b->arena;
  for (int i = 0; i < count; ++i) {
    hdf::Img& m = b->im[i];
    const std::vector<size_t>& v = off[i];
    m.ctrl = (int*)(a + v[0]);
    m.mu = (float*)(a + v[1]);
    m.mu64 = (double*)(a + v[2]);
    m.pinv64 = (double*)(a + v[3]);
    m.pinv32 = (float*)(a + v[4]);
    m.ek = (double*)(a + v[5]);
    m.B = (float*)(a + v[6]);
    m.C = (float*)(a + v[7]);
    m.s = (uint8_t*)(a + v[8]);
    m.den = (float*)(a + v[9]);
    m.rmax = (float*)(a + v[10]);
    m.fix_list = (int*)(a + v[11]);
    m.labels = (int32_t*)(a + v[12]);
    m.g16 = v[13] ? (__nv_bfloat16*)(a + v[13]) : nullptr;
    m.cl_ws = a + v[14];
  }
  b->d_cl = (hdf::clus::ClArgs*)(a + t_cl);
  b->d_grp = (int4*)(a + t_grp);
  b->d_ord = (int*)(a + t_ord);
  b->d_cl_list = (int*)(a + t_cll);
  b->d_fit = (hdf::FitJob*)(a + t_fit);
  b->d_fit1 = (hdf::FitJob*)(a + t_fit1);
  b->d_rm = (hdf::RmJob*)(a + t_rm);
  b->d_rm_block0 = (int*)(a + t_rmb);
  b->d_g16 = (hdf::GuideJob*)(a + t_g16);
  b->d_g16_block0 = (int*)(a + t_g16b);
  b->d_img = (hdf::BatchImg*)(a + t_img);
  b->d_div_block0 = (int*)(a + t_divb);
  b->d_items = (int4*)(a + t_items);
  b->d_counter = (int*)(a + t_cnt);
  bool ok = cudaMemset(b->arena, 0, o) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&b->st_int, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k <= hdf::kStages && ok; ++k) ok = cudaEventCreate(&b->ev[k]) == cudaSuccess;
  ok = ok && cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    hdf_status s = cuda_fail(cudaGetLastError(), "hdf_batch_create");
    hdf_batch_destroy(b);
    return s;
  }
  hdf::plan_cluster(b);
  *out = b;
  return HDF_OK;
}

void hdf_batch_destroy(hdf_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  hdf::drop_graph(b);
  if (b->st_int) cudaStreamDestroy(b->st_int);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (int k = 0; k <= hdf::kStages; ++k)
    if (b->ev[k]) cudaEventDestroy(b->ev[k]);
  cudaFree(b->arena);
  delete b;
}

hdf_status hdf_batch_bind(hdf_batch* b, const float* const* d_f, const void* const* d_p,
                          float* const* d_g) {
  if (!b || !d_f || !d_g) return HDF_EINVAL;
  for (int i = 0; i < b->count; ++i) {
    hdf::Img& m = b->im[i];
    const void* p = d_p ? d_p[i] : nullptr;
    if (!d_f[i] || !d_g[i]) return HDF_EINVAL;
    if ((const void*)d_g[i] == (const void*)d_f[i] || (p && (const void*)d_g[i] == p))
      return HDF_EINVAL;
    if (!p) {
      if (m.d.rho != m.d.n) return HDF_EINVAL;
      if (m.d.guide_dtype == HDF_GUIDE_BF16 && !m.g16) return HDF_EINVAL;
    }
  }
  for (int i = 0; i < b->count; ++i) {
    hdf::Img& m = b->im[i];
    const void* p = d_p ? d_p[i] : nullptr;
    m.f = d_f[i];
    m.g = d_g[i];
    m.bf16_own = (!p && m.d.guide_dtype == HDF_GUIDE_BF16) ? 1 : 0;
    m.p = p ? p : (const void*)d_f[i];
  }
  HDF_CUDA(cudaDeviceSynchronize(), "sync");   // no run in flight reads the tables
  hdf::drop_graph(b);
  HDF_CUDA(hdf::upload_tables(b), "batch tables");
  HDF_CUDA(hdf::upload_items(b, hdf::build_items(b, hdf::all_images(b))), "batch items");
  b->bound = true;
  return HDF_OK;
}

hdf_status hdf_batch_set_centers(hdf_batch* b, int i, const float* h_mu, int K) {
  if (!b || !h_mu || i < 0 || i >= b->count) return HDF_EINVAL;
  hdf::Img& m = b->im[i];
  if (K < 1 || K > m.d.K) return HDF_EINVAL;
  HDF_CUDA(cudaDeviceSynchronize(), "sync");
  HDF_CUDA(cudaMemcpy(m.mu, h_mu, sizeof(float) * (size_t)K * m.d.rho, cudaMemcpyHostToDevice),
           "set_centers copy");
  HDF_CUDA(cudaMemcpy(m.ctrl + hdf::CTRL_K_EFF, &K, sizeof(int), cudaMemcpyHostToDevice),
           "set_centers K");
  const hdf::FitJob job{m.mu, m.d.rho, m.ctrl, 1.0 / (2.0 * m.d.sigma_r * m.d.sigma_r), m.pinv64,
                        m.pinv32};
  HDF_CUDA(cudaMemcpy(b->d_fit1, &job, sizeof(job), cudaMemcpyHostToDevice), "set_centers job");
  HDF_CUDA(hdf::launch_fit_batch(b->d_fit1, 1, m.d.K, b->st_int), "fit");
  HDF_CUDA(cudaStreamSynchronize(b->st_int), "sync");
  if (!m.user_centers) {
    m.user_centers = 1;
    hdf::plan_cluster(b);
    hdf::drop_graph(b);
    if (b->bound) HDF_CUDA(hdf::upload_tables(b), "batch tables");
  }
  return HDF_OK;
}

hdf_status hdf_batch_run(hdf_batch* b, int flags, void* stream) {
  if (!b || !b->bound) return HDF_EINVAL;
  hdf::NvtxRange r("hdf batch run");
  cudaStream_t user = (cudaStream_t)stream;
  const int key = flags & HDF_BATCH_SKIP_CLUSTER;
  if (flags & HDF_BATCH_TIMED) {
    HDF_CUDA(hdf::enqueue(b, flags, user, b->ev), "batch run");
    b->timed_valid = true;
    return HDF_OK;
  }
  if (!(flags & HDF_BATCH_GRAPH) || b->graph_state < 0) {
    HDF_CUDA(hdf::enqueue(b, flags, user, nullptr), "batch run");
    return HDF_OK;
  }
  if (!b->exec || b->exec_flags != key) {
    hdf::drop_graph(b);
    cudaGraph_t graph = nullptr;
    HDF_CUDA(cudaStreamBeginCapture(b->st_int, cudaStreamCaptureModeThreadLocal), "capture");
    const cudaError_t e1 = hdf::enqueue(b, flags, b->st_int, nullptr);
    const cudaError_t e2 = cudaStreamEndCapture(b->st_int, &graph);
    cudaError_t e3 = cudaErrorUnknown;
    if (e1 == cudaSuccess && e2 == cudaSuccess && graph)
      e3 = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
      // a stage this device or driver cannot capture: run without a graph from now on
      cudaGetLastError();
      b->exec = nullptr;
      b->graph_state = -1;
      HDF_CUDA(hdf::enqueue(b, flags, user, nullptr), "batch run");
      return HDF_OK;
    }
    b->exec_flags = key;
    b->graph_state = 1;
  }
  HDF_CUDA(cudaEventRecord(b->ev_in, user), "event");
  HDF_CUDA(cudaStreamWaitEvent(b->st_int, b->ev_in, 0), "wait");
  HDF_CUDA(cudaGraphLaunch(b->exec, b->st_int), "graph launch");
  HDF_CUDA(cudaEventRecord(b->ev_out, b->st_int), "event");
  HDF_CUDA(cudaStreamWaitEvent(user, b->ev_out, 0), "wait");
  return HDF_OK;
}

hdf_status hdf_batch_tune(hdf_batch* b, int reps, void* stream) {
  if (!b || !b->bound || reps < 1) return HDF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  HDF_CUDA(cudaDeviceSynchronize(), "sync");
  hdf::drop_graph(b);
  HDF_CUDA(hdf::enqueue(b, 0, st, nullptr), "tune run");
  HDF_CUDA(cudaStreamSynchronize(st), "sync");
  b->trials.clear();
  std::vector<std::pair<int, int>> keys;
  for (auto& m : b->im) keys.push_back({m.SB, m.planes});
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  cudaEvent_t e0, e1;
  HDF_CUDA(cudaEventCreate(&e0), "event");
  HDF_CUDA(cudaEventCreate(&e1), "event");
  hdf_status status = HDF_OK;
  // clustering plan: one group per image, or M equal groups taking their
  // images one after the other; each timed once on the bound guides
  if (!b->cl_list.empty()) {
    const int L = (int)b->cl_list.size();
    std::vector<int> cand = {0};
    for (int M = 1; M < L && M <= b->sms; M *= 2) cand.push_back(M);
    float best_ms = 1e30f;
    int best = b->cl_groups;
    const size_t first = b->trials.size();
    for (int M : cand) {
      b->cl_groups = M;
      hdf::plan_cluster(b);
      cudaError_t e = hdf::upload_tables(b);
      if (e == cudaSuccess)
        e = hdf::launch_batch_prep(b->d_img, b->count, b->d_cl, b->d_cl_list, L, b->d_counter, st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess)
        e = hdf::clus::launch_table(b->rho_max_cl, b->d_cl, b->d_grp, (int)b->groups.size(),
                                    b->d_ord, nullptr, b->grid_cluster,
                                    hdf::clus::DEFAULT_WAIT_NS, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e != cudaSuccess) { status = cuda_fail(e, "tune clustering"); break; }
      const int gsz = M == 0 ? 0 : b->sms / M;
      b->trials.push_back({0, M, gsz, 0, t, 0});
      if (t < best_ms) { best_ms = t; best = M; }
    }
    if (status == HDF_OK) {
      for (size_t t = first; t < b->trials.size(); ++t) b->trials[t].chosen = b->trials[t].planes == best;
      b->cl_groups = best;
      hdf::plan_cluster(b);
    }
  }
  for (auto& key : keys) {
    if (status != HDF_OK) break;
    std::vector<int> sel;
    for (int i = 0; i < b->count; ++i)
      if (b->im[i].SB == key.first && b->im[i].planes == key.second) sel.push_back(i);
    const auto cands = hdf::shape_candidates(key.first, b->smem_max);
    float best_ms = 1e30f;
    std::pair<int, int> best = {b->im[sel[0]].P, b->im[sel[0]].TY};
    const size_t first = b->trials.size();
    for (auto& c : cands) {
      for (int i : sel) { b->im[i].P = c.first; b->im[i].TY = c.second; }
      cudaError_t e = hdf::upload_tables(b);
      const std::vector<int4> items = hdf::build_items(b, sel);
      if (e == cudaSuccess) e = hdf::upload_items(b, items);
      const size_t smem = hdf::batch_smem(key.first, c.first, c.second);
      float ms = 1e30f;
      for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = hdf::tile_launch(b, (int)items.size(), smem, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && r > 0) ms = std::min(ms, t);   // r = 0 warms up
      }
      if (e != cudaSuccess) { status = cuda_fail(e, "tune"); break; }
      b->trials.push_back({key.first, key.second, c.first, c.second, ms, 0});
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
    if (status != HDF_OK) break;
    for (size_t t = first; t < b->trials.size(); ++t)
      b->trials[t].chosen = b->trials[t].P == best.first && b->trials[t].TY == best.second;
    for (int i : sel) { b->im[i].P = best.first; b->im[i].TY = best.second; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != HDF_OK) return status;
  HDF_CUDA(hdf::upload_tables(b), "batch tables");
  HDF_CUDA(hdf::upload_items(b, hdf::build_items(b, hdf::all_images(b))), "batch items");
  return HDF_OK;
}

hdf_status hdf_batch_get_tuning(hdf_batch* b, hdf_tile_trial* out, int cap, int* count) {
  if (!b || !count || cap < 0 || (cap > 0 && !out)) return HDF_EINVAL;
  const int n = std::min(cap, (int)b->trials.size());
  for (int k = 0; k < n; ++k) out[k] = b->trials[k];
  *count = (int)b->trials.size();
  return HDF_OK;
}

hdf_status hdf_batch_set_shape(hdf_batch* b, int SB, int planes, int P, int TY) {
  if (!b) return HDF_EINVAL;
  bool ok = false;
  for (auto& c : hdf::shape_candidates(SB, b->smem_max)) ok |= c.first == P && c.second == TY;
  if (!ok) return HDF_EINVAL;
  HDF_CUDA(cudaDeviceSynchronize(), "sync");
  for (auto& m : b->im)
    if (m.SB == SB && m.planes == planes) { m.P = P; m.TY = TY; }
  hdf::drop_graph(b);
  if (b->bound) {
    HDF_CUDA(hdf::upload_tables(b), "batch tables");
    HDF_CUDA(hdf::upload_items(b, hdf::build_items(b, hdf::all_images(b))), "batch items");
  }
  return HDF_OK;
}

hdf_status hdf_batch_get_times(hdf_batch* b, float* h_ms, int cap, int* count) {
  if (!b || !count || cap < 0 || (cap > 0 && !h_ms)) return HDF_EINVAL;
  if (!b->timed_valid) return HDF_EINVAL;
  HDF_CUDA(cudaEventSynchronize(b->ev[hdf::kStages]), "sync");
  const int n = std::min(cap, hdf::kStages);
  for (int k = 0; k < n; ++k) HDF_CUDA(cudaEventElapsedTime(h_ms + k, b->ev[k], b->ev[k + 1]), "elapsed");
  *count = n;
  return HDF_OK;
}

hdf_status hdf_batch_get_centers(hdf_batch* b, int i, float* h_mu, int* K_eff) {
  if (!b || !h_mu || !K_eff || i < 0 || i >= b->count) return HDF_EINVAL;
  const hdf::Img& m = b->im[i];
  HDF_CUDA(cudaDeviceSynchronize(), "sync");
  HDF_CUDA(cudaMemcpy(K_eff, m.ctrl + hdf::CTRL_K_EFF, sizeof(int), cudaMemcpyDeviceToHost), "get K");
  HDF_CUDA(cudaMemcpy(h_mu, m.mu, sizeof(float) * (size_t)m.d.K * m.d.rho, cudaMemcpyDeviceToHost),
           "get centers");
  return HDF_OK;
}

hdf_status hdf_batch_get_stats(hdf_batch* b, int i, hdf_stats* out) {
  if (!b || !out || i < 0 || i >= b->count) return HDF_EINVAL;
  const hdf::Img& m = b->im[i];
  int c[hdf::CTRL_WORDS];
  double ek = 0.0;
  HDF_CUDA(cudaDeviceSynchronize(), "sync");
  HDF_CUDA(cudaMemcpy(c, m.ctrl, sizeof(c), cudaMemcpyDeviceToHost), "stats");
  HDF_CUDA(cudaMemcpy(&ek, m.ek, sizeof(double), cudaMemcpyDeviceToHost), "stats");
  out->K_eff = c[hdf::CTRL_K_EFF];
  out->device_error = c[hdf::CTRL_ERROR];
  out->fallback_pixels = c[hdf::CTRL_FALLBACK];
  out->lloyd_iters_max = c[hdf::CTRL_LLOYD_MAX];
  out->rounds = c[hdf::CTRL_ROUNDS];
  out->cluster_error = ek;
  out->rescued_pixels = 0;   // the batch keeps every pixel on the float32 path
  out->nlm_sweeps = 0;
  return (hdf_status)c[hdf::CTRL_ERROR];
}

hdf_status hdf_batch_get_info(hdf_batch* b, hdf_batch_info* out) {
  if (!b || !out) return HDF_EINVAL;
  out->count = b->count;
  out->graph_state = b->graph_state;
  out->launches_per_run = hdf::launches_per_run(b, 0);
  out->nitems = b->nitems;
  out->ngroups = (int)b->groups.size();
  out->grid_cluster = b->grid_cluster;
  out->grid_tile = b->grid_tile;
  out->smem_tile = b->smem_tile;
  out->device_bytes = b->arena_bytes;
  return HDF_OK;
}

}  // extern "C"
