// Device code of Algorithm 1 "cluster": bisecting K-means of the range set
// Theta = {p(i)} (Eq. (8), Sec. II-C), entirely on the device in one
// cooperative persistent launch (no host round trip, graph-capturable).
//
// Method (paper): start from one cluster; repeatedly split the cluster of
// largest variance into two by 2-means, initialised with a pair of points
// of largest separation, until there are K clusters.  Readings shared with
// the FP64 oracle: variance = sum of squared deviations (SSE), ties -> lowest
// cluster index, stop early when the largest SSE is 0; initial pair a = the
// point farthest from the mean, b = the point farthest from a (ties -> first
// in raster order); Lloyd iterations assign each point to the nearer centre
// (ties -> a), stop when no assignment changes or after 20 assignments, and
// keep the previous assignment if a side would become empty; child 1 keeps
// the parent's index, child 2 takes the next one.
//
// GPU design.  The split of a cluster depends only on that cluster's points,
// so the split tree is a deterministic function of the data.  Each round
// replays the sequential greedy rule (largest SSE first) on the part of the
// tree computed so far and collects every node the replay would split next
// without knowing its children; all of them are split together in that round
// (segments of one permutation array, one pass over all their points per
// Lloyd iteration).  The final replay on the complete tree yields exactly the
// sequential algorithm's clusters and numbering.  Splits a later replay does
// not use are simply ignored.
//
// Precision: distances in FP32 from direct differences; every integer
// decision is taken in FP64 where FP32 cannot settle it (Lloyd assignments
// within 2^-14 relative of a tie, farthest-point candidates within 2^-12 of
// the maximum).  Coordinate sums are accumulated error-free per thread
// (TwoSum pairs), then in FP64 across threads and blocks in a fixed order, so
// the means match a plain FP64 evaluation to rounding and are exact for
// clusters of identical points (deterministic for a given grid).  The points
// are kept in a planar copy permuted with the clusters, so every pass reads
// them coalesced.
//
// Synchronisation: a grid barrier with a bounded wait (2 s unless the launch
// sets another limit), after which the
// device status records HDF_ETIMEOUT and every block returns.  Reductions
// across blocks are replayed identically by every block from the per-block
// partial results, so block-local copies of the control state agree.
#pragma once

#include <math.h>

#include <type_traits>

#include "cluster_args.cuh"

namespace hdf {

namespace clus {
namespace {

// Threads per block of this translation unit's instantiation (one block per
// SM): the instantiations for guides of few dimensions keep few coordinates
// per point in registers and run 32 warps per SM; those for many dimensions
// run fewer, larger threads.  A chunk is CH points, PPT per thread.
#ifndef HDF_CL_THREADS
#define HDF_CL_THREADS 256
#endif
constexpr int CL_THREADS = HDF_CL_THREADS;
constexpr int CL_WARPS = CL_THREADS / 32;
constexpr int PPT = CH / CL_THREADS;    // points per thread per chunk
static_assert(PPT * CL_THREADS == CH && PPT >= 1, "a chunk is a whole number of points per thread");

// Points whose coordinates one thread loads together (registers permitting).
template <int RMAX>
__host__ __device__ constexpr int load_batch() {
  return (RMAX <= 4 ? 8 : (RMAX <= 16 ? 2 : 1)) < PPT
             ? (RMAX <= 4 ? 8 : (RMAX <= 16 ? 2 : 1))
             : PPT;
}

struct ClShared {
  int seg_start[MAXSEG], seg_count[MAXSEG], seg_chunk0[MAXSEG + 1], seg_on[MAXSEG];
  int seg_act[MAXSEG];    // splits still iterating (the Lloyd loop keeps its chunk table)
  int nseg, nchunks;
  SlotRec slot[MAXACT];
  int nslots;
  double sim_sse[MAXNODES];
  int sim_child0[MAXNODES];
  int leaf_node[HDF_MAX_K], leaf_cl[HDF_MAX_K];
  int nleaves, nclusters, nneeded;
  int needed[MAXACT];
  float redg[CL_WARPS][2 * HDF_MAX_RHO];
  float redf[CL_WARPS][1];
  int redi[CL_WARPS][2];
  float redd[CL_WARPS];
  double redD[CL_WARPS];
  int redx[CL_WARPS];
  int scanw[CL_WARPS];
  int hlist[CH];          // positions of a chunk that need the full test
  int wtab[PPT * CL_WARPS];   // per (u, warp) counts, then their exclusive prefix
  int wtotal;
  int ccnt[4];               // side-b counts of a group of chunks (partition count pass)
  int mypre[64];             // partition: side-b points before each of the block's chunks
  int segpre[MAXSEG];        //   and before each segment's first chunk
  float segmax[MAXSEG];
  float slack[MAXACT];   // centre movement of the last update
  double cum[MAXACT];    // total centre movement since the split started
  float cabs[MAXACT];    // absolute allowance for the float32 rounding of the centres
  double segsse[MAXSEG];
  int segarg[MAXSEG];
  int ok;
  int all_done;
  int tr_n;              // trace events recorded (block 0)
  float bmax;            // block maximum of the last block_max_sum
  int last;              // this block is the last contributor of a split
};

__device__ __forceinline__ bool better(double d1, int i1, double d2, int i2) {
  return d1 > d2 || (d1 == d2 && i1 < i2);
}

// Trace event of the group's block 0 (thread 0): the event count lives in
// shared memory, so recording is two stores and no global round trip.
__device__ __forceinline__ void trace_event(long long* trace, int bid, int& count, int phase) {
  if (bid == 0 && threadIdx.x == 0 && count < TRACE_CAP) {
    trace[1 + 2 * count] = phase;
    trace[2 + 2 * count] = (long long)globaltimer_ns();
    ++count;
    trace[0] = count;
  }
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier with a bounded wait.  One monotonically growing arrival
// counter per launch: the gen-th barrier is passed once it reaches gen * G,
// so a block arrives with a single atomic and nobody resets anything.  The
// wait gives up after a.wait_ns (recording HDF_ETIMEOUT), or as soon as the
// device status records an error from another block.  Returns false if the
// device status records an error, in which case the caller returns.
__device__ bool grid_barrier(const ClArgs& a, unsigned& gen, ClShared& s, int phase) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* cnt = (unsigned*)(a.ctrl + CTRL_BARRIER);
    ++gen;
    const unsigned target = gen * (unsigned)a.G;
    __threadfence();
    const unsigned arrived = atomicAdd(cnt, 1u) + 1u;
    if (arrived < target) {
      const unsigned long long t0 = globaltimer_ns();
      unsigned k = 0;
      while (ld_acquire_gpu(cnt) < target) {
        if ((++k & 31u) == 0) {
          if (*(volatile int*)(a.ctrl + CTRL_ERROR) != 0) break;
          if (globaltimer_ns() - t0 > a.wait_ns) {
            record_error(a.ctrl, HDF_ETIMEOUT);
            break;
          }
        }
      }
    }
    __threadfence();
    s.ok = (*(volatile int*)(a.ctrl + CTRL_ERROR) == 0);
    trace_event(a.trace, a.bid, s.tr_n, phase);
  }
  __syncthreads();
  return s.ok != 0;
}

// Guide element (raster layout) as float, for either storage type.
__device__ __forceinline__ float guide_at(const ClArgs& a, size_t i) {
  return a.p_bf16 ? __bfloat162float(((const __nv_bfloat16*)a.p)[i]) : __ldg((const float*)a.p + i);
}

// Chunk prefix of the current segment table (thread 0), then sync.
__device__ void build_chunks(ClShared& s) {
  if (threadIdx.x == 0) {
    int c = 0;
    for (int i = 0; i < s.nseg; ++i) {
      s.seg_chunk0[i] = c;
      if (s.seg_on[i]) c += (s.seg_count[i] + CH - 1) / CH;
    }
    s.seg_chunk0[s.nseg] = c;
    s.nchunks = c;
  }
  __syncthreads();
}

// Double-float value hi + lo.  Sums run in FP32 pairs: FP64 issues at 1/64 of
// the FP32 rate on this GPU, so warp-wide FP64 reductions would dominate.
struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const float s = a.hi + b.hi;                      // TwoSum of the high parts
  const float bp = s - a.hi;
  float e = (a.hi - (s - bp)) + (b.hi - bp);
  e += a.lo + b.lo;
  F2 r;
  r.hi = s + e;                                     // FastTwoSum renormalisation
  r.lo = e - (r.hi - s);
  return r;
}

__device__ __forceinline__ double f2_to_d(F2 x) { return (double)x.hi + (double)x.lo; }

struct ArgMax {
  double d;
  int i;
};

__device__ __forceinline__ F2 shfl_xor_t(F2 x, int o) {
  F2 r;
  r.hi = __shfl_xor_sync(0xffffffffu, x.hi, o);
  r.lo = __shfl_xor_sync(0xffffffffu, x.lo, o);
  return r;
}
__device__ __forceinline__ double shfl_xor_t(double x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
__device__ __forceinline__ float shfl_xor_t(float x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
__device__ __forceinline__ ArgMax shfl_xor_t(ArgMax x, int o) {
  ArgMax r;
  r.d = __shfl_xor_sync(0xffffffffu, x.d, o);
  r.i = __shfl_xor_sync(0xffffffffu, x.i, o);
  return r;
}

// Side of the accepted 2-means assignment at position pos; rv = 1 + the
// iteration whose changes were undone (0: none).
__device__ __forceinline__ int accepted_side(const ClArgs& a, int pos, int rv) {
  const int sd = (int)__ldcg(a.side + pos);
  return (rv > 0 && (int)__ldcg(a.side + a.N + pos) == rv) ? sd ^ 1 : sd;
}

// x / y in FP64 from the correctly rounded reciprocal (__drcp_rn) and one
// remainder correction (Markstein's FMA refinement: e = x - q y exactly,
// q += e / y); exact when the quotient is representable, as for the mean of
// identical points.  Cheaper than the FP64 division sequence.
__device__ __forceinline__ double quotient(double x, double y) {
  const double r = __drcp_rn(y);
  double q = x * r;
  const double e = fma(-q, y, x);
  return fma(e, r, q);
}

// An upper bound of sqrt(x), x >= 0: FP32 square root (the FP64 one is slow
// on this GPU) of the rounded value, scaled up by 2^-20 relative, which covers
// the < 2^-23 relative error of the conversion and of sqrtf; FP64 where the
// FP32 value would be subnormal.
__device__ __forceinline__ double sqrt_up(double x) {
  if (!(x >= 1e-36 && x <= 1e36)) return sqrt(x);
  return (double)sqrtf((float)x) * ROUND_UP;
}

// Deterministic replay of a cross-block reduction, run identically by every
// block: for each value v, lane l of a warp combines the contributors
// i = l, l + 32, ... of v, and the lanes are combined by a fixed xor tree.
// The loads of IPW values per warp are independent, so their latencies
// overlap.  combine(a, b) must be commutative; init is its identity.
template <int IPW, class T, class NC, class SRC, class COMB, class DST>
__device__ void replay(int nvals, T init, NC nc_of, SRC src, COMB combine, DST dst) {
  constexpr int SMALL = 8;   // at most this many contributors: one thread per value
  for (int v = threadIdx.x; v < nvals; v += CL_THREADS) {
    const int n = nc_of(v);
    if (n > SMALL) continue;
    T buf[SMALL];
#pragma unroll
    for (int i = 0; i < SMALL; ++i) buf[i] = (i < n) ? src(v, i) : init;
    T acc = init;
#pragma unroll
    for (int i = 0; i < SMALL; ++i) acc = combine(acc, buf[i]);
    dst(v, acc);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = warp * IPW; base < nvals; base += CL_WARPS * IPW) {
    T part[IPW];
    bool big[IPW];
#pragma unroll
    for (int k = 0; k < IPW; ++k) {
      part[k] = init;
      const int v = base + k;
      const int n = v < nvals ? nc_of(v) : 0;
      big[k] = n > SMALL;
      if (big[k]) {
#pragma unroll 4
        for (int i = lane; i < n; i += 32) part[k] = combine(part[k], src(v, i));
      }
    }
#pragma unroll
    for (int k = 0; k < IPW; ++k) {
      if (!big[k]) continue;
      T x = part[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x = combine(x, shfl_xor_t(x, o));
      if (lane == 0) dst(base + k, x);
    }
  }
}

// Iterate over this block's chunks at chunk granularity: f(seg, base, end, j)
// with the chunk's positions base + u * CL_THREADS + tid (u < PPT), < end;
// flush(seg) once per segment after its last chunk in this block.
template <class F, class Flush>
__device__ void for_blocks(const ClArgs& a, const ClShared& s, F f, Flush flush) {
  int cur = -1, seg = 0;
  for (int j = a.bid; j < s.nchunks; j += a.G) {
    while (s.seg_chunk0[seg + 1] <= j) ++seg;
    if (seg != cur) {
      if (cur >= 0) flush(cur);
      cur = seg;
    }
    const int base = s.seg_start[seg] + (j - s.seg_chunk0[seg]) * CH;
    f(seg, base, s.seg_start[seg] + s.seg_count[seg], j);
  }
  if (cur >= 0) flush(cur);
}

// Blocks whose partial results cover segment `seg`, in a fixed order.
__device__ __forceinline__ int contrib_count(const ClArgs& a, const ClShared& s, int seg) {
  const int nch = s.seg_chunk0[seg + 1] - s.seg_chunk0[seg];
  return nch < a.G ? nch : a.G;
}
__device__ __forceinline__ int contrib_block(const ClArgs& a, const ClShared& s, int seg, int i) {
  return (s.seg_chunk0[seg] + i) % a.G;
}

// hi + x = t + e exactly (Knuth's TwoSum); the error terms are summed in lo.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float t = hi + x;
  const float bp = t - hi;
  const float e = (hi - (t - bp)) + (x - bp);
  hi = t;
  lo += e;
}

// Block sum of NV per-thread double-float values, fixed order.  Within a warp
// the values are reduced by recursive halving (each lane keeps half of its
// values and adds its partner's copy of them), so a warp needs NV - 1 pair
// additions per lane instead of 5 NV; lane l ends with value (l >> (5-L)) & (NV-1)
// (L = log2 NV <= 5).  The warp results are then added across warps.  out
// receives nv pairs (hi, lo).
template <int NV>
__device__ void block_sum_f2(const float (&hi)[NV], const float (&lo)[NV], int nv, ClShared& s,
                             float* out) {
  static_assert((NV & (NV - 1)) == 0, "power of two");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int H = NV > 32 ? NV / 32 : 1;          // values per lane after the halving
  constexpr int NV1 = NV > 32 ? 32 : NV;            // values per group of the halving
#pragma unroll
  for (int h = 0; h < H; ++h) {
    F2 v[NV1];
#pragma unroll
    for (int i = 0; i < NV1; ++i) {
      v[i].hi = hi[h * NV1 + i];
      v[i].lo = lo[h * NV1 + i];
    }
    int n = NV1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (n > 1) {
        const int half = n / 2;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < NV1 / 2; ++i) {
          if (i < half) {
            const F2 send = up ? v[i] : v[i + half];
            const F2 keep = up ? v[i + half] : v[i];
            v[i] = f2_add(keep, shfl_xor_t(send, o));
          }
        }
        n = half;
      } else {
        v[0] = f2_add(v[0], shfl_xor_t(v[0], o));
      }
    }
    constexpr int L = NV1 == 32 ? 5 : NV1 == 16 ? 4 : NV1 == 8 ? 3 : NV1 == 4 ? 2 : NV1 == 2 ? 1 : 0;
    const int idx = h * NV1 + ((lane >> (5 - L)) & (NV1 - 1));
    if ((lane & ((1 << (5 - L)) - 1)) == 0) {
      s.redg[warp][2 * idx] = v[0].hi;
      s.redg[warp][2 * idx + 1] = v[0].lo;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += CL_THREADS) {
    F2 t;
    t.hi = s.redg[0][2 * i];
    t.lo = s.redg[0][2 * i + 1];
#pragma unroll
    for (int w = 1; w < CL_WARPS; ++w) {
      F2 u;
      u.hi = s.redg[w][2 * i];
      u.lo = s.redg[w][2 * i + 1];
      t = f2_add(t, u);
    }
    out[2 * i] = t.hi;
    out[2 * i + 1] = t.lo;
  }
  __syncthreads();
}

__device__ void block_sum_i2(int v0, int v1, ClShared& s, int* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
  }
  if (lane == 0) { s.redi[warp][0] = v0; s.redi[warp][1] = v1; }
  __syncthreads();
  if (threadIdx.x < 2) {
    int t = 0;
    for (int w = 0; w < CL_WARPS; ++w) t += s.redi[w][threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// Exclusive scan of one int per thread across the block; *total = sum.
__device__ int block_excl_scan(int v, ClShared& s, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s.scanw[warp] = x;
  __syncthreads();
  int before = 0, t = 0;
#pragma unroll
  for (int w = 0; w < CL_WARPS; ++w) {
    if (w < warp) before += s.scanw[w];
    t += s.scanw[w];
  }
  __syncthreads();
  *total = t;
  return before + x - v;
}

// Ranks in position order of the flagged points of a chunk whose positions
// are base + u * CL_THREADS + tid (u < PPT): rank[u] = number of flagged
// points at smaller positions (valid where flag[u]); returns the total.  The
// per-(u, warp) ballot counts are prefixed over the 64 (u, warp) pairs in
// position order by warp 0.  Three block barriers.
__device__ int position_ranks(const bool (&flag)[PPT], int (&rank)[PPT], ClShared& s) {
  static_assert(PPT * CL_WARPS == 64, "the prefix runs over 64 (u, warp) counts");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int pre[PPT];
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const unsigned bal = __ballot_sync(0xffffffffu, flag[u]);
    pre[u] = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) s.wtab[u * CL_WARPS + warp] = __popc(bal);
  }
  __syncthreads();
  if (warp == 0) {
    const int v0 = s.wtab[2 * lane], v1 = s.wtab[2 * lane + 1];
    int x = v0 + v1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const int ex = x - v0 - v1;
    s.wtab[2 * lane] = ex;
    s.wtab[2 * lane + 1] = ex + v0;
    if (lane == 31) s.wtotal = x;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < PPT; ++u) rank[u] = s.wtab[u * CL_WARPS + warp] + pre[u];
  const int total = s.wtotal;
  __syncthreads();   // wtab / wtotal may be rewritten by the next call
  return total;
}

// Block max of a float and sum of a float; results written by thread 0.
__device__ void block_max_sum(float m, F2 sum, ClShared& s, float* out_max, float* out_sum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    sum = f2_add(sum, shfl_xor_t(sum, o));
  }
  if (lane == 0) { s.redd[warp] = m; s.redg[warp][0] = sum.hi; s.redg[warp][1] = sum.lo; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = s.redd[0];
    F2 ss;
    ss.hi = s.redg[0][0];
    ss.lo = s.redg[0][1];
    for (int w = 1; w < CL_WARPS; ++w) {
      F2 u;
      u.hi = s.redg[w][0];
      u.lo = s.redg[w][1];
      mm = fmaxf(mm, s.redd[w]);
      ss = f2_add(ss, u);
    }
    *out_max = mm;
    s.bmax = mm;
    out_sum[0] = ss.hi;
    out_sum[1] = ss.lo;
  }
  __syncthreads();
}

__device__ void block_argmax(double d, int idx, ClShared& s, double* out_d, int* out_i) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double d2 = __shfl_xor_sync(0xffffffffu, d, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (better(d2, i2, d, idx)) { d = d2; idx = i2; }
  }
  if (lane == 0) { s.redD[warp] = d; s.redx[warp] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bd = s.redD[0];
    int bi = s.redx[0];
    for (int w = 1; w < CL_WARPS; ++w)
      if (better(s.redD[w], s.redx[w], bd, bi)) { bd = s.redD[w]; bi = s.redx[w]; }
    *out_d = bd;
    *out_i = bi;
  }
  __syncthreads();
}

// Coordinate d of the point at permutation position pos.
__device__ __forceinline__ float xat(const float* X, size_t N, int d, int pos) {
  return __ldcg(X + (size_t)d * N + pos);
}

// Replay of the sequential greedy rule on the known tree (warp 0).  Leaves
// carry their cluster index; the leaf of largest SSE (ties -> lowest
// cluster index) is split next.  A leaf whose split is not known yet is
// recorded as needed, removed, and counted as split, and the replay goes on.
__device__ void simulate(ClShared& s, int K, int maxneeded) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  if (lane == 0) {
    s.leaf_node[0] = 0;
    s.leaf_cl[0] = 0;
    s.nleaves = 1;
    s.nclusters = 1;
    s.nneeded = 0;
  }
  __syncwarp();
  while (true) {
    const int nl = s.nleaves;
    if (s.nclusters >= K || nl == 0 || s.nneeded >= maxneeded) break;
    double bd = -1.0;
    int bc = 0x7fffffff, bl = -1;
    for (int i = lane; i < nl; i += 32) {
      const double v = s.sim_sse[s.leaf_node[i]];
      const int c = s.leaf_cl[i];
      if (v > bd || (v == bd && c < bc)) { bd = v; bc = c; bl = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, bd, o);
      const int c2 = __shfl_xor_sync(0xffffffffu, bc, o);
      const int l2 = __shfl_xor_sync(0xffffffffu, bl, o);
      if (v2 > bd || (v2 == bd && c2 < bc)) { bd = v2; bc = c2; bl = l2; }
    }
    if (!(bd > 0.0)) break;
    if (lane == 0) {
      const int nd = s.leaf_node[bl];
      const int c0 = s.sim_child0[nd];
      if (c0 >= 0) {
        s.leaf_node[bl] = c0;
        s.leaf_node[nl] = c0 + 1;
        s.leaf_cl[nl] = s.nclusters;
        s.nleaves = nl + 1;
      } else {
        s.needed[s.nneeded++] = nd;
        s.leaf_node[bl] = s.leaf_node[nl - 1];
        s.leaf_cl[bl] = s.leaf_cl[nl - 1];
        s.nleaves = nl - 1;
      }
      s.nclusters += 1;
    }
    __syncwarp();
  }
}

__host__ __device__ constexpr size_t dyn_c64_offset(int rho) {
  return ((sizeof(float) * MAXSEG * (size_t)rho + 15) / 16) * 16;
}

__host__ __device__ constexpr size_t dyn_red_offset(int rho) {
  return dyn_c64_offset(rho) + sizeof(double) * ((size_t)MAXSEG * rho + (size_t)MAXACT * (rho + 2) +
                                                 3 * (size_t)MAXACT * rho);
}

// ... plus the staging area of one split's partial records (MAXG records)
// and the per-class partial sums of their reduction (CL_THREADS pairs).
__host__ __device__ constexpr size_t dyn_smem_bytes(int rho) {
  return ((dyn_red_offset(rho) + 127) / 128) * 128 +
         sizeof(float) * ((size_t)MAXG * record_floats(rho) + 2 * CL_THREADS);
}

// Lloyd passes of guides of up to 8 dimensions keep the margins (rounded
// down to half precision: the skip test stays conservative) and sides of the
// block's points in shared memory for the whole Lloyd loop of a round, when
// the block holds at most RES_CHUNKS chunks.
constexpr int RES_CHUNKS = 16;
template <int RMAX>
__host__ __device__ constexpr size_t resident_bytes() {
  return RMAX <= 8 ? (size_t)RES_CHUNKS * CH * (sizeof(unsigned short) + 1) : 0;
}
__host__ __device__ constexpr size_t dyn_stage_offset(int rho) {
  return (dyn_smem_bytes(rho) + 127) / 128 * 128;
}

// Distance statistics of every segment of the table against the centres
// c32[seg] / c64[seg]: SSE, then the farthest point decided in FP64 among
// the FP32 candidates (ties -> lowest raster index).  Results in s.segmax /
// s.segsse / s.segarg.  `from_scratch` reads the points (and raster
// indices) from the scatter buffers and moves them into place.  One grid
// barrier: each block takes its own FP64
// candidates relative to its own FP32 maximum; the global FP64 maximiser
// lies within 2^-12 of the global FP32 maximum, hence of its block's
// maximum, so it is its block's winner and the replay of the block winners
// returns it.
template <int RMAX>
__device__ __noinline__ bool dist_stats_fn(const ClArgs& a, ClShared& s, unsigned& gen,
                                           const float* c32, const double* c64, float* X,
                                           const float* Xn, uint32_t* P, const uint32_t* Pn,
                                           bool from_scratch) {
  constexpr int UB = load_batch<RMAX>();
  const int rho = a.rho;
  const int PS = record_floats(rho);
  const int tid = threadIdx.x, bid = a.bid;
  const size_t N = (size_t)a.N;

  {
    float mx = -1.0f;
    F2 sse{0.0f, 0.0f};
    int seg_first_chunk = -1;
    // distances of a batch of points of segment seg (positions >= end skipped)
    auto visit = [&](int seg, auto& posv, int end) {
      constexpr int NB = std::extent<std::remove_reference_t<decltype(posv)>>::value;
      const float* c = c32 + seg * rho;
      float x[NB][RMAX];
      uint32_t pid[NB];
      const float* src = from_scratch ? Xn : X;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int pos = posv[b];
        const bool v = pos < end;
        pid[b] = (v && from_scratch) ? __ldcg(Pn + pos) : 0u;
#pragma unroll
        for (int d = 0; d < RMAX; ++d)
          x[b][d] = (v && d < rho) ? __ldcg(src + (size_t)d * N + pos) : 0.0f;
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int pos = posv[b];
        if (pos >= end) continue;
        float d2 = 0.0f;
#pragma unroll
        for (int d = 0; d < RMAX; ++d) {
          if (d < rho) {
            if (from_scratch) X[(size_t)d * N + pos] = x[b][d];
            const float t = x[b][d] - c[d];
            d2 = fmaf(t, t, d2);
          }
        }
        if (from_scratch) P[pos] = pid[b];
        a.d32[pos] = d2;
        mx = fmaxf(mx, d2);
        two_sum_acc(sse.hi, sse.lo, d2);
      }
    };
    auto dflush = [&](int seg) {
          const size_t off = (size_t)bid * MAXSEG + seg;
          block_max_sum(mx, sse, s, a.pd + off, a.pf + off * PS);   // ends with a block sync
          const float m = s.bmax;                                   // this block's maximum
          // FP64 candidates of this block's chunks of the segment
          double bd = -1.0;
          int bi = 0x7fffffff;
          const int c1 = s.seg_chunk0[seg + 1];
          const int end = s.seg_start[seg] + s.seg_count[seg];
          for (int j = seg_first_chunk; j < c1; j += a.G) {
            constexpr int NQ = PPT;
            float dd[NQ];
            int pp[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
              const int jj = j + (q / PPT) * a.G;
              const int pos = jj < c1 ? s.seg_start[seg] + (jj - s.seg_chunk0[seg]) * CH +
                                            (q % PPT) * CL_THREADS + tid
                                      : end;
              pp[q] = pos;
              dd[q] = (pos < end) ? __ldcg(a.d32 + pos) : -1.0f;
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
              const int pos = pp[q];
              if (pos >= end) continue;
              if (m > 0.0f && dd[q] < m * (1.0f - CAND_REL)) continue;
              const int idx = (int)__ldcg(P + pos);
              double e = 0.0;
              if (m > 0.0f) {
                const double* cc = c64 + (size_t)seg * rho;
                float xv[RMAX];
#pragma unroll
                for (int d = 0; d < RMAX; ++d) xv[d] = (d < rho) ? xat(X, N, d, pos) : 0.0f;
#pragma unroll
                for (int d = 0; d < RMAX; ++d) {
                  if (d < rho) {
                    const double t = (double)xv[d] - cc[d];
                    e = fma(t, t, e);
                  }
                }
              }
              if (better(e, idx, bd, bi)) { bd = e; bi = idx; }
            }
          }
          block_argmax(bd, bi, s, a.pdd + off, a.px + off);
          mx = -1.0f;
          sse = F2{0.0f, 0.0f};
          seg_first_chunk = -1;
    };
    for_blocks(a, s,
        [&](int seg, int base, int end, int j) {
          if (seg_first_chunk < 0) seg_first_chunk = j;
#pragma unroll
          for (int u0 = 0; u0 < PPT; u0 += UB) {
            int pv[UB];
#pragma unroll
            for (int b2 = 0; b2 < UB; ++b2) pv[b2] = base + (u0 + b2) * CL_THREADS + tid;
            visit(seg, pv, end);
          }
        },
        dflush);
  }
  trace_event(a.trace, a.bid, s.tr_n, TR_DPASS);
  if (!grid_barrier(a, gen, s, TR_DIST1)) return false;
  {
    // One fused replay of the blocks' maxima, SSE and FP64 arg-maxima: warp
    // per segment, lanes over the contributors (all loads of a lane issued
    // together), xor trees; every block computes the same values.
    constexpr int MAXC = (MAXG + 31) / 32;
    const int lane = tid & 31, warp = tid >> 5;
    for (int seg = warp; seg < s.nseg; seg += CL_WARPS) {
      if (!s.seg_on[seg]) {
        if (lane == 0) {
          s.segmax[seg] = -1.0f;
          s.segsse[seg] = 0.0;
          s.segarg[seg] = 0x7fffffff;
        }
        continue;
      }
      const int nc = contrib_count(a, s, seg);
      float m = -1.0f;
      F2 t{0.0f, 0.0f};
      ArgMax r;
      r.d = -1.0;
      r.i = 0x7fffffff;
      {
        float pm[MAXC], ph[MAXC], pl[MAXC];
#pragma unroll
        for (int k = 0; k < MAXC; ++k) {
          const int c = lane + 32 * k;
          if (c < nc) {
            const size_t o = (size_t)contrib_block(a, s, seg, c) * MAXSEG + seg;
            pm[k] = __ldcg(a.pd + o);
            ph[k] = __ldcg(a.pf + o * PS);
            pl[k] = __ldcg(a.pf + o * PS + 1);
          }
        }
#pragma unroll
        for (int k = 0; k < MAXC; ++k) {
          if (lane + 32 * k < nc) {
            m = fmaxf(m, pm[k]);
            t = f2_add(t, F2{ph[k], pl[k]});
          }
        }
      }
      {
        double pd[MAXC];
        int px[MAXC];
#pragma unroll
        for (int k = 0; k < MAXC; ++k) {
          const int c = lane + 32 * k;
          if (c < nc) {
            const size_t o = (size_t)contrib_block(a, s, seg, c) * MAXSEG + seg;
            pd[k] = __ldcg(a.pdd + o);
            px[k] = __ldcg(a.px + o);
          }
        }
#pragma unroll
        for (int k = 0; k < MAXC; ++k)
          if (lane + 32 * k < nc && better(pd[k], px[k], r.d, r.i)) { r.d = pd[k]; r.i = px[k]; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        t = f2_add(t, shfl_xor_t(t, o));
        const ArgMax q = shfl_xor_t(r, o);
        if (better(q.d, q.i, r.d, r.i)) r = q;
      }
      if (lane == 0) {
        s.segmax[seg] = m;
        s.segsse[seg] = f2_to_d(t);
        s.segarg[seg] = r.i;
      }
    }
  }
  __syncthreads();
  return true;
}

// The clustering of one guide by the blocks of its group.
template <int RMAX>
__device__ void cluster_run(const ClArgs& a, ClShared& s, unsigned char* dyn) {
  const int rho = a.rho;
  const int PS = record_floats(rho);   // floats per partial record (pairs, padded)
  float* c32 = (float*)dyn;                                   // MAXSEG x rho
  double* c64 = (double*)(dyn + dyn_c64_offset(rho));         // MAXSEG x rho
  double* tmp = c64 + MAXSEG * rho;                           // MAXACT x (rho + 2)
  double* acc_sum = tmp + MAXACT * (rho + 2);                 // MAXACT x rho
  double* nsum = acc_sum + MAXACT * rho;                      // MAXACT x rho sums of the split nodes
  double* mean_a = nsum + MAXACT * rho;                       // MAXACT x rho
  // partial-record regions (distance passes; Lloyd even / odd iterations)
  const size_t pf_stride = (size_t)a.G * MAXSEG * PS;
  float* const pf_root = a.pf + 2 * pf_stride;
  auto acc_sum_a = [&](int i, int d) -> double& { return mean_a[i * rho + d]; };
  float* red = (float*)(dyn + ((dyn_red_offset(rho) + 127) / 128) * 128);   // MAXG records
  float* parts = red + (size_t)MAXG * PS;                                    // CL_THREADS pairs
  unsigned gen = 0;
  const int tid = threadIdx.x, bid = a.bid;
  const size_t N = (size_t)a.N;
  // Points in permutation order (X, raster indices P) and the scatter
  // targets of the partition (Xn, Pn).  Only the split segments are moved,
  // so the children's points are copied back into X / P by the next
  // distance pass (the other leaves never leave X).
  float* const X = a.X;
  float* const Xn = a.X2;
  uint32_t* const P = a.perm;
  uint32_t* const Pn = a.perm2;
  int nnodes = 1, rounds = 0, lloyd_max = 0;
  // points whose coordinates are loaded together (registers permitting)
  constexpr int UB = load_batch<RMAX>();
  static_assert(PPT % UB == 0, "load batch must divide the points per thread");
  static_assert(PPT * CL_WARPS == 64, "the partition's prefix runs over 64 (u, warp) counts");

  // ------------------------------------------------------------ root node
  if (bid == 0 && tid < MAXACT) a.arrive[tid] = 0u;   // ordered before any use by the root barrier
  if (tid == 0) s.tr_n = 0;
  if (tid == 0) {
    s.nseg = 1;
    s.seg_start[0] = 0;
    s.seg_count[0] = a.N;
    s.seg_on[0] = 1;
  }
  __syncthreads();
  build_chunks(s);
  {
    float hi[RMAX], lo[RMAX];
#pragma unroll
    for (int d = 0; d < RMAX; ++d) hi[d] = lo[d] = 0.0f;
    for_blocks(a, s,
        [&](int, int base, int end, int) {
#pragma unroll
          for (int u0 = 0; u0 < PPT; u0 += UB) {
            float x[UB][RMAX];
#pragma unroll
            for (int b = 0; b < UB; ++b) {
              const int pos = base + (u0 + b) * CL_THREADS + tid;
#pragma unroll
              for (int d = 0; d < RMAX; ++d)
                x[b][d] = (pos < end && d < rho) ? guide_at(a, (size_t)d * N + pos) : 0.0f;
            }
#pragma unroll
            for (int b = 0; b < UB; ++b) {
              const int pos = base + (u0 + b) * CL_THREADS + tid;
              if (pos >= end) continue;
              P[pos] = (uint32_t)pos;
#pragma unroll
              for (int d = 0; d < RMAX; ++d) {
                if (d < rho) {
                  X[(size_t)d * N + pos] = x[b][d];
                  two_sum_acc(hi[d], lo[d], x[b][d]);
                }
              }
            }
          }
        },
        [&](int seg) {
          block_sum_f2<RMAX>(hi, lo, rho, s, pf_root + ((size_t)bid * MAXSEG + seg) * PS);
#pragma unroll
          for (int d = 0; d < RMAX; ++d) hi[d] = lo[d] = 0.0f;
        });
  }
  if (!grid_barrier(a, gen, s, TR_ROOT)) return;
  replay<8>(rho, F2{0.0f, 0.0f}, [&](int) { return contrib_count(a, s, 0); },
      [&](int d, int i) {
        const float* q = pf_root + ((size_t)contrib_block(a, s, 0, i) * MAXSEG) * PS + 2 * d;
        return F2{__ldcg(q), __ldcg(q + 1)};
      },
      [](F2 x, F2 y) { return f2_add(x, y); },
      [&](int d, F2 tf) {
        const double t = f2_to_d(tf);
        const double m = t / (double)a.N;
        c64[d] = m;
        c32[d] = (float)m;
        if (bid == 0) a.node_sum[d] = t;
      });
  __syncthreads();

  auto dist_stats = [&](bool from_scratch) -> bool {
    return dist_stats_fn<RMAX>(a, s, gen, c32, c64, X, Xn, P, Pn, from_scratch);
  };

  if (!dist_stats(false)) return;
  if (bid == 0 && tid == 0) {
    NodeRec r;
    r.start = 0;
    r.count = a.N;
    r.child0 = -1;
    r.far_idx = s.segarg[0];
    r.sse = s.segsse[0];
    a.nodes[0] = r;
  }
  if (!grid_barrier(a, gen, s, TR_NODE)) return;

  // ------------------------------------------------------------ rounds
  while (true) {
    for (int i = tid; i < nnodes; i += CL_THREADS) {
      s.sim_sse[i] = __ldcg(&a.nodes[i].sse);
      s.sim_child0[i] = __ldcg(&a.nodes[i].child0);
    }
    __syncthreads();
    int room = (MAXNODES - nnodes) / 2;
    if (room > MAXACT) room = MAXACT;
    simulate(s, a.K, room);
    __syncthreads();
    if (s.nneeded == 0) break;
    if (room == 0) {                       // node table full: cannot go on
      if (bid == 0 && tid == 0) record_error(a.ctrl, HDF_EUNSUPPORTED);
      return;
    }
    ++rounds;
    // ---- slots, and the point farthest from a (segments = slots)
    if (tid == 0) {
      s.nslots = s.nneeded;
      s.nseg = s.nneeded;
    }
    {   // one thread per slot: its node's loads are independent of the others'
      const int i = tid;
      if (i < s.nneeded) {
        const int nd = s.needed[i];
        SlotRec& sl = s.slot[i];
        sl.node = nd;
        sl.start = __ldcg(&a.nodes[nd].start);
        sl.count = __ldcg(&a.nodes[nd].count);
        sl.a_idx = __ldcg(&a.nodes[nd].far_idx);
        sl.b_idx = -1;
        sl.done = 0;
        sl.iters = 0;
        sl.rev_it = -1;
        sl.cnt_b_cur = 0;
        sl.cnt_b_acc = 0;
        sl.split = 1;
        sl.recompute = 0;
        s.seg_start[i] = sl.start;
        s.seg_count[i] = sl.count;
        s.seg_on[i] = 1;
      }
    }
    __syncthreads();
    build_chunks(s);
    trace_event(a.trace, a.bid, s.tr_n, TR_SETUP);
    for (int v = tid; v < s.nslots * rho; v += CL_THREADS) {
      const int sl = v / rho, d = v % rho;
      const float x = guide_at(a, (size_t)d * N + s.slot[sl].a_idx);
      c32[sl * rho + d] = x;
      c64[sl * rho + d] = (double)x;
      nsum[v] = __ldcg(a.node_sum + (size_t)s.slot[sl].node * rho + d);
    }
    __syncthreads();
    if (!dist_stats(false)) return;
    if (tid == 0) {
      for (int i = 0; i < s.nslots; ++i) {
        SlotRec& sl = s.slot[i];
        sl.b_idx = s.segarg[i];
        if (!(s.segmax[i] > 0.0f) || sl.b_idx < 0 || sl.b_idx >= a.N) {   // all points coincide
          sl.split = 0;
          sl.done = 1;
          sl.b_idx = sl.a_idx;
        }
      }
    }
    __syncthreads();
    // centres a, b of split i at [2i], [2i + 1]
    for (int v = tid; v < s.nslots * 2 * rho; v += CL_THREADS) {
      const int sl = v / (2 * rho), w = (v / rho) % 2, d = v % rho;
      const int idx = w == 0 ? s.slot[sl].a_idx : s.slot[sl].b_idx;
      c64[(2 * sl + w) * rho + d] = (double)guide_at(a, (size_t)d * N + idx);
    }
    __syncthreads();
    for (int v = tid; v < s.nslots * 2 * rho; v += CL_THREADS) c32[v] = (float)c64[v];
    if (tid < s.nslots) s.seg_on[tid] = !s.slot[tid].done;
    __syncthreads();
    for (int i = tid >> 5; i < s.nslots; i += CL_WARPS) {     // |c_a| + |c_b| per split
      double na = 0.0, nb = 0.0;
      for (int d = tid & 31; d < rho; d += 32) {
        na += c64[(2 * i) * rho + d] * c64[(2 * i) * rho + d];
        nb += c64[(2 * i + 1) * rho + d] * c64[(2 * i + 1) * rho + d];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        na += __shfl_xor_sync(0xffffffffu, na, o);
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
      }
      if ((tid & 31) == 0) {
        s.cabs[i] = (float)((sqrt(na) + sqrt(nb)) * (1.0 / 1048576.0));
        s.slack[i] = 0.0f;
        s.cum[i] = 0.0;
      }
    }
    __syncthreads();
    build_chunks(s);   // the chunk table of the whole Lloyd loop: a block keeps its points
    if (tid < s.nslots) s.seg_act[tid] = !s.slot[tid].done;
    __syncthreads();

    // Arrival of this block's partial sums of split sl (written by the block
    // before the barrier): one release-add, nobody waits for it.
    auto arrive = [&](int sl) {
      __syncthreads();
      if (tid == 0) red_release_add(a.arrive + sl, 1u);
    };
    // The finishing block of split sl: one of the blocks with the fewest
    // chunks (chunk j belongs to block j mod G), distinct for distinct splits.
    auto finisher_of = [&](int sl) { return a.G - 1 - sl % a.G; };
    // Wait (bounded) until every contributor of split sl has arrived.
    auto wait_arrivals = [&](int sl) -> bool {
      if (tid == 0) {
        const unsigned need = (unsigned)contrib_count(a, s, sl);
        int ok = 1;
        if (ld_acquire_gpu(a.arrive + sl) < need) {
          const unsigned long long t0 = globaltimer_ns();
          unsigned k = 0;
          while (ld_acquire_gpu(a.arrive + sl) < need) {
            if ((++k & 31u) == 0) {
              if (*(volatile int*)(a.ctrl + CTRL_ERROR) != 0) { ok = 0; break; }
              if (globaltimer_ns() - t0 > a.wait_ns) {
                record_error(a.ctrl, HDF_ETIMEOUT);
                ok = 0;
                break;
              }
            }
          }
        }
        a.arrive[sl] = 0u;   // the next arrivals come after the grid barrier
        s.last = ok;
      }
      __syncthreads();
      return s.last != 0;
    };
    // The nc partial records of split i (record of contributor c at block
    // contrib_block(c)) into dst: 16-byte loads spread over the block, all in
    // flight at once.  Thread 0's acquire of the arrival count and the block
    // barrier after it make the records visible.
    auto stage_records = [&](int i, int it, int nc, float* dst) {
      const float* lpf = a.pf + (1 + (it & 1)) * pf_stride;
      const int Q = PS / 4;   // 16-byte words per record
      // words per thread in flight together: the long records of guides of
      // 16 or more dimensions need several per thread
      constexpr int U = RMAX >= 16 ? 8 : 1;
      for (int v0 = tid; v0 < nc * Q; v0 += U * CL_THREADS) {
        float4 x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int v = v0 + u * CL_THREADS;
          if (v < nc * Q) {
            const int c = v / Q, w = v - c * Q;
            x[u] = __ldcg(reinterpret_cast<const float4*>(
                              lpf + ((size_t)contrib_block(a, s, i, c) * MAXSEG + i) * PS) + w);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int v = v0 + u * CL_THREADS;
          if (v < nc * Q) {
            const int c = v / Q, w = v - c * Q;
            reinterpret_cast<float4*>(dst + (size_t)c * PS)[w] = x[u];
          }
        }
      }
      __syncthreads();
    };
    // Lloyd update of split i from its reduced sums fin = tmp + i (rho + 2),
    // by one warp (lanes over the coordinates): accept, revert or stop, the
    // new FP64 centres and the movement bounds behind the skip test, then
    // the state published to global memory for the other blocks.
    auto update_split = [&](int i, int it, int lane) {
      const double* fin = tmp + i * (rho + 2);
      SlotRec& sl = s.slot[i];
      int recompute = 0;
      if (lane == 0) {
        sl.recompute = 0;
        const int cb = (it == 0 ? 0 : sl.cnt_b_acc) + (int)fin[rho];
        const int changed = (int)fin[rho + 1];
        if (it == 0 && (cb == 0 || cb == sl.count)) {          // degenerate pair: not splittable
          sl.done = 1;
          sl.split = 0;
        } else if (it > 0 && (cb == 0 || cb == sl.count)) {    // a side would be empty:
          sl.done = 1;                                          // keep the previous assignment
          sl.rev_it = it;
          sl.iters = it;
        } else if (it > 0 && changed == 0) {                   // converged
          sl.done = 1;
          sl.iters = it;
        } else {                                                // accept this assignment
          sl.cnt_b_cur = cb;
          sl.iters = it + 1;
          sl.recompute = 1;
          if (it + 1 == MAX_LLOYD) sl.done = 1;
        }
        recompute = sl.recompute;
      }
      __syncwarp();
      recompute = __shfl_sync(0xffffffffu, recompute, 0);
      if (recompute) {
        // accepted sums, the new means (a, b) and the distance each centre moved
        const double nb_cnt = (double)sl.cnt_b_cur, na_cnt = (double)(sl.count - sl.cnt_b_cur);
        // The centres in FP64; the norms behind the skip bounds in FP32 (FP64
        // issues at a small fraction of the FP32 rate).  Rounded up: the
        // FP32 sums of <= 2 rho nonnegative terms and the square roots are
        // within 2^-19 relative, covered by the factor 1 + 2^-16; squares
        // that underflow lose less than 1e-18 in a norm, covered by the
        // absolute 1e-18.  Upper bounds only decide which points are
        // re-examined, never an assignment.
        float ma2 = 0.0f, mb2 = 0.0f, na = 0.0f, nb = 0.0f;
        for (int d = lane; d < rho; d += 32) {
          const double sb = fin[d] + (it > 0 ? acc_sum[i * rho + d] : 0.0);
          acc_sum[i * rho + d] = sb;
          const double mb = quotient(sb, nb_cnt);
          const double ma = quotient(nsum[i * rho + d] - sb, na_cnt);
          const float ua = (float)(ma - c64[(2 * i) * rho + d]);
          const float ub = (float)(mb - c64[(2 * i + 1) * rho + d]);
          const float fa = (float)ma, fb = (float)mb;
          ma2 = fmaf(ua, ua, ma2);
          mb2 = fmaf(ub, ub, mb2);
          na = fmaf(fa, fa, na);
          nb = fmaf(fb, fb, nb);
          c64[(2 * i) * rho + d] = ma;
          c64[(2 * i + 1) * rho + d] = mb;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          ma2 += __shfl_xor_sync(0xffffffffu, ma2, o);
          mb2 += __shfl_xor_sync(0xffffffffu, mb2, o);
          na += __shfl_xor_sync(0xffffffffu, na, o);
          nb += __shfl_xor_sync(0xffffffffu, nb, o);
        }
        if (lane == 0) {
          constexpr float UP32 = 1.0f + 1.0f / 65536.0f;
          s.slack[i] = (sqrtf(ma2) + sqrtf(mb2)) * UP32 + 1e-18f;
          s.cum[i] = (s.cum[i] + (double)s.slack[i]) * ROUND_UP;
          s.cabs[i] = (sqrtf(na) + sqrtf(nb)) * (UP32 / 1048576.0f);
          sl.cnt_b_acc = sl.cnt_b_cur;
        }
      }
      __syncwarp();
      // publish
      for (int v = lane; v < 3 * rho; v += 32) {
        if (v < 2 * rho) a.gcen[(size_t)i * 2 * rho + v] = c64[2 * i * rho + v];
        else a.gacc[(size_t)i * rho + v - 2 * rho] = acc_sum[i * rho + v - 2 * rho];
      }
      if (lane == 0) {
        SlotOut o;
        o.r = sl;
        o.slack = s.slack[i];
        o.cabs = s.cabs[i];
        o.cum = s.cum[i];
        a.sout[i] = o;
      }
    };

    auto finish_split = [&](int i, int it) -> bool {
      const int nc = contrib_count(a, s, i);
      const int V = rho + 2;
      // Fetch the nc records into shared memory, then reduce them in a
      // fixed order: thread (g, v)
      // sums value v of the records c = g, g + NG, ... (ascending), and
      // fin[v] = ((part_0 + part_1) + ...) + part_{NG-1}.
      stage_records(i, it, nc, red);
      const int VS = V <= 32 ? 32 : (V <= 64 ? 64 : 128);   // value slots
      const int NG = CL_THREADS / VS;                        // record classes
      {
        const int v = tid % VS, g = tid / VS;
        F2 t{0.0f, 0.0f};
        if (v < V) {
          for (int c = g; c < nc; c += NG) {
            const float* r = red + (size_t)c * PS;
            t = f2_add(t, v < rho ? F2{r[2 * v], r[2 * v + 1]}
                                  : F2{(float)reinterpret_cast<const int*>(r)[2 * rho + (v - rho)], 0.0f});
          }
        }
        reinterpret_cast<float2*>(parts)[g * VS + v] = make_float2(t.hi, t.lo);
      }
      __syncthreads();
      trace_event(a.trace, a.bid, s.tr_n, TR_FSTAGE);
      double* fin = tmp + i * (rho + 2);
      for (int v = tid; v < V; v += CL_THREADS) {
        F2 t{parts[2 * v], parts[2 * v + 1]};
        for (int g = 1; g < NG; ++g) t = f2_add(t, F2{parts[2 * (g * VS + v)], parts[2 * (g * VS + v) + 1]});
        fin[v] = f2_to_d(t);
      }
      __syncthreads();
      // the update, by warp 0 alone
      if (tid < 32) update_split(i, it, tid);
      __syncthreads();
      return true;
    };

    // ---- Lloyd iterations, all splits of the round together
    for (int it = 0; it < MAX_LLOYD; ++it) {
      const int all_done = __syncthreads_and(tid < s.nslots ? s.slot[tid].done : 1);
      if (all_done) break;
      float* const lpf = a.pf + (1 + (it & 1)) * pf_stride;   // this iteration's records
      {
        // it == 0: full side-b sums; it > 0: change of the side-b sums (points
        // that switched), so that skipped points need no coordinates at all.
        float hi[RMAX], lo[RMAX];
        int cnt = 0, chg = 0;
#pragma unroll
        for (int d = 0; d < RMAX; ++d) hi[d] = lo[d] = 0.0f;
        // The assignment cannot change while the margin bound (stored margin
        // minus the centre movement since it was computed) is positive.
        auto needs_test = [&](int seg, int pos, int end) -> bool {
          const float cum = (float)s.cum[seg];
          const float m0 = (pos < end && it > 0) ? __ldcg(a.marg + pos) : -1.0f;
          return pos < end && !(m0 - cum > 1e-6f * (fabsf(m0) + cum));
        };
        // The full test of one point of split seg with coordinates x: nearer
        // centre (FP64 within 2^-14 of a tie), new margin, side change, sums.
        // Returns the new margin; stores a side change (and its iteration).
        auto test_point = [&](int seg, int pos, const float (&x)[RMAX], int sdp, int& sd_out) -> float {
          const float cum = (float)s.cum[seg];
          const float* ca = c32 + (2 * seg) * rho;
          const float* cb = ca + rho;
          float da = 0.0f, db = 0.0f;
#pragma unroll
          for (int d = 0; d < RMAX; ++d) {
            if (d < rho) {
              const float ta = x[d] - ca[d], tb = x[d] - cb[d];
              da = fmaf(ta, ta, da);
              db = fmaf(tb, tb, db);
            }
          }
          bool sd = db < da;
          if (fabsf(da - db) <= TIE_REL * (da + db)) {
            const double* ea = c64 + (2 * seg) * rho;
            const double* eb = ea + rho;
            double e_a = 0.0, e_b = 0.0;
#pragma unroll
            for (int d = 0; d < RMAX; ++d) {
              if (d < rho) {
                const double xd = (double)x[d];
                e_a = fma(xd - ea[d], xd - ea[d], e_a);
                e_b = fma(xd - eb[d], xd - eb[d], e_b);
              }
            }
            sd = e_b < e_a;
          }
          const float ra = sqrtf(da), rb = sqrtf(db);
          const float marg = fabsf(rb - ra) - MARGIN_REL * (ra + rb) - s.cabs[seg] + cum;
          sd_out = (int)sd;
          if ((int)sd != sdp) {
            a.side[pos] = (uint8_t)sd;
            a.side[N + pos] = (uint8_t)(it + 1);   // iteration of the last change
          }
          if (it == 0) {
            if (sd) {
              ++cnt;
#pragma unroll
              for (int d = 0; d < RMAX; ++d)
                if (d < rho) two_sum_acc(hi[d], lo[d], x[d]);
            }
          } else if ((int)sd != sdp) {
            ++chg;
            cnt += sd ? 1 : -1;
#pragma unroll
            for (int d = 0; d < RMAX; ++d)
              if (d < rho) two_sum_acc(hi[d], lo[d], sd ? x[d] : -x[d]);
          }
          return marg;
        };
        auto flush_split = [&](int seg) {
          if (!s.seg_act[seg]) return;   // converged split: no record, no arrival
          const size_t off = (size_t)bid * MAXSEG + seg;
          if (__syncthreads_or(cnt != 0 || chg != 0)) {
            block_sum_f2<RMAX>(hi, lo, rho, s, lpf + off * PS);
            block_sum_i2(cnt, chg, s, reinterpret_cast<int*>(lpf + off * PS + 2 * rho));
          } else {   // nothing moved to or from side b here: a zero record
            for (int v = tid; v < PS; v += CL_THREADS) lpf[off * PS + v] = 0.0f;
          }
#pragma unroll
          for (int d = 0; d < RMAX; ++d) hi[d] = lo[d] = 0.0f;
          cnt = 0;
          chg = 0;
          arrive(seg);
        };
      const int nmine = bid < s.nchunks ? (s.nchunks - bid + a.G - 1) / a.G : 0;
      bool resident = false;
      if constexpr (resident_bytes<RMAX>() > 0) resident = nmine <= RES_CHUNKS;
      if constexpr (resident_bytes<RMAX>() > 0) if (resident) {
        // Each thread tests its own points.  Their margins and sides live in
        // shared memory (slot c of the block's c-th chunk), so the margin
        // test reads no global memory; the points that fail it are taken in
        // batches of HB from groups of up to 4 chunks of one split, their
        // coordinates loaded together (one round trip per batch).
        constexpr int HB = RMAX <= 4 ? 4 : 2;
        unsigned short* rmarg = (unsigned short*)(dyn + dyn_stage_offset(rho));
        unsigned char* rside = (unsigned char*)(rmarg + (size_t)RES_CHUNKS * CH);
        int cur = -1, sg = 0;
        for (int c = 0; c < nmine;) {
          const int j = bid + c * a.G;
          while (s.seg_chunk0[sg + 1] <= j) ++sg;
          if (sg != cur) {
            if (cur >= 0) flush_split(cur);
            cur = sg;
          }
          int ng = 1;
          while (ng < 4 && c + ng < nmine && s.seg_chunk0[sg + 1] > j + ng * a.G) ++ng;
          if (!s.seg_act[sg]) {   // uniform: shared flag
            c += ng;
            continue;
          }
          const int base0 = s.seg_start[sg] + (j - s.seg_chunk0[sg]) * CH;
          const int end = s.seg_start[sg] + s.seg_count[sg];
          const float cum = (float)s.cum[sg];
          // bit k * PPT + u: point u of chunk c + k fails the margin test
          unsigned hm = 0u;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int u = 0; u < PPT; ++u) {
              const int p = u * CL_THREADS + tid;
              const int pos = base0 + k * a.G * CH + p;
              if (k < ng && pos < end) {
                bool hv = true;
                if (it > 0) {
                  const float m0 = __half2float(__ushort_as_half(rmarg[(size_t)(c + k) * CH + p]));
                  hv = !(m0 - cum > 1e-6f * (fabsf(m0) + cum));
                }
                if (hv) hm |= 1u << (k * PPT + u);
              }
            }
          }
          while (hm) {
            int slot[HB], pos[HB], sdp[HB];
            float x[HB][RMAX];
#pragma unroll
            for (int b = 0; b < HB; ++b) {
              slot[b] = -1;
              if (hm) {
                const int bit = __ffs(hm) - 1;
                hm &= hm - 1u;
                const int k = bit / PPT, u = bit % PPT;
                const int p = u * CL_THREADS + tid;
                slot[b] = (c + k) * CH + p;
                pos[b] = base0 + k * a.G * CH + p;
              }
              sdp[b] = (slot[b] >= 0 && it > 0) ? (int)rside[slot[b]] : -1;
#pragma unroll
              for (int d = 0; d < RMAX; ++d)
                x[b][d] = (slot[b] >= 0 && d < rho) ? xat(X, N, d, pos[b]) : 0.0f;
            }
#pragma unroll
            for (int b = 0; b < HB; ++b) {
              if (slot[b] < 0) continue;
              int sd;
              const float m = test_point(sg, pos[b], x[b], sdp[b], sd);
              rmarg[slot[b]] = __half_as_ushort(__float2half_rd(m));
              rside[slot[b]] = (unsigned char)sd;
            }
          }
          c += ng;
        }
        if (cur >= 0) flush_split(cur);
      }
      if (!resident) {
        // compact each chunk's points that need the full test in position
        // order (coalesced coordinate loads where they are dense) and spread
        // them over the block
        for_blocks(a, s,
            [&](int seg, int base, int end, int) {
              if (!s.seg_act[seg]) return;   // uniform: shared flag
              bool heavy[PPT];
#pragma unroll
              for (int u = 0; u < PPT; ++u) heavy[u] = needs_test(seg, base + u * CL_THREADS + tid, end);
              int hr[PPT];
              const int nheavy = position_ranks(heavy, hr, s);
#pragma unroll
              for (int u = 0; u < PPT; ++u)
                if (heavy[u]) s.hlist[hr[u]] = base + u * CL_THREADS + tid;
              __syncthreads();
              for (int q0 = 0; q0 < nheavy; q0 += UB * CL_THREADS) {
                int hp[UB];
                float x[UB][RMAX];
#pragma unroll
                for (int b = 0; b < UB; ++b) {
                  const int q = q0 + b * CL_THREADS + tid;
                  hp[b] = q < nheavy ? s.hlist[q] : -1;
#pragma unroll
                  for (int d = 0; d < RMAX; ++d)
                    x[b][d] = (hp[b] >= 0 && d < rho) ? xat(X, N, d, hp[b]) : 0.0f;
                }
#pragma unroll
                for (int b = 0; b < UB; ++b)
                  if (hp[b] >= 0) {
                    int sd;
                    a.marg[hp[b]] = test_point(seg, hp[b], x[b],
                                               it > 0 ? (int)__ldcg(a.side + hp[b]) : -1, sd);
                  }
              }
              __syncthreads();   // hlist is reused by the next chunk
            },
            flush_split);
      }
      }
      // finish the splits this block is the finishing block of
      for (int sl = 0; sl < s.nslots; ++sl) {
        if (!s.seg_act[sl] || finisher_of(sl) != bid) continue;
        if (!wait_arrivals(sl)) return;
        trace_event(a.trace, a.bid, s.tr_n, TR_FWAIT);
        if (!finish_split(sl, it)) return;
        trace_event(a.trace, a.bid, s.tr_n, TR_FDONE);
      }
      trace_event(a.trace, a.bid, s.tr_n, TR_LPASS);
      if (!grid_barrier(a, gen, s, TR_LLOYD)) return;
      // every block takes the published state of the splits that were active
      for (int v = tid; v < s.nslots * 3 * rho; v += CL_THREADS) {
        const int i = v / (3 * rho), r = v % (3 * rho);
        if (!s.seg_act[i]) continue;
        if (r < 2 * rho) c64[2 * i * rho + r] = __ldcg(a.gcen + (size_t)i * 2 * rho + r);
        else acc_sum[i * rho + r - 2 * rho] = __ldcg(a.gacc + (size_t)i * rho + r - 2 * rho);
      }
      for (int i = tid; i < s.nslots; i += CL_THREADS) {
        if (!s.seg_act[i]) continue;
        const SlotOut* o = a.sout + i;
        SlotRec& sl = s.slot[i];
        sl.done = __ldcg(&o->r.done);
        sl.iters = __ldcg(&o->r.iters);
        sl.rev_it = __ldcg(&o->r.rev_it);
        sl.cnt_b_cur = __ldcg(&o->r.cnt_b_cur);
        sl.cnt_b_acc = __ldcg(&o->r.cnt_b_acc);
        sl.split = __ldcg(&o->r.split);
        sl.recompute = __ldcg(&o->r.recompute);
        s.slack[i] = __ldcg(&o->slack);
        s.cabs[i] = __ldcg(&o->cabs);
        s.cum[i] = __ldcg(&o->cum);
      }
      __syncthreads();
      for (int v = tid; v < s.nslots * 2 * rho; v += CL_THREADS)
        if (s.seg_act[v / (2 * rho)]) c32[v] = (float)c64[v];
      __syncthreads();
      if (tid < s.nslots) s.seg_act[tid] = !s.slot[tid].done;
      __syncthreads();
      trace_event(a.trace, a.bid, s.tr_n, TR_LUPDATE);
    }
    if (tid == 0) {
      for (int i = 0; i < s.nslots; ++i) {
        if (s.slot[i].iters > lloyd_max) lloyd_max = s.slot[i].iters;
        s.seg_on[i] = s.slot[i].split;
      }
    }
    __syncthreads();
    build_chunks(s);

    // ---- stable partition of every split segment: side-a points first.
    // A chunk's positions are base + u * CL_THREADS + tid (u < PPT), so the
    // loads are coalesced; a point's rank among the chunk's side-b points is
    // the prefix over (u, warp) of the warps' ballot counts plus its rank in
    // its warp's ballot.
    auto chunk_geom = [&](int j, int& seg, int& base, int& end) {
      while (s.seg_chunk0[seg + 1] <= j) ++seg;
      base = s.seg_start[seg] + (j - s.seg_chunk0[seg]) * CH;
      end = s.seg_start[seg] + s.seg_count[seg];
    };
    // exclusive block scan of v (one value per thread); also returns the total
    auto block_scan = [&](int v, int& total) -> int {
      const int lane = tid & 31, warp = tid >> 5;
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s.scanw[warp] = x;
      __syncthreads();
      int before = 0;
      total = 0;
#pragma unroll
      for (int w = 0; w < CL_WARPS; ++w) {
        if (w < warp) before += s.scanw[w];
        total += s.scanw[w];
      }
      __syncthreads();
      return before + x - v;
    };
    {
      // side-b counts of the block's chunks, 4 chunks per round of loads;
      // warp sums added up in shared memory (integer: order-free)
      if (tid < 4) s.ccnt[tid] = 0;
      __syncthreads();
      int seg = 0;
      for (int j0 = bid; j0 < s.nchunks; j0 += 4 * a.G) {
        int c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int j = j0 + k * a.G;
          c[k] = 0;
          if (j < s.nchunks) {
            int base, end;
            chunk_geom(j, seg, base, end);
            const int rv = s.slot[seg].rev_it + 1;   // 0: nothing undone
#pragma unroll
            for (int u = 0; u < PPT; ++u) {
              const int pos = base + u * CL_THREADS + tid;
              if (pos < end) c[k] += accepted_side(a, pos, rv);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int w = __reduce_add_sync(0xffffffffu, c[k]);
          if ((tid & 31) == 0 && w != 0) atomicAdd(&s.ccnt[k], w);
        }
        __syncthreads();
        if (tid < 4) {
          const int j = j0 + tid * a.G;
          if (j < s.nchunks) a.chunk_cnt[j] = s.ccnt[tid];
          s.ccnt[tid] = 0;
        }
        __syncthreads();
      }
    }
    if (!grid_barrier(a, gen, s, TR_COUNT)) return;
    {
      // Side-b points before each of the block's chunks within its segment,
      // from one block scan of the whole count table: P[q] = sum of the
      // counts of the chunks before q; the segment's share is
      // P[j] - P[first chunk of the segment].  Blocks with more than
      // MAXMINE chunks add the counts up chunk by chunk instead.
      constexpr int MAXMINE = 64;
      const int nmine = bid < s.nchunks ? (s.nchunks - bid + a.G - 1) / a.G : 0;
      const bool tab = nmine <= MAXMINE;
      if (tab) {
        const int R = (s.nchunks + CL_THREADS - 1) / CL_THREADS;
        const int q0 = tid * R < s.nchunks ? tid * R : s.nchunks;
        const int q1 = q0 + R < s.nchunks ? q0 + R : s.nchunks;
        int loc = 0;
        for (int q = q0; q < q1; ++q) loc += __ldcg(a.chunk_cnt + q);
        int total;
        int pq = block_scan(loc, total);
        for (int sg = 0; sg < s.nseg; ++sg) {
          const int q = s.seg_chunk0[sg];
          if (q == s.nchunks && tid == 0) s.segpre[sg] = total;
        }
        for (int q = q0; q < q1; ++q) {
          if (q >= bid && (q - bid) % a.G == 0) s.mypre[(q - bid) / a.G] = pq;
          for (int sg = 0; sg < s.nseg; ++sg)
            if (s.seg_chunk0[sg] == q) s.segpre[sg] = pq;
          pq += __ldcg(a.chunk_cnt + q);
        }
        __syncthreads();
      }
      int seg = 0;
      for (int j = bid; j < s.nchunks; j += a.G) {
        int base, end;
        chunk_geom(j, seg, base, end);
        const SlotRec& sl = s.slot[seg];
        const int rv = sl.rev_it + 1;
        int before_b_chunk;
        if (tab) {
          before_b_chunk = s.mypre[(j - bid) / a.G] - s.segpre[seg];
        } else {
          // side-b points in the earlier chunks of this segment
          int pb = 0;
          for (int q = s.seg_chunk0[seg] + tid; q < j; q += CL_THREADS) pb += __ldcg(a.chunk_cnt + q);
          block_scan(pb, before_b_chunk);
        }
        bool sdv[PPT];
        int rk[PPT];
        // guides of up to 8 dimensions: the coordinates and raster indices are
        // loaded together with the sides, before the ranks
        constexpr bool EARLY = RMAX <= 8;
        float xe[EARLY ? PPT : 1][RMAX];
        uint32_t pe[EARLY ? PPT : 1];
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
          const int pos = base + u * CL_THREADS + tid;
          sdv[u] = (pos < end) && accepted_side(a, pos, rv) != 0;
          if constexpr (EARLY) {
            pe[u] = pos < end ? __ldcg(P + pos) : 0u;
#pragma unroll
            for (int d = 0; d < RMAX; ++d) xe[u][d] = (pos < end && d < rho) ? xat(X, N, d, pos) : 0.0f;
          }
        }
        position_ranks(sdv, rk, s);
        const int cnt_a = sl.count - sl.cnt_b_acc;
        int np[PPT];
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
          const int pos = base + u * CL_THREADS + tid;
          np[u] = -1;
          if (pos >= end) continue;
          const int rank_b = before_b_chunk + rk[u];   // side-b points before pos (valid for either side)
          if (sdv[u]) np[u] = sl.start + cnt_a + rank_b;
          else np[u] = sl.start + (pos - sl.start - rank_b);   // side-a points before = offset - side-b before
          if (np[u] < sl.start || np[u] >= sl.start + sl.count) {
            record_error(a.ctrl, HDF_EDOMAIN);   // inconsistent counts: never write outside
            np[u] = -1;
          }
        }
        if constexpr (EARLY) {
#pragma unroll
          for (int u = 0; u < PPT; ++u) {
            const int q = np[u];
            if (q < 0) continue;
            Pn[q] = pe[u];
#pragma unroll
            for (int d = 0; d < RMAX; ++d)
              if (d < rho) Xn[(size_t)d * N + q] = xe[u][d];
          }
        } else {
#pragma unroll
          for (int u0 = 0; u0 < PPT; u0 += UB) {
            float x[UB][RMAX];
            uint32_t pid[UB];
#pragma unroll
            for (int b = 0; b < UB; ++b) {
              const int pos = base + (u0 + b) * CL_THREADS + tid;
              const bool v = np[u0 + b] >= 0;
              pid[b] = v ? __ldcg(P + pos) : 0u;
#pragma unroll
              for (int d = 0; d < RMAX; ++d) x[b][d] = (v && d < rho) ? xat(X, N, d, pos) : 0.0f;
            }
#pragma unroll
            for (int b = 0; b < UB; ++b) {
              const int q = np[u0 + b];
              if (q < 0) continue;
              Pn[q] = pid[b];
#pragma unroll
              for (int d = 0; d < RMAX; ++d)
                if (d < rho) Xn[(size_t)d * N + q] = x[b][d];
            }
          }
        }
      }
    }
    if (!grid_barrier(a, gen, s, TR_SCATTER)) return;

    // ---- children: segments, sums, SSE and farthest points
    const int first = nnodes;
    if (tid == 0) {
      s.nseg = 2 * s.nslots;
      for (int i = 0; i < s.nslots; ++i) {
        const SlotRec& sl = s.slot[i];
        const int ca = sl.count - sl.cnt_b_acc;
        s.seg_start[2 * i] = sl.start;
        s.seg_count[2 * i] = ca;
        s.seg_start[2 * i + 1] = sl.start + ca;
        s.seg_count[2 * i + 1] = sl.cnt_b_acc;
        s.seg_on[2 * i] = sl.split;
        s.seg_on[2 * i + 1] = sl.split;
      }
    }
    __syncthreads();
    // the centres of the accepted assignment are the children's means
    for (int v = tid; v < s.nslots * rho; v += CL_THREADS) {
      const int i = v / rho, d = v % rho;
      const SlotRec& sl = s.slot[i];
      if (!sl.split || bid != 0) continue;
      const double tot = nsum[i * rho + d];
      const double sb = acc_sum[i * rho + d];
      a.node_sum[(size_t)(first + 2 * i) * rho + d] = tot - sb;
      a.node_sum[(size_t)(first + 2 * i + 1) * rho + d] = sb;
    }
    __syncthreads();
    build_chunks(s);
    if (!dist_stats(true)) return;
    if (bid == 0 && tid == 0) {
      for (int i = 0; i < s.nslots; ++i) {
        const SlotRec& sl = s.slot[i];
        if (!sl.split) {
          a.nodes[sl.node].sse = 0.0;   // not splittable: never chosen again
          continue;
        }
        for (int w = 0; w < 2; ++w) {
          NodeRec r;
          r.start = s.seg_start[2 * i + w];
          r.count = s.seg_count[2 * i + w];
          r.child0 = -1;
          r.far_idx = s.segarg[2 * i + w];
          r.sse = s.segsse[2 * i + w];
          a.nodes[first + 2 * i + w] = r;
        }
        a.nodes[sl.node].child0 = first + 2 * i;
      }
    }
    nnodes += 2 * s.nslots;
    if (!grid_barrier(a, gen, s, TR_CHILD)) return;
  }

  // ------------------------------------------------------------ outputs
  // Leaves of the final replay are the clusters; s.leaf_cl holds the index.
  if (tid == 0) s.nseg = s.nleaves;
  for (int i = tid; i < s.nleaves; i += CL_THREADS) {
    const int nd = s.leaf_node[i];
    s.seg_start[i] = __ldcg(&a.nodes[nd].start);
    s.seg_count[i] = __ldcg(&a.nodes[nd].count);
    s.seg_on[i] = 1;
  }
  __syncthreads();
  if (bid == 0) {
    for (int v = tid; v < s.nleaves * rho; v += CL_THREADS) {
      const int i = v / rho, d = v % rho;
      const double m = __ldcg(a.node_sum + (size_t)s.leaf_node[i] * rho + d) / (double)s.seg_count[i];
      a.mu64[s.leaf_cl[i] * rho + d] = m;
      a.mu[s.leaf_cl[i] * rho + d] = (float)m;
    }
    for (int i = tid; i < s.nleaves; i += CL_THREADS)   // SSE of the leaves by cluster index
      s.sim_sse[s.leaf_cl[i]] = __ldcg(&a.nodes[s.leaf_node[i]].sse);
    __syncthreads();
    if (tid == 0) {
      double ek = 0.0;
      for (int c = 0; c < s.nleaves; ++c) ek += s.sim_sse[c];
      *a.ek = ek;
      a.ctrl[CTRL_K_EFF] = s.nclusters;
      a.ctrl[CTRL_LLOYD_MAX] = lloyd_max;
      a.ctrl[CTRL_ROUNDS] = rounds;
    }
  }
  // labels: one segment per cluster (MAXSEG >= HDF_MAX_K)
  build_chunks(s);
  for_blocks(a, s,
      [&](int seg, int base, int end, int) {
        uint32_t idx[PPT];
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
          const int pos = base + u * CL_THREADS + tid;
          idx[u] = (pos < end) ? __ldcg(P + pos) : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < PPT; ++u)
          if (idx[u] < (uint32_t)a.N) a.labels[idx[u]] = s.leaf_cl[seg];
      },
      [&](int) {});
}


// One cooperative launch clusters a table of guides.  The grid is split into
// groups of consecutive blocks, groups[g] = (first block, block count, first
// and one-past-last entry of `order`); the group clusters the guides
// order[z..w) one after the other, each with its own control words (grid
// barrier counters) and workspace, so groups never wait on one another.
// p_override (if not null) replaces the guide pointer of every entry.
template <int RMAX>
__global__ void __launch_bounds__(CL_THREADS, 1)
cluster_kernel(const ClArgs* __restrict__ table, const int4* __restrict__ groups, int ngroups,
               const int* __restrict__ order, const void* p_override,
               unsigned long long wait_ns) {
  __shared__ ClShared s;
  __shared__ ClArgs sa;
  __shared__ int4 s_grp;
  extern __shared__ __align__(128) unsigned char dyn[];
  if (threadIdx.x == 0) {
    s_grp = make_int4(0, 0, 0, 0);
    for (int g = 0; g < ngroups; ++g) {
      const int4 gr = groups[g];
      if ((int)blockIdx.x >= gr.x && (int)blockIdx.x < gr.x + gr.y) s_grp = gr;
    }
  }
  __syncthreads();
  const int4 gr = s_grp;
  for (int t = gr.z; t < gr.w; ++t) {
    if (threadIdx.x == 0) {
      sa = table[order[t]];
      sa.bid = (int)blockIdx.x - gr.x;
      sa.wait_ns = wait_ns;
      if (p_override) sa.p = p_override;
    }
    __syncthreads();
    cluster_run<RMAX>(sa, s, dyn);
    __syncthreads();
  }
}

// Host: cooperative launch of one instantiation over `grid` blocks.
template <int RMAX>
cudaError_t launch_cl(const ClArgs* table, const int4* groups, int ngroups, const int* order,
                      const void* p_override, int rho_max, int grid, unsigned long long wait_ns,
                      cudaStream_t st) {
  const size_t smem = dyn_stage_offset(rho_max) + resident_bytes<RMAX>();
  cudaError_t e = cudaFuncSetAttribute(cluster_kernel<RMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cluster_kernel<RMAX>, CL_THREADS,
                                                    smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(CL_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cluster_kernel<RMAX>, table, groups, ngroups, order, p_override,
                            wait_ns);
}

}  // namespace
}  // namespace clus
}  // namespace hdf
