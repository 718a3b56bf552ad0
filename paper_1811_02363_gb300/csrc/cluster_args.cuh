// Constants and records shared by the clustering kernel (cluster_kernel.cuh)
// and the host code that lays out its workspace for one guide or a batch.
#pragma once

#include "hdf_internal.cuh"

namespace hdf {
namespace clus {

constexpr int CH = 2048;                // points per chunk (the workspace layout depends on it)
constexpr int MAXACT = 32;              // splits per round
constexpr int MAXSEG = 2 * MAXACT;
constexpr int MAXNODES = 16 * HDF_MAX_K;
constexpr int MAX_LLOYD = 20;
constexpr int MAXG = 160;               // blocks of one group (one per SM)
// Partial-record regions of a guide's workspace (each G x MAXSEG records):
// 0 the distance passes, 1 and 2 the Lloyd passes of even and odd
// iterations (region 2 also the root sums).  A region is rewritten only
// after a grid barrier that every reader of its previous contents has passed.
constexpr int PF_REGIONS = 3;
constexpr unsigned long long DEFAULT_WAIT_NS = kDefaultWaitNs;
constexpr float TIE_REL = 1.0f / 16384.0f;      // 2^-14: Lloyd recheck band
constexpr float CAND_REL = 1.0f / 4096.0f;      // 2^-12: farthest-point candidates
constexpr int TRACE_CAP = 2048;                  // trace events per launch
constexpr float MARGIN_REL = 1.0f / 4096.0f;    // 2^-12: rounding allowance of a stored margin
constexpr double ROUND_UP = 1.0 + 1.0 / 1048576.0;

// Phases recorded in the trace (one event per grid barrier passed by block 0).
// Events 9 and up are recorded by block 0 between barriers (its own progress).
enum TracePhase { TR_ROOT = 1, TR_DIST1 = 2, TR_NODE = 4, TR_LLOYD = 5, TR_COUNT = 6,
                  TR_SCATTER = 7, TR_CHILD = 8, TR_LPASS = 9, TR_LUPDATE = 11,
                  TR_FWAIT = 12, TR_FSTAGE = 13, TR_FDONE = 14, TR_SETUP = 15, TR_DPASS = 16 };

struct NodeRec {
  int start, count;   // segment of the permutation
  int child0;         // first child (-1: not split); child 2 = child0 + 1
  int far_idx;        // raster index of the point farthest from the mean
  double sse;         // sum of squared deviations (0: never split)
};

struct SlotRec {      // a split in flight (block-local copy, identical in every block)
  int node, start, count;
  int a_idx, b_idx;
  int done, iters, rev_it;   // rev_it: iteration whose changes were undone (-1: none)
  int cnt_b_cur, cnt_b_acc;
  int split;          // produces children
  int recompute;      // centres to be recomputed from the assignment just made
};

struct SlotOut {      // a split after a Lloyd update, published by its finishing block
  SlotRec r;
  float slack, cabs;  // centre movement of the update; rounding allowance of the centres
  double cum;         // total centre movement since the split started
};

struct ClArgs {
  const void* p;
  int p_bf16;         // guide stored as bfloat16
  int N, rho, K, G;   // G: blocks of the group that clusters this guide
  int bid;            // this block's rank in the group (set per block on the device)
  unsigned long long wait_ns;   // limit of each device-side wait (set per launch)
  int* ctrl;
  float* mu;          // out: K x rho
  double* mu64;       // out: K x rho
  int32_t* labels;    // out: N
  double* ek;         // out: E_K
  uint32_t* perm;     // N
  uint32_t* perm2;    // N
  float* X;           // rho x N points in permutation order
  float* X2;          // rho x N scatter target
  uint8_t* side;      // 2 x N
  float* marg;        // N margin bound + total centre movement when it was computed
  float* d32;         // N
  NodeRec* nodes;     // MAXNODES
  double* node_sum;   // MAXNODES x rho coordinate sums
  float* pf;          // G x MAXSEG records of record_floats(rho) floats
  int* pi;            // G x MAXSEG x 2
  float* pd;          // G x MAXSEG
  double* pdd;        // G x MAXSEG
  int* px;            // G x MAXSEG
  int* chunk_cnt;     // max chunks
  long long* trace;   // [0] = count, then (phase, ns) pairs, block 0 only
  unsigned* arrive;   // MAXACT arrival counters of the Lloyd partial sums (0 between passes)
  SlotOut* sout;      // MAXACT splits after the last Lloyd update
  double* gcen;       // MAXACT x 2 x rho centres after the last Lloyd update
  double* gacc;       // MAXACT x rho accepted side-b coordinate sums
};

// Floats per partial record of a block: rho double-float pairs and one more
// pair, padded to 16 bytes (records are fetched in 16-byte words).
__host__ __device__ constexpr int record_floats(int rho) { return ((2 * (rho + 1) + 3) / 4) * 4; }

// Host helpers (k_cluster.cu).
int grid_blocks(int dev);
size_t ws_bytes(int N, int rho, int G);   // workspace of one guide clustered by G blocks
ClArgs make_args(void* ws, int N, int rho, int K, int G, int* ctrl, float* mu, double* mu64,
                 int32_t* labels, double* ek, const void* p, int p_bf16);
cudaError_t launch_table(int rho_max, const ClArgs* table, const int4* groups, int ngroups,
                         const int* order, const void* p_override, int grid,
                         unsigned long long wait_ns, cudaStream_t st);

}  // namespace clus
}  // namespace hdf
