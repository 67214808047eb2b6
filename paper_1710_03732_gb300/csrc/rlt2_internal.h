// Internal interfaces shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "rlt2.h"

namespace rlt2 {

// Bounds-checked build (-DRLT2_BOUNDS_CHECK, `build.build(checked=True)`): the
// indices the kernels compute pass through RLT2_IDX(i, n), which counts an
// index outside [0, n) in a per-file device counter and uses 0 instead, so a
// bad index is reported (rlt2_debug_bounds_violations) and never dereferenced.
// In the normal build RLT2_IDX(i, n) is i.
#ifdef RLT2_BOUNDS_CHECK
static __device__ unsigned long long g_oob_count;
template <typename I, typename N>
__device__ __forceinline__ I checked_index(I i, N n) {
  if ((unsigned long long)(long long)i < (unsigned long long)(long long)n) return i;
  atomicAdd(&g_oob_count, 1ull);
  return I(0);
}
#define RLT2_IDX(i, n) ::rlt2::checked_index((i), (n))
#else
#define RLT2_IDX(i, n) (i)
#endif
// Host: this file's counter (defined once per translation unit by
// RLT2_DEFINE_OOB_QUERY; 0 in the normal build, ~0 if it cannot be read).
#ifdef RLT2_BOUNDS_CHECK
#define RLT2_DEFINE_OOB_QUERY(name)                                                  \
  unsigned long long name() {                                                        \
    unsigned long long v = 0;                                                        \
    return cudaMemcpyFromSymbol(&v, g_oob_count, sizeof v) == cudaSuccess ? v : ~0ull; \
  }
#else
#define RLT2_DEFINE_OOB_QUERY(name) \
  unsigned long long name() { return 0; }
#endif
unsigned long long oob_lap();
unsigned long long oob_ascent();
unsigned long long oob_nodes();
unsigned long long oob_fused();

struct MoveZArgs;
struct DevScalars;

// One launch solves `batch` LAPs of size m; LAP b has cost A[b*m*m..] (+ Badd[b*m*m..]).
struct LapArgs {
  long long batch;
  int m;
  const double* A;
  const double* Badd;        // nullable: cost = A + Badd (the Z->Y and Y->X folds)
  const double* u0;          // nullable: starting row duals (batch*m)
  const int* warm_gate;      // nullable: if set and *warm_gate == 0 the start is cold
  double* value;             // batch
  double* u;                 // nullable, batch*m
  double* v;                 // nullable, batch*m
  int* r2c;                  // nullable, batch*m
  int* naug;                 // nullable, batch
  double* pi;                // nullable, batch*m*m reduced costs ((cost - u_r) - v_c)
  int dual_mode;             // 0 raw (FP64), 1 canonical (fixed point), 2 canonical (FP64)
  unsigned long long* stats; // nullable, [0] += augmentations, [1] += relaxations
  const int* skip;           // nullable: kernel does nothing when *skip != 0
  int group;                 // lanes per LAP (8, 16 or 32); 0 = smallest that fits m
  int warps_per_block;       // 4 or 8; 0 = 8
  const int* map;            // nullable: LAP b works on slot map[b] of every array (a subset of tiles)
  int prefetch;              // set by launch_lap: the fixed-point form without Badd and pi stages
                             // the next tile by cp.async while it solves the current one
  unsigned long long* head;  // nullable: device counter of the prefetching form's LAP queue
                             // (launch_lap zeroes it on the stream before the launch)
  int head_zeroed;           // an earlier launch on the stream has zeroed *head: no memset
};

// The LAPs of one stage of one branch-and-bound node.
struct NodeLapItem {
  long long count;     // LAPs of this node in this stage
  int m;               // their size
  const double* A;     // cost tiles (+ Badd if set)
  const double* Badd;
  const double* u0;    // warm-start row duals or nullptr
  const int* warm_gate;
  const int* skip;     // the node's done flag
  double* value;
  double* u;
  double* v;
  int* r2c;
  double* pi;
};

constexpr int kMaxWaveNodes = 1024;

// One stage of all nodes of a wave as one persistent launch: warps take LAPs
// from a device queue (head must be zero at launch), nodes looked up by prefix.
struct NodeLapArgs {
  int nnodes;
  const NodeLapItem* items;  // device [nnodes]
  const long long* prefix;   // device [nnodes + 1]
  long long total;
  int max_m;
  int dual_mode;
  unsigned long long* head;
  unsigned long long* stats;  // device [2]: augmentations, relaxations (nullable)
  int group, warps_per_block;
  bool pre;  // no node of the stage writes reduced costs (the tile may be reduced in place);
             // such stages (the Z stages) have no Badd either
  int prefetch;  // set by launch_lap_nodes: fixed-point pre stages copy each warp's next
                 // queue item into shared memory by cp.async while the current one is solved
  int cold;      // no item has start duals: fixed-point LAPs reduce their rows first
};
cudaError_t launch_lap_nodes(const NodeLapArgs& a, cudaStream_t s);

// The z move of one ascent step and the Z-stage LAPs that follow it as one
// persistent launch (fused.cu): a few warps of every block run the move's
// (triple, p) blocks while the others solve the Z-LAPs, tiles grouped by
// facility pair in the order the move finishes the pairs.  A tile's LAP waits
// until every move block whose facility triple holds the tile's two
// facilities is done (its pair counter reaches (n-2) n), so the FP64 move and
// the integer LAPs overlap on the SMs while each LAP sees exactly the costs and
// start duals of the two-kernel sequence.
struct PipePlan {
  int n = 0;
  const int* order = nullptr;  // device, T tiles in pair-completion order
  long long nmove = 0;         // move blocks: triples * n
  int grid = 0;                // blocks (resident on every SM), 8 warps each
};
// The plan for residual size n on the current device: kernel attributes,
// occupancy and tile order, built once per (device, n) and kept for the life
// of the process.  Call outside stream capture.
const PipePlan* prepare_pipe(int n, cudaError_t* err);
struct PipeArgs {
  const int* order;
  long long nmove;
  unsigned long long* ctr;   // [0] move head, [1] warps done, [2] LAP head, [4 + a*n + b] blocks done for pair a < b
  DevScalars* sc;            // stop flags (a wait that gives up sets done, reason 4)
  int spin_limit;            // polls of a pair counter before a LAP warp gives up
  unsigned long long extra;  // added to the pair target: 0, or 1 in the failure-detection check
};
// check: the failure-detection form (rlt2_pipeline_check_wait_timeout): the
// pair targets are raised by one, so no wait can be satisfied, and the polls
// are capped low so that the first wait gives up within a few milliseconds.
cudaError_t launch_move_lap_z(const MoveZArgs& mz, const LapArgs& z, const PipePlan& plan, unsigned long long* ctr,
                              DevScalars* sc, cudaStream_t s, bool check = false);

// Lanes per LAP the launcher would pick for size m (8, 16 or 32).
int default_group(int m);

// Configure the LAP kernel for size m (shared-memory limit, occupancy); call
// outside stream capture before the first launch of that size.
cudaError_t prepare_lap(int m, int group = 0, int warps_per_block = 0);

// Enqueue the batched LAP kernel (grid sized for the device); returns the CUDA error.
cudaError_t launch_lap(const LapArgs& a, cudaStream_t s);

constexpr int kRing = 1 << 16;  // bound-history ring (entries)

// Device-resident scalars of one dual ascent.
constexpr int kStallRing = 64;  // best-bound history for the stall rule
struct DevScalars {
  double lb, best_lb, ub, gap;
  double lb_base;  // F variant: the bound the next X-LAP value is added to
  int iter, done, have_snap, reason;
  int sa_on;       // the pending ascent step applies a Type 4 draw
  unsigned long long stats[6];  // Z aug, Z relax, Y aug, Y relax, X aug, X relax
  unsigned long long lap_head;  // queue counter of the Z-stage LAP launch
  double best_hist[kStallRing];  // best bound after iteration it, at it % kStallRing
};

// Every device buffer one dual ascent works on (layouts as in rlt2.h).
struct IterView {
  rlt2_mlp* mlp;   // learned warm start (warm == 2)
  double* u0buf;   // its predictions, T*m
  int n, m;
  long long T, E;
  int ntrip;
  rlt2_params prm;
  double *d_cst, *Fr, *Dr, *bprime, *Chat, *Dhat, *Theta, *xi, *psi, *Delta, *gamma, *delta;
  double *alpha, *beta, *pix, *piy, *tterm, *xval, *ring;
  double* xcost;   // X-LAP costs: b' (S variant, may alias bprime) or the incremental x costs (F)
  double* saterm;  // n*n Type 4 amount per (first facility, first location) of the pending step
  const double *sa_kf, *sa_kl, *sa_K, *sa_thr;  // Type 4 draws (count*n, count*n, count, count)
  int sa_count;
  const int* zmap;  // half-Z scheme: the tiles with first facility < second facility
  long long Tz;     // number of Z-LAPs solved (T, or T/2 with the half scheme)
  const PipePlan* pplan;   // nullable: pipelined z move + Z-LAPs (see PipePlan)
  unsigned long long* pipe;  // their queues and pair counters (4 + n*n)
  int pipe_check;            // 1: the pipelined launch in its failure-detection form
  const double* bqap;     // nullable: QAP linear costs for upper bounds (default bprime)
  const double* cst_qap;  // nullable: QAP constant for upper bounds (default d_cst)
  int *xperm, *ubperm, *trips;
  DevScalars* sc;
};

// Up to `iters` iterations of several ascents (one view each, nn <= 1024) in
// lockstep, every stage one launch over all of them (the batched node kernels
// of rlt2_bound_nodes); stops early once every view's ascent has stopped
// (checked between chunks of 8, 16, ... iterations).  *ran: iterations
// enqueued.  Synchronises s.  Not for the half-Z scheme, the learned start or
// Type 4 draws; the views' augmentation counters are not updated.
cudaError_t iterate_views(const IterView* views, int nn, const rlt2_params& prm, int iters, cudaStream_t s,
                          int* ran);

// Step A0 (setup kernels) and one iteration (seven to nine kernels) on a view.
cudaError_t enqueue_setup(const IterView& v, int n_full, const double* dF, const double* dD, const double* dB,
                          const int* dfac, const int* dloc, const int* dfixf, const int* dfixl, int nfix,
                          cudaStream_t s);
// launched (nullable, kKinds entries): incremented by the kernels launched per timing kind.
cudaError_t enqueue_iteration(const IterView& v, cudaStream_t s, cudaEvent_t* ev, int* launched = nullptr);

// Predicted Z-LAP row duals for ntiles tiles of size mz (mlp.cu).
cudaError_t mlp_predict_enqueue(rlt2_mlp* m, long long ntiles, int mz, const double* tiles, const double* prev_u,
                                double* u0, cudaStream_t s, int* launched = nullptr);

// Parameter validation shared by the entry points.
bool params_valid(const rlt2_params& p);

// Thread-local last error text.
void set_error(const std::string& msg);
rlt2_status cuda_fail(cudaError_t e, const char* what);

}  // namespace rlt2
