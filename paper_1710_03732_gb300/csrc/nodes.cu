// Batched bounding of branch-and-bound nodes (rlt2_bound_nodes).
//
// Nodes of a QAP branch-and-bound tree (Section 4: level l fixes l facilities)
// have uneven residual sizes.  Instead of one context per node, the nodes are
// admitted into waves that fit a device-memory budget, each node gets its own
// arena (D^, C^, duals, scalars) carved from one pool, and every stage of an
// iteration runs as one launch over all nodes of the wave:
//   k_move_y_nodes / k_move_z_nodes  grid.y = node
//   k_lap_nodes (Z, Y, X)            persistent warps pulling LAPs of all nodes
//                                    from a device queue (lap.cu)
//   k_finalize_nodes                 one block per node
// The per-iteration sequence is captured once into a CUDA graph and replayed.
// The Z stages' items are sorted by LAP size; each size has its own launch
// shape (lanes per LAP, warps per block), picked by an autotuner that times the
// candidates on live iterations, one launch per size (every candidate gives
// bit-identical results, so tuning costs no accuracy), and kept in a
// process-wide table keyed by the Z-LAP size (rlt2_node_tuning reports it).
// After tuning, adjacent sizes with the same shape share one launch.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rlt2_ascent.cuh"
#include "rlt2_internal.h"

namespace rlt2 {
namespace {

// blockDim.x a multiple of 32 (the folded form's warps move 32 tiles together)
__global__ void k_move_y_nodes(const MoveYArgs* nodes) {
  const MoveYArgs a = nodes[blockIdx.y];
  if (!a.sc->have_snap || a.sc->done) return;
  const long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  if (a.shift_psi) move_y_shift_range(a, start, stride);
  else move_y_range(a, start, stride);
}

__global__ void __launch_bounds__(352, 3) k_move_z_nodes(const MoveZArgs* nodes, const int* nblocks) {
  if ((int)blockIdx.x >= nblocks[blockIdx.y]) return;
  const MoveZArgs a = nodes[blockIdx.y];
  if (!a.sc->have_snap || a.sc->done) return;
  move_z_block(a, blockIdx.x, threadIdx.x, blockDim.x);
}

__global__ void __launch_bounds__(512) k_phase2_nodes(const Phase2Args* nodes, const int* nblocks) {
  if ((int)blockIdx.x >= nblocks[blockIdx.y]) return;
  const Phase2Args a = nodes[blockIdx.y];
  if (a.sc->done) return;
  phase2_block(a, blockIdx.x);
}

__global__ void __launch_bounds__(256) k_finalize_nodes(const FinArgs* nodes) {
  const FinArgs a = nodes[blockIdx.x];
  if (a.sc->done) return;
  finalize_block(a);
}

// Sub-arrays of one node's arena, 256-byte aligned.  With base == nullptr it
// only counts bytes, so sizing and carving cannot disagree.
struct Arena {
  char* base;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += (count * sizeof(T) + 255) & ~size_t(255);
    return p;
  }
};

struct NodeHost {
  int nr = 0;
  std::vector<int> fac, loc, fixf, fixl;
  IterView v{};
  int* dfac = nullptr;  // fac | loc | fixf | fixl | trips on the device
  size_t bytes = 0;
};

void carve(NodeHost& h, char* base, const rlt2_params& prm) {
  Arena ar{base};
  IterView& v = h.v;
  const int n = h.nr;
  v.n = n;
  v.m = n - 2;
  v.T = (long long)n * n * (n - 1) * (n - 1);
  v.E = v.T * v.m * v.m;
  v.ntrip = n * (n - 1) * (n - 2) / 6;
  v.prm = prm;
  const size_t T = v.T, m = v.m, n2 = (size_t)n * n;
  v.Dhat = ar.take<double>(v.E);
  v.xi = ar.take<double>(T * m);
  v.psi = ar.take<double>(T * m);
  v.Chat = ar.take<double>(T);
  v.Theta = ar.take<double>(T);
  v.piy = ar.take<double>(T);
  v.tterm = ar.take<double>(T);
  v.d_cst = ar.take<double>(1);
  v.Fr = ar.take<double>(n2);
  v.Dr = ar.take<double>(n2);
  v.bprime = ar.take<double>(n2);
  v.xcost = ar.take<double>(n2);
  v.Delta = ar.take<double>(n2);
  v.pix = ar.take<double>(n2);
  v.gamma = ar.take<double>(n2 * (n - 1));
  v.delta = ar.take<double>(n2 * (n - 1));
  v.alpha = ar.take<double>(n);
  v.beta = ar.take<double>(n);
  v.xval = ar.take<double>(1);
  v.ring = ar.take<double>(kRing);
  v.sc = ar.take<DevScalars>(1);
  v.xperm = ar.take<int>(n);
  v.ubperm = ar.take<int>(n);
  v.u0buf = prm.warm == 2 ? ar.take<double>(T * m) : nullptr;
  h.dfac = ar.take<int>((size_t)2 * n + h.fixf.size() * 2 + v.ntrip);
  v.trips = h.dfac ? h.dfac + 2 * n + 2 * h.fixf.size() : nullptr;
  h.bytes = ar.used;
}

struct Tuned {
  int group, wpb;
  double ms;  // the chosen shape's Z-stage time for this size when it was tuned
};
std::mutex g_tune_mu;
std::map<int, Tuned> g_tuned;  // Z-LAP size -> Z-stage launch shape

// Device-side descriptors of one wave.
// LAP stages of a wave: Z, Y, X and the second Z phase.
constexpr int kStages = 4;
// Launches per Z stage: at most one per Z-LAP size (1..32)
constexpr int kMaxRuns = 33;
// Per stage: the prefix arrays of all launches of the stage, each starting at 0
constexpr int kPrefixStride = kMaxWaveNodes + kMaxRuns + 1;

// One launch of a Z stage: sorted items [first, last), their LAP sizes up to max_m.
struct ZRun {
  int first = 0, last = 0, max_m = 0, group = 0, wpb = 0;
  long long total = 0;
};

struct WaveDev {
  NodeLapItem* items = nullptr;  // [kStages][kMaxWaveNodes]; Z stages sorted by LAP size
  long long* prefix = nullptr;   // [kStages][kPrefixStride]; Z stages: one array per launch
  MoveYArgs* my = nullptr;
  MoveZArgs* mz = nullptr;
  Phase2Args* p2 = nullptr;
  int* mz_blocks = nullptr;
  FinArgs* fin = nullptr;
  unsigned long long* heads = nullptr;  // [kStages][kMaxRuns]
  unsigned long long* stats = nullptr;  // [6]
  int* live = nullptr;                  // nodes not stopped (k_count_live)
};

struct LearnedStart {
  long long T;
  int m;
  const double* Dhat;
  const double* xi;
  double* u0;
};

struct Wave {
  rlt2_mlp* mlp = nullptr;
  std::vector<LearnedStart> learned;  // one per node when warm == 2
  int nn = 0;
  int two_phase = 0;
  int cold = 0;  // warm == 0: no LAP of the wave has start duals
  long long total[kStages] = {0, 0, 0, 0};
  int max_m[kStages] = {0, 0, 0, 0};
  int max_blocks = 0;
  int max_T = 0;
  int max_n = 0;
  std::vector<int> zm;     // Z-LAP size of each sorted Z item
  std::vector<ZRun> runs;  // the Z stages' launches
};

// The Z stages' launches for `runs`: prefix arrays (each from 0) for stages 0
// and 3, uploaded synchronously (outside capture, before the launches use them).
cudaError_t upload_runs(Wave& w, const WaveDev& d, const std::vector<NodeLapItem>& items, cudaStream_t s) {
  std::vector<long long> pre((size_t)kPrefixStride * 2, 0);
  for (int si = 0; si < 2; ++si) {
    const int stage = si == 0 ? 0 : 3;
    size_t off = 0;
    for (ZRun& r : w.runs) {
      long long acc = 0;
      pre[si * kPrefixStride + off] = 0;
      for (int j = r.first; j < r.last; ++j) {
        acc += items[stage * kMaxWaveNodes + j].count;
        pre[si * kPrefixStride + off + (j - r.first) + 1] = acc;
      }
      r.total = acc;  // the same count in both Z stages
      off += (size_t)(r.last - r.first) + 1;
    }
  }
  cudaError_t e = cudaMemcpyAsync(d.prefix, pre.data(), sizeof(long long) * kPrefixStride, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(d.prefix + 3 * kPrefixStride, pre.data() + kPrefixStride, sizeof(long long) * kPrefixStride,
                      cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

// One launch per Z-LAP size present (sorted items), each with shape `shape(m)`.
template <class F>
std::vector<ZRun> size_runs(const Wave& w, F shape) {
  std::vector<ZRun> runs;
  for (int j = 0; j < (int)w.zm.size(); ++j) {
    if (runs.empty() || w.zm[j] != runs.back().max_m) {
      ZRun r;
      r.first = j;
      r.max_m = w.zm[j];
      const std::pair<int, int> gw = shape(w.zm[j]);
      r.group = gw.first;
      r.wpb = gw.second;
      runs.push_back(r);
    }
    runs.back().last = j + 1;
  }
  return runs;
}

// Adjacent runs with the same shape merged into one launch.
std::vector<ZRun> merge_runs(const std::vector<ZRun>& in) {
  std::vector<ZRun> out;
  for (const ZRun& r : in) {
    if (!out.empty() && out.back().group == r.group && out.back().wpb == r.wpb && out.back().last == r.first) {
      out.back().last = r.last;
      out.back().max_m = std::max(out.back().max_m, r.max_m);
    } else {
      out.push_back(r);
    }
  }
  return out;
}

// zev (nullable): 2 events per Z run, recorded around that run's first-phase launch.
cudaError_t enqueue_wave_iteration(const Wave& w, const WaveDev& d, int dual_mode, cudaStream_t s,
                                   const cudaEvent_t* zev) {
  cudaError_t e;
  {
    const int bx = std::max(1, std::min(1024, (w.max_T + 255) / 256));
    k_move_y_nodes<<<dim3(bx, w.nn), 256, 0, s>>>(d.my);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_move_z_nodes<<<dim3(w.max_blocks, w.nn), move_z_threads(w.max_n), 0, s>>>(d.mz, d.mz_blocks);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (const LearnedStart& ls : w.learned)
    if ((e = mlp_predict_enqueue(w.mlp, ls.T, ls.m, ls.Dhat, ls.xi, ls.u0, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(d.heads, 0, kStages * kMaxRuns * sizeof(unsigned long long), s)) != cudaSuccess) return e;
  // Z, [second phase move, Z again], Y, X
  const int order[kStages] = {0, 3, 1, 2};
  for (int oi = 0; oi < kStages; ++oi) {
    const int stage = order[oi];
    if (stage == 3) {
      if (!w.two_phase) continue;
      k_phase2_nodes<<<dim3(w.max_blocks, w.nn), move_z_threads(w.max_n), 0, s>>>(d.p2, d.mz_blocks);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    NodeLapArgs a{};
    a.dual_mode = dual_mode;
    a.cold = w.cold;
    a.stats = d.stats + 2 * (stage == 3 ? 0 : stage);
    if (stage == 1 || stage == 2) {  // Y, X: one launch over all nodes, node order
      a.nnodes = w.nn;
      a.items = d.items + stage * kMaxWaveNodes;
      a.prefix = d.prefix + stage * kPrefixStride;
      a.total = w.total[stage];
      a.max_m = w.max_m[stage];
      a.head = d.heads + stage * kMaxRuns;
      a.pre = false;
      if ((e = launch_lap_nodes(a, s)) != cudaSuccess) return e;
      continue;
    }
    // Z stages: one launch per run of sizes, items sorted by size; no reduced costs
    size_t off = 0;
    for (size_t ri = 0; ri < w.runs.size(); ++ri) {
      const ZRun& r = w.runs[ri];
      a.nnodes = r.last - r.first;
      a.items = d.items + stage * kMaxWaveNodes + r.first;
      a.prefix = d.prefix + stage * kPrefixStride + off;
      a.total = r.total;
      a.max_m = r.max_m;
      a.head = d.heads + stage * kMaxRuns + ri;
      a.group = r.group;
      a.warps_per_block = r.wpb;
      a.pre = true;
      off += (size_t)a.nnodes + 1;
      if (stage == 0 && zev && (e = cudaEventRecord(zev[2 * ri], s)) != cudaSuccess) return e;
      if ((e = launch_lap_nodes(a, s)) != cudaSuccess) return e;
      if (stage == 0 && zev && (e = cudaEventRecord(zev[2 * ri + 1], s)) != cudaSuccess) return e;
    }
  }
  k_finalize_nodes<<<w.nn, 256, 0, s>>>(d.fin);
  return cudaGetLastError();
}


// Host-side descriptors of one wave.
struct WaveHost {
  std::vector<NodeLapItem> items = std::vector<NodeLapItem>(kStages * kMaxWaveNodes);
  std::vector<long long> prefix = std::vector<long long>((size_t)kStages * kPrefixStride, 0);
  std::vector<MoveYArgs> my;
  std::vector<MoveZArgs> mz;
  std::vector<Phase2Args> p2;
  std::vector<int> mzb;
  std::vector<FinArgs> fin;
  explicit WaveHost(int nn) : my(nn), mz(nn), p2(nn), mzb(nn), fin(nn) {}
};

// The stage descriptors of node j of a wave, whose buffers and scalars are v.
void add_node(Wave& w, WaveHost& h, int j, const IterView& v, const rlt2_params& prm) {
  const int nr = v.n;
  NodeLapItem z{}, y{}, x{}, z2{};
  z.count = v.T;
  z.m = nr - 2;
  z.A = v.Dhat;
  z.u0 = prm.warm == 1 ? v.xi : (prm.warm == 2 ? v.u0buf : nullptr);
  z.warm_gate = prm.warm == 2 ? nullptr : &v.sc->have_snap;
  if (prm.warm == 2) w.learned.push_back(LearnedStart{v.T, nr - 2, v.Dhat, v.xi, v.u0buf});
  z.skip = &v.sc->done;
  z.value = v.Theta;
  z.u = v.xi;
  z.v = v.psi;
  y.count = (long long)nr * nr;
  y.m = nr - 1;
  y.A = v.Chat;
  y.Badd = v.Theta;
  y.u0 = prm.warm >= 1 ? v.gamma : nullptr;
  y.warm_gate = &v.sc->have_snap;
  y.skip = &v.sc->done;
  y.value = v.Delta;
  y.u = v.gamma;
  y.v = v.delta;
  y.pi = v.piy;
  x.count = 1;
  x.m = nr;
  x.A = v.xcost;
  x.Badd = v.Delta;
  x.u0 = prm.warm >= 1 ? v.alpha : nullptr;
  x.warm_gate = &v.sc->have_snap;
  x.skip = &v.sc->done;
  x.value = v.xval;
  x.u = v.alpha;
  x.v = v.beta;
  x.r2c = v.xperm;
  x.pi = v.pix;
  z2 = z;
  z2.u0 = prm.warm >= 1 ? v.xi : nullptr;  // second phase: from the first phase's row duals
  z2.warm_gate = nullptr;
  const NodeLapItem st3[kStages] = {z, y, x, z2};
  for (int sg = 0; sg < kStages; ++sg) {
    h.items[sg * kMaxWaveNodes + j] = st3[sg];  // Z stages are sorted by size in sort_z
    h.prefix[sg * kPrefixStride + j + 1] = h.prefix[sg * kPrefixStride + j] + st3[sg].count;
    w.total[sg] += st3[sg].count;
    w.max_m[sg] = std::max(w.max_m[sg], st3[sg].m);
  }
  h.my[j] = make_move_y(v);
  h.mz[j] = make_move_z(v);
  h.p2[j] = make_phase2(v);
  h.mzb[j] = v.ntrip * nr;
  h.fin[j] = make_fin(v);
  w.max_blocks = std::max(w.max_blocks, h.mzb[j]);
  w.max_T = std::max(w.max_T, (int)v.T);
  w.max_n = std::max(w.max_n, nr);
}

// The Z stages' items sorted by LAP size (stable: node order within a size).
void sort_z(Wave& w, WaveHost& h) {
  std::vector<int> ord(w.nn);
  for (int j = 0; j < w.nn; ++j) ord[j] = j;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return h.items[x].m < h.items[y].m; });
  std::vector<NodeLapItem> zs(w.nn), z2s(w.nn);
  w.zm.assign(w.nn, 0);
  for (int pos = 0; pos < w.nn; ++pos) {
    zs[pos] = h.items[ord[pos]];
    z2s[pos] = h.items[3 * kMaxWaveNodes + ord[pos]];
    w.zm[pos] = zs[pos].m;
  }
  std::copy(zs.begin(), zs.end(), h.items.begin());
  std::copy(z2s.begin(), z2s.end(), h.items.begin() + 3 * kMaxWaveNodes);
}

// Copies a wave's descriptors to the device and waits for the copies.
cudaError_t upload_wave(const Wave& w, const WaveHost& h, const WaveDev& d, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d.items, h.items.data(), sizeof(NodeLapItem) * h.items.size(), cudaMemcpyHostToDevice,
                           s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d.prefix, h.prefix.data(), sizeof(long long) * h.prefix.size(), cudaMemcpyHostToDevice,
                           s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d.my, h.my.data(), sizeof(MoveYArgs) * w.nn, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d.mz, h.mz.data(), sizeof(MoveZArgs) * w.nn, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d.p2, h.p2.data(), sizeof(Phase2Args) * w.nn, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d.mz_blocks, h.mzb.data(), sizeof(int) * w.nn, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(d.fin, h.fin.data(), sizeof(FinArgs) * w.nn, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  return cudaStreamSynchronize(s);  // the host vectors must outlive the copies
}

cudaError_t alloc_wave_dev(WaveDev& d) {
  cudaError_t e;
  if ((e = cudaMalloc((void**)&d.items, sizeof(NodeLapItem) * kStages * kMaxWaveNodes)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d.prefix, sizeof(long long) * kStages * kPrefixStride)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d.my, sizeof(MoveYArgs) * kMaxWaveNodes)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d.mz, sizeof(MoveZArgs) * kMaxWaveNodes)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d.p2, sizeof(Phase2Args) * kMaxWaveNodes)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d.mz_blocks, sizeof(int) * kMaxWaveNodes)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d.fin, sizeof(FinArgs) * kMaxWaveNodes)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d.heads, sizeof(unsigned long long) * kStages * kMaxRuns)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d.stats, sizeof(unsigned long long) * 6)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d.live, sizeof(int))) != cudaSuccess)
    return e;
  return cudaSuccess;
}

void free_wave_dev(WaveDev& d) {
  void* frees[] = {d.items, d.prefix, d.my, d.mz, d.p2, d.mz_blocks, d.fin, d.heads, d.stats, d.live};
  for (void* q : frees)
    if (q) cudaFree(q);
  d = WaveDev{};
}

// Tunes, on live iterations, the Z-stage shape of every size of the wave not
// in the process table yet (iteration 1, then one iteration per candidate:
// these are iterations of the ascent like any other), then sets the wave's Z
// launches (sizes with equal shapes merged).  *ran: iterations enqueued.
cudaError_t plan_z(Wave& w, const WaveDev& d, const WaveHost& h, int dual_mode, int iters, cudaStream_t s,
                   const cudaEvent_t* zev, int* ran) {
  *ran = 0;
  auto cands = [](int m) {
    std::vector<std::pair<int, int>> c;
    const int g0 = default_group(m);
    c.push_back({g0, 8});
    c.push_back({g0, 4});
    if (g0 != 32) c.push_back({32, 8});
    return c;
  };
  std::map<int, Tuned> table;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    table = g_tuned;
  }
  std::vector<int> todo;
  for (int mz : w.zm)
    if (!table.count(mz) && (todo.empty() || todo.back() != mz)) todo.push_back(mz);
  auto known = [&](int mz) -> std::pair<int, int> {
    auto it = table.find(mz);
    return it != table.end() ? std::make_pair(it->second.group, it->second.wpb) : std::make_pair(default_group(mz), 8);
  };
  int ncand = 0;
  for (int mz : todo) ncand = std::max(ncand, (int)cands(mz).size());
  cudaError_t e;
  if (!todo.empty() && iters >= ncand + 1) {
    w.runs = size_runs(w, known);
    if ((e = upload_runs(w, d, h.items, s)) != cudaSuccess) return e;
    if ((e = enqueue_wave_iteration(w, d, dual_mode, s, nullptr)) != cudaSuccess) return e;
    ++*ran;
    std::map<int, Tuned> best;
    for (int c = 0; c < ncand; ++c) {
      w.runs = size_runs(w, [&](int mz) {
        if (std::find(todo.begin(), todo.end(), mz) == todo.end()) return known(mz);
        const auto cs = cands(mz);
        return cs[std::min(c, (int)cs.size() - 1)];
      });
      if ((e = upload_runs(w, d, h.items, s)) != cudaSuccess) return e;
      if ((e = enqueue_wave_iteration(w, d, dual_mode, s, zev)) != cudaSuccess) return e;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
      ++*ran;
      for (size_t ri = 0; ri < w.runs.size(); ++ri) {
        const ZRun& r = w.runs[ri];
        if (std::find(todo.begin(), todo.end(), r.max_m) == todo.end()) continue;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, zev[2 * ri], zev[2 * ri + 1])) != cudaSuccess) return e;
        auto it = best.find(r.max_m);
        if (it == best.end() || ms < it->second.ms) best[r.max_m] = Tuned{r.group, r.wpb, ms};
      }
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto& kv : best) {
      g_tuned[kv.first] = kv.second;
      table[kv.first] = kv.second;
    }
  }
  w.runs = merge_runs(size_runs(w, known));
  return upload_runs(w, d, h.items, s);
}

// Number of nodes of a wave that have not stopped.
__global__ void k_count_live(const FinArgs* nodes, int nn, int* live) {
  int c = 0;
  for (int j = threadIdx.x; j < nn; j += blockDim.x) c += nodes[j].sc->done == 0;
  c = __reduce_add_sync(0xffffffffu, c);
  __shared__ int part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
    *live = t;
  }
}
std::mutex g_views_mu;  // iterate_views' device descriptors, one set per device
constexpr int kViewDevices = 64;
WaveDev g_views_dev[kViewDevices];

}  // namespace

cudaError_t iterate_views(const IterView* views, int nn, const rlt2_params& prm, int iters, cudaStream_t s,
                          int* ran) {
  *ran = 0;
  if (nn < 1 || nn > kMaxWaveNodes || iters < 0) return cudaErrorInvalidValue;
  if (iters == 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kViewDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_views_mu);
  WaveDev& d = g_views_dev[dev];
  if (!d.items && (e = alloc_wave_dev(d)) != cudaSuccess) {
    free_wave_dev(d);
    return e;
  }
  Wave w;
  w.nn = nn;
  w.two_phase = prm.two_phase;
  w.cold = prm.warm == 0;
  WaveHost h(nn);
  for (int j = 0; j < nn; ++j) add_node(w, h, j, views[j], prm);
  sort_z(w, h);
  if ((e = upload_wave(w, h, d, s)) != cudaSuccess) return e;
  std::vector<cudaEvent_t> zev(2 * kMaxRuns, nullptr);
  for (cudaEvent_t& ev : zev)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) break;
  int done = 0;
  if (e == cudaSuccess) e = plan_z(w, d, h, prm.dual_mode, iters, s, zev.data(), &done);
  // chunks of 8, 16, 32, ... iterations, the nodes' stop flags checked between
  // chunks: a batch whose nodes have all stopped ends early
  int step = 8, live = 1;
  while (e == cudaSuccess && done < iters) {
    k_count_live<<<1, 256, 0, s>>>(d.fin, nn, d.live);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(&live, d.live, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      break;
    if (live == 0) break;
    const int chunk = std::min(step, iters - done);
    for (int it = 0; it < chunk && e == cudaSuccess; ++it) e = enqueue_wave_iteration(w, d, prm.dual_mode, s, nullptr);
    done += chunk;
    step = std::min(2 * step, 1024);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (cudaEvent_t ev : zev)
    if (ev) cudaEventDestroy(ev);
  *ran = done;
  return e;
}

RLT2_DEFINE_OOB_QUERY(oob_nodes)
}  // namespace rlt2

using namespace rlt2;

#define CKN(call)                                         \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) {                              \
      st = cuda_fail(e_, #call);                          \
      goto done;                                          \
    }                                                     \
  } while (0)

extern "C" rlt2_status rlt2_bound_nodes(int n, const double* F, const double* D, const double* B, int n_nodes,
                                        const int* partials, const rlt2_params* p, rlt2_mlp* mlp, int iters,
                                        size_t mem_budget,
                                        double* lb_out, double* lb_hist, int* iters_out, long long* stats_out,
                                        void* stream) {
  if (n < 3 || n > 64 || !F || !D || n_nodes < 1 || !partials || iters < 1 || iters > kRing || !lb_out) {
    set_error("rlt2_bound_nodes: invalid argument");
    return RLT2_EINVAL;
  }
  const size_t nn2 = (size_t)n * n;
  for (size_t i = 0; i < nn2; ++i)
    if (!std::isfinite(F[i]) || !std::isfinite(D[i]) || (B && !std::isfinite(B[i]))) {
      set_error("rlt2_bound_nodes: non-finite input");
      return RLT2_EINVAL;
    }
  rlt2_params prm;
  rlt2_params_default(&prm);
  if (p) prm = *p;
  if (!params_valid(prm)) {
    set_error("rlt2_bound_nodes: parameters out of range");
    return RLT2_EINVAL;
  }
  if (prm.warm == 2 && !mlp) {
    set_error("rlt2_bound_nodes: warm == 2 needs a network");
    return RLT2_EINVAL;
  }
  if (prm.half_z) {
    set_error("rlt2_bound_nodes: the half-Z scheme runs on single contexts only");
    return RLT2_EINVAL;
  }
  // per-node residual problems
  std::vector<NodeHost> nodes(n_nodes);
  for (int k = 0; k < n_nodes; ++k) {
    const int* part = partials + (size_t)k * n;
    std::vector<char> used(n, 0);
    NodeHost& h = nodes[k];
    for (int i = 0; i < n; ++i) {
      if (part[i] >= 0) {
        if (part[i] >= n || used[part[i]]) {
          set_error("rlt2_bound_nodes: node " + std::to_string(k) + " has a non-injective partial assignment");
          return RLT2_EINVAL;
        }
        used[part[i]] = 1;
        h.fixf.push_back(i);
        h.fixl.push_back(part[i]);
      } else if (part[i] < -1) {
        set_error("rlt2_bound_nodes: partial entries must be -1 or a location");
        return RLT2_EINVAL;
      }
    }
    for (int i = 0; i < n; ++i)
      if (part[i] < 0) h.fac.push_back(i);
    for (int q = 0; q < n; ++q)
      if (!used[q]) h.loc.push_back(q);
    h.nr = (int)h.fac.size();
    if (h.nr < 3 || h.nr > 32) {
      set_error("rlt2_bound_nodes: node " + std::to_string(k) + " has residual size outside [3, 32]");
      return RLT2_EINVAL;
    }
    carve(h, nullptr, prm);
  }
  size_t fr = 0, tot = 0;
  cudaError_t e0 = cudaMemGetInfo(&fr, &tot);
  if (e0 != cudaSuccess) return cuda_fail(e0, "cudaMemGetInfo");
  const size_t budget = mem_budget ? mem_budget : (size_t)(0.8 * (double)fr);
  // admission: consecutive nodes join a wave while its arenas fit the budget
  std::vector<std::pair<int, int>> waves;  // [first, last)
  {
    int first = 0;
    size_t acc = 0;
    for (int k = 0; k < n_nodes; ++k) {
      if (nodes[k].bytes > budget) {
        set_error("rlt2_bound_nodes: node " + std::to_string(k) + " needs " + std::to_string(nodes[k].bytes) +
                  " bytes, more than the memory budget");
        return RLT2_EADMIT;
      }
      if (acc + nodes[k].bytes > budget || k - first >= kMaxWaveNodes) {
        waves.push_back({first, k});
        first = k;
        acc = 0;
      }
      acc += nodes[k].bytes;
    }
    waves.push_back({first, n_nodes});
  }
  size_t pool_bytes = 0;
  for (auto& w : waves) {
    size_t b = 0;
    for (int k = w.first; k < w.second; ++k) b += nodes[k].bytes;
    pool_bytes = std::max(pool_bytes, b);
  }
  if (pool_bytes + (64u << 20) > fr) {
    set_error("rlt2_bound_nodes: not enough free device memory for the budget");
    return RLT2_ENOMEM;
  }

  cudaStream_t s = (cudaStream_t)stream;
  rlt2_status st = RLT2_OK;
  char* pool = nullptr;
  double *dF = nullptr, *dD = nullptr, *dB = nullptr;
  WaveDev d;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<cudaEvent_t> zev(2 * kMaxRuns, nullptr);
  long long tot_aug = 0, tot_relax = 0;
  CKN(cudaMalloc((void**)&pool, pool_bytes));
  CKN(cudaMalloc((void**)&dF, nn2 * 8));
  CKN(cudaMalloc((void**)&dD, nn2 * 8));
  if (B) CKN(cudaMalloc((void**)&dB, nn2 * 8));
  CKN(alloc_wave_dev(d));
  CKN(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  for (cudaEvent_t& ev : zev) CKN(cudaEventCreate(&ev));
  CKN(cudaMemcpyAsync(dF, F, nn2 * 8, cudaMemcpyHostToDevice, s));
  CKN(cudaMemcpyAsync(dD, D, nn2 * 8, cudaMemcpyHostToDevice, s));
  if (B) CKN(cudaMemcpyAsync(dB, B, nn2 * 8, cudaMemcpyHostToDevice, s));
  CKN(cudaMemsetAsync(d.stats, 0, sizeof(unsigned long long) * 6, s));

  for (auto& wr : waves) {
    Wave w;
    w.nn = wr.second - wr.first;
    w.mlp = prm.warm == 2 ? mlp : nullptr;
    // carve the arenas and upload each node's index lists
    char* cur = pool;
    w.two_phase = prm.two_phase;
    w.cold = prm.warm == 0;
    WaveHost hw(w.nn);
    std::vector<DevScalars> init(1);
    init[0] = DevScalars{};
    init[0].ub = INFINITY;
    init[0].best_lb = -INFINITY;
    init[0].lb = -INFINITY;
    CKN(cudaMemsetAsync(pool, 0, pool_bytes, s));  // D^ = 0 (Algorithm 1 step 1), scalars cleared
    for (int j = 0; j < w.nn; ++j) {
      NodeHost& h = nodes[wr.first + j];
      carve(h, cur, prm);
      cur += h.bytes;
      const IterView& v = h.v;
      std::vector<int> ints;
      ints.insert(ints.end(), h.fac.begin(), h.fac.end());
      ints.insert(ints.end(), h.loc.begin(), h.loc.end());
      ints.insert(ints.end(), h.fixf.begin(), h.fixf.end());
      ints.insert(ints.end(), h.fixl.begin(), h.fixl.end());
      for (int i = 0; i < h.nr; ++i)
        for (int jj = i + 1; jj < h.nr; ++jj)
          for (int kk = jj + 1; kk < h.nr; ++kk) ints.push_back(i | (jj << 8) | (kk << 16));
      CKN(cudaMemcpyAsync(h.dfac, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      CKN(cudaMemcpyAsync(v.sc, init.data(), sizeof(DevScalars), cudaMemcpyHostToDevice, s));
      const int nfix = (int)h.fixf.size();
      CKN(enqueue_setup(v, n, dF, dD, dB, h.dfac, h.dfac + h.nr, h.dfac + 2 * h.nr, h.dfac + 2 * h.nr + nfix, nfix,
                        s));
      // X-LAP costs start as b' (the F variant then updates them); F's bound starts at the constant
      CKN(cudaMemcpyAsync(v.xcost, v.bprime, sizeof(double) * h.nr * h.nr, cudaMemcpyDeviceToDevice, s));
      CKN(cudaMemcpyAsync(&v.sc->lb_base, v.d_cst, sizeof(double), cudaMemcpyDeviceToDevice, s));
      add_node(w, hw, j, v, prm);
    }
    sort_z(w, hw);
    CKN(upload_wave(w, hw, d, s));
    // autotune the Z stage per LAP size on live iterations 2.. (iteration 1
    // has D^ = 0), then plan the Z launches
    int done_iters = 0;
    CKN(plan_z(w, d, hw, prm.dual_mode, iters, s, zev.data(), &done_iters));
    // the rest of the iterations: one CUDA graph per wave, replayed
    if (done_iters < iters) {
      cudaGraph_t g = nullptr;
      CKN(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      cudaError_t ec = enqueue_wave_iteration(w, d, prm.dual_mode, cap, nullptr);
      cudaError_t ee = cudaStreamEndCapture(cap, &g);
      if (ec != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        st = cuda_fail(ec != cudaSuccess ? ec : ee, "wave capture");
        goto done;
      }
      cudaError_t ei = cudaGraphInstantiate(&gexec, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) {
        gexec = nullptr;
        st = cuda_fail(ei, "cudaGraphInstantiate");
        goto done;
      }
      for (int it = done_iters; it < iters; ++it) CKN(cudaGraphLaunch(gexec, s));
      CKN(cudaStreamSynchronize(s));
      cudaGraphExecDestroy(gexec);
      gexec = nullptr;
    }
    // results
    for (int j = 0; j < w.nn; ++j) {
      const int k = wr.first + j;
      const IterView& v = nodes[k].v;
      DevScalars h;
      CKN(cudaMemcpy(&h, v.sc, sizeof h, cudaMemcpyDeviceToHost));
      lb_out[k] = h.best_lb;
      if (iters_out) iters_out[k] = h.iter;
      if (lb_hist) {
        CKN(cudaMemcpy(lb_hist + (size_t)k * iters, v.ring, sizeof(double) * std::min(h.iter, iters),
                       cudaMemcpyDeviceToHost));
        for (int it = h.iter; it < iters; ++it) lb_hist[(size_t)k * iters + it] = NAN;
      }
    }
  }
  {
    unsigned long long hs[6];
    CKN(cudaMemcpy(hs, d.stats, sizeof hs, cudaMemcpyDeviceToHost));
    tot_aug = (long long)hs[0];
    tot_relax = (long long)hs[1];
  }
  if (stats_out) {
    stats_out[0] = (long long)waves.size();
    stats_out[1] = tot_aug;
    stats_out[2] = tot_relax;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    int mz_all = 0;
    for (auto& h : nodes) mz_all = std::max(mz_all, h.nr - 2);
    auto it = g_tuned.find(mz_all);
    stats_out[3] = it != g_tuned.end() ? it->second.group : 0;
    stats_out[4] = it != g_tuned.end() ? it->second.wpb : 0;
  }
done:
  if (gexec) cudaGraphExecDestroy(gexec);
  for (cudaEvent_t ev : zev)
    if (ev) cudaEventDestroy(ev);
  if (cap) cudaStreamDestroy(cap);
  cudaStreamSynchronize(s);
  void* frees[] = {pool, dF, dD, dB};
  for (void* q : frees)
    if (q) cudaFree(q);
  free_wave_dev(d);
  return st;
}

extern "C" rlt2_status rlt2_node_tuning(int cap, int* m, int* group, int* wpb, double* ms, int* count) {
  if (cap < 0 || !count || (cap > 0 && (!m || !group || !wpb))) {
    set_error("rlt2_node_tuning: invalid argument");
    return RLT2_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  *count = (int)g_tuned.size();
  int k = 0;
  for (const auto& kv : g_tuned) {
    if (k >= cap) break;
    m[k] = kv.first;
    group[k] = kv.second.group;
    wpb[k] = kv.second.wpb;
    if (ms) ms[k] = kv.second.ms;
    ++k;
  }
  return RLT2_OK;
}
