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
// The Z stage's launch shape (lanes per LAP, warps per block) is picked by an
// autotuner that times the candidates on live iterations (every candidate gives
// bit-identical results, so tuning costs no accuracy) and caches the choice per
// largest Z-LAP size.
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

__global__ void k_move_y_nodes(const MoveYArgs* nodes) {
  const MoveYArgs a = nodes[blockIdx.y];
  if (!a.sc->have_snap || a.sc->done) return;
  move_y_range(a, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(352, 3) k_move_z_nodes(const MoveZArgs* nodes, const int* nblocks) {
  if ((int)blockIdx.x >= nblocks[blockIdx.y]) return;
  const MoveZArgs a = nodes[blockIdx.y];
  if (!a.sc->have_snap || a.sc->done) return;
  move_z_block(a, blockIdx.x, threadIdx.x, blockDim.x);
}

__global__ void k_shift_psi_nodes(const MoveYArgs* nodes) {
  const MoveYArgs a = nodes[blockIdx.y];
  if (!a.shift_psi || !a.sc->have_snap || a.sc->done) return;
  shift_psi_range(a, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
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
  double ms;
};
std::mutex g_tune_mu;
std::map<int, Tuned> g_tuned;  // largest Z-LAP size of a wave -> Z-stage launch shape

// Device-side descriptors of one wave.
// LAP stages of a wave: Z, Y, X and the second Z phase.
constexpr int kStages = 4;

struct WaveDev {
  NodeLapItem* items = nullptr;  // [kStages][kMaxWaveNodes]
  long long* prefix = nullptr;   // [kStages][kMaxWaveNodes + 1]
  MoveYArgs* my = nullptr;
  MoveZArgs* mz = nullptr;
  Phase2Args* p2 = nullptr;
  int* mz_blocks = nullptr;
  FinArgs* fin = nullptr;
  unsigned long long* heads = nullptr;  // [kStages]
  unsigned long long* stats = nullptr;  // [6]
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
  long long total[kStages] = {0, 0, 0, 0};
  int max_m[kStages] = {0, 0, 0, 0};
  int max_blocks = 0;
  int max_T = 0;
  int max_n = 0;
};

cudaError_t enqueue_wave_iteration(const Wave& w, const WaveDev& d, int dual_mode, int zgroup, int zwpb,
                                   cudaStream_t s, cudaEvent_t zev0, cudaEvent_t zev1) {
  cudaError_t e;
  {
    const int bx = std::max(1, std::min(1024, (w.max_T + 255) / 256));
    k_move_y_nodes<<<dim3(bx, w.nn), 256, 0, s>>>(d.my);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int bx2 = std::max(1, std::min(4096, (int)(((long long)w.max_T * (w.max_n - 2) + 255) / 256)));
    k_shift_psi_nodes<<<dim3(bx2, w.nn), 256, 0, s>>>(d.my);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_move_z_nodes<<<dim3(w.max_blocks, w.nn), move_z_threads(w.max_n), 0, s>>>(d.mz, d.mz_blocks);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (const LearnedStart& ls : w.learned)
    if ((e = mlp_predict_enqueue(w.mlp, ls.T, ls.m, ls.Dhat, ls.xi, ls.u0, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(d.heads, 0, kStages * sizeof(unsigned long long), s)) != cudaSuccess) return e;
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
    a.nnodes = w.nn;
    a.items = d.items + stage * kMaxWaveNodes;
    a.prefix = d.prefix + stage * (kMaxWaveNodes + 1);
    a.total = w.total[stage];
    a.max_m = w.max_m[stage];
    a.dual_mode = dual_mode;
    a.head = d.heads + stage;
    a.stats = d.stats + 2 * (stage == 3 ? 0 : stage);
    a.group = (stage == 0 || stage == 3) ? zgroup : 0;
    a.warps_per_block = (stage == 0 || stage == 3) ? zwpb : 0;
    a.pre = stage == 0 || stage == 3;  // the Z stages write no reduced costs
    if (stage == 0 && zev0 && (e = cudaEventRecord(zev0, s)) != cudaSuccess) return e;
    if ((e = launch_lap_nodes(a, s)) != cudaSuccess) return e;
    if (stage == 0 && zev1 && (e = cudaEventRecord(zev1, s)) != cudaSuccess) return e;
  }
  k_finalize_nodes<<<w.nn, 256, 0, s>>>(d.fin);
  return cudaGetLastError();
}

}  // namespace

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
  cudaEvent_t zev0 = nullptr, zev1 = nullptr;
  long long tot_aug = 0, tot_relax = 0;
  CKN(cudaMalloc((void**)&pool, pool_bytes));
  CKN(cudaMalloc((void**)&dF, nn2 * 8));
  CKN(cudaMalloc((void**)&dD, nn2 * 8));
  if (B) CKN(cudaMalloc((void**)&dB, nn2 * 8));
  CKN(cudaMalloc((void**)&d.items, sizeof(NodeLapItem) * kStages * kMaxWaveNodes));
  CKN(cudaMalloc((void**)&d.prefix, sizeof(long long) * kStages * (kMaxWaveNodes + 1)));
  CKN(cudaMalloc((void**)&d.my, sizeof(MoveYArgs) * kMaxWaveNodes));
  CKN(cudaMalloc((void**)&d.mz, sizeof(MoveZArgs) * kMaxWaveNodes));
  CKN(cudaMalloc((void**)&d.p2, sizeof(Phase2Args) * kMaxWaveNodes));
  CKN(cudaMalloc((void**)&d.mz_blocks, sizeof(int) * kMaxWaveNodes));
  CKN(cudaMalloc((void**)&d.fin, sizeof(FinArgs) * kMaxWaveNodes));
  CKN(cudaMalloc((void**)&d.heads, sizeof(unsigned long long) * kStages));
  CKN(cudaMalloc((void**)&d.stats, sizeof(unsigned long long) * 6));
  CKN(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  CKN(cudaEventCreate(&zev0));
  CKN(cudaEventCreate(&zev1));
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
    std::vector<NodeLapItem> items(kStages * kMaxWaveNodes);
    std::vector<long long> prefix(kStages * (kMaxWaveNodes + 1), 0);
    std::vector<MoveYArgs> my(w.nn);
    std::vector<MoveZArgs> mz(w.nn);
    std::vector<Phase2Args> p2(w.nn);
    std::vector<int> mzb(w.nn);
    std::vector<FinArgs> fin(w.nn);
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
      // stage descriptors
      const int nr = h.nr;
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
        items[sg * kMaxWaveNodes + j] = st3[sg];
        prefix[sg * (kMaxWaveNodes + 1) + j + 1] = prefix[sg * (kMaxWaveNodes + 1) + j] + st3[sg].count;
        w.total[sg] += st3[sg].count;
        w.max_m[sg] = std::max(w.max_m[sg], st3[sg].m);
      }
      my[j] = make_move_y(v);
      mz[j] = make_move_z(v);
      p2[j] = make_phase2(v);
      mzb[j] = v.ntrip * nr;
      fin[j] = make_fin(v);
      w.max_blocks = std::max(w.max_blocks, mzb[j]);
      w.max_T = std::max(w.max_T, (int)v.T);
      w.max_n = std::max(w.max_n, nr);
    }
    CKN(cudaMemcpyAsync(d.items, items.data(), sizeof(NodeLapItem) * items.size(), cudaMemcpyHostToDevice, s));
    CKN(cudaMemcpyAsync(d.prefix, prefix.data(), sizeof(long long) * prefix.size(), cudaMemcpyHostToDevice, s));
    CKN(cudaMemcpyAsync(d.my, my.data(), sizeof(MoveYArgs) * w.nn, cudaMemcpyHostToDevice, s));
    CKN(cudaMemcpyAsync(d.mz, mz.data(), sizeof(MoveZArgs) * w.nn, cudaMemcpyHostToDevice, s));
    CKN(cudaMemcpyAsync(d.p2, p2.data(), sizeof(Phase2Args) * w.nn, cudaMemcpyHostToDevice, s));
    CKN(cudaMemcpyAsync(d.mz_blocks, mzb.data(), sizeof(int) * w.nn, cudaMemcpyHostToDevice, s));
    CKN(cudaMemcpyAsync(d.fin, fin.data(), sizeof(FinArgs) * w.nn, cudaMemcpyHostToDevice, s));
    CKN(cudaStreamSynchronize(s));  // host vectors above must outlive the copies

    // autotune the Z stage on live iterations 2.. (iteration 1 has D^ = 0)
    const int mz_max = w.max_m[0];
    Tuned tuned{0, 0, 0.0};
    bool have_tuned = false;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tuned.find(mz_max);
      if (it != g_tuned.end()) {
        tuned = it->second;
        have_tuned = true;
      }
    }
    int done_iters = 0;
    if (!have_tuned) {
      std::vector<std::pair<int, int>> cand;
      const int g0 = default_group(mz_max);
      cand.push_back({g0, 8});
      cand.push_back({g0, 4});
      if (g0 != 32) cand.push_back({32, 8});
      if (iters >= (int)cand.size() + 1) {
        CKN(enqueue_wave_iteration(w, d, prm.dual_mode, cand[0].first, cand[0].second, s, nullptr, nullptr));
        ++done_iters;
        double best = 1e30;
        for (auto& c : cand) {
          CKN(enqueue_wave_iteration(w, d, prm.dual_mode, c.first, c.second, s, zev0, zev1));
          CKN(cudaEventSynchronize(zev1));
          float ms = 0.f;
          CKN(cudaEventElapsedTime(&ms, zev0, zev1));
          ++done_iters;
          if (ms < best) {
            best = ms;
            tuned = Tuned{c.first, c.second, ms};
          }
        }
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[mz_max] = tuned;
      } else {
        tuned = Tuned{g0, 8, 0.0};
      }
    }
    // the rest of the iterations: one CUDA graph per wave, replayed
    if (done_iters < iters) {
      cudaGraph_t g = nullptr;
      CKN(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      cudaError_t ec = enqueue_wave_iteration(w, d, prm.dual_mode, tuned.group, tuned.wpb, cap, nullptr, nullptr);
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
  if (zev0) cudaEventDestroy(zev0);
  if (zev1) cudaEventDestroy(zev1);
  if (cap) cudaStreamDestroy(cap);
  cudaStreamSynchronize(s);
  void* frees[] = {pool, dF, dD, dB, d.items, d.prefix, d.my, d.mz, d.p2, d.mz_blocks, d.fin, d.heads, d.stats};
  for (void* q : frees)
    if (q) cudaFree(q);
  return st;
}
