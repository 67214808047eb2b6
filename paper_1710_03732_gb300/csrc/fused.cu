// The z move of an ascent step (Eq. 2.20-2.23, Section 3.3) and the Z-stage
// LAPs of the next solve (Algorithm 1, Section 3.2) as one persistent launch.
//
// On GB300 the z move is bound by the FP64 pipe and the fixed-point Z-LAPs by
// the integer ALU pipe.  Run back to back, each leaves the other pipe idle;
// here warps of the same SMs run both at once.  The data dependence between
// them is narrow enough to allow it: the entries of Z tile (i,j,p,q) belong to
// the classes {(i,p),(j,q),(k,r)}, which the move handles in its blocks
// (triple, location) whose facility triple holds both i and j, and those same
// blocks are the only readers of the tile's duals.  So once the (n-2) n move
// blocks of facility pair {i,j} are done, the pair's 2 n (n-1) tiles hold their
// final costs and no move reads their duals any more: their LAPs may run
// while the move continues on other pairs.  Every LAP then sees exactly the
// costs and start duals of the two-kernel sequence, so results are identical
// bit for bit.
//
// Warps have roles.  The first kMoveWarps warps of every block take the move's
// (triple, p) blocks from one queue, in triple order, and increment the pair
// counters of each triple they finish; they never wait.  The other warps take
// the Z-LAPs from a second queue, 32/G tiles at a time, tiles grouped by
// facility pair in the order the move completes the pairs, and wait (bounded)
// until their tiles' pair counters are full; once the move queue is empty the
// movers join them.  Every move block is taken by a warp that finishes it
// without waiting, so every wait ends.  The last warp to leave resets the
// queues and counters for the next launch.  (Letting LAP warps run move blocks
// while theirs are not ready was tried: it starts the integer LAPs later and
// was slower.)
//
// Used with rlt2_params.pipeline = 1, off by default: it pays for cold starts
// near n = 20, while elsewhere the LAPs miss the warp slots the movers hold.
#include <algorithm>
#include <mutex>
#include <vector>

#include "rlt2_ascent.cuh"
#include "rlt2_internal.h"
#include "rlt2_lap.cuh"

namespace rlt2 {

// Polls of a pair counter before a LAP warp gives up (about a second with the
// back-off below); a move block takes microseconds, so only a fault gets here.
constexpr int kPipeSpinLimit = 1 << 22;
// The same limit in the failure-detection check, whose waits can never end.
constexpr int kPipeCheckSpinLimit = 1 << 12;
// Warps per block that run the move first (of kMaxWarpsPerBlock): 12 per SM
// keep the FP64 pipe busy through the move's load latencies, the other 20 run
// the integer LAPs (n = 20: 1, 2, 3, 4 tried, 3 fastest).
constexpr int kMoveWarps = 3;

// 64 registers: four blocks of eight warps per SM (80 unbounded: three)
template <int G, bool FX, bool RR = false>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32, 4) k_move_lap_z(MoveZArgs mz, LapArgs a, PipeArgs pa) {
  DevScalars* sc = pa.sc;
  if (sc->done) return;  // stopped: no work, counters untouched
  using A = typename std::conditional<FX, ArithFx, ArithF64>::type;
  using T = typename A::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int per = 32 / G;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane & (G - 1);
  const int m = a.m, n = mz.n, n1 = n - 1;
  const int ld = tile_ld(m);
  unsigned char* base = smem_raw + (size_t)wib * warp_smem_bytes(m, G);
  T* tile = reinterpret_cast<T*>(base) + (size_t)grp * m * ld;
  T* uv = reinterpret_cast<T*>(base) + (size_t)per * m * ld;
  int* scr = reinterpret_cast<int*>(uv + 64) + grp * G;
  const bool moving = sc->have_snap != 0;  // the first solve has no pending move
  const bool warm = moving && a.u0 != nullptr;
  const int mm = m * m;
  const unsigned long long target = (unsigned long long)(n - 2) * n;
  const unsigned long long nmove = (unsigned long long)pa.nmove;
  const unsigned long long nlap = (unsigned long long)((a.batch + per - 1) / per);
  unsigned long long* pair_done = pa.ctr + 4;
  unsigned long long aug_acc = 0, relax_acc = 0;
  bool mover = moving && wib < kMoveWarps;

  for (;;) {
    unsigned long long q = 0;
    if (mover) {
      if (lane == 0) q = atomicAdd(pa.ctr + 0, 1ull);
      q = __shfl_sync(kFull, q, 0);
      if (q >= nmove) {
        mover = false;  // the move is handed out: join the LAPs
        continue;
      }
      // move block (triple, p) = q, its classes across the warp's lanes, then
      // the counters of the triple's three facility pairs
      move_z_block<false, false>(mz, (int)q, lane, 32);  // one warp per block: plain class order
      __threadfence();  // this lane's D^ writes before the pair counters move
      __syncwarp();
      if (lane == 0) {
        const int packed = mz.trips[q / (unsigned long long)n];
        const int f0 = packed & 255, f1 = (packed >> 8) & 255, f2 = packed >> 16;
        atomicAdd(pair_done + f0 * n + f1, 1ull);
        atomicAdd(pair_done + f0 * n + f2, 1ull);
        atomicAdd(pair_done + f1 * n + f2, 1ull);
      }
      continue;
    }
    if (lane == 0) q = atomicAdd(pa.ctr + 2, 1ull);
    q = __shfl_sync(kFull, q, 0);
    if (q >= nlap) break;
    const long long tb = (long long)q * per + grp;
    const bool have = tb < a.batch;
    const long long t = have ? RLT2_IDX((long long)pa.order[tb], a.batch) : 0;
    if (have && moving && gl == 0) {
      // tile t = ((i n + p) (n-1) + j') (n-1) + q': wait for facility pair {i, j}
      const int i = (int)(t / ((long long)n * n1 * n1));
      const int jj = (int)((t / n1) % n1);
      const int j = jj + (jj >= i);
      const volatile unsigned long long* cnt = pair_done + RLT2_IDX(i < j ? i * n + j : j * n + i, n * n);
      const volatile int* stop = &sc->done;
      int spins = 0;
      while (*cnt < target + pa.extra) {
        if (++spins > pa.spin_limit) {
          sc->reason = 4;  // reported as RLT2_ETIMEOUT; the step's results are not used
          sc->done = 1;
          break;
        }
        if (*stop) break;  // another warp gave up: this launch's LAPs are void
        __nanosleep(200);
      }
    }
    __syncwarp();
    __threadfence();
    // after a wait gave up (sc->done is set only then during this launch) the
    // remaining LAPs are skipped, so the launch drains its queue and ends
    const bool live = have && !*(const volatile int*)&sc->done;
    const int L = stage_tile<G, FX, true>(tile, ld, m, gl, live ? a.A + t * mm : nullptr, nullptr);
    T u0 = T(0);
    if (warm && live && gl < m) u0 = start_dual<FX>(a.u0[t * m + gl], L);
    __syncwarp();
    const WarpLapResult<T> R =
        group_lap<G, true, A, RR && FX>(tile, ld, live ? m : 0, lane, warm, u0, a.dual_mode, scr, uv + grp * G);
    if (live && gl < m) {
      a.u[t * m + gl] = out_value<FX>(R.u, L);
      a.v[t * m + gl] = out_value<FX>(R.v, L);
    }
    if (live && gl == 0) {
      a.value[t] = out_value<FX>(R.value, L);
      aug_acc += R.naug;
      relax_acc += R.nrelax;
    }
    __syncwarp();
  }
  if (a.stats && gl == 0 && (aug_acc | relax_acc)) {
    atomicAdd(a.stats + 0, aug_acc);
    atomicAdd(a.stats + 1, relax_acc);
  }
  // the last warp out (every other warp has left the loop) resets the queue
  if (lane == 0) {
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    __threadfence();
    if (atomicAdd(pa.ctr + 1, 1ull) == warps - 1) {
      pa.ctr[0] = 0;
      pa.ctr[1] = 0;
      pa.ctr[2] = 0;
      for (int k = 0; k < n * n; ++k) pair_done[k] = 0;
    }
  }
}

using PipeKernel = void (*)(MoveZArgs, LapArgs, PipeArgs);

// rr: a cold fixed-point launch reduces the rows first (as k_lap does)
template <int G>
static PipeKernel pipe_kernel(bool fx, bool rr) {
  if (fx && rr) return k_move_lap_z<G, true, true>;
  return fx ? k_move_lap_z<G, true> : k_move_lap_z<G, false>;
}
static PipeKernel pipe_kernel(int G, bool fx, bool rr) {
  return G == 8 ? pipe_kernel<8>(fx, rr) : (G == 16 ? pipe_kernel<16>(fx, rr) : pipe_kernel<32>(fx, rr));
}

// Tiles of an n-facility problem sorted by the last move triple of their
// facility pair (triples i < j < k in lexicographic order, as the move's queue
// hands them out).
static void build_pipe_order(int n, std::vector<int>& order) {
  const int n1 = n - 1;
  std::vector<long long> last((size_t)n * n, -1);
  long long ntrip = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      for (int k = j + 1; k < n; ++k, ++ntrip) {
        last[(size_t)i * n + j] = ntrip;
        last[(size_t)i * n + k] = ntrip;
        last[(size_t)j * n + k] = ntrip;
      }
  const long long T = (long long)n * n * n1 * n1;
  std::vector<std::pair<long long, int>> key((size_t)T);
  for (long long t = 0; t < T; ++t) {
    const int i = (int)(t / ((long long)n * n1 * n1));
    const int jj = (int)((t / n1) % n1);
    const int j = jj + (jj >= i);
    key[(size_t)t] = {last[(size_t)std::min(i, j) * n + std::max(i, j)], (int)t};
  }
  std::sort(key.begin(), key.end());
  order.resize((size_t)T);
  for (long long t = 0; t < T; ++t) order[(size_t)t] = key[(size_t)t].second;
}

RLT2_DEFINE_OOB_QUERY(oob_fused)

static std::mutex g_pipe_mu;

const PipePlan* prepare_pipe(int n, cudaError_t* err) {
  static std::vector<std::pair<std::pair<int, int>, PipePlan*>> cache;
  *err = cudaSuccess;
  if (n < 3 || n > 34) {
    *err = cudaErrorInvalidValue;
    return nullptr;
  }
  int dev = 0;
  if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(g_pipe_mu);
  for (auto& kv : cache)
    if (kv.first.first == dev && kv.first.second == n) return kv.second;
  const int m = n - 2, G = default_group(m);
  int sms = 0;
  if ((*err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return nullptr;
  const size_t smem = warp_smem_bytes(m, G) * kMaxWarpsPerBlock;
  const int cap = (int)(warp_smem_bytes(32, 32) * kMaxWarpsPerBlock);
  int occ = 1 << 20;
  for (int k = 0; k < 3; ++k) {  // every form the launch may pick: all co-resident
    const PipeKernel kern = pipe_kernel(G, k >= 1, k == 2);
    if ((*err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cap)) != cudaSuccess)
      return nullptr;
    int o = 0;
    if ((*err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kMaxWarpsPerBlock * 32, smem)) !=
        cudaSuccess)
      return nullptr;
    occ = std::min(occ, o);
  }
  occ = std::max(occ, 1);
  const int grid = sms * occ;
  std::vector<int> order;
  build_pipe_order(n, order);
  int* dorder = nullptr;
  if ((*err = cudaMalloc(&dorder, sizeof(int) * order.size())) != cudaSuccess) return nullptr;
  if ((*err = cudaMemcpy(dorder, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice)) !=
      cudaSuccess) {
    cudaFree(dorder);
    return nullptr;
  }
  PipePlan* plan = new PipePlan();
  plan->n = n;
  plan->order = dorder;
  plan->nmove = (long long)n * (n - 1) * (n - 2) / 6 * n;
  plan->grid = grid;
  cache.push_back({{dev, n}, plan});
  return plan;
}

cudaError_t launch_move_lap_z(const MoveZArgs& mz, const LapArgs& a, const PipePlan& plan, unsigned long long* ctr,
                              DevScalars* sc, cudaStream_t s, bool check) {
  if (a.m < 1 || a.m > 32 || mz.n != a.m + 2 || plan.n != mz.n || mz.half || a.map || a.Badd || a.pi || a.r2c ||
      !a.u || !a.v || !ctr || !sc)
    return cudaErrorInvalidValue;
  const int G = default_group(a.m);
  PipeArgs pa{};
  pa.order = plan.order;
  pa.nmove = plan.nmove;
  pa.ctr = ctr;
  pa.sc = sc;
  pa.spin_limit = check ? kPipeCheckSpinLimit : kPipeSpinLimit;
  pa.extra = check ? 1ull : 0ull;
  const PipeKernel kern = pipe_kernel(G, a.dual_mode == 1, a.dual_mode == 1 && a.u0 == nullptr);
  kern<<<plan.grid, kMaxWarpsPerBlock * 32, warp_smem_bytes(a.m, G) * kMaxWarpsPerBlock, s>>>(mz, a, pa);
  return cudaGetLastError();
}

}  // namespace rlt2
