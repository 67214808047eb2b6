// Batched LAP kernel (one warp per LAP) and the rlt2_lap_batched entry point.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <type_traits>

#include "rlt2_internal.h"
#include "rlt2_lap.cuh"

namespace rlt2 {

int default_group(int m) { return m <= 8 ? 8 : (m <= 16 ? 16 : 32); }

// Grid-stride over LAPs, 32/G LAPs per warp per step.  FX selects the exact
// fixed-point arithmetic (canonical duals), else FP64.
template <int G, bool PRE, bool FX>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32) k_lap(LapArgs a) {
  if (a.skip && *a.skip) return;
  using A = typename std::conditional<FX, ArithFx, ArithF64>::type;
  using T = typename A::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int per = 32 / G;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int grp = lane / G, gl = lane & (G - 1);
  const int m = a.m;
  const int ld = tile_ld(m);
  unsigned char* base = smem_raw + (size_t)wib * warp_smem_bytes(m, G);
  T* tile = reinterpret_cast<T*>(base) + (size_t)grp * m * ld;
  T* uv = reinterpret_cast<T*>(base) + (size_t)per * m * ld;  // [0..31] u, [32..63] v
  int* scr = reinterpret_cast<int*>(uv + 64) + grp * G;
  const bool warm = a.u0 != nullptr && (a.warm_gate == nullptr || *a.warm_gate != 0);
  const long long nwarps = (long long)gridDim.x * wpb;
  const int mm = m * m;
  unsigned long long aug_acc = 0, relax_acc = 0;

  for (long long t0 = ((long long)blockIdx.x * wpb + wib) * per; t0 < a.batch; t0 += nwarps * per) {
    const long long tb = t0 + grp;
    const bool have = tb < a.batch;
    const long long t = (have && a.map) ? (long long)a.map[tb] : tb;
    const int L = stage_tile<G, FX>(tile, ld, m, gl, have ? a.A + t * mm : nullptr,
                                    (have && a.Badd) ? a.Badd + t * mm : nullptr);
    T u0 = T(0);
    if (warm && have && gl < m) u0 = start_dual<FX>(a.u0[t * m + gl], L);
    __syncwarp();
    // without a reduced-cost output (PRE) the tile may be overwritten by the canonical pass
    const WarpLapResult<T> R =
        group_lap<G, PRE, A>(tile, ld, have ? m : 0, lane, warm, u0, a.dual_mode, scr, uv + grp * G);
    if (have && gl < m) {
      if (a.u) a.u[t * m + gl] = out_value<FX>(R.u, L);
      if (a.v) a.v[t * m + gl] = out_value<FX>(R.v, L);
      if (a.r2c) a.r2c[t * m + gl] = R.r2c;
    }
    if (have && gl == 0) {
      a.value[t] = out_value<FX>(R.value, L);
      if (a.naug) a.naug[t] = R.naug;
      aug_acc += R.naug;
      relax_acc += R.nrelax;
    }
    if (a.pi) {
      uv[lane] = R.u;
      uv[32 + lane] = R.v;
      __syncwarp();
      if (have) {
        double* dst = a.pi + t * mm;
        const T* ug = uv + grp * G;
        const T* vg = uv + 32 + grp * G;
        for (int e = gl; e < mm; e += G) {
          const int r = e / m, c = e - r * m;
          dst[e] = out_value<FX>(A::sub(A::sub(tile[r * ld + c], ug[r]), vg[c]), L);
        }
      }
    }
    __syncwarp();
  }
  if (a.stats && gl == 0 && (aug_acc | relax_acc)) {
    atomicAdd(a.stats + 0, aug_acc);
    atomicAdd(a.stats + 1, relax_acc);
  }
}

// blocks per SM for (m, G, warps per block), 0 = not configured
// Launch configuration (occupancy per size, shared-memory attributes), set once
// per (size, group, warps) under g_cfg_mu: contexts may be created and used
// from different host threads.
static std::mutex g_cfg_mu;
static int g_occ[33][3][2];

static int gidx(int G) { return G == 8 ? 0 : (G == 16 ? 1 : 2); }

using LapKernel = void (*)(LapArgs);

// The kernel for (group, in-place canonical pass, fixed-point arithmetic).
template <int G>
static LapKernel lap_kernel(bool pre, bool fx) {
  if (pre) return fx ? k_lap<G, true, true> : k_lap<G, true, false>;
  return fx ? k_lap<G, false, true> : k_lap<G, false, false>;
}
static LapKernel lap_kernel(int G, bool pre, bool fx) {
  return G == 8 ? lap_kernel<8>(pre, fx) : (G == 16 ? lap_kernel<16>(pre, fx) : lap_kernel<32>(pre, fx));
}

// Occupancy of the slowest of the four forms, so that one grid size serves all.
static cudaError_t prepare_one(int G, int m, int wpb) {
  int& slot = g_occ[m][gidx(G)][wpb == 4 ? 0 : 1];
  if (slot > 0) return cudaSuccess;
  static bool attr_set[3] = {false, false, false};
  cudaError_t e;
  const int cap = (int)(warp_smem_bytes(32, 32) * kMaxWarpsPerBlock);
  int occ = 1 << 20;
  for (int k = 0; k < 4; ++k) {
    const LapKernel kern = lap_kernel(G, (k & 1) != 0, (k & 2) != 0);
    if (!attr_set[gidx(G)]) {
      if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cap)) != cudaSuccess)
        return e;
    }
    int o = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, wpb * 32, warp_smem_bytes(m, G) * wpb);
    if (e != cudaSuccess) return e;
    occ = o < occ ? o : occ;
  }
  attr_set[gidx(G)] = true;
  slot = occ < 1 ? 1 : occ;
  return cudaSuccess;
}

static int g_sms = 0;

cudaError_t prepare_lap(int m, int group, int warps_per_block) {
  if (m < 1 || m > 32) return cudaErrorInvalidValue;
  const int G = group ? group : default_group(m);
  const int wpb = warps_per_block ? warps_per_block : kMaxWarpsPerBlock;
  if (G < m || (G != 8 && G != 16 && G != 32) || (wpb != 4 && wpb != 8)) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lock(g_cfg_mu);
  cudaError_t e;
  if (!g_sms) {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  }
  return prepare_one(G, m, wpb);
}

cudaError_t launch_lap(const LapArgs& a, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  const int G = a.group ? a.group : default_group(a.m);
  const int wpb = a.warps_per_block ? a.warps_per_block : kMaxWarpsPerBlock;
  cudaError_t e = prepare_lap(a.m, G, wpb);
  if (e != cudaSuccess) return e;
  const size_t smem = warp_smem_bytes(a.m, G) * wpb;
  const long long per_block = (long long)wpb * (32 / G);
  const long long need = (a.batch + per_block - 1) / per_block;
  const long long cap = (long long)g_sms * g_occ[a.m][gidx(G)][wpb == 4 ? 0 : 1];
  const int grid = (int)(need < cap ? need : cap);
  const LapKernel kern = lap_kernel(G, a.pi == nullptr, a.dual_mode == 1);
  kern<<<grid, wpb * 32, smem, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched branch-and-bound nodes: one persistent launch per stage over the LAPs
// of every node of a wave.  Warps pull 32/G LAPs at a time from a device queue
// (atomic head, no waiting), so nodes of uneven size share the GPU.
template <int G, bool PRE, bool FX>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32) k_lap_nodes(NodeLapArgs a) {
  using A = typename std::conditional<FX, ArithFx, ArithF64>::type;
  using T = typename A::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int per = 32 / G;
  long long* s_prefix = reinterpret_cast<long long*>(smem_raw);
  for (int i = threadIdx.x; i <= a.nnodes; i += blockDim.x) s_prefix[i] = a.prefix[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane & (G - 1);
  const size_t pre = (((size_t)(a.nnodes + 1) * sizeof(long long)) + 255) & ~size_t(255);
  const int MM = a.max_m;
  unsigned char* base = smem_raw + pre + (size_t)wib * warp_smem_bytes(MM, G);
  T* tile = reinterpret_cast<T*>(base) + (size_t)grp * MM * tile_ld(MM);
  T* uv = reinterpret_cast<T*>(base) + (size_t)per * MM * tile_ld(MM);
  int* scr = reinterpret_cast<int*>(uv + 64) + grp * G;
  unsigned long long aug_acc = 0, relax_acc = 0;
  for (;;) {
    unsigned long long b0 = 0;
    if (lane == 0) b0 = atomicAdd(a.head, (unsigned long long)per);
    b0 = __shfl_sync(kFull, b0, 0);
    if (b0 >= (unsigned long long)a.total) break;
    const long long t = (long long)b0 + grp;
    bool have = t < a.total;
    int k = 0;
    long long li = 0;
    NodeLapItem it{};
    if (have) {
      int lo = 0, hi = a.nnodes - 1;
      while (lo < hi) {  // largest k with prefix[k] <= t
        const int mid = (lo + hi + 1) >> 1;
        if (s_prefix[mid] <= t) lo = mid;
        else hi = mid - 1;
      }
      k = lo;
      it = a.items[k];
      li = RLT2_IDX(t - s_prefix[k], it.count);
      if (*it.skip) have = false;
    }
    const int m = have ? it.m : 0;
    const int ld = tile_ld(m);
    const int mm = m * m;
    const int L = stage_tile<G, FX>(tile, ld, m, gl, have ? it.A + li * mm : nullptr,
                                    (have && it.Badd) ? it.Badd + li * mm : nullptr);
    const bool warm = have && it.u0 != nullptr && (it.warm_gate == nullptr || *it.warm_gate != 0);
    const T u0 = (warm && gl < m) ? start_dual<FX>(it.u0[li * m + gl], L) : T(0);
    __syncwarp();
    const WarpLapResult<T> R = group_lap<G, PRE, A>(tile, ld, m, lane, warm, u0, a.dual_mode, scr, uv + grp * G);
    if (have && gl < m) {
      if (it.u) it.u[li * m + gl] = out_value<FX>(R.u, L);
      if (it.v) it.v[li * m + gl] = out_value<FX>(R.v, L);
      if (it.r2c) it.r2c[li * m + gl] = R.r2c;
    }
    if (have && gl == 0) {
      it.value[li] = out_value<FX>(R.value, L);
      aug_acc += R.naug;
      relax_acc += R.nrelax;
    }
    uv[lane] = R.u;
    uv[32 + lane] = R.v;
    __syncwarp();
    if (have && it.pi) {
      double* dst = it.pi + li * mm;
      const T* ug = uv + grp * G;
      const T* vg = uv + 32 + grp * G;
      for (int e = gl; e < mm; e += G) {
        const int r = e / m, c = e - r * m;
        dst[e] = out_value<FX>(A::sub(A::sub(tile[r * ld + c], ug[r]), vg[c]), L);
      }
    }
    __syncwarp();
  }
  if (a.stats && gl == 0 && (aug_acc | relax_acc)) {
    atomicAdd(a.stats + 0, aug_acc);
    atomicAdd(a.stats + 1, relax_acc);
  }
}

using NodeLapKernel = void (*)(NodeLapArgs);

template <int G>
static NodeLapKernel node_lap_kernel(bool pre, bool fx) {
  if (pre) return fx ? k_lap_nodes<G, true, true> : k_lap_nodes<G, true, false>;
  return fx ? k_lap_nodes<G, false, true> : k_lap_nodes<G, false, false>;
}
static NodeLapKernel node_lap_kernel(int G, bool pre, bool fx) {
  return G == 8 ? node_lap_kernel<8>(pre, fx) : (G == 16 ? node_lap_kernel<16>(pre, fx) : node_lap_kernel<32>(pre, fx));
}

static int g_occ_nodes[33][3][2];

cudaError_t launch_lap_nodes(const NodeLapArgs& a, cudaStream_t s) {
  if (a.total <= 0) return cudaSuccess;
  if (a.max_m < 1 || a.max_m > 32 || a.nnodes < 1 || a.nnodes > kMaxWaveNodes) return cudaErrorInvalidValue;
  const int G = a.group ? a.group : default_group(a.max_m);
  const int wpb = a.warps_per_block ? a.warps_per_block : kMaxWarpsPerBlock;
  if (G < a.max_m || (wpb != 4 && wpb != 8)) return cudaErrorInvalidValue;
  const size_t pre = (((size_t)(a.nnodes + 1) * sizeof(long long)) + 255) & ~size_t(255);
  const size_t smem = pre + warp_smem_bytes(a.max_m, G) * wpb;
  cudaError_t e;
  std::unique_lock<std::mutex> lock(g_cfg_mu);
  if (!g_sms) {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  }
  static bool attr_set[3] = {false, false, false};
  const size_t cap_smem = (((size_t)(kMaxWaveNodes + 1) * sizeof(long long)) + 255) / 256 * 256 +
                          warp_smem_bytes(32, 32) * kMaxWarpsPerBlock;
  int& occ = g_occ_nodes[a.max_m][gidx(G)][wpb == 4 ? 0 : 1];
  // occupancy of the slowest of the four forms, computed once per size (the
  // prefix table's share of shared memory varies with the node count; a grid
  // above the resident count only queues blocks, which never wait on others)
  if (!occ) {
    int lo = 1 << 20;
    for (int k = 0; k < 4; ++k) {
      const NodeLapKernel kern = node_lap_kernel(G, (k & 1) != 0, (k & 2) != 0);
      if (!attr_set[gidx(G)]) {
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap_smem)) !=
            cudaSuccess)
          return e;
      }
      int o = 0;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, wpb * 32, smem)) != cudaSuccess) return e;
      lo = o < lo ? o : lo;
    }
    attr_set[gidx(G)] = true;
    occ = lo < 1 ? 1 : lo;
  }
  const long long cap = (long long)g_sms * occ;
  lock.unlock();
  const long long per_block = (long long)wpb * (32 / G);
  const long long need = (a.total + per_block - 1) / per_block;
  const int grid = (int)(need < cap ? need : cap);
  const NodeLapKernel kern = node_lap_kernel(G, a.pre, a.dual_mode == 1);
  kern<<<grid, wpb * 32, smem, s>>>(a);
  return cudaGetLastError();
}

RLT2_DEFINE_OOB_QUERY(oob_lap)

}  // namespace rlt2

using namespace rlt2;

extern "C" rlt2_status rlt2_lap_batched(int batch, int m, const double* cost, const double* u0, double* value,
                                        double* u, double* v, int* row_to_col, int* n_aug, int dual_mode,
                                        void* stream) {
  if (batch < 0 || m < 1 || m > 32 || (batch > 0 && (!cost || !value)) || dual_mode < 0 || dual_mode > 2) {
    set_error("rlt2_lap_batched: invalid argument");
    return RLT2_EINVAL;
  }
  if (batch == 0) return RLT2_OK;
  LapArgs a{};
  a.batch = batch;
  a.m = m;
  a.A = cost;
  a.u0 = u0;
  a.value = value;
  a.u = u;
  a.v = v;
  a.r2c = row_to_col;
  a.naug = n_aug;
  a.dual_mode = dual_mode;
  cudaError_t e = launch_lap(a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "rlt2_lap_batched");
  return RLT2_OK;
}
