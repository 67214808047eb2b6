// Batched LAP kernel (one warp per LAP) and the rlt2_lap_batched entry point.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <type_traits>

#include "rlt2_internal.h"
#include "rlt2_lap.cuh"

namespace rlt2 {

int default_group(int m) { return m <= 8 ? 8 : (m <= 16 ? 16 : 32); }

// The fixed-point Z stage with prefetching (a.prefetch): each group's next tile
// and start duals are copied into shared memory by cp.async while the current
// LAP is solved, so the tile's HBM latency is off the warp's path.  The copy
// of tile k+1 is issued as soon as the column reduction of tile k has
// converted its raw entries (group_lap's hook); the grid exponent of a tile is
// the largest exponent field of its raw entries, as in stage_tile.  Results
// are those of the staged form bit for bit.  With a.head set, warps claim
// their next step of 32/G LAPs from that counter (zero at launch) when they
// issue its copies, so that warps whose LAPs needed few searches take more of
// them and all warps end together; otherwise they take a fixed grid stride.
template <int G, bool RR>
__device__ __forceinline__ void k_lap_prefetching(const LapArgs& a, unsigned char* base, int lane, bool warm,
                                                  long long first, long long stride) {
  using A = ArithFx;
  using T = long long;
  constexpr int per = 32 / G;
  const int grp = lane / G, gl = lane & (G - 1);
  const int m = a.m, ld = tile_ld(m), mm = m * m;
  T* tile = reinterpret_cast<T*>(base) + (size_t)grp * m * ld;
  T* uv = reinterpret_cast<T*>(base) + (size_t)per * m * ld;  // [0..31] u, [32..63] v
  int* scr = reinterpret_cast<int*>(uv + 64) + grp * G;
  double* raw = reinterpret_cast<double*>(base + warp_smem_bytes(m, G)) + (size_t)grp * raw_group_doubles(m);
  unsigned long long aug_acc = 0, relax_acc = 0;
  // copies of group grp's tile of the step starting at LAP t0 (nothing past the batch)
  auto issue = [&](long long t0) {
    const long long tb = t0 + grp;
    if (tb < a.batch) {
      const long long t = a.map ? (long long)a.map[tb] : tb;
      const double* src = a.A + t * mm;
      for (int e = gl; e < mm; e += G) cp_async8(raw + e, src + e);
      if (warm && gl < m) cp_async8(raw + mm + gl, a.u0 + t * m + gl);
    }
    cp_async_commit();
  };
  // the first LAP of this warp's next step (every lane of the warp)
  auto claim = [&](long long t_static) -> long long {
    if (a.head == nullptr) return t_static;
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(a.head, (unsigned long long)per);
    return (long long)__shfl_sync(kFull, b, 0);
  };
  long long t0 = claim(first);
  issue(t0);
  while (t0 < a.batch) {
    const long long tb = t0 + grp;
    const bool have = tb < a.batch;
    const long long t = (have && a.map) ? (long long)a.map[tb] : tb;
    cp_async_wait_all();
    __syncwarp();
    unsigned eb = 0;
    if (have)
      for (int e = gl; e < mm; e += G) eb = max(eb, fx_expfield_hi(raw + e));
    if constexpr (G == 32) {
      eb = __reduce_max_sync(kFull, eb);
    } else {
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) eb = max(eb, __shfl_xor_sync(kFull, eb, off));
    }
    const int L = fx_grid(eb);
    T u0 = T(0);
    if (warm && have && gl < m) u0 = start_dual<true>(raw[mm + gl], L);
    long long next = a.batch;  // claimed in the hook, which group_lap calls once (raw is set)
    const WarpLapResult<T> R = group_lap<G, true, A, RR>(tile, ld, have ? m : 0, lane, warm, u0, a.dual_mode, scr,
                                                     uv + grp * G, raw, L, [&]() {
                                                       next = claim(t0 + stride);
                                                       issue(next);
                                                     });
    if (have && gl < m) {
      if (a.u) a.u[t * m + gl] = out_value<true>(R.u, L);
      if (a.v) a.v[t * m + gl] = out_value<true>(R.v, L);
      if (a.r2c) a.r2c[t * m + gl] = R.r2c;
    }
    if (have && gl == 0) {
      a.value[t] = out_value<true>(R.value, L);
      if (a.naug) a.naug[t] = R.naug;
      aug_acc += R.naug;
      relax_acc += R.nrelax;
    }
    __syncwarp();
    t0 = next;
  }
  cp_async_wait_all();  // nothing may be in flight when the warp leaves
  if (a.stats && gl == 0 && (aug_acc | relax_acc)) {
    atomicAdd(a.stats + 0, aug_acc);
    atomicAdd(a.stats + 1, relax_acc);
  }
}

// Grid-stride over LAPs, 32/G LAPs per warp per step.  FX selects the exact
// fixed-point arithmetic (canonical duals), else FP64; RR (fixed point, cold
// launches) reduces the rows of a cold start first.
template <int G, bool PRE, bool FX, bool RR = false>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32) k_lap(LapArgs a) {
  if (a.skip && *a.skip) return;
  using A = typename std::conditional<FX, ArithFx, ArithF64>::type;
  using T = typename A::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if constexpr (FX && PRE) {
    if (a.prefetch) {
      const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
      const bool warm = a.u0 != nullptr && (a.warm_gate == nullptr || *a.warm_gate != 0);
      const long long nwarps = (long long)gridDim.x * wpb;
      k_lap_prefetching<G, RR>(a, smem_raw + (size_t)wib * warp_smem_bytes_async(a.m, G), lane, warm,
                           ((long long)blockIdx.x * wpb + wib) * (32 / G), nwarps * (32 / G));
      return;
    }
  }
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
    // with a reduced-cost output (the Y and X stages: few LAPs, one per warp)
    // the tile's loads are batched
    const int L = stage_tile<G, FX, false, PRE ? 1 : 4>(tile, ld, m, gl, have ? a.A + t * mm : nullptr,
                                                        (have && a.Badd) ? a.Badd + t * mm : nullptr);
    T u0 = T(0);
    if (warm && have && gl < m) u0 = start_dual<FX>(a.u0[t * m + gl], L);
    __syncwarp();
    // without a reduced-cost output (PRE) the tile may be overwritten by the canonical pass
    const WarpLapResult<T> R =
        group_lap<G, PRE, A, RR && FX>(tile, ld, have ? m : 0, lane, warm, u0, a.dual_mode, scr, uv + grp * G);
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
#pragma unroll 4
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

// Launch configuration (SM count, occupancy per size, shared-memory
// attributes), kept per device and set once per (device, size, group, warps)
// under g_cfg_mu: contexts may be created and used from different host threads
// and on different devices.  Like every per-device cache of the library it is
// not valid across a cudaDeviceReset.
static std::mutex g_cfg_mu;
constexpr int kMaxCfgDevices = 64;
struct LapDevCfg {
  int sms = 0;                 // multiprocessors of the device
  int occ[33][3][2] = {};      // blocks per SM for (m, G, warps per block), 0 = not configured
  int occ_nodes[33][3][2] = {};
  bool attr[3] = {};           // dynamic shared-memory attribute set (k_lap, per G)
  bool attr_nodes[3] = {};     // the same for k_lap_nodes
};
static LapDevCfg g_devcfg[kMaxCfgDevices];

// The current device's entry, its SM count read on first use (g_cfg_mu held).
static cudaError_t current_cfg(LapDevCfg** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxCfgDevices) return cudaErrorInvalidDevice;
  LapDevCfg& c = g_devcfg[dev];
  if (!c.sms && (e = cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  *out = &c;
  return cudaSuccess;
}

static int gidx(int G) { return G == 8 ? 0 : (G == 16 ? 1 : 2); }

using LapKernel = void (*)(LapArgs);

// The kernel for (group, in-place canonical pass, fixed-point arithmetic, row
// reduction of cold starts; the last only with fixed point).
template <int G>
static LapKernel lap_kernel(bool pre, bool fx, bool rr) {
  if (fx && rr) return pre ? k_lap<G, true, true, true> : k_lap<G, false, true, true>;
  if (pre) return fx ? k_lap<G, true, true> : k_lap<G, true, false>;
  return fx ? k_lap<G, false, true> : k_lap<G, false, false>;
}
static LapKernel lap_kernel(int G, bool pre, bool fx, bool rr) {
  return G == 8 ? lap_kernel<8>(pre, fx, rr) : (G == 16 ? lap_kernel<16>(pre, fx, rr) : lap_kernel<32>(pre, fx, rr));
}

// Occupancy of the slowest of the six forms, so that one grid size serves all.
static cudaError_t prepare_one(LapDevCfg& cfg, int G, int m, int wpb) {
  int& slot = cfg.occ[m][gidx(G)][wpb == 4 ? 0 : 1];
  if (slot > 0) return cudaSuccess;
  bool* attr_set = cfg.attr;
  cudaError_t e;
  const int cap = (int)(warp_smem_bytes_async(32, 32) * kMaxWarpsPerBlock);
  int occ = 1 << 20;
  for (int k = 0; k < 6; ++k) {
    const bool pre = (k & 1) != 0, fx = (k & 2) != 0 || k >= 4, rr = k >= 4;
    const LapKernel kern = lap_kernel(G, pre, fx, rr);
    if (!attr_set[gidx(G)]) {
      if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cap)) != cudaSuccess)
        return e;
    }
    int o = 0;
    // the prefetching form (fixed point, no reduced-cost output) needs more shared memory
    const size_t per_warp = (pre && fx) ? warp_smem_bytes_async(m, G) : warp_smem_bytes(m, G);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, wpb * 32, per_warp * wpb);
    if (e != cudaSuccess) return e;
    occ = o < occ ? o : occ;
  }
  attr_set[gidx(G)] = true;
  slot = occ < 1 ? 1 : occ;
  return cudaSuccess;
}

// Configures (once per device) the launch of an m-column LAP; *cap (nullable)
// receives the resident block count of that launch on the current device.
static cudaError_t prepare_cap(int m, int group, int warps_per_block, long long* cap) {
  if (m < 1 || m > 32) return cudaErrorInvalidValue;
  const int G = group ? group : default_group(m);
  const int wpb = warps_per_block ? warps_per_block : kMaxWarpsPerBlock;
  if (G < m || (G != 8 && G != 16 && G != 32) || (wpb != 4 && wpb != 8)) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lock(g_cfg_mu);
  LapDevCfg* cfg = nullptr;
  cudaError_t e = current_cfg(&cfg);
  if (e != cudaSuccess) return e;
  if ((e = prepare_one(*cfg, G, m, wpb)) != cudaSuccess) return e;
  if (cap) *cap = (long long)cfg->sms * cfg->occ[m][gidx(G)][wpb == 4 ? 0 : 1];
  return cudaSuccess;
}

cudaError_t prepare_lap(int m, int group, int warps_per_block) {
  return prepare_cap(m, group, warps_per_block, nullptr);
}

cudaError_t launch_lap(const LapArgs& a, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  const int G = a.group ? a.group : default_group(a.m);
  const int wpb = a.warps_per_block ? a.warps_per_block : kMaxWarpsPerBlock;
  long long cap = 0;
  cudaError_t e = prepare_cap(a.m, G, wpb, &cap);
  if (e != cudaSuccess) return e;
  LapArgs b = a;
  b.prefetch = (a.dual_mode == 1 && a.pi == nullptr && a.Badd == nullptr) ? 1 : 0;
  const size_t smem = (b.prefetch ? warp_smem_bytes_async(a.m, G) : warp_smem_bytes(a.m, G)) * wpb;
  const long long per_block = (long long)wpb * (32 / G);
  const long long need = (a.batch + per_block - 1) / per_block;
  const int grid = (int)(need < cap ? need : cap);
  // a cold fixed-point launch reduces the rows first (the same canonical result)
  const LapKernel kern = lap_kernel(G, a.pi == nullptr, a.dual_mode == 1, a.dual_mode == 1 && a.u0 == nullptr);
  if (!b.prefetch) b.head = nullptr;
  if (b.head && !b.head_zeroed && (e = cudaMemsetAsync(b.head, 0, sizeof(unsigned long long), s)) != cudaSuccess)
    return e;
  kern<<<grid, wpb * 32, smem, s>>>(b);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched branch-and-bound nodes: one persistent launch per stage over the LAPs
// of every node of a wave.  Warps pull 32/G LAPs at a time from a device queue
// (atomic head, no waiting), so nodes of uneven size share the GPU.
// The queue-fed node form of k_lap_prefetching (fixed point, Z stages): a
// warp claims its next queue slot before it solves the current one and copies
// that slot's tiles and start duals into shared memory by cp.async (issued by
// group_lap's hook once the current raw tiles are converted).  The raw buffers
// are sized for the largest LAP of the stage.  Results are those of the staged
// form bit for bit (each LAP is independent of which warp solves it).
template <int G, bool RR>
__device__ __forceinline__ void k_lap_nodes_prefetching(const NodeLapArgs& a, const long long* s_prefix,
                                                        unsigned char* base, int lane) {
  using A = ArithFx;
  using T = long long;
  constexpr int per = 32 / G;
  const int grp = lane / G, gl = lane & (G - 1);
  const int MM = a.max_m;
  T* tile = reinterpret_cast<T*>(base) + (size_t)grp * MM * tile_ld(MM);
  T* uv = reinterpret_cast<T*>(base) + (size_t)per * MM * tile_ld(MM);
  int* scr = reinterpret_cast<int*>(uv + 64) + grp * G;
  double* raw = reinterpret_cast<double*>(base + warp_smem_bytes(MM, G)) + (size_t)grp * raw_group_doubles(MM);
  unsigned long long aug_acc = 0, relax_acc = 0;
  // the queue slot's LAP of this group: node k, LAP li of that node (have = false past the end or for a
  // stopped node)
  struct Slot {
    bool have, warm;
    int k;
    long long li;
  };
  auto lookup = [&](unsigned long long b0) {
    Slot sl{false, false, 0, 0};
    const long long t = (long long)b0 + grp;
    if (b0 < (unsigned long long)a.total && t < a.total) {
      int lo = 0, hi = a.nnodes - 1;
      while (lo < hi) {  // largest k with prefix[k] <= t
        const int mid = (lo + hi + 1) >> 1;
        if (s_prefix[mid] <= t) lo = mid;
        else hi = mid - 1;
      }
      sl.k = lo;
      const NodeLapItem& it = a.items[lo];
      sl.li = RLT2_IDX(t - s_prefix[lo], it.count);
      sl.have = *it.skip == 0;
      sl.warm = sl.have && it.u0 != nullptr && (it.warm_gate == nullptr || *it.warm_gate != 0);
    }
    return sl;
  };
  auto grab = [&]() {
    unsigned long long b0 = 0;
    if (lane == 0) b0 = atomicAdd(a.head, (unsigned long long)per);
    return __shfl_sync(kFull, b0, 0);
  };
  auto issue = [&](const Slot& sl) {
    if (sl.have) {
      const NodeLapItem& it = a.items[sl.k];
      const int m = it.m, mm = m * m;
      const double* src = it.A + sl.li * mm;
      for (int e = gl; e < mm; e += G) cp_async8(raw + e, src + e);
      if (sl.warm && gl < m) cp_async8(raw + mm + gl, it.u0 + sl.li * m + gl);
    }
    cp_async_commit();
  };
  unsigned long long b0 = grab();
  Slot cur = lookup(b0);
  issue(cur);
  while (b0 < (unsigned long long)a.total) {
    const unsigned long long b1 = grab();
    const Slot nxt = lookup(b1);
    cp_async_wait_all();
    __syncwarp();
    const int m = cur.have ? a.items[cur.k].m : 0;
    const int mm = m * m;
    unsigned eb = 0;
    for (int e = gl; e < mm; e += G) eb = max(eb, fx_expfield_hi(raw + e));
    if constexpr (G == 32) {
      eb = __reduce_max_sync(kFull, eb);
    } else {
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) eb = max(eb, __shfl_xor_sync(kFull, eb, off));
    }
    const int L = fx_grid(eb);
    const T u0 = (cur.warm && gl < m) ? start_dual<true>(raw[mm + gl], L) : T(0);
    const WarpLapResult<T> R = group_lap<G, true, A, RR>(tile, tile_ld(m), m, lane, cur.warm, u0, a.dual_mode, scr,
                                                     uv + grp * G, raw, L, [&]() { issue(nxt); });
    if (cur.have) {
      const NodeLapItem& it = a.items[cur.k];
      if (gl < m) {
        if (it.u) it.u[cur.li * m + gl] = out_value<true>(R.u, L);
        if (it.v) it.v[cur.li * m + gl] = out_value<true>(R.v, L);
        if (it.r2c) it.r2c[cur.li * m + gl] = R.r2c;
      }
      if (gl == 0) {
        it.value[cur.li] = out_value<true>(R.value, L);
        aug_acc += R.naug;
        relax_acc += R.nrelax;
      }
    }
    __syncwarp();
    b0 = b1;
    cur = nxt;
  }
  cp_async_wait_all();  // nothing may be in flight when the warp leaves
  if (a.stats && gl == 0 && (aug_acc | relax_acc)) {
    atomicAdd(a.stats + 0, aug_acc);
    atomicAdd(a.stats + 1, relax_acc);
  }
}

template <int G, bool PRE, bool FX, bool RR = false>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32) k_lap_nodes(NodeLapArgs a) {
  using A = typename std::conditional<FX, ArithFx, ArithF64>::type;
  using T = typename A::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int per = 32 / G;
  long long* s_prefix = reinterpret_cast<long long*>(smem_raw);
  for (int i = threadIdx.x; i <= a.nnodes; i += blockDim.x) s_prefix[i] = a.prefix[i];
  __syncthreads();
  if constexpr (PRE && FX) {
    if (a.prefetch) {
      const size_t pre = (((size_t)(a.nnodes + 1) * sizeof(long long)) + 255) & ~size_t(255);
      k_lap_nodes_prefetching<G, RR>(a, s_prefix,
                                 smem_raw + pre + (size_t)(threadIdx.x >> 5) * warp_smem_bytes_async(a.max_m, G),
                                 threadIdx.x & 31);
      return;
    }
  }
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
    const WarpLapResult<T> R =
        group_lap<G, PRE, A, RR && FX>(tile, ld, m, lane, warm, u0, a.dual_mode, scr, uv + grp * G);
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
static NodeLapKernel node_lap_kernel(bool pre, bool fx, bool rr) {
  if (fx && rr) return pre ? k_lap_nodes<G, true, true, true> : k_lap_nodes<G, false, true, true>;
  if (pre) return fx ? k_lap_nodes<G, true, true> : k_lap_nodes<G, true, false>;
  return fx ? k_lap_nodes<G, false, true> : k_lap_nodes<G, false, false>;
}
static NodeLapKernel node_lap_kernel(int G, bool pre, bool fx, bool rr) {
  return G == 8 ? node_lap_kernel<8>(pre, fx, rr)
                : (G == 16 ? node_lap_kernel<16>(pre, fx, rr) : node_lap_kernel<32>(pre, fx, rr));
}

cudaError_t launch_lap_nodes(const NodeLapArgs& a, cudaStream_t s) {
  if (a.total <= 0) return cudaSuccess;
  if (a.max_m < 1 || a.max_m > 32 || a.nnodes < 1 || a.nnodes > kMaxWaveNodes) return cudaErrorInvalidValue;
  const int G = a.group ? a.group : default_group(a.max_m);
  const int wpb = a.warps_per_block ? a.warps_per_block : kMaxWarpsPerBlock;
  if (G < a.max_m || (wpb != 4 && wpb != 8)) return cudaErrorInvalidValue;
  const size_t pre = (((size_t)(a.nnodes + 1) * sizeof(long long)) + 255) & ~size_t(255);
  NodeLapArgs b = a;
  b.prefetch = (a.pre && a.dual_mode == 1) ? 1 : 0;
  const size_t per_warp = b.prefetch ? warp_smem_bytes_async(a.max_m, G) : warp_smem_bytes(a.max_m, G);
  const size_t smem = pre + per_warp * wpb;
  cudaError_t e;
  std::unique_lock<std::mutex> lock(g_cfg_mu);
  LapDevCfg* cfg = nullptr;
  if ((e = current_cfg(&cfg)) != cudaSuccess) return e;
  bool* attr_set = cfg->attr_nodes;
  const size_t cap_smem = (((size_t)(kMaxWaveNodes + 1) * sizeof(long long)) + 255) / 256 * 256 +
                          warp_smem_bytes_async(32, 32) * kMaxWarpsPerBlock;
  int& occ = cfg->occ_nodes[a.max_m][gidx(G)][wpb == 4 ? 0 : 1];
  // occupancy of the slowest of the six forms, computed once per size (the
  // prefix table's share of shared memory varies with the node count; a grid
  // above the resident count only queues blocks, which never wait on others)
  if (!occ) {
    int lo = 1 << 20;
    for (int k = 0; k < 6; ++k) {
      const bool kpre = (k & 1) != 0, kfx = (k & 2) != 0 || k >= 4;
      const NodeLapKernel kern = node_lap_kernel(G, kpre, kfx, k >= 4);
      if (!attr_set[gidx(G)]) {
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap_smem)) !=
            cudaSuccess)
          return e;
      }
      int o = 0;
      const size_t ksmem =
          pre + (kpre && kfx ? warp_smem_bytes_async(a.max_m, G) : warp_smem_bytes(a.max_m, G)) * wpb;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, wpb * 32, ksmem)) != cudaSuccess) return e;
      lo = o < lo ? o : lo;
    }
    attr_set[gidx(G)] = true;
    occ = lo < 1 ? 1 : lo;
  }
  const long long cap = (long long)cfg->sms * occ;
  lock.unlock();
  const long long per_block = (long long)wpb * (32 / G);
  const long long need = (a.total + per_block - 1) / per_block;
  const int grid = (int)(need < cap ? need : cap);
  const NodeLapKernel kern = node_lap_kernel(G, a.pre, a.dual_mode == 1, a.cold && a.dual_mode == 1);
  kern<<<grid, wpb * 32, smem, s>>>(b);
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
  const cudaStream_t s = (cudaStream_t)stream;
  // the fixed-point form's LAP queue: 8 stream-ordered bytes, freed after the launch
  // (without them the warps take a fixed stride; the results are the same)
  unsigned long long* head = nullptr;
  if (dual_mode == 1 && cudaMallocAsync((void**)&head, sizeof(unsigned long long), s) != cudaSuccess) {
    (void)cudaGetLastError();
    head = nullptr;
  }
  a.head = head;
  cudaError_t e = launch_lap(a, s);
  if (head) {
    const cudaError_t ef = cudaFreeAsync(head, s);
    if (e == cudaSuccess) e = ef;
  }
  if (e != cudaSuccess) return cuda_fail(e, "rlt2_lap_batched");
  return RLT2_OK;
}
