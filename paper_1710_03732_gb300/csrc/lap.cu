// Batched LAP kernel (one warp per LAP) and the rlt2_lap_batched entry point.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "rlt2_internal.h"
#include "rlt2_lap.cuh"

namespace rlt2 {

constexpr int kMaxWarpsPerBlock = 8;

__host__ __device__ inline int tile_ld(int m) { return m | 1; }  // odd stride: conflict-free rows and columns

// Shared memory per warp: 32/G tiles, u/v staging (64 doubles) and 32 ints.
__host__ __device__ inline size_t warp_smem_bytes(int m, int G) {
  return (size_t)(32 / G) * m * tile_ld(m) * sizeof(double) + 64 * sizeof(double) + 32 * sizeof(int);
}

int default_group(int m) { return m <= 8 ? 8 : (m <= 16 ? 16 : 32); }

// Grid-stride over LAPs, 32/G LAPs per warp per step; each group of G lanes
// stages its own tile (coalesced: a group reads a contiguous m*m run).
template <int G, bool PRE>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32) k_lap(LapArgs a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int per = 32 / G;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int grp = lane / G, gl = lane & (G - 1);
  const int m = a.m;
  const int ld = tile_ld(m);
  unsigned char* base = smem_raw + (size_t)wib * warp_smem_bytes(m, G);
  double* tile = reinterpret_cast<double*>(base) + (size_t)grp * m * ld;
  double* uv = reinterpret_cast<double*>(base) + (size_t)per * m * ld;  // [0..31] u, [32..63] v
  int* scr = reinterpret_cast<int*>(uv + 64) + grp * G;
  const bool warm = a.u0 != nullptr && (a.warm_gate == nullptr || *a.warm_gate != 0);
  const long long nwarps = (long long)gridDim.x * wpb;
  const int mm = m * m;
  unsigned long long aug_acc = 0, relax_acc = 0;

  for (long long t0 = ((long long)blockIdx.x * wpb + wib) * per; t0 < a.batch; t0 += nwarps * per) {
    const long long tb = t0 + grp;
    const bool have = tb < a.batch;
    const long long t = (have && a.map) ? (long long)a.map[tb] : tb;
    if (have) {
      const double* src = a.A + t * mm;
      const double* add = a.Badd ? a.Badd + t * mm : nullptr;
      for (int e = gl; e < mm; e += G) {
        const int r = e / m, c = e - r * m;
        double x = __ldcs(src + e);
        if (add) x = __dadd_rn(x, __ldcs(add + e));
        tile[r * ld + c] = x;
      }
    }
    double u0 = 0.0;
    if (warm && have && gl < m) u0 = a.u0[t * m + gl];
    __syncwarp();
    // without a reduced-cost output (PRE) the tile may be overwritten by the canonical pass
    const WarpLapResult R = group_lap<G, PRE>(tile, ld, have ? m : 0, lane, warm, u0, a.dual_mode, scr, uv + grp * G);
    if (have && gl < m) {
      if (a.u) a.u[t * m + gl] = R.u;
      if (a.v) a.v[t * m + gl] = R.v;
      if (a.r2c) a.r2c[t * m + gl] = R.r2c;
    }
    if (have && gl == 0) {
      a.value[t] = R.value;
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
        const double* ug = uv + grp * G;
        const double* vg = uv + 32 + grp * G;
        for (int e = gl; e < mm; e += G) {
          const int r = e / m, c = e - r * m;
          dst[e] = __dsub_rn(__dsub_rn(tile[r * ld + c], ug[r]), vg[c]);
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

template <int G>
static cudaError_t prepare_one(int m, int wpb) {
  int& slot = g_occ[m][gidx(G)][wpb == 4 ? 0 : 1];
  if (slot > 0) return cudaSuccess;
  static bool attr_set[3] = {false, false, false};
  cudaError_t e;
  const int cap = (int)(warp_smem_bytes(32, 32) * kMaxWarpsPerBlock);
  if (!attr_set[gidx(G)]) {
    if ((e = cudaFuncSetAttribute(k_lap<G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_lap<G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap)) != cudaSuccess)
      return e;
    attr_set[gidx(G)] = true;
  }
  int occ = 0, occ2 = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lap<G, true>, wpb * 32, warp_smem_bytes(m, G) * wpb);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_lap<G, false>, wpb * 32, warp_smem_bytes(m, G) * wpb);
  if (e != cudaSuccess) return e;
  occ = occ < occ2 ? occ : occ2;
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
  if (G == 8) return prepare_one<8>(m, wpb);
  if (G == 16) return prepare_one<16>(m, wpb);
  return prepare_one<32>(m, wpb);
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
  const bool pre = a.pi == nullptr;
  if (G == 8) {
    if (pre) k_lap<8, true><<<grid, wpb * 32, smem, s>>>(a);
    else k_lap<8, false><<<grid, wpb * 32, smem, s>>>(a);
  } else if (G == 16) {
    if (pre) k_lap<16, true><<<grid, wpb * 32, smem, s>>>(a);
    else k_lap<16, false><<<grid, wpb * 32, smem, s>>>(a);
  } else {
    if (pre) k_lap<32, true><<<grid, wpb * 32, smem, s>>>(a);
    else k_lap<32, false><<<grid, wpb * 32, smem, s>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched branch-and-bound nodes: one persistent launch per stage over the LAPs
// of every node of a wave.  Warps pull 32/G LAPs at a time from a device queue
// (atomic head, no waiting), so nodes of uneven size share the GPU.
template <int G, bool PRE>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32) k_lap_nodes(NodeLapArgs a) {
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
  double* tile = reinterpret_cast<double*>(base) + (size_t)grp * MM * tile_ld(MM);
  double* uv = reinterpret_cast<double*>(base) + (size_t)per * MM * tile_ld(MM);
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
      li = t - s_prefix[k];
      it = a.items[k];
      if (*it.skip) have = false;
    }
    const int m = have ? it.m : 0;
    const int ld = tile_ld(m);
    const int mm = m * m;
    if (have) {
      const double* src = it.A + li * mm;
      const double* add = it.Badd ? it.Badd + li * mm : nullptr;
      for (int e = gl; e < mm; e += G) {
        const int r = e / m, c = e - r * m;
        double x = __ldcs(src + e);
        if (add) x = __dadd_rn(x, __ldcs(add + e));
        tile[r * ld + c] = x;
      }
    }
    const bool warm = have && it.u0 != nullptr && (it.warm_gate == nullptr || *it.warm_gate != 0);
    const double u0 = (warm && gl < m) ? it.u0[li * m + gl] : 0.0;
    __syncwarp();
    const WarpLapResult R = group_lap<G, PRE>(tile, ld, m, lane, warm, u0, a.dual_mode, scr, uv + grp * G);
    if (have && gl < m) {
      if (it.u) it.u[li * m + gl] = R.u;
      if (it.v) it.v[li * m + gl] = R.v;
      if (it.r2c) it.r2c[li * m + gl] = R.r2c;
    }
    if (have && gl == 0) {
      it.value[li] = R.value;
      aug_acc += R.naug;
      relax_acc += R.nrelax;
    }
    uv[lane] = R.u;
    uv[32 + lane] = R.v;
    __syncwarp();
    if (have && it.pi) {
      double* dst = it.pi + li * mm;
      const double* ug = uv + grp * G;
      const double* vg = uv + 32 + grp * G;
      for (int e = gl; e < mm; e += G) {
        const int r = e / m, c = e - r * m;
        dst[e] = __dsub_rn(__dsub_rn(tile[r * ld + c], ug[r]), vg[c]);
      }
    }
    __syncwarp();
  }
  if (a.stats && gl == 0 && (aug_acc | relax_acc)) {
    atomicAdd(a.stats + 0, aug_acc);
    atomicAdd(a.stats + 1, relax_acc);
  }
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
  auto setup = [&](auto kern) -> cudaError_t {
    cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap_smem);
    if (e2 != cudaSuccess) return e2;
    int o = 0;
    e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, wpb * 32, smem);
    if (e2 != cudaSuccess) return e2;
    if (!occ || o < occ) occ = o;
    return cudaSuccess;
  };
  if (!attr_set[gidx(G)]) {
    if (G == 8) {
      if ((e = setup(k_lap_nodes<8, true>)) != cudaSuccess || (e = setup(k_lap_nodes<8, false>)) != cudaSuccess) return e;
    } else if (G == 16) {
      if ((e = setup(k_lap_nodes<16, true>)) != cudaSuccess || (e = setup(k_lap_nodes<16, false>)) != cudaSuccess)
        return e;
    } else {
      if ((e = setup(k_lap_nodes<32, true>)) != cudaSuccess || (e = setup(k_lap_nodes<32, false>)) != cudaSuccess)
        return e;
    }
    attr_set[gidx(G)] = true;
  } else if (!occ) {
    int o1 = 0, o2 = 0;
    if (G == 8) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_lap_nodes<8, true>, wpb * 32, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_lap_nodes<8, false>, wpb * 32, smem);
    } else if (G == 16) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_lap_nodes<16, true>, wpb * 32, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_lap_nodes<16, false>, wpb * 32, smem);
    } else {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_lap_nodes<32, true>, wpb * 32, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_lap_nodes<32, false>, wpb * 32, smem);
    }
    occ = o1 < o2 ? o1 : o2;
  }
  if (occ < 1) occ = 1;
  const long long cap = (long long)g_sms * occ;
  lock.unlock();
  const long long per_block = (long long)wpb * (32 / G);
  const long long need = (a.total + per_block - 1) / per_block;
  const int grid = (int)(need < cap ? need : cap);
  if (G == 8) {
    if (a.pre) k_lap_nodes<8, true><<<grid, wpb * 32, smem, s>>>(a);
    else k_lap_nodes<8, false><<<grid, wpb * 32, smem, s>>>(a);
  } else if (G == 16) {
    if (a.pre) k_lap_nodes<16, true><<<grid, wpb * 32, smem, s>>>(a);
    else k_lap_nodes<16, false><<<grid, wpb * 32, smem, s>>>(a);
  } else {
    if (a.pre) k_lap_nodes<32, true><<<grid, wpb * 32, smem, s>>>(a);
    else k_lap_nodes<32, false><<<grid, wpb * 32, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace rlt2

using namespace rlt2;

extern "C" rlt2_status rlt2_lap_batched(int batch, int m, const double* cost, const double* u0, double* value,
                                        double* u, double* v, int* row_to_col, int* n_aug, int dual_mode,
                                        void* stream) {
  if (batch < 0 || m < 1 || m > 32 || (batch > 0 && (!cost || !value)) || (dual_mode != 0 && dual_mode != 1)) {
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
