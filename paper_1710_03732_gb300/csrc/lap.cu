// Batched LAP kernel (one warp per LAP) and the rlt2_lap_batched entry point.
#include <cmath>
#include <cstdio>

#include "rlt2_internal.h"
#include "rlt2_lap.cuh"

namespace rlt2 {

constexpr int kWarpsPerBlock = 8;

__host__ __device__ inline int tile_ld(int m) { return m | 1; }  // odd stride: conflict-free rows and columns

// Shared memory per warp: the tile, u/v staging (64 doubles) and 32 ints.
__host__ __device__ inline size_t warp_smem_bytes(int m) {
  return (size_t)m * tile_ld(m) * sizeof(double) + 64 * sizeof(double) + 32 * sizeof(int);
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_lap(LapArgs a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int m = a.m;
  const int ld = tile_ld(m);
  unsigned char* base = smem_raw + (size_t)wib * warp_smem_bytes(m);
  double* cs = reinterpret_cast<double*>(base);
  double* uv = cs + (size_t)m * ld;  // [0..31] u, [32..63] v
  int* scr = reinterpret_cast<int*>(uv + 64);
  const bool warm = a.u0 != nullptr && (a.warm_gate == nullptr || *a.warm_gate != 0);
  const long long nwarps = (long long)gridDim.x * kWarpsPerBlock;
  const int mm = m * m;
  unsigned long long aug_acc = 0, relax_acc = 0;

  for (long long t = (long long)blockIdx.x * kWarpsPerBlock + wib; t < a.batch; t += nwarps) {
    const double* src = a.A + t * mm;
    const double* add = a.Badd ? a.Badd + t * mm : nullptr;
    for (int e = lane; e < mm; e += 32) {
      const int r = e / m, c = e - r * m;
      double x = __ldcs(src + e);
      if (add) x = __dadd_rn(x, __ldcs(add + e));
      cs[r * ld + c] = x;
    }
    double u0 = 0.0;
    if (warm && lane < m) u0 = a.u0[t * m + lane];
    __syncwarp();
    const WarpLapResult R = warp_lap(cs, ld, m, lane, warm, u0, a.dual_mode, scr);
    if (lane < m) {
      if (a.u) a.u[t * m + lane] = R.u;
      if (a.v) a.v[t * m + lane] = R.v;
      if (a.r2c) a.r2c[t * m + lane] = R.r2c;
    }
    if (lane == 0) {
      a.value[t] = R.value;
      if (a.naug) a.naug[t] = R.naug;
    }
    if (a.pi) {
      uv[lane] = R.u;
      uv[32 + lane] = R.v;
      __syncwarp();
      double* dst = a.pi + t * mm;
      for (int e = lane; e < mm; e += 32) {
        const int r = e / m, c = e - r * m;
        dst[e] = __dsub_rn(__dsub_rn(cs[r * ld + c], uv[r]), uv[32 + c]);
      }
    }
    aug_acc += R.naug;
    relax_acc += R.nrelax;
    __syncwarp();
  }
  if (a.stats && lane == 0 && (aug_acc | relax_acc)) {
    atomicAdd(a.stats + 0, aug_acc);
    atomicAdd(a.stats + 1, relax_acc);
  }
}

static int g_grid_cap[33];  // blocks per device for each LAP size (0 = not configured)

cudaError_t prepare_lap(int m) {
  if (m < 1 || m > 32) return cudaErrorInvalidValue;
  if (g_grid_cap[m] > 0) return cudaSuccess;
  static bool attr_set = false;
  cudaError_t e;
  if (!attr_set) {
    e = cudaFuncSetAttribute(k_lap, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(warp_smem_bytes(32) * kWarpsPerBlock));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int dev = 0, sms = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lap, kWarpsPerBlock * 32,
                                                    warp_smem_bytes(m) * kWarpsPerBlock);
  if (e != cudaSuccess) return e;
  g_grid_cap[m] = sms * (occ < 1 ? 1 : occ);
  return cudaSuccess;
}

cudaError_t launch_lap(const LapArgs& a, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  cudaError_t e = prepare_lap(a.m);
  if (e != cudaSuccess) return e;
  const size_t smem = warp_smem_bytes(a.m) * kWarpsPerBlock;
  const long long need = (a.batch + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const long long cap = g_grid_cap[a.m];
  const int grid = (int)(need < cap ? need : cap);
  k_lap<<<grid, kWarpsPerBlock * 32, smem, s>>>(a);
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
