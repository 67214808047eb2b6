// Throughput probes for the roofline denominators (no counterpart in the
// paper).  The dual ascent's two hot kernels are bound by instruction pipes,
// not by HBM: the z move by the FP64 pipe (subtractions, additions and fused
// multiply-adds that the oracle's rounding order fixes) and the fixed-point
// LAPs by the integer ALU pipe.  GB300's data sheet gives a nominal FP64 rate
// but no per-instruction figures, so the bench measures them here with CUDA
// events, on the same device and in the same run as the kernels it rates.
//
// Each probe runs a grid of resident warps in which every thread keeps kChains
// independent accumulators and applies one operation to each per loop trip, so
// that the pipe, not the latency of a dependent chain, sets the pace.  The
// operations are inline PTX so that the compiler can neither fold the loop nor
// change the instruction; the accumulators are stored at the end so that
// nothing is dead.
#include <cuda_runtime.h>

#include "rlt2_fp64emu.cuh"
#include "rlt2_internal.h"

namespace rlt2 {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

enum ProbeOp { kDadd = 0, kDfma = 1, kIadd64 = 2, kIadd32 = 3, kEmuAdd = 4, kNumProbes = 5 };

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_probe(int trips, unsigned long long seed, double* sink_d,
                                                          unsigned long long* sink_i) {
  const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  if constexpr (OP == kDadd || OP == kDfma) {
    double acc[kChains];
    const double x = 1.0 + 1e-9 * (double)(tid & 7), y = 0.999999 + 1e-12 * (double)(seed & 15);
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (double)(c + 1);
    for (int t = 0; t < trips; ++t) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        if constexpr (OP == kDadd) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(acc[c]) : "d"(x));
        else asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(acc[c]) : "d"(y), "d"(x));
      }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    sink_d[tid] = s;
  } else if constexpr (OP == kEmuAdd) {
    // the integer-pipe binary64 addition (rlt2_fp64emu.cuh), 8 independent chains
    uint64_t acc[kChains];
    const uint64_t x = (uint64_t)__double_as_longlong(1.0 + 1e-9 * (double)(tid & 7));
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (uint64_t)__double_as_longlong((double)(c + 1));
    for (int t = 0; t < trips; ++t) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) acc[c] = emu_add_bits(acc[c], x);
    }
    uint64_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= acc[c];
    sink_i[tid] = s;
  } else if constexpr (OP == kIadd64) {
    unsigned long long acc[kChains];
    const unsigned long long x = seed | 1ull;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = tid * (c + 3);
    for (int t = 0; t < trips; ++t) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("add.s64 %0, %0, %1;" : "+l"(acc[c]) : "l"(x));
    }
    unsigned long long s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= acc[c];
    sink_i[tid] = s;
  } else {
    unsigned acc[kChains];
    const unsigned x = (unsigned)seed | 1u;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (unsigned)tid * (c + 3);
    for (int t = 0; t < trips; ++t) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("add.s32 %0, %0, %1;" : "+r"(acc[c]) : "r"(x));
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= acc[c];
    sink_i[tid] = s;
  }
}

__global__ void k_emu_add(long long count, const double* a, const double* b, double* sum, double* diff) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    sum[i] = emu_dadd(a[i], b[i]);
    diff[i] = emu_dsub(a[i], b[i]);
  }
}

template <int OP>
cudaError_t launch_probe(int blocks, int trips, double* sd, unsigned long long* si, cudaStream_t s) {
  k_probe<OP><<<blocks, kProbeThreads, 0, s>>>(trips, 0x9e3779b97f4a7c15ull, sd, si);
  return cudaGetLastError();
}

cudaError_t launch_any(int op, int blocks, int trips, double* sd, unsigned long long* si, cudaStream_t s) {
  switch (op) {
    case kDadd: return launch_probe<kDadd>(blocks, trips, sd, si, s);
    case kDfma: return launch_probe<kDfma>(blocks, trips, sd, si, s);
    case kIadd64: return launch_probe<kIadd64>(blocks, trips, sd, si, s);
    case kEmuAdd: return launch_probe<kEmuAdd>(blocks, trips, sd, si, s);
    default: return launch_probe<kIadd32>(blocks, trips, sd, si, s);
  }
}

}  // namespace
}  // namespace rlt2

using namespace rlt2;

extern "C" rlt2_status rlt2_probe_rates(double* rates, double* sm_clock_ghz, void* stream) {
  if (!rates) {
    set_error("rlt2_probe_rates: rates must not be NULL");
    return RLT2_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, occ = 0, clk_khz = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount,
                                                                               dev)) != cudaSuccess)
    return cuda_fail(e, "rlt2_probe_rates: device");
  if ((e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev)) != cudaSuccess) clk_khz = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_probe<kDfma>, kProbeThreads, 0)) != cudaSuccess)
    return cuda_fail(e, "rlt2_probe_rates: occupancy");
  const int blocks = sms * (occ < 1 ? 1 : (occ > 4 ? 4 : occ));
  const size_t nthreads = (size_t)blocks * kProbeThreads;
  double* sd = nullptr;
  unsigned long long* si = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rlt2_status st = RLT2_OK;
  if ((e = cudaMalloc(&sd, sizeof(double) * nthreads)) != cudaSuccess ||
      (e = cudaMalloc(&si, sizeof(unsigned long long) * nthreads)) != cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    st = cuda_fail(e, "rlt2_probe_rates: buffers");
  }
  // trips per op: FP64 runs at a few lanes per clock per SM, the integer adds at
  // tens, so each probe lasts a few milliseconds
  const int trips[kNumProbes] = {256, 256, 8192, 16384, 256};
  for (int op = 0; op < kNumProbes && st == RLT2_OK; ++op) {
    float best = 1e30f;
    for (int rep = 0; rep < 4 && st == RLT2_OK; ++rep) {  // the first is a warm-up
      if ((e = cudaEventRecord(e0, s)) != cudaSuccess ||
          (e = launch_any(op, blocks, trips[op], sd, si, s)) != cudaSuccess ||
          (e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
        st = cuda_fail(e, "rlt2_probe_rates: probe");
        break;
      }
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
        st = cuda_fail(e, "rlt2_probe_rates: timing");
        break;
      }
      if (rep > 0 && ms < best) best = ms;
    }
    if (st == RLT2_OK) rates[op] = (double)nthreads * trips[op] * kChains / (best * 1e-3) / 1e9;
  }
  if (sm_clock_ghz) *sm_clock_ghz = clk_khz * 1e-6;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sd) cudaFree(sd);
  if (si) cudaFree(si);
  return st;
}

extern "C" rlt2_status rlt2_fp64_add_emulated(long long count, const double* a, const double* b, double* sum,
                                              double* diff, void* stream) {
  if (count < 0 || (count > 0 && (!a || !b || !sum || !diff))) {
    set_error("rlt2_fp64_add_emulated: invalid argument");
    return RLT2_EINVAL;
  }
  if (count == 0) return RLT2_OK;
  const long long blocks = (count + 255) / 256;
  k_emu_add<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(count, a, b, sum, diff);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rlt2_fp64_add_emulated");
  return RLT2_OK;
}
