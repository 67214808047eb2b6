// rlt2_iterate_noalloc: the dual ascent of a small QAP with no device allocation.
//
// Some callers cannot call cudaMalloc: code running under a framework that owns
// the whole device memory pool (an extra cudaMalloc fails or breaks its
// accounting), loops that must never hit the allocator's implicit device
// synchronisation, and deployments that forbid allocation after start-up.  For
// them this file keeps every working buffer of one dual ascent in a single
// file-scope device array of fixed size, which each GPU that loads the library
// holds until the process exits.  The arithmetic is the same kernels as the
// context path (rlt2_create / rlt2_iterate).
#include <cmath>
#include <mutex>
#include <string>

#include "rlt2_internal.h"

namespace rlt2 {
namespace {

// 8 MiB: enough for a residual size of at most kNoallocMaxN = 10.
constexpr size_t kScratchDoubles = size_t(1) << 20;
constexpr int kNoallocMaxN = 10;
constexpr int kMaxDevices = 64;

// The workspace.  In host code `g_scratch` is only a host-side stand-in for the
// symbol, never a device address: host code passes the address obtained with
// cudaGetSymbolAddress below.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

std::mutex g_setup_mu;
double* g_scratch_addr[kMaxDevices];  // device address of g_scratch on each device

// Sub-arrays carved from the workspace, each aligned to 256 bytes.
struct Carver {
  double* base;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    const size_t doubles = (count * sizeof(T) + sizeof(double) - 1) / sizeof(double);
    T* p = reinterpret_cast<T*>(base + used);
    used += (doubles + 31) & ~size_t(31);
    return p;
  }
};

// Identity lists (root node: every facility and location is free), the facility
// triples of the z move, fresh scalars and a NaN-filled bound history.
__global__ void k_noalloc_init(int n, int* fac, int* loc, int* trips, int ntrip, DevScalars* sc, double* lb_hist,
                               int iters) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  for (int i = tid; i < n; i += nth) {
    fac[i] = i;
    loc[i] = i;
  }
  for (int t = tid; t < ntrip; t += nth) {
    // t-th triple i<j<k in lexicographic order
    int rem = t, i = 0;
    for (;; ++i) {
      const int cnt = (n - 1 - i) * (n - 2 - i) / 2;
      if (rem < cnt) break;
      rem -= cnt;
    }
    int j = i + 1;
    for (;; ++j) {
      const int cnt = n - 1 - j;
      if (rem < cnt) break;
      rem -= cnt;
    }
    const int k = j + 1 + rem;
    trips[t] = i | (j << 8) | (k << 16);
  }
  for (int it = tid; it < iters; it += nth) lb_hist[it] = NAN;
  if (tid == 0) {
    sc->lb = -INFINITY;
    sc->best_lb = -INFINITY;
    sc->ub = INFINITY;
    sc->gap = 0.0;
    sc->iter = 0;
    sc->done = 0;
    sc->have_snap = 0;
    sc->reason = 0;
    sc->sa_on = 0;
    sc->lb_base = 0.0;  // set to the constant after setup
    for (int k = 0; k < 6; ++k) sc->stats[k] = 0;
  }
}

// Device address of the workspace on the current device, looked up once per
// device (the first call on a device does it, with that device current).  A
// cudaDeviceReset unloads the module, so the cached address (like the LAP
// launch set-up) is not valid across a reset: do not use the library after one.
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    double* ptr = nullptr;
    e = cudaGetSymbolAddress((void**)&ptr, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace rlt2

using namespace rlt2;

extern "C" rlt2_status rlt2_iterate_noalloc(int n, const double* F, const double* D, const double* B,
                                            const rlt2_params* p, int iters, double* lb_hist, void* stream) {
  if (n < 3 || n > kNoallocMaxN) {
    set_error("rlt2_iterate_noalloc: n must be in [3, " + std::to_string(kNoallocMaxN) +
              "] (fixed 8 MiB workspace); use rlt2_create for larger problems");
    return RLT2_EINVAL;
  }
  if (!F || !D || !lb_hist || iters < 1 || iters > kRing) {
    set_error("rlt2_iterate_noalloc: need device F, D, lb_hist and 1 <= iters <= 65536");
    return RLT2_EINVAL;
  }
  rlt2_params prm;
  rlt2_params_default(&prm);
  if (p) prm = *p;
  if (!params_valid(prm) || prm.half_z) {
    set_error("rlt2_iterate_noalloc: parameters out of range (the half-Z scheme needs a context)");
    return RLT2_EINVAL;
  }
  if (prm.warm == 2) {
    // the learned start needs a network (rlt2_set_mlp) and its prediction buffer
    set_error("rlt2_iterate_noalloc: warm = 2 (learned start) needs a context with rlt2_set_mlp; use warm 0 or 1");
    return RLT2_EINVAL;
  }
  double* base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess) return cuda_fail(e, "rlt2_iterate_noalloc: workspace address");

  IterView v{};
  v.n = n;
  v.m = n - 2;
  v.T = (long long)n * n * (n - 1) * (n - 1);
  v.E = v.T * v.m * v.m;
  v.ntrip = n * (n - 1) * (n - 2) / 6;
  v.prm = prm;
  const size_t T = v.T, m = v.m, n2 = (size_t)n * n;
  Carver cv{base};
  v.Dhat = cv.take<double>(v.E);
  v.xi = cv.take<double>(T * m);
  v.psi = cv.take<double>(T * m);
  v.Chat = cv.take<double>(T);
  v.Theta = cv.take<double>(T);
  v.piy = cv.take<double>(T);
  v.tterm = cv.take<double>(T);
  v.d_cst = cv.take<double>(1);
  v.Fr = cv.take<double>(n2);
  v.Dr = cv.take<double>(n2);
  v.bprime = cv.take<double>(n2);
  v.xcost = cv.take<double>(n2);
  v.saterm = cv.take<double>(n2);
  v.Delta = cv.take<double>(n2);
  v.pix = cv.take<double>(n2);
  v.gamma = cv.take<double>(n2 * (n - 1));
  v.delta = cv.take<double>(n2 * (n - 1));
  v.alpha = cv.take<double>(n);
  v.beta = cv.take<double>(n);
  v.xval = cv.take<double>(1);
  v.sc = cv.take<DevScalars>(1);
  v.xperm = cv.take<int>(n);
  v.ubperm = cv.take<int>(n);
  v.trips = cv.take<int>(v.ntrip);
  int* fac = cv.take<int>(n);
  int* loc = cv.take<int>(n);
  if (cv.used > kScratchDoubles) {
    set_error("rlt2_iterate_noalloc: problem does not fit the fixed workspace");
    return RLT2_EINVAL;
  }
  v.ring = lb_hist;  // the bound of iteration it goes to lb_hist[it]

  cudaStream_t s = (cudaStream_t)stream;
  // the workspace keeps the previous call's contents: clear what must start at zero
  if ((e = cudaMemsetAsync(v.Dhat, 0, sizeof(double) * (size_t)v.E, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(v.xi, 0, sizeof(double) * T * m, s)) != cudaSuccess)
    return cuda_fail(e, "rlt2_iterate_noalloc: clear");
  k_noalloc_init<<<8, 128, 0, s>>>(n, fac, loc, v.trips, v.ntrip, v.sc, lb_hist, iters);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "rlt2_iterate_noalloc: init");
  if ((e = enqueue_setup(v, n, F, D, B, fac, loc, nullptr, nullptr, 0, s)) != cudaSuccess)
    return cuda_fail(e, "rlt2_iterate_noalloc: setup");
  if ((e = cudaMemcpyAsync(v.xcost, v.bprime, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&v.sc->lb_base, v.d_cst, sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return cuda_fail(e, "rlt2_iterate_noalloc: x costs");
  for (int mm : {n - 2, n - 1, n})
    if ((e = prepare_lap(mm)) != cudaSuccess) return cuda_fail(e, "rlt2_iterate_noalloc: prepare");
  if ((e = prepare_lap(n - 1, 0, 4)) != cudaSuccess) return cuda_fail(e, "rlt2_iterate_noalloc: prepare");
  for (int it = 0; it < iters; ++it)
    if ((e = enqueue_iteration(v, s, nullptr)) != cudaSuccess) return cuda_fail(e, "rlt2_iterate_noalloc: iterate");
  return RLT2_OK;
}
