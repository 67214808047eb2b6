// RLT2 dual ascent on one GPU: context, setup, ascent moves, stage driver,
// branch-and-bound child derivation and the C ABI.
//
// One iteration (Algorithm 2 on one GPU, no MPI; S or F variant, Section 3.4)
// is these kernels on the context's stream:
//   k_move_y     per tile: pending y move (Eq. 2.21; the F and half-Z forms)
//                and the tile term cy*pi_y + cx*pi_x that rules 2 and 3
//                (Eq. 2.22, 2.23) add to every z pool, plus an accepted Type 4
//                amount (Section 2.3 rule 4); for the folded z move (kz = 1,
//                equal phi) also psi <- psi - tile term, and it zeroes the Z
//                stage's LAP queue counter
//   k_move_z     class-owned z move (Eq. 2.20 + 2.22 + 2.23, combined as in the
//                proof of Theorem 1), in place on D^ (Section 3.3)
//   k_lap(Z)     n^2 (n-1)^2 LAPs of size n-2 on the tiles of D^ (half of them
//                with the half-Z scheme, Section 5)
//   [k_phase2, k_lap(Z)]  the two-phase Z solve (Section 3.4)
//   k_lap(Y)     n^2 LAPs of size n-1 on C^ + Theta (fold fused into the tile
//                load), writes pi_y
//   k_lap(X)     one LAP of size n on b' + Delta, writes pi_x
//   k_finalize   bound, best bound, upper bound of the X primal, the feasibility
//                check that follows Algorithm 1, stop flags, bound history
// A context's first 64 iterations are launched kernel by kernel, later ones as
// replays of captured CUDA graphs (eight iterations each, one for the rest of a
// call).  The ascent step of iteration m runs at
// the start of iteration m+1, so after every call the state, duals and reduced
// costs describe the same multipliers.  Device-side flags (done / have_snap)
// make every kernel a no-op after a stop, so whole batches of iterations can
// be enqueued without host round trips.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "rlt2_ascent.cuh"
#include "rlt2_internal.h"

namespace rlt2 {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
rlt2_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return RLT2_ECUDA;
}

constexpr int kKinds = 8;

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }

// ------------------------------------------------------------------ setup ----
// b'_ip = b_ip + f_ii d_pp + sum_{a fixed} (f_ia d_{p,phi a} + f_ai d_{phi a,p})
// (Eq. 1.1 with the fixed facilities of a branch-and-bound node moved into b),
// plus the residual F and D used for the upper bound.
__global__ void k_setup_b(int n, int nr, const double* F, const double* D, const double* B, const int* fac,
                          const int* loc, const int* fixf, const int* fixl, int nfix, double* bprime, double* Fr,
                          double* Dr) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nr * nr) return;
  const int ii = e / nr, pp = e - ii * nr;
  const int i = fac[ii], p = loc[pp];
  double s = dadd(B ? B[i * n + p] : 0.0, dmul(F[i * n + i], D[p * n + p]));
  for (int x = 0; x < nfix; ++x) {
    const int a = fixf[x], pa = fixl[x];
    s = dadd(s, dadd(dmul(F[i * n + a], D[p * n + pa]), dmul(F[a * n + i], D[pa * n + p])));
  }
  bprime[e] = s;
  Fr[e] = F[fac[ii] * n + fac[pp]];
  Dr[e] = D[loc[ii] * n + loc[pp]];
}

// const = sum_a b_{a,phi a} + sum_{a,a'} f_aa' d_{phi a, phi a'} over fixed facilities.
__global__ void k_setup_const(int n, const double* F, const double* D, const double* B, const int* fixf,
                              const int* fixl, int nfix, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double c = 0.0;
  for (int x = 0; x < nfix; ++x) {
    const int a = fixf[x], pa = fixl[x];
    if (B) c = dadd(c, B[a * n + pa]);
    for (int y = 0; y < nfix; ++y) c = dadd(c, dmul(F[a * n + fixf[y]], D[pa * n + fixl[y]]));
  }
  *out = c;
}

// C^_ijpq = f_ij d_pq on the tile layout (RLT1 cost, Eq. 2.1).
__global__ void k_setup_c(int nr, long long T, const double* Fr, const double* Dr, double* Chat) {
  const int n1 = nr - 1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T; t += (long long)gridDim.x * blockDim.x) {
    const int ip = (int)(t / (n1 * n1));
    const int rem = (int)(t - (long long)ip * n1 * n1);
    const int jj = rem / n1, qq = rem - jj * n1;
    const int i = ip / nr, p = ip - i * nr;
    const int j = jj + (jj >= i), q = qq + (qq >= p);
    Chat[t] = dmul(Fr[i * nr + j], Dr[p * nr + q]);
  }
}

// ------------------------------------------------------------------ moves ----
static const int h_widx[5] = {0, 1, 3, 2, 4};

// blockDim.x a multiple of 32 (the folded form's warps move 32 tiles together)
__global__ void k_move_y(MoveYArgs a) {
  // the Z stage's launch comes after this one on the stream
  if (a.lap_head && blockIdx.x == 0 && threadIdx.x == 0) *a.lap_head = 0;
  if (!a.sc->have_snap || a.sc->done) return;
  const long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  if (a.shift_psi) move_y_shift_range(a, start, stride);
  else move_y_range(a, start, stride);
}

// at most 352 threads (move_z_threads) and 62 registers: three blocks per SM
__global__ void __launch_bounds__(352, 3) k_move_z(MoveZArgs a) {
  if (!a.sc->have_snap || a.sc->done) return;
  move_z_block(a, blockIdx.x, threadIdx.x, blockDim.x);
}

// Second phase of the two-phase Z solve; runs on every iteration (the first
// phase's duals are always fresh).
__global__ void __launch_bounds__(512) k_phase2(Phase2Args a) {
  if (a.sc->done) return;
  phase2_block(a, blockIdx.x);
}

// pi_z = (D^ - xi_k') - psi_r' for every z entry (reduced costs on demand).
__global__ void k_pi_z(long long E, int m, const double* Dhat, const double* xi, const double* psi, double* out) {
  const long long mm = (long long)m * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / mm;
    const int w = (int)(e - t * mm);
    const int k = w / m, r = w - k * m;
    out[e] = dsub(dsub(Dhat[e], xi[t * m + k]), psi[t * m + r]);
  }
}

// ---------------------------------------------------------------- finalize ----
__global__ void __launch_bounds__(256) k_finalize(FinArgs a) {
  if (a.sc->done) return;
  finalize_block(a);
}

// Step A0 on the device: b', the residual F and D, the constant of the fixed
// facilities and C^ (D^ is cleared by the caller).
cudaError_t enqueue_setup(const IterView& v, int n_full, const double* dF, const double* dD, const double* dB,
                          const int* dfac, const int* dloc, const int* dfixf, const int* dfixl, int nfix,
                          cudaStream_t s) {
  const int nr = v.n;
  const long long n2 = (long long)nr * nr;
  k_setup_b<<<(int)((n2 + 127) / 128), 128, 0, s>>>(n_full, nr, dF, dD, dB, dfac, dloc, dfixf, dfixl, nfix, v.bprime,
                                                     v.Fr, v.Dr);
  k_setup_const<<<1, 32, 0, s>>>(n_full, dF, dD, dB, dfixf, dfixl, nfix, v.d_cst);
  const long long blocks = (v.T + 255) / 256;
  k_setup_c<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(nr, v.T, v.Fr, v.Dr, v.Chat);
  return cudaGetLastError();
}

// ------------------------------------------------ parent -> child warm start --
// A branch-and-bound child fixes residual facility f at location l of its
// parent (Section 4).  In the parent's Lagrangian LRLT2(v), y_{i f p l} and
// y_{f i l p} become x_ip and every z with (f,l) in one position becomes the y
// of the other two, so the child starts from the parent's multipliers:
//   D^_c(i,j,k|p,q,r) = D^_p(I,J,K|P,Q,R)        (I = i + (i >= f), P = p + (p >= l))
//   C^_c(i,j|p,q) = ((C^_p(I,J|P,Q) + D^_p(I,J,f|P,Q,l)) + D^_p(I,f,J|P,l,Q)) + D^_p(f,I,J|l,P,Q)
//   b'_c(i|p) = (b'_p(I|P) + C^_p(I,f|P,l)) + C^_p(f,I|l,P),  const_c = const_p + b'_p(f|l)
// and, for upper bounds, the QAP's own reduction of b and the constant.
__device__ __forceinline__ long long ptile(int n, int i, int p, int j, int q) {
  return ((long long)(i * n + p) * (n - 1) + (j - (j > i))) * (n - 1) + (q - (q > p));
}
__device__ __forceinline__ long long pz(int n, int i, int j, int k, int p, int q, int r) {
  const int m = n - 2;
  return ptile(n, i, p, j, q) * m * m + (long long)(k - (k > i) - (k > j)) * m + (r - (r > p) - (r > q));
}

__global__ void k_child_z(int np, int f, int l, const double* __restrict__ Dp, double* __restrict__ Dc, long long Ec) {
  const int nc = np - 1, n1 = nc - 1, mc = nc - 2;
  const long long mm = (long long)mc * mc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < Ec; e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / mm;
    const int w = (int)(e - t * mm);
    const int kk = w / mc, rr = w - kk * mc;
    const int ip = (int)(t / (n1 * n1));
    const int rem = (int)(t - (long long)ip * n1 * n1);
    const int jj = rem / n1, qq = rem - jj * n1;
    const int i = ip / nc, p = ip - i * nc;
    const int j = jj + (jj >= i), q = qq + (qq >= p);
    int k = kk;
    k += (k >= (i < j ? i : j));
    k += (k >= (i < j ? j : i));
    int r = rr;
    r += (r >= (p < q ? p : q));
    r += (r >= (p < q ? q : p));
    Dc[e] = Dp[pz(np, i + (i >= f), j + (j >= f), k + (k >= f), p + (p >= l), q + (q >= l), r + (r >= l))];
  }
}

__global__ void k_child_yx(int np, int f, int l, const double* __restrict__ Dp, const double* __restrict__ Cp,
                           const double* __restrict__ bp, const double* __restrict__ bqp, const double* __restrict__ Frp,
                           const double* __restrict__ Drp, const double* cst_p, const double* cstq_p,
                           double* __restrict__ Cc, double* __restrict__ bc, double* __restrict__ bqc,
                           double* __restrict__ Frc, double* __restrict__ Drc, double* cst_c, double* cstq_c,
                           long long Tc) {
  const int nc = np - 1, n1 = nc - 1;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long t = t0; t < Tc; t += stride) {
    const int ip = (int)(t / (n1 * n1));
    const int rem = (int)(t - (long long)ip * n1 * n1);
    const int jj = rem / n1, qq = rem - jj * n1;
    const int i = ip / nc, p = ip - i * nc;
    const int j = jj + (jj >= i), q = qq + (qq >= p);
    const int I = i + (i >= f), J = j + (j >= f), P = p + (p >= l), Q = q + (q >= l);
    double c = Cp[ptile(np, I, P, J, Q)];
    c = dadd(c, Dp[pz(np, I, J, f, P, Q, l)]);
    c = dadd(c, Dp[pz(np, I, f, J, P, l, Q)]);
    c = dadd(c, Dp[pz(np, f, I, J, l, P, Q)]);
    Cc[t] = c;
  }
  for (long long e = t0; e < (long long)nc * nc; e += stride) {
    const int i = (int)e / nc, p = (int)e - i * nc;
    const int I = i + (i >= f), P = p + (p >= l);
    bc[e] = dadd(dadd(bp[I * np + P], Cp[ptile(np, I, P, f, l)]), Cp[ptile(np, f, l, I, P)]);
    bqc[e] = dadd(dadd(bqp[I * np + P], dmul(Frp[I * np + f], Drp[P * np + l])), dmul(Frp[f * np + I], Drp[l * np + P]));
    Frc[e] = Frp[I * np + (p + (p >= f))];
    Drc[e] = Drp[(i + (i >= l)) * np + P];
  }
  if (t0 == 0) {
    *cst_c = dadd(*cst_p, bp[f * np + l]);
    *cstq_c = dadd(*cstq_p, bqp[f * np + l]);
  }
}

RLT2_DEFINE_OOB_QUERY(oob_ascent)

}  // namespace rlt2

using namespace rlt2;

extern "C" long long rlt2_debug_bounds_violations(void) {
#ifdef RLT2_BOUNDS_CHECK
  unsigned long long total = 0;
  for (auto query : {oob_lap, oob_ascent, oob_nodes, oob_fused}) {
    const unsigned long long v = query();
    if (v == ~0ull) return -2;
    total += v;
  }
  return (long long)total;
#else
  return -1;
#endif
}

// ------------------------------------------------------------------ context ---
struct rlt2_ctx {
  int n_full = 0, n = 0, m = 0;
  long long T = 0, E = 0;
  rlt2_params prm{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // created when the first graph is captured
  char* arena = nullptr;              // every fixed-size buffer, one pool allocation
  std::vector<int> fac, loc;  // free facilities / locations (host)
  std::vector<int> fixf, fixl;
  double* d_cst = nullptr;
  double *Fr = nullptr, *Dr = nullptr, *bprime = nullptr, *Chat = nullptr, *Dhat = nullptr;
  double *Theta = nullptr, *xi = nullptr, *psi = nullptr, *Delta = nullptr, *gamma = nullptr, *delta = nullptr;
  double *alpha = nullptr, *beta = nullptr, *pix = nullptr, *piy = nullptr, *tterm = nullptr, *xval = nullptr;
  double* ring = nullptr;
  double* xcost = nullptr;   // F variant: own buffer; S variant: aliases bprime
  double* saterm = nullptr;
  double* sa_buf = nullptr;  // Type 4 draws: kf[count*n] | kl[count*n] | K[count] | thr[count]
  int sa_count = 0;
  int* zmap = nullptr;       // half-Z scheme: upper tiles
  long long Tz = 0;
  double* bqap = nullptr;    // QAP linear costs of the residual problem (upper bounds); aliases bprime
  double* d_cst_qap = nullptr;  // QAP constant of the fixed facilities; aliases d_cst
  int *xperm = nullptr, *ubperm = nullptr, *trips = nullptr;
  int ntrip = 0;
  DevScalars* sc = nullptr;
  cudaGraphExec_t graph = nullptr;       // one iteration
  cudaGraphExec_t graph_many = nullptr;  // kGraphIters iterations (fewer launch gaps)
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // timing mode: 2 events per kernel launch
  double kms[kKinds] = {};
  long long kcount[kKinds] = {};
  int iter_host = 0;
  long long enqueued = 0;  // iterations enqueued so far (the graph is captured past kDirectIters)
  double cst_host = 0.0;
  rlt2_mlp* mlp = nullptr;
  double* u0buf = nullptr;
  const PipePlan* pplan = nullptr;     // pipelined z move + Z-LAPs: shared plan (not owned)
  unsigned long long* pipe = nullptr;  // its queue head, exit count and pair counters
};

// Device memory of contexts.  A branch and bound creates and destroys a
// context per node, and cudaMalloc / cudaFree (which waits for the whole
// device) cost about a millisecond per node for the twenty-odd buffers; so a
// context takes all its fixed-size buffers as one arena from a stream-ordered
// memory pool of the library (one per device), allocated and freed in order on
// the context's stream.  The pool keeps up to a quarter of the device's memory
// cached for reuse after contexts are destroyed.
static std::mutex g_pool_mu;
constexpr int kPoolDevices = 64;
static cudaMemPool_t g_pool[kPoolDevices];

static cudaError_t ctx_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kPoolDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
    size_t fr = 0, tot = 0;
    if ((e = cudaMemGetInfo(&fr, &tot)) != cudaSuccess) return e;
    unsigned long long keep = tot / 4;
    if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) return e;
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

// Bytes the pool holds but no context uses (available to the next context).
static size_t ctx_pool_idle(cudaMemPool_t pool) {
  unsigned long long reserved = 0, used = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess)
    return 0;
  return reserved > used ? (size_t)(reserved - used) : 0;
}

static void ctx_free(rlt2_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph_many) cudaGraphExecDestroy(c->graph_many);
  for (auto e : c->ev) cudaEventDestroy(e);
  if (c->arena) cudaFreeAsync(c->arena, c->stream);
  if (c->sa_buf) cudaFree(c->sa_buf);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->u0buf) cudaFree(c->u0buf);
  delete c;
}

static IterView view_of(const rlt2_ctx* c) {
  IterView v{};
  v.mlp = c->mlp;
  v.u0buf = c->u0buf;
  v.n = c->n;
  v.m = c->m;
  v.T = c->T;
  v.E = c->E;
  v.ntrip = c->ntrip;
  v.prm = c->prm;
  v.d_cst = c->d_cst;
  v.Fr = c->Fr;
  v.Dr = c->Dr;
  v.bprime = c->bprime;
  v.Chat = c->Chat;
  v.Dhat = c->Dhat;
  v.Theta = c->Theta;
  v.xi = c->xi;
  v.psi = c->psi;
  v.Delta = c->Delta;
  v.gamma = c->gamma;
  v.delta = c->delta;
  v.alpha = c->alpha;
  v.beta = c->beta;
  v.pix = c->pix;
  v.piy = c->piy;
  v.tterm = c->tterm;
  v.xval = c->xval;
  v.ring = c->ring;
  v.xperm = c->xperm;
  v.ubperm = c->ubperm;
  v.trips = c->trips;
  v.sc = c->sc;
  v.xcost = c->xcost;
  v.saterm = c->saterm;
  v.zmap = c->zmap;
  v.Tz = c->Tz;
  v.bqap = c->bqap;
  v.cst_qap = c->d_cst_qap;
  v.pplan = c->pplan;
  v.pipe = c->pipe;
  v.sa_count = c->sa_count;
  if (c->sa_count > 0) {
    const long long cn = (long long)c->sa_count * c->n;
    v.sa_kf = c->sa_buf;
    v.sa_kl = c->sa_buf + cn;
    v.sa_K = c->sa_buf + 2 * cn;
    v.sa_thr = c->sa_buf + 2 * cn + c->sa_count;
  }
  return v;
}

static bool finite_all(const double* x, size_t k) {
  for (size_t i = 0; i < k; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

extern "C" void rlt2_params_default(rlt2_params* p) {
  if (!p) return;
  p->kz = 1.0;
  p->ky = 0.5;
  p->kx = 1.0;
  p->phi_y = 0.5;
  for (int l = 0; l < 5; ++l) p->phi_z[l] = 0.2;
  p->dual_mode = 1;
  p->warm = 0;
  p->min_gap = 0.0;
  p->ub = 0.0;
  p->feas_tol = 1e-9;
  p->stall_window = 0;
  p->stall_tol = 0.0002;
  p->variant = 0;
  p->two_phase = 0;
  p->phase2_tol = 1e-9;
  p->sa_t0 = 0.04;
  p->sa_cool = 0.99;
  p->sa_period = 100;
  p->half_z = 0;
  p->pipeline = 0;
}

bool rlt2::params_valid(const rlt2_params& p) {
  auto in01 = [](double x) { return std::isfinite(x) && x >= 0.0 && x <= 1.0; };
  if (!in01(p.kz) || !in01(p.ky) || !in01(p.kx) || !in01(p.phi_y)) return false;
  if (p.half_z != 0 && p.half_z != 1) return false;
  // the half scheme moves an upper y's slack (ky) and a lower y's slack (phi_y): different y
  if (!p.half_z && p.phi_y + p.ky > 1.0) return false;
  if (p.half_z && (p.variant != 0 || p.two_phase != 0)) return false;
  double s = 0.0;
  for (int l = 0; l < 5; ++l) {
    if (!in01(p.phi_z[l])) return false;
    s += p.phi_z[l];
  }
  if (std::fabs(s - 1.0) > 1e-12) return false;
  if (p.dual_mode < 0 || p.dual_mode > 2) return false;
  if (p.warm < 0 || p.warm > 2) return false;
  if (p.pipeline != 0 && p.pipeline != 1) return false;
  if (!std::isfinite(p.min_gap) || !std::isfinite(p.ub) || !std::isfinite(p.feas_tol)) return false;
  if (p.stall_window < 0 || p.stall_window >= kStallRing || !std::isfinite(p.stall_tol)) return false;
  if (p.variant != 0 && p.variant != 1) return false;
  if (p.two_phase != 0 && p.two_phase != 1) return false;
  if (!std::isfinite(p.phase2_tol) || p.phase2_tol < 0.0) return false;
  if (!std::isfinite(p.sa_t0) || !std::isfinite(p.sa_cool) || p.sa_period < 1) return false;
  return true;
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

template <class T>
static cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

// Sub-arrays of a context's arena, each 256-byte aligned; with base == nullptr
// it only counts, so sizing and carving cannot disagree.
struct CtxCarver {
  char* base;
  size_t used = 0;
  template <class T>
  void take(T** p, size_t count) {
    *p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += (sizeof(T) * (count ? count : 1) + 255) & ~size_t(255);
  }
};

// Device buffers of a context whose sizes (n, m, T, E, ntrip) and parameters
// are set: memory admission, allocation, the capture stream, cleared D^, duals
// and Theta, fresh scalars, the facility triples and (half-Z scheme) the tile
// map.  own_qap: the QAP linear costs and constant used for upper bounds get
// their own buffers (child contexts, whose b' carries multipliers); otherwise
// they are b' and the constant.  Frees c and returns the status on failure.
static rlt2_status ctx_alloc(rlt2_ctx* c, bool own_qap) {
  const int nr = c->n;
  const rlt2_params& prm = c->prm;
  size_t need = sizeof(double) * ((size_t)c->E + 6 * (size_t)c->T + 2 * (size_t)c->T * c->m + 10 * (size_t)nr * nr +
                                  2 * (size_t)nr * nr * nr + kRing) +
                sizeof(int) * (size_t)(c->ntrip + nr + (prm.half_z ? c->T / 2 : 0)) + (64u << 20);
  size_t fr = 0, tot = 0;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = ctx_pool(&pool);
  if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaMemGetInfo");
  }
  fr += ctx_pool_idle(pool);
  if (need > fr) {
    delete c;
    set_error("rlt2_create: not enough free device memory");
    return RLT2_ENOMEM;
  }
  rlt2_status st = RLT2_OK;
  auto fail = [&](cudaError_t err, const char* what) {
    st = (err == cudaErrorMemoryAllocation) ? RLT2_ENOMEM : RLT2_ECUDA;
    cuda_fail(err, what);
    ctx_free(c);
    return st;
  };
  const size_t T = c->T, m = c->m, n2 = (size_t)nr * nr;
  // the arena: sized by a counting pass, then allocated once and carved
  auto carve = [&](CtxCarver& cv) {
#define AL(ptr, cnt) cv.take(&(ptr), (cnt))
  AL(c->d_cst, 1);
  AL(c->Fr, n2);
  AL(c->Dr, n2);
  AL(c->bprime, n2);
  AL(c->Chat, T);
  AL(c->Dhat, (size_t)c->E);
  AL(c->Theta, T);
  AL(c->xi, T * m);
  AL(c->psi, T * m);
  AL(c->Delta, n2);
  AL(c->gamma, n2 * (nr - 1));
  AL(c->delta, n2 * (nr - 1));
  AL(c->alpha, nr);
  AL(c->beta, nr);
  AL(c->pix, n2);
  AL(c->piy, T);
  AL(c->tterm, T);
  AL(c->xval, 1);
  AL(c->ring, kRing);
  AL(c->xperm, nr);
  AL(c->ubperm, nr);
  AL(c->trips, c->ntrip);
  AL(c->sc, 1);
  AL(c->saterm, n2);
  if (prm.variant == 1) AL(c->xcost, n2);
  if (prm.half_z) AL(c->zmap, T / 2);
  if (own_qap) {
    AL(c->bqap, n2);
    AL(c->d_cst_qap, 1);
  }
  if (prm.pipeline && !prm.half_z) AL(c->pipe, 4 + n2);
#undef AL
  };
  {
    CtxCarver count{nullptr};
    carve(count);
    if ((e = cudaMallocFromPoolAsync((void**)&c->arena, count.used, pool, c->stream)) != cudaSuccess) {
      c->arena = nullptr;
      return fail(e, "context arena");
    }
    CtxCarver cv{c->arena};
    carve(cv);
  }
  if (prm.pipeline && !prm.half_z) {
    cudaError_t e2 = cudaSuccess;
    c->pplan = prepare_pipe(nr, &e2);
    if (!c->pplan) return fail(e2, "pipelined move and Z-LAP plan");
  }
  if (!c->xcost) c->xcost = c->bprime;  // S variant: the X-LAP reads b' itself
  if (!c->bqap) c->bqap = c->bprime;
  if (!c->d_cst_qap) c->d_cst_qap = c->d_cst;
  std::vector<int> trips;
  trips.reserve(c->ntrip);
  for (int i = 0; i < nr; ++i)
    for (int j = i + 1; j < nr; ++j)
      for (int k = j + 1; k < nr; ++k) trips.push_back(i | (j << 8) | (k << 16));
  // half-Z scheme: the tiles (i,p,j',q') with j > i, i.e. j' >= i; the others keep
  // D^ = 0, Theta = 0 and zero duals forever
  std::vector<int> up;
  c->Tz = (long long)T;
  if (prm.half_z) {
    up.reserve(T / 2);
    for (int i = 0; i < nr; ++i)
      for (int p2 = 0; p2 < nr; ++p2)
        for (int jj = i; jj < nr - 1; ++jj)
          for (int qq = 0; qq < nr - 1; ++qq) up.push_back(((i * nr + p2) * (nr - 1) + jj) * (nr - 1) + qq);
    c->Tz = (long long)up.size();
  }
  DevScalars init{};
  init.ub = INFINITY;
  init.best_lb = -INFINITY;
  init.lb = -INFINITY;
  cudaStream_t s = c->stream;
  if ((e = cudaMemcpyAsync(c->trips, trips.data(), trips.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->sc, &init, sizeof init, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->Dhat, 0, sizeof(double) * (size_t)c->E, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->xi, 0, sizeof(double) * T * m, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->psi, 0, sizeof(double) * T * m, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->Theta, 0, sizeof(double) * T, s)) != cudaSuccess ||
      (c->pipe && (e = cudaMemsetAsync(c->pipe, 0, sizeof(unsigned long long) * (4 + n2), s)) != cudaSuccess) ||
      (prm.half_z &&
       (e = cudaMemcpyAsync(c->zmap, up.data(), up.size() * sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess)) {
    cudaStreamSynchronize(s);
    return fail(e, "upload");
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "upload sync");  // host vectors outlive the copies
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_create(int n, const double* F, const double* D, const double* B, const int* partial,
                                   const rlt2_params* p, void* stream, rlt2_ctx** out) {
  if (!out) {
    set_error("rlt2_create: out is NULL");
    return RLT2_EINVAL;
  }
  *out = nullptr;
  if (n < 3 || n > 64 || !F || !D) {
    set_error("rlt2_create: need 3 <= n <= 64 and non-NULL F, D");
    return RLT2_EINVAL;
  }
  const size_t nn = (size_t)n * n;
  if (!finite_all(F, nn) || !finite_all(D, nn) || (B && !finite_all(B, nn))) {
    set_error("rlt2_create: non-finite input");
    return RLT2_EINVAL;
  }
  rlt2_params prm;
  rlt2_params_default(&prm);
  if (p) prm = *p;
  if (!params_valid(prm)) {
    set_error("rlt2_create: parameters out of range (kappa, phi in [0,1], phi_y+ky<=1, sum phi_z = 1)");
    return RLT2_EINVAL;
  }
  rlt2_ctx* c = new rlt2_ctx();
  c->n_full = n;
  c->prm = prm;
  c->stream = (cudaStream_t)stream;
  std::vector<char> used(n, 0);
  for (int i = 0; i < n; ++i) {
    if (partial && partial[i] >= 0) {
      if (partial[i] >= n || used[partial[i]]) {
        delete c;
        set_error("rlt2_create: partial assignment is not injective / out of range");
        return RLT2_EINVAL;
      }
      used[partial[i]] = 1;
      c->fixf.push_back(i);
      c->fixl.push_back(partial[i]);
    } else if (partial && partial[i] < -1) {
      delete c;
      set_error("rlt2_create: partial entries must be -1 or a location");
      return RLT2_EINVAL;
    }
  }
  for (int i = 0; i < n; ++i)
    if (!partial || partial[i] < 0) c->fac.push_back(i);
  for (int q = 0; q < n; ++q)
    if (!used[q]) c->loc.push_back(q);
  const int nr = (int)c->fac.size();
  if (nr < 3 || nr > 32) {
    delete c;
    set_error("rlt2_create: residual size must be in [3, 32]");
    return RLT2_EINVAL;
  }
  c->n = nr;
  c->m = nr - 2;
  c->T = (long long)nr * nr * (nr - 1) * (nr - 1);
  c->E = c->T * c->m * c->m;
  c->ntrip = nr * (nr - 1) * (nr - 2) / 6;
  rlt2_status st = ctx_alloc(c, false);
  if (st != RLT2_OK) return st;
  auto fail = [&](cudaError_t err, const char* what) {
    st = (err == cudaErrorMemoryAllocation) ? RLT2_ENOMEM : RLT2_ECUDA;
    cuda_fail(err, what);
    ctx_free(c);
    return st;
  };
  // inputs to the device, then the setup kernels (step A0) on the stream
  cudaError_t e = cudaSuccess;
  const size_t n2 = (size_t)nr * nr;
  double *dF = nullptr, *dD = nullptr, *dB = nullptr;
  int* dint = nullptr;
  const int nfix = (int)c->fixf.size();
  std::vector<int> ints;
  ints.insert(ints.end(), c->fac.begin(), c->fac.end());
  ints.insert(ints.end(), c->loc.begin(), c->loc.end());
  ints.insert(ints.end(), c->fixf.begin(), c->fixf.end());
  ints.insert(ints.end(), c->fixl.begin(), c->fixl.end());
  cudaStream_t s = c->stream;
  auto cleanup_tmp = [&]() {
    if (dF) cudaFree(dF);
    if (dD) cudaFree(dD);
    if (dB) cudaFree(dB);
    if (dint) cudaFree(dint);
  };
  if ((e = dalloc(&dF, nn)) != cudaSuccess || (e = dalloc(&dD, nn)) != cudaSuccess ||
      (B && (e = dalloc(&dB, nn)) != cudaSuccess) || (e = dalloc(&dint, ints.size())) != cudaSuccess) {
    cleanup_tmp();
    return fail(e, "cudaMalloc");
  }
  if ((e = cudaMemcpyAsync(dF, F, nn * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dD, D, nn * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (B && (e = cudaMemcpyAsync(dB, B, nn * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess) ||
      (e = cudaMemcpyAsync(dint, ints.data(), ints.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
    cudaStreamSynchronize(s);
    cleanup_tmp();
    return fail(e, "upload");
  }
  const int* dfac = dint;
  const int* dloc = dint + nr;
  const int* dfixf = dint + 2 * nr;
  const int* dfixl = dint + 2 * nr + nfix;
  e = enqueue_setup(view_of(c), n, dF, dD, dB, dfac, dloc, dfixf, dfixl, nfix, s);
  if (e == cudaSuccess) e = cudaGetLastError();
  // F variant: the first solve runs on b' and its bound starts from the constant
  if (e == cudaSuccess && c->xcost != c->bprime)
    e = cudaMemcpyAsync(c->xcost, c->bprime, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c->sc->lb_base, c->d_cst, sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaError_t e3 = cudaStreamSynchronize(s);
  cleanup_tmp();
  if (e != cudaSuccess) return fail(e, "setup kernels");
  if (e3 != cudaSuccess) return fail(e3, "setup sync");
  if ((e = cudaMemcpy(&c->cst_host, c->d_cst, 8, cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(e, "cst");
  for (int mm2 : {nr - 2, nr - 1, nr})
    if ((e = prepare_lap(mm2)) != cudaSuccess) return fail(e, "prepare_lap");
  if ((e = prepare_lap(nr - 1, 0, 4)) != cudaSuccess) return fail(e, "prepare_lap");
  *out = c;
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_create_child(rlt2_ctx* parent, int facility, int location, const rlt2_params* p,
                                         rlt2_ctx** out) {
  if (!out) {
    set_error("rlt2_create_child: out is NULL");
    return RLT2_EINVAL;
  }
  *out = nullptr;
  if (!parent) {
    set_error("rlt2_create_child: parent is NULL");
    return RLT2_EINVAL;
  }
  if (parent->prm.variant != 0) {
    set_error("rlt2_create_child: the parent must run the S variant (its costs carry the multipliers)");
    return RLT2_EINVAL;
  }
  int f = -1, l = -1;
  for (int a = 0; a < parent->n; ++a) {
    if (parent->fac[a] == facility) f = a;
    if (parent->loc[a] == location) l = a;
  }
  if (f < 0 || l < 0) {
    set_error("rlt2_create_child: facility or location is not free in the parent");
    return RLT2_EINVAL;
  }
  const int nr = parent->n - 1;
  if (nr < 3) {
    set_error("rlt2_create_child: the child's residual size would be below 3");
    return RLT2_EINVAL;
  }
  rlt2_params prm = parent->prm;
  if (p) prm = *p;
  if (!params_valid(prm) || prm.variant != 0) {
    set_error("rlt2_create_child: parameters out of range (S variant only)");
    return RLT2_EINVAL;
  }
  rlt2_ctx* c = new rlt2_ctx();
  c->n_full = parent->n_full;
  c->prm = prm;
  c->stream = parent->stream;
  for (int a = 0; a < parent->n; ++a) {
    if (a != f) c->fac.push_back(parent->fac[a]);
    if (a != l) c->loc.push_back(parent->loc[a]);
  }
  c->fixf = parent->fixf;
  c->fixl = parent->fixl;
  c->fixf.push_back(facility);
  c->fixl.push_back(location);
  c->n = nr;
  c->m = nr - 2;
  c->T = (long long)nr * nr * (nr - 1) * (nr - 1);
  c->E = c->T * c->m * c->m;
  c->ntrip = nr * (nr - 1) * (nr - 2) / 6;
  rlt2_status st = ctx_alloc(c, true);
  if (st != RLT2_OK) return st;
  cudaStream_t s = c->stream;
  cudaError_t e;
  {
    const long long blocks = (c->E + 255) / 256;
    k_child_z<<<(int)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(parent->n, f, l, parent->Dhat, c->Dhat, c->E);
    const long long b2 = (c->T + 255) / 256;
    k_child_yx<<<(int)(b2 < 4096 ? b2 : 4096), 256, 0, s>>>(
        parent->n, f, l, parent->Dhat, parent->Chat, parent->bprime, parent->bqap, parent->Fr, parent->Dr,
        parent->d_cst, parent->d_cst_qap, c->Chat, c->bprime, c->bqap, c->Fr, c->Dr, c->d_cst, c->d_cst_qap, c->T);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c->sc->lb_base, c->d_cst, sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&c->cst_host, c->d_cst, 8, cudaMemcpyDeviceToHost);
  for (int mm2 : {nr - 2, nr - 1, nr})
    if (e == cudaSuccess) e = prepare_lap(mm2);
  if (e == cudaSuccess) e = prepare_lap(nr - 1, 0, 4);
  if (e != cudaSuccess) {
    rlt2_status r = cuda_fail(e, "rlt2_create_child");
    ctx_free(c);
    return r;
  }
  *out = c;
  return RLT2_OK;
}

MoveYArgs rlt2::make_move_y(const IterView& v) {
  const rlt2_params& p = v.prm;
  const int n = v.n;
  MoveYArgs a{};
  a.n = n;
  a.T = v.T;
  a.cy = p.ky / (double)(n - 2);
  a.cx = p.kx / ((double)(n - 1) * (double)(n - 2));
  a.phi_y = p.phi_y;
  a.fast = p.variant == 1;
  a.half = p.half_z;
  a.cxy = p.kx / (double)(n - 1);
  a.shift_psi = make_move_z(v).folded;
  a.psi = v.psi;
  a.keep_y = (1.0 - p.ky) - p.phi_y;
  a.keep_x = 1.0 - p.kx;
  a.piy = v.piy;
  a.pix = v.pix;
  a.Chat = v.Chat;
  a.tterm = v.tterm;
  a.xcost = v.xcost;
  a.saterm = v.saterm;
  a.sa_kf = v.sa_kf;
  a.sa_kl = v.sa_kl;
  a.sa_K = v.sa_K;
  a.sa_thr = v.sa_thr;
  a.sa_count = v.sa_count;
  a.c4 = 1.0 / (((double)n * (double)(n - 1)) * (double)(n - 2));
  a.sc = v.sc;
  a.lap_head = &v.sc->lap_head;
  return a;
}

Phase2Args rlt2::make_phase2(const IterView& v) {
  Phase2Args a{};
  a.n = v.n;
  a.m = v.m;
  a.tol = v.prm.phase2_tol;
  a.Dhat = v.Dhat;
  a.xi = v.xi;
  a.psi = v.psi;
  a.trips = v.trips;
  a.sc = v.sc;
  return a;
}

MoveZArgs rlt2::make_move_z(const IterView& v) {
  const rlt2_params& p = v.prm;
  MoveZArgs mz{};
  mz.n = v.n;
  mz.m = v.m;
  mz.kz = p.kz;
  for (int l = 0; l < 5; ++l) mz.w[l] = p.phi_z[h_widx[l]];
  mz.kz_one = (p.kz == 1.0);
  mz.uniform = (p.phi_z[0] == p.phi_z[1] && p.phi_z[0] == p.phi_z[2] && p.phi_z[0] == p.phi_z[3] &&
                p.phi_z[0] == p.phi_z[4]);
  mz.fast = p.variant == 1;
  mz.half = p.half_z;
  mz.folded = p.variant == 0 && !p.half_z && mz.kz_one && mz.uniform;
  mz.c1 = -(1.0 + p.phi_z[0]);
  mz.saterm = v.saterm;
  mz.Dhat = v.Dhat;
  mz.xi = v.xi;
  mz.psi = v.psi;
  mz.tterm = v.tterm;
  mz.trips = v.trips;
  mz.sc = v.sc;
  return mz;
}

FinArgs rlt2::make_fin(const IterView& v) {
  const rlt2_params& p = v.prm;
  FinArgs f{};
  f.n = v.n;
  f.m = v.m;
  f.cst = v.d_cst;
  f.xval = v.xval;
  f.xperm = v.xperm;
  f.ubperm = v.ubperm;
  f.piy = v.piy;
  f.Dhat = v.Dhat;
  f.xi = v.xi;
  f.psi = v.psi;
  f.Fr = v.Fr;
  f.Dr = v.Dr;
  f.bprime = v.bprime;
  f.bqap = v.bqap ? v.bqap : v.bprime;
  f.cst_qap = v.cst_qap ? v.cst_qap : v.d_cst;
  f.ring = v.ring;
  f.min_gap = p.min_gap;
  f.ub_known = p.ub;
  f.feas_tol = p.feas_tol;
  f.stall_window = p.stall_window;
  f.stall_tol = p.stall_tol;
  f.fast = p.variant == 1;
  f.sc = v.sc;
  return f;
}

// Enqueue one iteration on stream s.  With ev != nullptr, the 2 kKinds events
// ev[2k], ev[2k+1] bracket timing kind k (kinds 6 and 7, the second Z phase,
// are empty intervals without two_phase); launched[k] counts the kernels.
cudaError_t rlt2::enqueue_iteration(const IterView& v, cudaStream_t s, cudaEvent_t* ev, int* launched) {
  auto count = [&](int k, int nk) {
    if (launched) launched[k] += nk;
  };
  const int n = v.n, m = v.m;
  const long long T = v.T;
  const rlt2_params& p = v.prm;
  const int* done = &v.sc->done;
  cudaError_t e;
  auto rec = [&](int k, int which) -> cudaError_t {
    if (!ev) return cudaSuccess;
    return cudaEventRecord(ev[2 * k + which], s);
  };
  // 1) y move (and F's x move) + tile terms
  if ((e = rec(0, 0)) != cudaSuccess) return e;
  {
    const MoveYArgs my = make_move_y(v);
    const long long blocks = (T + 255) / 256;
    k_move_y<<<(int)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(my);
    count(0, 1);
  }
  if ((e = cudaGetLastError()) != cudaSuccess || (e = rec(0, 1)) != cudaSuccess) return e;
  // 2) z move (inside the Z-stage launch when pipelined)
  const MoveZArgs mz = make_move_z(v);
  const bool pipelined = v.pplan && v.pipe && !p.half_z && p.warm != 2;
  if ((e = rec(1, 0)) != cudaSuccess) return e;
  if (!pipelined) {
    // one thread per (q, r) class of the block's (triple, p): round to whole warps
    k_move_z<<<v.ntrip * n, move_z_threads(n), 0, s>>>(mz);
    count(1, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = rec(1, 1)) != cudaSuccess) return e;
  // 3) Z stage
  LapArgs z{};
  z.batch = v.zmap ? v.Tz : T;
  z.map = v.zmap;
  z.m = m;
  z.A = v.Dhat;
  z.u0 = p.warm == 1 ? v.xi : nullptr;
  z.warm_gate = &v.sc->have_snap;
  if (p.warm == 2 && v.mlp && v.u0buf) {
    // learned start from the tile and the row's previous dual (zero before the first solve)
    if ((e = mlp_predict_enqueue(v.mlp, T, m, v.Dhat, v.xi, v.u0buf, s, launched ? launched + 2 : nullptr)) !=
        cudaSuccess)
      return e;
    z.u0 = v.u0buf;
    z.warm_gate = nullptr;
  }
  z.value = v.Theta;
  z.u = v.xi;
  z.v = v.psi;
  z.dual_mode = p.dual_mode;
  z.stats = v.sc->stats + 0;
  z.head = &v.sc->lap_head;
  z.head_zeroed = 1;  // by k_move_y
  z.skip = done;
  if ((e = rec(2, 0)) != cudaSuccess) return e;
  if (pipelined) {
    if ((e = launch_move_lap_z(mz, z, *v.pplan, v.pipe, v.sc, s, v.pipe_check != 0)) != cudaSuccess) return e;
  } else if ((e = launch_lap(z, s)) != cudaSuccess) {
    return e;
  }
  count(2, 1);
  if ((e = rec(2, 1)) != cudaSuccess) return e;
  // 3b) two-phase Z solve: move slack onto the zero-slack members, solve again
  if ((e = rec(6, 0)) != cudaSuccess) return e;
  if (p.two_phase) {
    k_phase2<<<v.ntrip * n, move_z_threads(n), 0, s>>>(make_phase2(v));
    count(6, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = rec(6, 1)) != cudaSuccess || (e = rec(7, 0)) != cudaSuccess) return e;
  if (p.two_phase) {
    LapArgs z2 = z;
    z2.u0 = p.warm >= 1 ? v.xi : nullptr;  // from the first phase's row duals
    z2.warm_gate = nullptr;
    z2.head_zeroed = 0;  // the first phase used the counter
    if ((e = launch_lap(z2, s)) != cudaSuccess) return e;
    count(7, 1);
  }
  if ((e = rec(7, 1)) != cudaSuccess) return e;
  // 4) Y stage on C^ + Theta, writes pi_y
  LapArgs y{};
  y.batch = (long long)n * n;
  y.m = n - 1;
  y.A = v.Chat;
  y.Badd = v.Theta;
  y.value = v.Delta;
  y.u = v.gamma;
  y.u0 = p.warm >= 1 ? v.gamma : nullptr;  // previous iteration's row duals
  y.warm_gate = &v.sc->have_snap;
  y.v = v.delta;
  y.pi = v.piy;
  y.dual_mode = p.dual_mode;
  y.stats = v.sc->stats + 2;
  y.skip = done;
  y.warps_per_block = 4;  // n^2 LAPs only: spread them over more SMs
  if ((e = rec(3, 0)) != cudaSuccess) return e;
  if ((e = launch_lap(y, s)) != cudaSuccess) return e;
  count(3, 1);
  if ((e = rec(3, 1)) != cudaSuccess) return e;
  // 5) X stage on b' + Delta, writes pi_x
  LapArgs x{};
  x.batch = 1;
  x.m = n;
  x.A = v.xcost;
  x.Badd = v.Delta;
  x.value = v.xval;
  x.u = v.alpha;
  x.u0 = p.warm >= 1 ? v.alpha : nullptr;
  x.warm_gate = &v.sc->have_snap;
  x.v = v.beta;
  x.r2c = v.xperm;
  x.pi = v.pix;
  x.dual_mode = p.dual_mode;
  x.stats = v.sc->stats + 4;
  x.skip = done;
  if ((e = rec(4, 0)) != cudaSuccess) return e;
  if ((e = launch_lap(x, s)) != cudaSuccess) return e;
  count(4, 1);
  if ((e = rec(4, 1)) != cudaSuccess) return e;
  // 6) finalize
  const FinArgs f = make_fin(v);
  if ((e = rec(5, 0)) != cudaSuccess) return e;
  k_finalize<<<1, 256, 0, s>>>(f);
  count(5, 1);
  if ((e = cudaGetLastError()) != cudaSuccess || (e = rec(5, 1)) != cudaSuccess) return e;
  return cudaSuccess;
}

static cudaError_t enqueue_iteration_ctx(rlt2_ctx* c, cudaStream_t s, int ev_base, int* launched = nullptr) {
  return enqueue_iteration(view_of(c), s, ev_base < 0 ? nullptr : c->ev.data() + ev_base, launched);
}

// Failure detection of the pipelined launch without a fault: one iteration
// whose Z-LAP warps wait for pair counts the move never reaches, with the
// polls capped low; the first wait to give up stops the context (reason 4)
// and the remaining LAPs of the launch are skipped.
extern "C" rlt2_status rlt2_pipeline_check_wait_timeout(rlt2_ctx* c) {
  if (!c || c->prm.pipeline != 1 || !c->pplan || !c->pipe || c->prm.warm == 2 || c->enqueued < 1) {
    set_error("rlt2_pipeline_check_wait_timeout: needs a context with pipeline = 1 (warm 0 or 1) that has "
              "run at least one iteration");
    return RLT2_EINVAL;
  }
  IterView v = view_of(c);
  v.pipe_check = 1;
  cudaError_t e = enqueue_iteration(v, c->stream, nullptr, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "rlt2_pipeline_check_wait_timeout");
  c->enqueued += 1;
  DevScalars h;
  CK(cudaMemcpyAsync(&h, c->sc, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->iter_host = h.iter;
  if (h.reason == 4) {
    set_error("rlt2_pipeline_check_wait_timeout: the pipelined wait gave up as intended; the context is stopped");
    return RLT2_ETIMEOUT;
  }
  return RLT2_OK;
}

// Iterations per replay of the longer graph: within one graph the kernels of
// consecutive iterations follow each other with the short intra-graph gap
// instead of a graph launch's.
constexpr int kGraphIters = 8;

// Captures `iters` iterations into *out.
static rlt2_status capture_graph(rlt2_ctx* c, int iters, cudaGraphExec_t* out) {
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < iters && e == cudaSuccess; ++it) e = enqueue_iteration_ctx(c, c->cap_stream, -1);
  cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e, "capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  return RLT2_OK;
}

static rlt2_status build_graph(rlt2_ctx* c) {
  if (c->graph) return RLT2_OK;
  rlt2_status st = capture_graph(c, 1, &c->graph);
  if (st != RLT2_OK) return st;
  if ((st = capture_graph(c, kGraphIters, &c->graph_many)) != RLT2_OK) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return st;
}

// The graphs hold the arguments they were captured with.
static void drop_graphs(rlt2_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph_many) cudaGraphExecDestroy(c->graph_many);
  c->graph = c->graph_many = nullptr;
}

constexpr int kEvChunk = 64;  // iterations per batch of timing events
// A context's first kDirectIters iterations are launched kernel by kernel:
// capturing and instantiating the CUDA graphs costs about as much as one
// iteration of a mid-size node, which short-lived branch-and-bound contexts
// never win back; the iterations are GPU-bound either way.
constexpr long long kDirectIters = 64;

static rlt2_status enqueue_many(rlt2_ctx* c, int iters) {
  if (c->prm.warm == 2 && !c->mlp) {
    set_error("warm == 2 needs a network: call rlt2_set_mlp first");
    return RLT2_EINVAL;
  }
  if (c->timing) {
    // the event pool was created by rlt2_set_timing; reuse it every kEvChunk iterations
    for (int base = 0; base < iters; base += kEvChunk) {
      const int cnt = (iters - base) < kEvChunk ? (iters - base) : kEvChunk;
      int launched[kKinds] = {};
      for (int it = 0; it < cnt; ++it) {
        cudaError_t e = enqueue_iteration_ctx(c, c->stream, it * kKinds * 2, launched);
        if (e != cudaSuccess) return cuda_fail(e, "enqueue_iteration");
      }
      for (int k = 0; k < kKinds; ++k) c->kcount[k] += launched[k];
      // finalize (kind 5) is the last interval recorded in an iteration
      CK(cudaEventSynchronize(c->ev[(cnt - 1) * kKinds * 2 + 2 * 5 + 1]));
      for (int it = 0; it < cnt; ++it)
        for (int k = 0; k < kKinds; ++k) {
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, c->ev[it * kKinds * 2 + 2 * k], c->ev[it * kKinds * 2 + 2 * k + 1]));
          c->kms[k] += ms;
        }
    }
    return RLT2_OK;
  }
  if (!c->graph && c->enqueued + iters <= kDirectIters) {
    for (int it = 0; it < iters; ++it) {
      cudaError_t e = enqueue_iteration_ctx(c, c->stream, -1);
      if (e != cudaSuccess) return cuda_fail(e, "enqueue_iteration");
    }
    c->enqueued += iters;
    return RLT2_OK;
  }
  rlt2_status st = build_graph(c);
  if (st != RLT2_OK) return st;
  int left = iters;
  for (; left >= kGraphIters; left -= kGraphIters) CK(cudaGraphLaunch(c->graph_many, c->stream));
  for (; left > 0; --left) CK(cudaGraphLaunch(c->graph, c->stream));
  c->enqueued += iters;
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_iterate_many(rlt2_ctx* const* ctxs, int count, int iters, int* done) {
  if (!ctxs || count < 1 || count > kMaxWaveNodes || iters < 0) {
    set_error("rlt2_iterate_many: need 1 <= count <= 1024 contexts and iters >= 0");
    return RLT2_EINVAL;
  }
  const rlt2_ctx* c0 = ctxs[0];
  for (int k = 0; k < count; ++k) {
    const rlt2_ctx* c = ctxs[k];
    if (!c) {
      set_error("rlt2_iterate_many: a context is NULL");
      return RLT2_EINVAL;
    }
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == c) {
        set_error("rlt2_iterate_many: a context appears twice");
        return RLT2_EINVAL;
      }
    if (c->prm.dual_mode != c0->prm.dual_mode || c->prm.warm != c0->prm.warm ||
        c->prm.two_phase != c0->prm.two_phase) {
      set_error("rlt2_iterate_many: the contexts must share dual_mode, warm and two_phase");
      return RLT2_EINVAL;
    }
    if (c->prm.half_z || c->prm.warm == 2 || c->sa_count > 0) {
      set_error("rlt2_iterate_many: the half-Z scheme, the learned start and Type 4 draws need rlt2_iterate");
      return RLT2_EINVAL;
    }
  }
  // the contexts' own streams first (their earlier work), then everything on the first one's
  for (int k = 0; k < count; ++k) CK(cudaStreamSynchronize(ctxs[k]->stream));
  std::vector<IterView> views;
  std::vector<int> before(count);
  views.reserve(count);
  for (int k = 0; k < count; ++k) {
    views.push_back(view_of(ctxs[k]));
    before[k] = ctxs[k]->iter_host;
  }
  int ran = 0;
  const cudaError_t e = iterate_views(views.data(), count, c0->prm, iters, c0->stream, &ran);
  if (e != cudaSuccess) return cuda_fail(e, "rlt2_iterate_many");
  for (int k = 0; k < count; ++k) {
    rlt2_ctx* c = ctxs[k];
    int it = 0;
    CK(cudaMemcpy(&it, &c->sc->iter, sizeof(int), cudaMemcpyDeviceToHost));
    c->enqueued += ran;
    c->iter_host = it;
    if (done) done[k] = it - before[k];
  }
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_iterate_async(rlt2_ctx* c, int iters) {
  if (!c || iters < 0) {
    set_error("rlt2_iterate_async: invalid argument");
    return RLT2_EINVAL;
  }
  if (iters == 0) return RLT2_OK;
  return enqueue_many(c, iters);
}

extern "C" rlt2_status rlt2_iterate(rlt2_ctx* c, int iters, double* lb_hist, int* done) {
  if (!c || iters < 0) {
    set_error("rlt2_iterate: invalid argument");
    return RLT2_EINVAL;
  }
  int total = 0;
  // chunks of 8, 16, 32, ... iterations: a stop on the device (feasibility,
  // min-gap, stall) ends the call after the chunk it falls in, so stopped
  // contexts (fathomed branch-and-bound nodes) do not run many no-op launches
  int step = 8;
  for (int off = 0; off < iters;) {
    int chunk = iters - off;
    if (chunk > step) chunk = step;
    if (chunk > kRing) chunk = kRing;
    step = step < 1024 ? 2 * step : step;
    const int it0 = c->iter_host;
    rlt2_status st = enqueue_many(c, chunk);
    if (st != RLT2_OK) return st;
    DevScalars h;
    CK(cudaMemcpyAsync(&h, c->sc, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int got = h.iter - it0;
    c->iter_host = h.iter;
    total += got;
    if (h.reason == 4) {
      set_error("rlt2_iterate: a pipelined Z-stage wait gave up (the step's results are not valid)");
      if (done) *done = total;
      return RLT2_ETIMEOUT;
    }
    if (lb_hist) {
      // copy only the entries of this chunk (at most two pieces around the ring's end)
      int k = 0;
      while (k < got) {
        const int pos = (it0 + k) & (kRing - 1);
        const int len = (got - k) < (kRing - pos) ? (got - k) : (kRing - pos);
        CK(cudaMemcpy(lb_hist + off + k, c->ring + pos, sizeof(double) * len, cudaMemcpyDeviceToHost));
        k += len;
      }
      for (k = got; k < chunk; ++k) lb_hist[off + k] = NAN;
    }
    if (got < chunk) {
      if (lb_hist)
        for (int k = off + chunk; k < iters; ++k) lb_hist[k] = NAN;
      break;
    }
    off += chunk;
  }
  if (done) *done = total;
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_bound(rlt2_ctx* c, double* lb, double* best_lb, double* ub, int* perm, int* ub_perm,
                                  int* iters) {
  if (!c) return RLT2_EINVAL;
  DevScalars h;
  std::vector<int> xp(c->n), up(c->n);
  CK(cudaMemcpyAsync(&h, c->sc, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(xp.data(), c->xperm, sizeof(int) * c->n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(up.data(), c->ubperm, sizeof(int) * c->n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (lb) *lb = h.lb;
  if (best_lb) *best_lb = h.best_lb;
  if (ub) *ub = h.ub;
  if (iters) *iters = h.iter;
  int* outs[2] = {perm, ub_perm};
  const std::vector<int>* srcs[2] = {&xp, &up};
  for (int w = 0; w < 2; ++w) {
    int* o = outs[w];
    if (!o) continue;
    for (int i = 0; i < c->n_full; ++i) o[i] = -1;
    for (size_t x = 0; x < c->fixf.size(); ++x) o[c->fixf[x]] = c->fixl[x];
    if (h.iter > 0)
      for (int i = 0; i < c->n; ++i) o[c->fac[i]] = c->loc[(*srcs[w])[i]];
  }
  return RLT2_OK;
}

static rlt2_status copy_out(rlt2_ctx* c, double* dst, const double* src, size_t count, int on_device) {
  if (!dst) return RLT2_OK;
  CK(cudaMemcpyAsync(dst, src, count * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->stream));
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_duals(rlt2_ctx* c, double* alpha, double* beta, double* gamma, double* delta, double* xi,
                                  double* psi, int on_device) {
  if (!c) return RLT2_EINVAL;
  const size_t n = c->n, yd = n * n * (n - 1), zd = (size_t)c->T * c->m;
  rlt2_status st;
  if ((st = copy_out(c, alpha, c->alpha, n, on_device)) != RLT2_OK) return st;
  if ((st = copy_out(c, beta, c->beta, n, on_device)) != RLT2_OK) return st;
  if ((st = copy_out(c, gamma, c->gamma, yd, on_device)) != RLT2_OK) return st;
  if ((st = copy_out(c, delta, c->delta, yd, on_device)) != RLT2_OK) return st;
  if ((st = copy_out(c, xi, c->xi, zd, on_device)) != RLT2_OK) return st;
  if ((st = copy_out(c, psi, c->psi, zd, on_device)) != RLT2_OK) return st;
  CK(cudaStreamSynchronize(c->stream));
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_reduced_costs(rlt2_ctx* c, double* pi_x, double* pi_y, double* pi_z, int on_device) {
  if (!c) return RLT2_EINVAL;
  rlt2_status st;
  if ((st = copy_out(c, pi_x, c->pix, (size_t)c->n * c->n, on_device)) != RLT2_OK) return st;
  if ((st = copy_out(c, pi_y, c->piy, (size_t)c->T, on_device)) != RLT2_OK) return st;
  if (pi_z) {
    double* dst = pi_z;
    double* tmp = nullptr;
    if (!on_device) {
      CK(cudaMalloc((void**)&tmp, sizeof(double) * (size_t)c->E));
      dst = tmp;
    }
    k_pi_z<<<4096, 256, 0, c->stream>>>(c->E, c->m, c->Dhat, c->xi, c->psi, dst);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && tmp)
      e = cudaMemcpyAsync(pi_z, tmp, sizeof(double) * (size_t)c->E, cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "pi_z");
    if (e2 != cudaSuccess) return cuda_fail(e2, "pi_z sync");
  }
  CK(cudaStreamSynchronize(c->stream));
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_export_state(rlt2_ctx* c, double* Dhat, double* Chat, int on_device) {
  if (!c) return RLT2_EINVAL;
  rlt2_status st;
  if ((st = copy_out(c, Dhat, c->Dhat, (size_t)c->E, on_device)) != RLT2_OK) return st;
  if ((st = copy_out(c, Chat, c->Chat, (size_t)c->T, on_device)) != RLT2_OK) return st;
  CK(cudaStreamSynchronize(c->stream));
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_import_state(rlt2_ctx* c, const double* Dhat, const double* Chat, int on_device) {
  if (!c) return RLT2_EINVAL;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (Dhat) CK(cudaMemcpyAsync(c->Dhat, Dhat, sizeof(double) * (size_t)c->E, k, c->stream));
  if (Chat) CK(cudaMemcpyAsync(c->Chat, Chat, sizeof(double) * (size_t)c->T, k, c->stream));
  const int zero = 0;
  CK(cudaMemcpyAsync(&c->sc->have_snap, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(&c->sc->done, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_export_xstate(rlt2_ctx* c, double* bx, double* lb_base) {
  if (!c) return RLT2_EINVAL;
  const size_t n2 = (size_t)c->n * c->n;
  if (bx) CK(cudaMemcpyAsync(bx, c->xcost, sizeof(double) * n2, cudaMemcpyDeviceToHost, c->stream));
  DevScalars h;
  CK(cudaMemcpyAsync(&h, c->sc, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (lb_base) *lb_base = (c->prm.variant == 1) ? h.lb_base : c->cst_host;
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_import_xstate(rlt2_ctx* c, const double* bx, double lb_base) {
  if (!c || !bx || !std::isfinite(lb_base)) {
    set_error("rlt2_import_xstate: invalid argument");
    return RLT2_EINVAL;
  }
  const size_t n2 = (size_t)c->n * c->n;
  if (!finite_all(bx, n2)) {
    set_error("rlt2_import_xstate: non-finite x costs");
    return RLT2_EINVAL;
  }
  if (c->prm.variant != 1) return RLT2_OK;  // S: b' and the constant never change
  CK(cudaMemcpyAsync(c->xcost, bx, sizeof(double) * n2, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(&c->sc->lb_base, &lb_base, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  const int zero = 0;
  CK(cudaMemcpyAsync(&c->sc->have_snap, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_set_sa(rlt2_ctx* c, int count, const double* kf, const double* kl,
                                   const double* neglog_u) {
  if (!c || count < 0) {
    set_error("rlt2_set_sa: invalid argument");
    return RLT2_EINVAL;
  }
  const int n = c->n;
  const rlt2_params& p = c->prm;
  if (count > 0 && p.half_z) {
    set_error("rlt2_set_sa: the Type 4 rule is not combined with the half-Z scheme");
    return RLT2_EINVAL;
  }
  if (count > 0) {
    if (!kf || !kl || !neglog_u) {
      set_error("rlt2_set_sa: NULL draws");
      return RLT2_EINVAL;
    }
    if (!(p.ub > 0.0) || !(p.sa_t0 > 0.0) || !(p.sa_cool > 0.0 && p.sa_cool <= 1.0) || p.sa_period < 1) {
      set_error("rlt2_set_sa: needs ub > 0, sa_t0 > 0, 0 < sa_cool <= 1, sa_period >= 1");
      return RLT2_EINVAL;
    }
  }
  // host side of the schedule: K[d] (facilities first, index order) and
  // thr[d] = neglog_u[d] * T_d, T_0 = sa_t0 * ub, times sa_cool every sa_period draws
  const long long cn = (long long)count * n;
  std::vector<double> buf((size_t)(2 * cn + 2 * (long long)count));
  double temp = p.sa_t0 * p.ub;
  for (int d = 0; d < count; ++d) {
    if (d > 0 && d % p.sa_period == 0) temp = temp * p.sa_cool;
    double k = 0.0;
    for (int i = 0; i < n; ++i) {
      const double x = kf[(long long)d * n + i];
      if (!std::isfinite(x) || x < 0.0 || x > 1.0) {
        set_error("rlt2_set_sa: kappa outside [0, 1]");
        return RLT2_EINVAL;
      }
      buf[(size_t)((long long)d * n + i)] = x;
      k = k + x;
    }
    for (int q = 0; q < n; ++q) {
      const double x = kl[(long long)d * n + q];
      if (!std::isfinite(x) || x < 0.0 || x > 1.0) {
        set_error("rlt2_set_sa: kappa outside [0, 1]");
        return RLT2_EINVAL;
      }
      buf[(size_t)(cn + (long long)d * n + q)] = x;
      k = k + x;
    }
    if (k > 1.0 || !std::isfinite(neglog_u[d]) || neglog_u[d] < 0.0) {
      set_error("rlt2_set_sa: kappa sum above 1 or bad -ln(u)");
      return RLT2_EINVAL;
    }
    buf[(size_t)(2 * cn + d)] = k;
    buf[(size_t)(2 * cn + count + d)] = neglog_u[d] * temp;
  }
  CK(cudaStreamSynchronize(c->stream));
  if (c->sa_buf) {
    cudaFree(c->sa_buf);
    c->sa_buf = nullptr;
  }
  c->sa_count = 0;
  if (count > 0) {
    cudaError_t e = cudaMalloc((void**)&c->sa_buf, sizeof(double) * buf.size());
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? (cuda_fail(e, "cudaMalloc"), RLT2_ENOMEM)
                                                                 : cuda_fail(e, "cudaMalloc");
    CK(cudaMemcpy(c->sa_buf, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice));
    c->sa_count = count;
  }
  drop_graphs(c);  // the graphs hold the old arguments
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_stats(rlt2_ctx* c, long long* out) {
  if (!c || !out) return RLT2_EINVAL;
  DevScalars h;
  CK(cudaMemcpyAsync(&h, c->sc, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  out[0] = h.iter;
  for (int k = 0; k < 6; ++k) out[1 + k] = (long long)h.stats[k];
  out[7] = h.reason;
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_sizes(rlt2_ctx* c, int* n_res, long long* T, long long* E, double* cst) {
  if (!c) return RLT2_EINVAL;
  if (n_res) *n_res = c->n;
  if (T) *T = c->T;
  if (E) *E = c->E;
  if (cst) *cst = c->cst_host;
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_set_timing(rlt2_ctx* c, int on) {
  if (!c) return RLT2_EINVAL;
  c->timing = on != 0;
  for (int k = 0; k < kKinds; ++k) {
    c->kms[k] = 0.0;
    c->kcount[k] = 0;
  }
  while (c->timing && c->ev.size() < (size_t)kEvChunk * kKinds * 2) {
    cudaEvent_t ev;
    CK(cudaEventCreate(&ev));
    c->ev.push_back(ev);
  }
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_kernel_times(rlt2_ctx* c, double* ms, long long* count, int nk) {
  if (!c || nk < 0) return RLT2_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < nk && k < kKinds; ++k) {
    if (ms) ms[k] = c->kms[k];
    if (count) count[k] = c->kcount[k];
  }
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_set_mlp(rlt2_ctx* c, rlt2_mlp* m) {
  if (!c) return RLT2_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  if (m && !c->u0buf) CK(cudaMalloc((void**)&c->u0buf, sizeof(double) * (size_t)c->T * c->m));
  c->mlp = m;
  drop_graphs(c);
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_destroy(rlt2_ctx* c) {
  if (!c) return RLT2_OK;
  cudaStreamSynchronize(c->stream);
  ctx_free(c);
  return RLT2_OK;
}

extern "C" const char* rlt2_strerror(rlt2_status s) {
  switch (s) {
    case RLT2_OK: return "ok";
    case RLT2_EINVAL: return "invalid argument";
    case RLT2_ENOMEM: return "out of device memory";
    case RLT2_ECUDA: return "CUDA error";
    case RLT2_ETIMEOUT: return "device wait timed out";
    case RLT2_EADMIT: return "node does not fit the memory budget";
  }
  return "unknown status";
}

extern "C" const char* rlt2_last_error(void) { return g_last_error.c_str(); }
