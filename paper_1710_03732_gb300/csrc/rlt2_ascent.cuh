// Device bodies of the ascent kernels, shared by the single-problem kernels
// (ascent.cu) and the batched branch-and-bound node kernels (nodes.cu).
#pragma once
#include <cuda_runtime.h>

#include <cmath>

#include "rlt2_internal.h"

namespace rlt2 {

__device__ __forceinline__ double dadd_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul_(double a, double b) { return __dmul_rn(a, b); }

// ------------------------------------------------------------------ moves ----
// Per tile (i,p,j,q): the pending y move of Eq. 2.21 on C^ and the term
// cy*pi_y(ijpq) + cx*pi_x(ip) that rules 2 and 3 add to each z of the tile.
__device__ __forceinline__ void move_y_range(int n, long long T, double cy, double cx, double phi_y,
                                             const double* __restrict__ piy, const double* __restrict__ pix,
                                             double* __restrict__ Chat, double* __restrict__ tterm, long long start,
                                             long long stride) {
  const int n1 = n - 1;
  for (long long t = start; t < T; t += stride) {
    const int ip = (int)(t / (n1 * n1));
    const int rem = (int)(t - (long long)ip * n1 * n1);
    const int jj = rem / n1, qq = rem - jj * n1;
    const int i = ip / n, p = ip - i * n;
    const int j = jj + (jj >= i), q = qq + (qq >= p);
    const long long tp = ((long long)(j * n + q) * n1 + (i - (i > j))) * n1 + (p - (p > q));
    const double py = piy[t];
    tterm[t] = dadd_(dmul_(cy, py), dmul_(cx, pix[ip]));
    Chat[t] = dadd_(dsub_(Chat[t], dmul_(phi_y, py)), dmul_(phi_y, piy[tp]));
  }
}

// The six members of a class {(i,p),(j,q),(k,r)} are the position orders of the
// triples, member 0 = (i,j,k | p,q,r) and members 1..5 = its partners 1..5 in
// the order of Eq. 2.20: (i,k,j|p,r,q), (j,i,k|q,p,r), (j,k,i|q,r,p),
// (k,i,j|r,p,q), (k,j,i|r,q,p).
// kOrd[b] is member b's order; kPart[a][l] is the member that is the l-th
// partner of member a (apply order l+1 to member a's order).  The weight that
// partner gives back to member a is phi_{h_widx[l]}: the swaps are their own
// inverse and the two 3-cycles are each other's inverse.
#define RLT2_CLASS_TABLES                                                                              \
  constexpr int kOrd[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};      \
  constexpr int kPart[6][5] = {{1, 2, 3, 4, 5}, {0, 4, 5, 2, 3}, {3, 0, 1, 5, 4},                    \
                               {2, 5, 4, 0, 1}, {5, 1, 0, 3, 2}, {4, 3, 2, 1, 0}};

struct MoveZArgs {
  int n, m;
  double kz;
  double w[5];  // weight received from partner l (phi permuted by h_widx)
  int kz_one;   // kz == 1: kz*x == x exactly, skip the product
  int uniform;  // all phi equal: member b gets phi * (class sum - s_b)
  double* Dhat;
  const double* xi;
  const double* psi;
  const double* tterm;
  const int* trips;  // i | j<<8 | k<<16 with i<j<k
  const DevScalars* sc;
};

// One thread per class; a block covers one facility triple and one location p
// of its first facility (all (q, r)).  Consecutive threads take consecutive r,
// so members (i,j,k|p,q,r) and (j,i,k|q,p,r) are read and written as contiguous
// rows; the other four members' rows are shared by the block or by the n blocks
// of the same triple, which run back to back.
__device__ __forceinline__ void move_z_block(const MoveZArgs& a, int blk) {
  RLT2_CLASS_TABLES
  const int n = a.n, m = a.m, n1 = n - 1;
  const int tr = blk / n, p = blk - tr * n;
  const int packed = a.trips[tr];
  const int F3[3] = {packed & 255, (packed >> 8) & 255, packed >> 16};
  const int npairs = n1 * m;
  const long long mm = (long long)m * m;
  for (int c = threadIdx.x; c < npairs; c += blockDim.x) {
    const int qq = c / m, rr = c - qq * m;
    const int q = qq + (qq >= p);
    const int lo = p < q ? p : q, hi = p < q ? q : p;
    int r = rr;
    r += (r >= lo);
    r += (r >= hi);
    const int L3[3] = {p, q, r};
    double s[6], Dv[6];
    long long idx[6];
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      const int f0 = F3[kOrd[b][0]], f1 = F3[kOrd[b][1]], f2 = F3[kOrd[b][2]];
      const int l0 = L3[kOrd[b][0]], l1 = L3[kOrd[b][1]], l2 = L3[kOrd[b][2]];
      const long long t = ((long long)(f0 * n + l0) * n1 + (f1 - (f1 > f0))) * n1 + (l1 - (l1 > l0));
      const int kr = f2 - (f2 > f0) - (f2 > f1), cc = l2 - (l2 > l0) - (l2 > l1);
      idx[b] = t * mm + kr * m + cc;
      Dv[b] = a.Dhat[idx[b]];
      const double pz = dsub_(dsub_(Dv[b], __ldg(a.xi + t * m + kr)), __ldg(a.psi + t * m + cc));
      // s = kz*pi_z + tile term in one rounding (kz = 1: an exact fma(1, x, y) is x + y)
      s[b] = a.kz_one ? dadd_(pz, __ldg(a.tterm + t)) : __fma_rn(a.kz, pz, __ldg(a.tterm + t));
    }
    if (a.uniform) {
      // all phi equal: member b receives phi * (S - s_b), S the class sum in member order
      double S = s[0];
#pragma unroll
      for (int b = 1; b < 6; ++b) S = dadd_(S, s[b]);
#pragma unroll
      for (int b = 0; b < 6; ++b) a.Dhat[idx[b]] = __fma_rn(a.w[0], dsub_(S, s[b]), dsub_(Dv[b], s[b]));
    } else {
      // partner inflows one fused multiply-add at a time, partners in Eq. 2.20 order
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        double acc = dsub_(Dv[b], s[b]);
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = __fma_rn(a.w[l], s[kPart[b][l]], acc);
        a.Dhat[idx[b]] = acc;
      }
    }
  }
}

// ---------------------------------------------------------------- finalize ----
struct FinArgs {
  int n, m;
  const double* cst;
  const double* xval;
  const int* xperm;
  int* ubperm;
  const double* piy;
  const double* Dhat;
  const double* xi;
  const double* psi;
  const double* Fr;
  const double* Dr;
  const double* bprime;
  double* ring;
  double min_gap, ub_known, feas_tol, stall_tol;
  int stall_window;
  DevScalars* sc;
};

// Must be called by every thread of a block of 256 threads.
__device__ __forceinline__ void finalize_block(const FinArgs& a) {
  __shared__ double red[256];
  __shared__ int bad, improve;
  const int n = a.n, m = a.m, n1 = n - 1, tid = threadIdx.x;
  const double lb = dadd_(*a.cst, a.xval[0]);
  if (tid == 0) bad = (a.feas_tol > 0.0) ? 0 : 1;
  // residual QAP value of the X-LAP primal (an upper bound)
  double part = 0.0;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    const int si = a.xperm[i], sj = a.xperm[j];
    part += (i == j) ? a.bprime[i * n + si] : a.Fr[i * n + j] * a.Dr[si * n + sj];
  }
  red[tid] = part;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  const double ub = *a.cst + red[0];
  // feasibility check: every y and z built from the X primal has zero slack (Eq. 2.19)
  if (a.feas_tol > 0.0) {
    const double tol = a.feas_tol * fmax(1.0, fabs(lb));
    for (int e = tid; e < n * n1; e += blockDim.x) {
      const int i = e / n1, jj = e - i * n1, j = jj + (jj >= i);
      const int si = a.xperm[i], sj = a.xperm[j];
      const long long t = ((long long)(i * n + si) * n1 + jj) * n1 + (sj - (sj > si));
      if (fabs(a.piy[t]) > tol) bad = 1;
    }
    const int per = n1 * m;
    for (int e = tid; e < n * per; e += blockDim.x) {
      if (bad) break;
      const int i = e / per, w = e - i * per, jj = w / m, kk = w - jj * m;
      const int j = jj + (jj >= i);
      const int lo = i < j ? i : j, hi = i < j ? j : i;
      int k = kk;
      k += (k >= lo);
      k += (k >= hi);
      const int si = a.xperm[i], sj = a.xperm[j], sk = a.xperm[k];
      const long long t = ((long long)(i * n + si) * n1 + jj) * n1 + (sj - (sj > si));
      const int rc = sk - (sk > si) - (sk > sj);
      const double pz = dsub_(dsub_(a.Dhat[t * m * m + (long long)kk * m + rc], a.xi[t * m + kk]), a.psi[t * m + rc]);
      if (fabs(pz) > tol) bad = 1;
    }
  }
  if (tid == 0) improve = ub < a.sc->ub;
  __syncthreads();
  if (improve)
    for (int i = tid; i < n; i += blockDim.x) a.ubperm[i] = a.xperm[i];
  if (tid == 0) {
    DevScalars* sc = a.sc;
    sc->lb = lb;
    if (sc->iter == 0 || lb > sc->best_lb) sc->best_lb = lb;
    if (improve) sc->ub = ub;
    const int it = sc->iter;
    a.ring[it & (kRing - 1)] = lb;
    sc->iter = it + 1;
    sc->have_snap = 1;
    double ubk = sc->ub;
    if (a.ub_known > 0.0 && a.ub_known < ubk) ubk = a.ub_known;
    sc->gap = (ubk - sc->best_lb) / fabs(ubk);
    sc->best_hist[it % kStallRing] = sc->best_lb;
    if (!bad) {
      sc->done = 1;
      sc->reason = 1;
    } else if (a.min_gap > 0.0 && sc->gap < a.min_gap) {
      sc->done = 1;
      sc->reason = 2;
    } else if (a.stall_window > 0 && it >= a.stall_window &&
               sc->best_lb - sc->best_hist[(it - a.stall_window) % kStallRing] <
                   a.stall_tol * fmax(1.0, fabs(ubk))) {
      sc->done = 1;
      sc->reason = 3;
    }
  }
}

// Threads of a z-move block: the (n-1)(n-2) classes of one (triple, p) in
// equal passes of at most 512 threads, rounded to whole warps.
inline int move_z_threads(int n) {
  const int c = (n - 1) * (n - 2);
  const int passes = (c + 511) / 512;
  return ((c + passes - 1) / passes + 31) / 32 * 32;
}

// Kernel arguments of one problem's z move and finalize step (host helpers).
MoveZArgs make_move_z(const IterView& v);
FinArgs make_fin(const IterView& v);

}  // namespace rlt2
