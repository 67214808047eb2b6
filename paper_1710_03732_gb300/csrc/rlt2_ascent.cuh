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

// 64-bit key that orders like the double (non-NaN; -0 == +0), for compares off the FP64 pipe.
__device__ __forceinline__ unsigned long long okey_(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  b = (b == 0x8000000000000000ull) ? 0ull : b;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// ------------------------------------------------------------------ moves ----
struct MoveYArgs {
  int n;
  long long T;
  double cy, cx, phi_y;
  int fast;              // F variant: new incremental y and x costs from the slacks
  int half;              // half-Z scheme (see move_y_range)
  double keep_y, keep_x;  // (1 - ky) - phi_y and 1 - kx (F variant)
  double cxy;             // half-Z scheme: kx / (n-1), Type 3 on the y level for the lower rows
  int shift_psi;          // folded z move: psi <- psi - tile term, in place (psi is rewritten by the next Z solve)
  double* psi;
  const double* piy;
  const double* pix;
  double* Chat;
  double* tterm;
  double* xcost;   // F: written with keep_x * pi_x
  double* saterm;  // n*n Type 4 amounts of an accepted draw
  const double *sa_kf, *sa_kl, *sa_K, *sa_thr;
  int sa_count;
  double c4;  // 1 / (n (n-1) (n-2))
  DevScalars* sc;
  unsigned long long* lap_head;  // nullable: the Z stage's LAP queue counter, zeroed by the y-move launch
};

// Per tile (i,p,j,q): the pending y move on C^ (S: Eq. 2.21 on the full cost;
// F: keep_y pi_y(ijpq) + phi_y pi_y(jiqp); half-Z scheme: Eq. 2.21 plus the
// lower rows' x slack moved on the y level), the term cy*pi_y(ijpq) + cx*pi_x(ip)
// that rules 2 and 3 add to each z pool of the tile, plus the Type 4 amount
// kf_i g + kl_p g of an accepted draw (rule 4, Section 5: accepted when
// kappa^lb * nu <= -ln(u) T).  Thread 0 records the draw's acceptance and, in
// F, makes the last bound the base of the next one (Eq. 3.7).
struct MoveYDraw {
  bool on;  // the Type 4 draw of this iteration was accepted
  double g;
  const double* kf;
  const double* kl;
};

__device__ __forceinline__ MoveYDraw move_y_draw(const MoveYArgs& a) {
  MoveYDraw r{false, 0.0, nullptr, nullptr};
  if (a.sa_count > 0) {
    const int d = a.sc->iter - 1;
    if (d >= 0 && d < a.sa_count) {
      const double nu = a.sc->lb;
      if (dmul_(a.sa_K[d], nu) <= a.sa_thr[d]) {
        r.on = true;
        r.g = dmul_(nu, a.c4);
        r.kf = a.sa_kf + (long long)d * a.n;
        r.kl = a.sa_kl + (long long)d * a.n;
      }
    }
  }
  return r;
}

// The y move of tile t; returns the tile's term (also written to tterm).
__device__ __forceinline__ double move_y_tile(const MoveYArgs& a, long long t, const MoveYDraw& dr) {
  const int n = a.n, n1 = n - 1;
  const bool on = dr.on;
  const double g = dr.g;
  const double* kf = dr.kf;
  const double* kl = dr.kl;
  // T = n^2 (n-1)^2 < 2^20 for n <= 32: 32-bit divisions (a 64-bit one is a
  // long subroutine)
  const int ip = RLT2_IDX((int)((unsigned)t / (unsigned)(n1 * n1)), n * n);
  const int rem = (int)(t - (long long)ip * n1 * n1);
  const int jj = rem / n1, qq = rem - jj * n1;
  const int i = ip / n, p = ip - i * n;
  const int j = jj + (jj >= i), q = qq + (qq >= p);
  const long long tp = RLT2_IDX(((long long)(j * n + q) * n1 + (i - (i > j))) * n1 + (p - (p > q)), a.T);
  const double py = a.piy[t];
  // half-Z scheme: the z pools of an upper tile take the y slack left after the y move
  const double pyz = a.half ? dadd_(dsub_(py, dmul_(a.phi_y, py)), dmul_(a.phi_y, a.piy[tp])) : py;
  double ty = dadd_(dmul_(a.cy, pyz), dmul_(a.cx, a.pix[ip]));
  if (on) ty = dadd_(ty, dadd_(dmul_(kf[i], g), dmul_(kl[p], g)));
  a.tterm[t] = ty;
  if (a.half) {
    // y move of Eq. 2.21, then Type 3 on the y level: a lower y (i > j) gives
    // kx pi_x(ip) / (n-1) to its mirror (the lower z stay at zero)
    const double c0 = dadd_(dsub_(a.Chat[t], dmul_(a.phi_y, py)), dmul_(a.phi_y, a.piy[tp]));
    a.Chat[t] = (i > j) ? dsub_(c0, dmul_(a.cxy, a.pix[ip])) : dadd_(c0, dmul_(a.cxy, a.pix[j * n + q]));
  } else if (a.fast)
    a.Chat[t] = dadd_(dmul_(a.keep_y, py), dmul_(a.phi_y, a.piy[tp]));
  else
    a.Chat[t] = dadd_(dsub_(a.Chat[t], dmul_(a.phi_y, py)), dmul_(a.phi_y, a.piy[tp]));
  if (t < (long long)n * n) {
    const int xi_ = (int)t / n, xp = (int)t - xi_ * n;
    if (a.fast) a.xcost[t] = dmul_(a.keep_x, a.pix[t]);
    if (on) a.saterm[t] = dadd_(dmul_(kf[xi_], g), dmul_(kl[xp], g));
  }
  return ty;
}

__device__ __forceinline__ void move_y_range(const MoveYArgs& a, long long start, long long stride) {
  const MoveYDraw dr = move_y_draw(a);
  for (long long t = start; t < a.T; t += stride) (void)move_y_tile(a, t, dr);
  if (start == 0) {
    a.sc->sa_on = dr.on ? 1 : 0;
    if (a.fast) a.sc->lb_base = a.sc->lb;
  }
}

// The y move and, for the folded z move, psi <- psi - tile term in the same
// pass: a warp moves 32 consecutive tiles (lane j tile tw + j) and then
// shifts their 32 m column duals, which are contiguous, in coalesced turns
// (each entry's term shuffled from the lane of its tile), six loads in flight
// per lane.  start is the global thread index and stride a multiple of 32.
__device__ __forceinline__ void move_y_shift_range(const MoveYArgs& a, long long start, long long stride) {
  constexpr int kU = 6;
  const int lane = (int)(start & 31), m = a.n - 2;
  const MoveYDraw dr = move_y_draw(a);
  for (long long tw = start - lane; tw < a.T; tw += stride) {
    const long long t = tw + lane;
    const double ty = t < a.T ? move_y_tile(a, t, dr) : 0.0;
    const int cnt = (int)(a.T - tw < 32 ? a.T - tw : 32) * m;
    double* p = a.psi + tw * m;
    for (int e0 = 0; e0 < cnt; e0 += 32 * kU) {
      double x[kU];
#pragma unroll
      for (int k = 0; k < kU; ++k) {
        const int e = e0 + 32 * k + lane;
        x[k] = e < cnt ? p[e] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < kU; ++k) {
        const int e = e0 + 32 * k + lane;
        // every lane shuffles (full mask); the source lane is e's tile, < 32 since e < 32 m
        const double tt = __shfl_sync(0xffffffffu, ty, (int)((unsigned)(e < cnt ? e : cnt - 1) / (unsigned)m));
        if (e < cnt) p[e] = dsub_(x[k], tt);
      }
    }
  }
  if (start == 0) {
    a.sc->sa_on = dr.on ? 1 : 0;
    if (a.fast) a.sc->lb_base = a.sc->lb;
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
  int uniform;  // all phi equal: member b gets phi * (S - s_b)
  int fast;     // F variant: the member keeps fma(-kz, pi_z, pi_z) (minus a Type 4 amount)
  int half;     // half-Z scheme: only the three upper members move (lower ones stay 0)
  int folded;   // S, kz = 1, all phi equal: psi holds psi - tile term, s = (D - xi) - psi,
                // D' = fma(c1, s, fma(phi, S, D)) with c1 = -(1 + phi)
  double c1;
  const double* saterm;  // n*n Type 4 amounts (F variant, when sc->sa_on)
  double* Dhat;
  const double* xi;
  const double* psi;
  const double* tterm;
  const int* trips;  // i | j<<8 | k<<16 with i<j<k
  const DevScalars* sc;
};

// The class (q, r) -- as indices qq < n-1, rr < n-2 with p (and q) skipped --
// of thread slot c of a (triple, p) block.  Two members of a class lie in rows
// along r, two in rows along q and two in a different tile for every (q, r):
// with lanes along r (slot c = qq (n-2) + rr) a warp's six loads touch 144
// 32-byte sectors.  For n >= 22 the slots run in bands of eight q with r
// outer, so a warp's lanes cover 8 q x 4 r and touch 96: the z array is then
// far larger than L2 and the move keeps its rate (n = 28: 3.60 instead of
// 5.58 ms).  Below that the plain order is as fast or faster (n = 20 equal,
// the batched nodes of residual 14..18 9 % faster without the bands' integer
// divisions).
template <bool BAND = true>
__device__ __forceinline__ void class_of(int c, int n1, int m, int& qq, int& rr) {
  constexpr int kBand = 8;
  if (!BAND || n1 < 21) {
    qq = c / m;
    rr = c - qq * m;
    return;
  }
  const int band = c / (kBand * m), cb = c - band * kBand * m;
  const int hb = min(kBand, n1 - kBand * band);
  qq = kBand * band + cb % hb;
  rr = cb / hb;
}

// One thread per class; a block covers one facility triple and one location p
// of its first facility (all (q, r)).  Consecutive threads take consecutive r,
// so members (i,j,k|p,q,r) and (j,i,k|q,p,r) are read and written as contiguous
// rows; the other four members' rows are shared by the block or by the n blocks
// of the same triple, which run back to back.
// Half-Z scheme (Section 5): the upper members (i,j,k|p,q,r), (i,k,j|p,r,q) and
// (j,k,i|q,r,p) -- members 0, 1, 3 -- pool s = kz pi_z + tile term and each
// receives half of the other two pools: D' = D - s + (S - s)/2 with S the sum
// of the three pools in member order, evaluated as fma(-3/2, s, fma(1/2, S, D)).
// Lower members are never touched.
__device__ __forceinline__ void move_z_half_block(const MoveZArgs& a, int blk) {
  RLT2_CLASS_TABLES
  (void)kPart;
  constexpr int kUp[3] = {0, 1, 3};
  const int n = a.n, m = a.m, n1 = n - 1;
  const int tr = blk / n, p = blk - tr * n;
  const int packed = a.trips[tr];
  const int F3[3] = {packed & 255, (packed >> 8) & 255, packed >> 16};
  const int npairs = n1 * m;
  const long long mm = (long long)m * m;
  for (int c = threadIdx.x; c < npairs; c += blockDim.x) {
    int qq, rr;
    class_of(c, n1, m, qq, rr);
    const int q = qq + (qq >= p);
    const int lo = p < q ? p : q, hi = p < q ? q : p;
    int r = rr;
    r += (r >= lo);
    r += (r >= hi);
    const int L3[3] = {p, q, r};
    double s[3], Dv[3];
    long long idx[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int b = kUp[u];
      const int f0 = F3[kOrd[b][0]], f1 = F3[kOrd[b][1]], f2 = F3[kOrd[b][2]];
      const int l0 = L3[kOrd[b][0]], l1 = L3[kOrd[b][1]], l2 = L3[kOrd[b][2]];
      const long long t = RLT2_IDX(((long long)(f0 * n + l0) * n1 + (f1 - (f1 > f0))) * n1 + (l1 - (l1 > l0)),
                                        (long long)n * n * n1 * n1);
      const int kr = RLT2_IDX(f2 - (f2 > f0) - (f2 > f1), m), cc = RLT2_IDX(l2 - (l2 > l0) - (l2 > l1), m);
      idx[u] = t * mm + kr * m + cc;
      Dv[u] = a.Dhat[idx[u]];
      const double pz = dsub_(dsub_(Dv[u], __ldg(a.xi + t * m + kr)), __ldg(a.psi + t * m + cc));
      s[u] = a.kz_one ? dadd_(pz, __ldg(a.tterm + t)) : __fma_rn(a.kz, pz, __ldg(a.tterm + t));
    }
    const double S = dadd_(dadd_(s[0], s[1]), s[2]);
#pragma unroll
    for (int u = 0; u < 3; ++u) a.Dhat[idx[u]] = __fma_rn(-1.5, s[u], __fma_rn(0.5, S, Dv[u]));
  }
}

// Loads of the duals and tile terms: through the read-only cache in the
// stand-alone move; plain loads where the same launch later rewrites the duals
// (the pipelined move + Z-LAP kernel, whose move reads of a tile's duals all
// precede that tile's LAP).
template <bool RO>
__device__ __forceinline__ double ldv(const double* p) {
  if constexpr (RO) return __ldg(p);
  else return *p;
}

// The classes (q, r) = first, first + stride, ... of block blk = (triple, p);
// BAND: the banded class order for n >= 22 (see class_of).
template <bool RO = true, bool BAND = true>
__device__ __forceinline__ void move_z_block(const MoveZArgs& a, int blk, int first, int stride) {
  if (a.half) {
    move_z_half_block(a, blk);
    return;
  }
  RLT2_CLASS_TABLES
  const int n = a.n, m = a.m, n1 = n - 1;
  const int tr = blk / n, p = blk - tr * n;
  const int packed = a.trips[tr];
  const int F3[3] = {packed & 255, (packed >> 8) & 255, packed >> 16};
  const int npairs = n1 * m;
  const long long mm = (long long)m * m;
  const bool sa = a.fast && a.sc->sa_on;
  for (int c = first; c < npairs; c += stride) {
    int qq, rr;
    class_of<BAND>(c, n1, m, qq, rr);
    const int q = qq + (qq >= p);
    const int lo = p < q ? p : q, hi = p < q ? q : p;
    int r = rr;
    r += (r >= lo);
    r += (r >= hi);
    const int L3[3] = {p, q, r};
    double s[6], base[6];
    long long idx[6];
    if (a.folded) {
      // the uniform pool of Eq. 2.20-2.23 with kz = 1, regrouped:
      // D' = D - s + phi (S - s) = (D + phi S) - (1 + phi) s
      double Dv[6];
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        const int f0 = F3[kOrd[b][0]], f1 = F3[kOrd[b][1]], f2 = F3[kOrd[b][2]];
        const int l0 = L3[kOrd[b][0]], l1 = L3[kOrd[b][1]], l2 = L3[kOrd[b][2]];
        const long long t = RLT2_IDX(((long long)(f0 * n + l0) * n1 + (f1 - (f1 > f0))) * n1 + (l1 - (l1 > l0)),
                                        (long long)n * n * n1 * n1);
        const int kr = RLT2_IDX(f2 - (f2 > f0) - (f2 > f1), m), cc = RLT2_IDX(l2 - (l2 > l0) - (l2 > l1), m);
        idx[b] = t * mm + kr * m + cc;
        Dv[b] = a.Dhat[idx[b]];
        s[b] = dsub_(dsub_(Dv[b], ldv<RO>(a.xi + t * m + kr)), ldv<RO>(a.psi + t * m + cc));
      }
      double S = s[0];
#pragma unroll
      for (int b = 1; b < 6; ++b) S = dadd_(S, s[b]);
#pragma unroll
      for (int b = 0; b < 6; ++b) a.Dhat[idx[b]] = __fma_rn(a.c1, s[b], __fma_rn(a.w[0], S, Dv[b]));
      continue;
    }
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      const int f0 = F3[kOrd[b][0]], f1 = F3[kOrd[b][1]], f2 = F3[kOrd[b][2]];
      const int l0 = L3[kOrd[b][0]], l1 = L3[kOrd[b][1]], l2 = L3[kOrd[b][2]];
      const long long t = RLT2_IDX(((long long)(f0 * n + l0) * n1 + (f1 - (f1 > f0))) * n1 + (l1 - (l1 > l0)),
                                        (long long)n * n * n1 * n1);
      const int kr = RLT2_IDX(f2 - (f2 > f0) - (f2 > f1), m), cc = RLT2_IDX(l2 - (l2 > l0) - (l2 > l1), m);
      idx[b] = t * mm + kr * m + cc;
      const double Dv = a.Dhat[idx[b]];
      const double pz = dsub_(dsub_(Dv, ldv<RO>(a.xi + t * m + kr)), ldv<RO>(a.psi + t * m + cc));
      // s = kz*pi_z + tile term in one rounding (kz = 1: an exact fma(1, x, y) is x + y)
      s[b] = a.kz_one ? dadd_(pz, ldv<RO>(a.tterm + t)) : __fma_rn(a.kz, pz, ldv<RO>(a.tterm + t));
      if (!a.fast) {
        base[b] = dsub_(Dv, s[b]);
      } else {
        // (1 - kz) pi_z in one rounding; fma(-1, x, x) is +0 exactly
        base[b] = a.kz_one ? 0.0 : __fma_rn(-a.kz, pz, pz);
        if (sa) base[b] = dsub_(base[b], ldv<RO>(a.saterm + f0 * n + l0));
      }
    }
    if (a.uniform) {
      // all phi equal: member b receives phi * (S - s_b), S the class sum in member order
      double S = s[0];
#pragma unroll
      for (int b = 1; b < 6; ++b) S = dadd_(S, s[b]);
#pragma unroll
      for (int b = 0; b < 6; ++b) a.Dhat[idx[b]] = __fma_rn(a.w[0], dsub_(S, s[b]), base[b]);
    } else {
      // partner inflows one fused multiply-add at a time, partners in Eq. 2.20 order
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        double acc = base[b];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = __fma_rn(a.w[l], s[kPart[b][l]], acc);
        a.Dhat[idx[b]] = acc;
      }
    }
  }
}

// Second phase of the two-phase Z solve (Section 3.4), class-owned like the z
// move: members with pi_z above tol (1 + |xi| + |psi|) (S_N) drop to D^ - pi_z,
// and the sum of their slacks (member order) times 1/|S_B| goes to each
// member with zero slack (S_B); classes with S_B or S_N empty stay as they are.
struct Phase2Args {
  int n, m;
  double tol;
  double* Dhat;
  const double* xi;
  const double* psi;
  const int* trips;
  const DevScalars* sc;
};

__device__ __forceinline__ void phase2_block(const Phase2Args& a, int blk) {
  RLT2_CLASS_TABLES
  (void)kPart;
  const int n = a.n, m = a.m, n1 = n - 1;
  const int tr = blk / n, p = blk - tr * n;
  const int packed = a.trips[tr];
  const int F3[3] = {packed & 255, (packed >> 8) & 255, packed >> 16};
  const int npairs = n1 * m;
  const long long mm = (long long)m * m;
  for (int c = threadIdx.x; c < npairs; c += blockDim.x) {
    int qq, rr;
    class_of(c, n1, m, qq, rr);
    const int q = qq + (qq >= p);
    const int lo = p < q ? p : q, hi = p < q ? q : p;
    int r = rr;
    r += (r >= lo);
    r += (r >= hi);
    const int L3[3] = {p, q, r};
    double pz[6], Dv[6];
    long long idx[6];
    int nb = 0;
    unsigned basic = 0;
    double sum = 0.0;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      const int f0 = F3[kOrd[b][0]], f1 = F3[kOrd[b][1]], f2 = F3[kOrd[b][2]];
      const int l0 = L3[kOrd[b][0]], l1 = L3[kOrd[b][1]], l2 = L3[kOrd[b][2]];
      const long long t = RLT2_IDX(((long long)(f0 * n + l0) * n1 + (f1 - (f1 > f0))) * n1 + (l1 - (l1 > l0)),
                                        (long long)n * n * n1 * n1);
      const int kr = RLT2_IDX(f2 - (f2 > f0) - (f2 > f1), m), cc = RLT2_IDX(l2 - (l2 > l0) - (l2 > l1), m);
      idx[b] = t * mm + kr * m + cc;
      Dv[b] = a.Dhat[idx[b]];
      const double xv = __ldg(a.xi + t * m + kr), pv = __ldg(a.psi + t * m + cc);
      pz[b] = dsub_(dsub_(Dv[b], xv), pv);
      const double lim = dmul_(a.tol, dadd_(dadd_(1.0, fabs(xv)), fabs(pv)));
      if (okey_(pz[b]) <= okey_(lim)) {
        basic |= 1u << b;
        ++nb;
      } else {
        sum = dadd_(sum, pz[b]);
      }
    }
    if (nb == 0 || nb == 6) continue;
    // 1/|S_B| as a correctly rounded constant, as in 1.0 / k
    const double inv = nb == 1 ? 1.0 : nb == 2 ? 0.5 : nb == 3 ? 1.0 / 3.0 : nb == 4 ? 0.25 : 0.2;
    const double share = dmul_(sum, inv);
#pragma unroll
    for (int b = 0; b < 6; ++b)
      a.Dhat[idx[b]] = ((basic >> b) & 1u) ? dadd_(Dv[b], share) : dsub_(Dv[b], pz[b]);
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
  const double* bqap;     // QAP linear costs (b' without multipliers) for the upper bound
  const double* cst_qap;  // QAP constant of the fixed facilities
  double* ring;
  double min_gap, ub_known, feas_tol, stall_tol;
  int stall_window;
  int fast;  // F variant: bound = previous bound + X-LAP value (Eq. 3.7)
  DevScalars* sc;
};

// Must be called by every thread of a block of 256 threads.
__device__ __forceinline__ void finalize_block(const FinArgs& a) {
  __shared__ double red[256];
  __shared__ int bad, improve;
  const int n = a.n, m = a.m, n1 = n - 1, tid = threadIdx.x;
  const double lb = dadd_(a.fast ? a.sc->lb_base : *a.cst, a.xval[0]);
  if (tid == 0) bad = (a.feas_tol > 0.0) ? 0 : 1;
  // residual QAP value of the X-LAP primal (an upper bound)
  double part = 0.0;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    const int si = RLT2_IDX(a.xperm[i], n), sj = RLT2_IDX(a.xperm[j], n);
    part += (i == j) ? a.bqap[i * n + si] : a.Fr[i * n + j] * a.Dr[si * n + sj];
  }
  red[tid] = part;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  const double ub = *a.cst_qap + red[0];
  // feasibility check: every y and z built from the X primal has zero slack (Eq. 2.19)
  if (a.feas_tol > 0.0) {
    const double tol = a.feas_tol * fmax(1.0, fabs(lb));
    for (int e = tid; e < n * n1; e += blockDim.x) {
      const int i = e / n1, jj = e - i * n1, j = jj + (jj >= i);
      const int si = RLT2_IDX(a.xperm[i], n), sj = RLT2_IDX(a.xperm[j], n);
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
      const int si = RLT2_IDX(a.xperm[i], n), sj = RLT2_IDX(a.xperm[j], n), sk = RLT2_IDX(a.xperm[k], n);
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
// equal passes of at most 352 threads, rounded to whole warps (n = 20: one
// pass of 352; three such blocks fit an SM at 62 registers, against two of
// up to 512 threads: 4 % faster).
inline int move_z_threads(int n) {
  const int c = (n - 1) * (n - 2);
  const int passes = (c + 351) / 352;
  return ((c + passes - 1) / passes + 31) / 32 * 32;
}

// Kernel arguments of one problem's moves and finalize step (host helpers).
MoveYArgs make_move_y(const IterView& v);
MoveZArgs make_move_z(const IterView& v);
Phase2Args make_phase2(const IterView& v);
FinArgs make_fin(const IterView& v);

}  // namespace rlt2
