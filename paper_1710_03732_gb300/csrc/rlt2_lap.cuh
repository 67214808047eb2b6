// Warp-per-LAP Hungarian for sm_103a (GB300).
//
// Every LAP of the RLT2 dual ascent is small (Z: n-2, Y: n-1, X: n; n <= 32), so
// one warp owns one LAP: lane c holds column c (dual v_c, Dijkstra label d_c,
// predecessor row, "scanned" flag, matched row) and lane r holds row r (dual
// u_r, matched column).  The cost tile sits in shared memory with an odd row
// stride so that both row reads (lanes = columns) and column reads (lanes =
// rows) are bank-conflict free.  This replaces the paper's tiled alternating-
// tree Hungarian (Section 3.2, written for Kepler): no cross-LAP coupling, no
// host round trips, one launch per stage.
//
// GB300 runs FP64 at ~1/70 of its FP32 rate, and FP64 compares and min/max use
// the same slow pipe, so every comparison below is done on 64-bit integer
// keys that order exactly like the doubles (okey), and every argmin is a
// two-step warp integer min reduction (redux.sync) plus a ballot.  The only
// FP64 instructions left are the additions the method needs.
//
// Arithmetic order (shared with the CPU oracle by specification, so raw-mode
// results match it bit for bit):
//   start     u = u0 or 0;  v_c = min_r (c_rc - u_r), ties to the lowest row
//   greedy    column c takes its argmin row if no lower column took that row
//   search    for every free row i (increasing): Dijkstra on reduced costs
//             pi(r,c) = (c_rc - u_r) - v_c; labels d_c = d_last + pi(r,c);
//             pick the unscanned column of least label (lowest index on ties);
//             relax only on strict '<'; stop at the first free column.
//   duals     v_c = v_c + (d_c - d_sink) on scanned columns, augment, then
//             u_r = c_{r,sigma(r)} - v_{sigma(r)} for every matched row
//   value     sum_r c_{r,sigma(r)} in increasing r
//   canonical (dual_mode 1) Dijkstra from row 0 over arcs r'->r with weight
//             pi(r, sigma(r')) (>= 0), u^c_r = dist_r + (u_r - u_0),
//             v^c_c = c_{sigma^-1(c),c} - u^c_{sigma^-1(c)}
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rlt2 {

constexpr unsigned kFull = 0xffffffffu;

// Order-preserving 64-bit key of a double (non-NaN): a < b  <=>  okey(a) < okey(b),
// with -0 and +0 equal, exactly as the IEEE comparison.
__device__ __forceinline__ unsigned long long okey(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  b = (b == 0x8000000000000000ull) ? 0ull : b;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Lane holding the least key; lowest lane on ties.
__device__ __forceinline__ int warp_argmin(unsigned long long key) {
  const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
  const unsigned mhi = __reduce_min_sync(kFull, hi);
  const unsigned mlo = __reduce_min_sync(kFull, hi == mhi ? lo : 0xffffffffu);
  const unsigned ball = __ballot_sync(kFull, hi == mhi && lo == mlo);
  return __ffs(ball) - 1;
}

__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }

struct WarpLapResult {
  double u;      // row dual of row `lane`
  double v;      // column dual of column `lane`
  int r2c;       // column matched to row `lane`
  int c2r;       // row matched to column `lane`
  double value;  // LAP optimum (all lanes)
  int naug;      // augmenting searches
  int nrelax;    // label relaxations (instrumentation for the roofline)
};

// Solve the m x m LAP in shared memory `cs` (row stride ld) with one warp.
// `scr` is 32 ints of per-warp scratch.  u0 is this lane's starting row dual
// (used only when warm).  Must be called by all 32 lanes.
__device__ __forceinline__ WarpLapResult warp_lap(const double* __restrict__ cs, int ld, int m, int lane, bool warm,
                                                  double u0, int dual_mode, int* scr) {
  const bool cv = lane < m;
  WarpLapResult R;
  double u = (cv && warm) ? u0 : 0.0;
  double v = 0.0;
  int naug = 0, nrelax = 0;

  // column reduction with the argmin row
  unsigned long long bestk = ~0ull;
  int arg = -1;
  for (int r = 0; r < m; ++r) {
    const double ur = __shfl_sync(kFull, u, r);
    if (cv) {
      const double c = cs[r * ld + lane];
      const double x = warm ? dsub(c, ur) : c;  // c - 0 == c exactly
      const unsigned long long k = okey(x);
      if (arg < 0 || k < bestk) {
        bestk = k;
        arg = r;
        v = x;
      }
    }
  }
  // greedy: the lowest column among those sharing an argmin row takes it
  const int marg = cv ? arg : (64 + lane);
  const unsigned same = __match_any_sync(kFull, marg);
  const bool win = cv && (__ffs(same) - 1) == lane;
  int c2r = win ? arg : -1;
  scr[lane] = -1;
  __syncwarp();
  if (win) scr[arg] = lane;
  __syncwarp();
  int r2c = cv ? scr[lane] : -1;
  __syncwarp();

  unsigned freerows = __ballot_sync(kFull, cv && r2c < 0);
  while (freerows) {
    const int i = __ffs(freerows) - 1;
    freerows &= freerows - 1;
    ++naug;
    const double ui = __shfl_sync(kFull, u, i);
    double d = cv ? dsub(dsub(cs[i * ld + lane], ui), v) : 0.0;
    unsigned long long dk = okey(d);
    int pred = i;
    bool scanned = !cv;
    nrelax += m;
    const unsigned freecols = __ballot_sync(kFull, cv && c2r < 0);
    int sink;
    double dlast;
    for (;;) {
      const int c = warp_argmin(scanned ? ~0ull : dk);
      const double dm = __shfl_sync(kFull, d, c);
      if (lane == c) scanned = true;
      if ((freecols >> c) & 1u) {
        sink = c;
        dlast = dm;
        break;
      }
      const int r = __shfl_sync(kFull, c2r, c);
      const double ur = __shfl_sync(kFull, u, r);
      if (!scanned) {
        const double nd = dadd(dm, dsub(dsub(cs[r * ld + lane], ur), v));
        const unsigned long long nk = okey(nd);
        if (nk < dk) {
          d = nd;
          dk = nk;
          pred = r;
        }
      }
      nrelax += __popc(__ballot_sync(kFull, !scanned));
    }
    if (cv && scanned) v = dadd(v, dsub(d, dlast));
    // augment back to row i
    int col = sink;
    for (;;) {
      const int r = __shfl_sync(kFull, pred, col);
      const int nxt = __shfl_sync(kFull, r2c, r);
      if (lane == col) c2r = r;
      if (lane == r) r2c = col;
      if (r == i) break;
      col = nxt;
    }
    const int mc = (cv && r2c >= 0) ? r2c : 0;
    const double vm = __shfl_sync(kFull, v, mc);
    if (cv && r2c >= 0) u = dsub(cs[lane * ld + r2c], vm);
  }

  // optimum, summed in increasing row order
  const double xr = cv ? cs[lane * ld + r2c] : 0.0;
  double val = 0.0;
  for (int r = 0; r < m; ++r) {
    const double t = __shfl_sync(kFull, xr, r);
    if (lane == 0) val = dadd(val, t);
  }
  val = __shfl_sync(kFull, val, 0);

  if (dual_mode == 1 && m > 1) {
    // shortest paths from row 0 on reduced weights pi(r, sigma(r')) >= 0
    const int s0 = __shfl_sync(kFull, r2c, 0);
    const double vs0 = __shfl_sync(kFull, v, s0);
    double dist = (cv && lane != 0) ? dsub(dsub(cs[lane * ld + s0], u), vs0) : 0.0;
    unsigned long long dk = okey(dist);
    bool done = !cv || lane == 0;
    for (int it = 0; it < m - 2; ++it) {
      const int rs = warp_argmin(done ? ~0ull : dk);
      const double dr = __shfl_sync(kFull, dist, rs);
      if (lane == rs) done = true;
      const int s = __shfl_sync(kFull, r2c, rs);
      const double vs = __shfl_sync(kFull, v, s);
      if (!done) {
        const double nd = dadd(dr, dsub(dsub(cs[lane * ld + s], u), vs));
        const unsigned long long nk = okey(nd);
        if (nk < dk) {
          dist = nd;
          dk = nk;
        }
      }
    }
    const double u0r = __shfl_sync(kFull, u, 0);
    const double ucan = cv ? dadd(dist, dsub(u, u0r)) : 0.0;
    const int rr = cv ? c2r : 0;
    const double ucr = __shfl_sync(kFull, ucan, rr);
    const double vcan = cv ? dsub(cs[rr * ld + lane], ucr) : 0.0;
    u = ucan;
    v = vcan;
  } else if (dual_mode == 1 && m == 1) {
    v = cv ? cs[0] : 0.0;
    u = 0.0;
  }
  R.u = u;
  R.v = v;
  R.r2c = r2c;
  R.c2r = c2r;
  R.value = val;
  R.naug = naug;
  R.nrelax = nrelax;
  return R;
}

}  // namespace rlt2
