// Warp-level (group-per-LAP) Hungarian for sm_103a (GB300).
//
// Every LAP of the RLT2 dual ascent is small (Z: n-2, Y: n-1, X: n; n <= 32), so
// a group of G = 8, 16 or 32 lanes owns one LAP (32/G LAPs per warp, in
// lockstep): lane c holds column c (dual v_c, Dijkstra label d_c,
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
//   value     sum_r c_{r,sigma(r)} as a pairwise tree (lane i += lane i+h, h = P/2..1)
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
  double u;      // row dual of row `gl` (group lane)
  double v;      // column dual of column `gl`
  int r2c;       // column matched to row `gl`
  int c2r;       // row matched to column `gl`
  double value;  // LAP optimum (all lanes of the group)
  int naug;      // augmenting searches
  int nrelax;    // label relaxations (instrumentation for the roofline)
};

// Lowest group lane holding the least key among the G lanes of this lane's
// group (aligned groups of G lanes).  Every lane of the warp must call it.
template <int G>
__device__ __forceinline__ int group_argmin(unsigned long long key, int gb) {
  if constexpr (G == 32) {
    return warp_argmin(key);
  } else {
    unsigned long long k = key;
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(kFull, k, off);
      k = o < k ? o : k;
    }
    const unsigned ball = __ballot_sync(kFull, key == k);
    return __ffs((ball >> gb) & ((1u << G) - 1u)) - 1;
  }
}

template <int G>
__device__ __forceinline__ unsigned group_bits(unsigned ball, int gb) {
  if constexpr (G == 32) return ball;
  else return (ball >> gb) & ((1u << G) - 1u);
}

// Solve one LAP per group of G lanes (32/G LAPs per warp) in lockstep: every
// intrinsic is executed by all 32 lanes with the full mask and all loops are
// warp-uniform (they run while any group still has work; idle groups only
// predicate their updates), so the LAPs of one warp share every instruction.
// Group lane gl = lane % G holds row gl and column gl of its LAP.  `cs` is the
// group's m x m tile (row stride ld) in shared memory, `scr` G ints of group
// scratch, m the group's LAP size (0 = no LAP, 1 <= m <= G otherwise).  The
// arithmetic is identical for every G.
// PRE: the caller does not need the tile afterwards, so the canonical pass may
// replace it by its reduced costs first (uvs: 64 doubles of group staging).
template <int G, bool PRE>
__device__ __forceinline__ WarpLapResult group_lap(double* __restrict__ cs, int ld, int m, int lane, bool warm,
                                                   double u0, int dual_mode, int* scr, double* uvs) {
  const int gl = lane & (G - 1);
  const int gb = lane - gl;
  const bool cv = gl < m;
  const int M = (G == 32) ? m : (int)__reduce_max_sync(kFull, (unsigned)m);
  WarpLapResult R;
  double u = (cv && warm) ? u0 : 0.0;
  double v = 0.0;
  int naug = 0, nrelax = 0;

  // column reduction with the argmin row
  unsigned long long bestk = ~0ull;
  int arg = -1;
  for (int r = 0; r < M; ++r) {
    const double ur = __shfl_sync(kFull, u, gb + r);
    if (cv && r < m) {
      const double c = cs[r * ld + gl];
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
  const int marg = cv ? ((lane / G) << 6) + arg : (1 << 20) + lane;
  const unsigned same = __match_any_sync(kFull, marg);
  const bool win = cv && (__ffs(same) - 1) == lane;
  int c2r = win ? arg : -1;
  scr[gl] = -1;
  __syncwarp();
  if (win) scr[arg] = gl;
  __syncwarp();
  int r2c = cv ? scr[gl] : -1;
  __syncwarp();

  unsigned freerows = group_bits<G>(__ballot_sync(kFull, cv && r2c < 0), gb);
  while (__any_sync(kFull, freerows != 0)) {
    const bool act = freerows != 0;  // this group runs a search in this round
    const int i = act ? __ffs(freerows) - 1 : 0;
    if (act) {
      freerows &= freerows - 1;
      ++naug;
      nrelax += m;
    }
    const double ui = __shfl_sync(kFull, u, gb + i);
    double d = (act && cv) ? dsub(dsub(cs[i * ld + gl], ui), v) : 0.0;
    unsigned long long dk = okey(d);
    int pred = i;
    bool scanned = !(act && cv);
    const unsigned freecols = group_bits<G>(__ballot_sync(kFull, cv && c2r < 0), gb);
    bool searching = act;
    int sink = 0;
    double dlast = 0.0;
    while (__any_sync(kFull, searching)) {
      const int c = group_argmin<G>(scanned ? ~0ull : dk, gb);
      const double dm = __shfl_sync(kFull, d, gb + c);
      if (searching && gl == c) scanned = true;
      const bool found = searching && ((freecols >> c) & 1u);
      if (found) {
        sink = c;
        dlast = dm;
      }
      const bool relaxing = searching && !found;
      const int r0 = __shfl_sync(kFull, c2r, gb + c);
      const int r = r0 < 0 ? 0 : r0;
      const double ur = __shfl_sync(kFull, u, gb + r);
      if (relaxing && !scanned) {
        const double nd = dadd(dm, dsub(dsub(cs[r * ld + gl], ur), v));
        const unsigned long long nk = okey(nd);
        if (nk < dk) {
          d = nd;
          dk = nk;
          pred = r;
        }
      }
      const int unsc = __popc(group_bits<G>(__ballot_sync(kFull, !scanned), gb));
      if (relaxing) nrelax += unsc;
      searching = relaxing;
    }
    if (act && cv && scanned) v = dadd(v, dsub(d, dlast));
    // augment back to row i (groups walk their own chains in lockstep)
    bool walking = act;
    int col = sink;
    while (__any_sync(kFull, walking)) {
      const int r = __shfl_sync(kFull, pred, gb + col);
      const int nxt = __shfl_sync(kFull, r2c, gb + r);
      if (walking) {
        if (gl == col) c2r = r;
        if (gl == r) r2c = col;
        if (r == i) walking = false;
        else col = nxt;
      }
    }
    const int mc = (cv && r2c >= 0) ? r2c : 0;
    const double vm = __shfl_sync(kFull, v, gb + mc);
    if (act && cv && r2c >= 0) u = dsub(cs[gl * ld + r2c], vm);
  }

  // optimum: pairwise tree over P = next power of two >= m rows (empty rows add
  // nothing), lane i adding lane i + h for h = P/2, ..., 1
  const double xr = cv ? cs[gl * ld + r2c] : 0.0;
  int P = 1;
  while (P < m) P <<= 1;
  const int PM = (G == 32) ? P : (int)__reduce_max_sync(kFull, (unsigned)P);
  double val = xr;
  for (int h = PM >> 1; h >= 1; h >>= 1) {
    const double o = __shfl_xor_sync(kFull, val, h);
    if (h < P) val = dadd(val, o);
  }
  val = __shfl_sync(kFull, val, gb);

  if (dual_mode == 1) {
    // canonical duals: shortest paths from row 0 on reduced weights
    // pi(r, sigma(r')) = (c_{r,sigma(r')} - u_r) - v_{sigma(r')} >= 0
    const int s0 = __shfl_sync(kFull, r2c, gb);
    if constexpr (PRE) {
      uvs[gl] = u;
      uvs[32 + gl] = v;
      __syncwarp();
      for (int e = gl; e < m * m; e += G) {
        const int r = e / m, c = e - r * m;
        cs[r * ld + c] = dsub(dsub(cs[r * ld + c], uvs[r]), uvs[32 + c]);
      }
      __syncwarp();
    }
    const double vs0 = __shfl_sync(kFull, v, gb + (s0 < 0 ? 0 : s0));
    double dist = 0.0;
    if (cv && gl != 0) {
      if constexpr (PRE) dist = cs[gl * ld + s0];
      else dist = dsub(dsub(cs[gl * ld + s0], u), vs0);
    }
    unsigned long long dk = okey(dist);
    bool done = !cv || gl == 0;
    for (int it = 0; it < M - 2; ++it) {
      const bool stepping = it < m - 2;
      const int rs = group_argmin<G>(done ? ~0ull : dk, gb);
      const double dr = __shfl_sync(kFull, dist, gb + rs);
      if (stepping && gl == rs) done = true;
      const int s = __shfl_sync(kFull, r2c, gb + rs);
      const double vs = __shfl_sync(kFull, v, gb + (s < 0 ? 0 : s));
      if (stepping && !done) {
        double w;
        if constexpr (PRE) w = cs[gl * ld + s];
        else w = dsub(dsub(cs[gl * ld + s], u), vs);
        const double nd = dadd(dr, w);
        const unsigned long long nk = okey(nd);
        if (nk < dk) {
          dist = nd;
          dk = nk;
        }
      }
    }
    const double u0r = __shfl_sync(kFull, u, gb);
    const double ucan = cv ? (m > 1 ? dadd(dist, dsub(u, u0r)) : 0.0) : 0.0;
    // v_c = c_{sigma^-1(c), c} - u_{sigma^-1(c)}, from the matched row's own entry
    const double wrow = dsub(xr, ucan);
    const int rr = cv ? c2r : 0;
    const double vcan = __shfl_sync(kFull, wrow, gb + rr);
    u = ucan;
    v = cv ? vcan : 0.0;
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
