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
// keys that order exactly like the values (okey for doubles), and every argmin
// is a two-step warp integer min reduction (redux.sync) plus a ballot.  In the
// FP64 form the only FP64 instructions left are the additions the method
// needs; the fixed-point form has none outside the output conversions.
//
// Two arithmetic forms, chosen per launch:
//   FP64      IEEE double, round to nearest, in the CPU oracle's operation order
//             (raw duals match it bit for bit); used for raw duals and for the
//             FP64 canonical mode.
//   fixed     exact 64-bit integer arithmetic on a per-tile grid (canonical
//             duals, the default).  The tile is rounded down onto the grid
//             2^L with L = E - 48, where 2^E bounds every |entry|; the start
//             duals are rounded down and clamped to |u0| <= 2^(E+1).  Every
//             quantity the Hungarian and the canonical pass form then stays
//             below 2^59 grid steps for m <= 32 (labels are bounded by the
//             growth of the matching cost, duals by the labels), so no
//             addition can overflow, and the result is the exact optimum and
//             the exact canonical dual of the rounded tile (whose entries are
//             within 2^-47 of the tile's magnitude of the given ones): the
//             same for every start, so warm and cold solves agree bit for bit,
//             and dual feasible for the given tile too (rounding down only
//             lowers costs).  GB300 issues integer additions ~40x faster than
//             FP64 ones.
//             The bounds, in grid steps: |c| < 2^48 and |u0| <= 2^49 give start
//             column duals below 2^49.6; a search's sink label is the growth
//             of the matching's cost minus u_i + v_sink, so the sink labels of
//             all searches sum below 2^56 and every dual stays below 2^56.2;
//             reduced costs are below 2^57.1 and labels below 2^57.6; the
//             canonical pass's distances are u^c_r - (u_r - u_0) with
//             |u^c| < 31 * 2^49 < 2^54, below 2^57.3, candidates below 2^58.3.
//
// Order of the operations (the oracle's, by specification; exact in fixed point):
//   start     u = u0 or 0;  v_c = min_r (c_rc - u_r), ties to the lowest row
//   greedy    column c takes its argmin row if no lower column took that row
//   search    for every free row i (increasing): Dijkstra on reduced costs
//             pi(r,c) = (c_rc - u_r) - v_c; labels d_c = d_last + pi(r,c);
//             pick the unscanned column of least label (lowest index on ties);
//             relax only on strict '<'; stop at the first free column.
//   duals     v_c = v_c + (d_c - d_sink) on scanned columns, augment, then
//             u_r = c_{r,sigma(r)} - v_{sigma(r)} for every matched row
//   value     sum_r c_{r,sigma(r)} as a pairwise tree (lane i += lane i+h, h = P/2..1);
//             exact in fixed point, where one LAP per warp sums by warp reductions
//   canonical (dual_mode 1, 2) Dijkstra from row 0 over arcs r'->r with weight
//             pi(r, sigma(r')) (>= 0), u^c_r = dist_r + (u_r - u_0),
//             v^c_c = c_{sigma^-1(c),c} - u^c_{sigma^-1(c)}
#pragma once
#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#include "rlt2_internal.h"

namespace rlt2 {

constexpr unsigned kFull = 0xffffffffu;

// Order-preserving 64-bit key of a double (non-NaN): a < b  <=>  okey(a) < okey(b),
// with -0 and +0 equal, exactly as the IEEE comparison.
__device__ __forceinline__ unsigned long long okey(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  b = (b == 0x8000000000000000ull) ? 0ull : b;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Lane holding the least key; lowest lane on ties.  The low words are compared
// only when several lanes share the least high word (a warp-uniform branch).
__device__ __forceinline__ int warp_argmin(unsigned long long key) {
  const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
  const unsigned mhi = __reduce_min_sync(kFull, hi);
  unsigned ball = __ballot_sync(kFull, hi == mhi);
  if (ball & (ball - 1u)) {
    const unsigned mlo = __reduce_min_sync(kFull, hi == mhi ? lo : 0xffffffffu);
    ball = __ballot_sync(kFull, hi == mhi && lo == mlo);
  }
  return __ffs(ball) - 1;
}

__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }

// Arithmetic of group_lap: value type, subtraction, addition and an
// order-preserving unsigned key.
struct ArithF64 {
  using T = double;
  static constexpr bool kExact = false;  // rounded: keys are cached next to the values
  static __device__ __forceinline__ T sub(T a, T b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ T add(T a, T b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ unsigned long long key(T x) { return okey(x); }
};
struct ArithFx {
  using T = long long;
  static constexpr bool kExact = true;  // exact: keys are the values with the sign bit flipped
  static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ unsigned long long key(T x) {
    return (unsigned long long)x ^ 0x8000000000000000ull;
  }
};

// ---- fixed-point grid of a tile -------------------------------------------
// Biased exponent field of a double (0 for zeros and subnormals).
__device__ __forceinline__ unsigned fx_expfield(double x) {
  return (unsigned)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffull);
}
// Grid exponent L of a tile whose largest exponent field is eb: every entry is
// below 2^E with E = max(eb, 1) - 1022, and L = E - 48.
__device__ __forceinline__ int fx_grid(unsigned eb) { return (int)(eb ? eb : 1u) - 1070; }

// floor(x / 2^L) for |x| < 2^(L + lim) (lim <= 53 + L - e_min keeps the shift
// positive); larger |x| clamp to +-2^lim.  Integer operations only: the signed
// mantissa shifted right arithmetically is the floor for either sign.
__device__ __forceinline__ long long fx_floor(double x, int L, int lim) {
  const long long b = __double_as_longlong(x);
  const int eb = (int)((b >> 52) & 0x7ff);
  const long long mant = (b & 0xFFFFFFFFFFFFFll) | (eb ? (1ll << 52) : 0ll);
  const int e = (eb ? eb : 1) - 1075;  // |x| = mant * 2^e
  if (e + 53 - L > lim) return b < 0 ? -(1ll << lim) : (1ll << lim);
  const int sh = min(L - e, 63);       // >= 53 - lim > 0
  return (b < 0 ? -mant : mant) >> sh;
}

// fx_floor for an entry of the tile whose grid is L: its exponent is at most
// the tile's largest, so |x| < 2^(L + 48) and the clamp of fx_floor cannot
// apply; the result is the same.
__device__ __forceinline__ long long fx_floor_entry(double x, int L) {
  const long long b = __double_as_longlong(x);
  const int eb = (int)((b >> 52) & 0x7ff);
  const long long mant = (b & 0xFFFFFFFFFFFFFll) | (eb ? (1ll << 52) : 0ll);
  const int sh = min(L + 1075 - (eb ? eb : 1), 63);  // >= 5
  return (b < 0 ? -mant : mant) >> sh;
}

// Biased exponent field from the high word of a double in shared memory.
__device__ __forceinline__ unsigned fx_expfield_hi(const double* p) {
  return (reinterpret_cast<const unsigned*>(p)[1] >> 20) & 0x7ffu;
}

// Asynchronous global -> shared copies of 8 bytes (cp.async, no registers held
// while in flight), committed as one group per call site and awaited with
// cp_async_wait_all (the copies of this thread; a __syncwarp then makes the
// group's copies visible to its lanes).
__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// q * 2^L rounded to the nearest double (L >= -1069 by construction of fx_grid).
__device__ __forceinline__ double fx_to_double(long long q, int L) {
  const double p2 = L >= -1022 ? __longlong_as_double((long long)(L + 1023) << 52)
                               : __longlong_as_double(1ll << (L + 1074));
  return __dmul_rn(__ll2double_rn(q), p2);
}

constexpr int kFxEntryBits = 48;  // |entry| < 2^48 grid steps
constexpr int kFxStartBits = 49;  // |u0| <= 2^49 grid steps

template <typename T>
struct WarpLapResult {
  T u;           // row dual of row `gl` (group lane)
  T v;           // column dual of column `gl`
  int r2c;       // column matched to row `gl`
  int c2r;       // row matched to column `gl`
  T value;       // LAP optimum (all lanes of the group)
  int naug;      // augmenting searches
  int nrelax;    // label relaxations (instrumentation for the roofline)
};

// Lowest group lane holding the least key among the G lanes of this lane's
// group (aligned groups of G lanes).  Every lane of the warp must call it.
template <int G>
__device__ __forceinline__ int group_argmin(unsigned long long key, int gb) {
  if constexpr (G == 32) {
    return warp_argmin(key);
  } else if constexpr (G == 16) {
    // two full-warp reductions of the high words, each with the other half's
    // lanes at the maximum (no divergence, unlike a redux.sync on a half-warp
    // mask), the low words only where a half has a tie on the high word
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const bool g0 = gb == 0;
    const unsigned m0 = __reduce_min_sync(kFull, g0 ? hi : 0xffffffffu);
    const unsigned m1 = __reduce_min_sync(kFull, g0 ? 0xffffffffu : hi);
    const unsigned mhi = g0 ? m0 : m1;
    unsigned mine = (__ballot_sync(kFull, hi == mhi) >> gb) & 0xffffu;
    if (__any_sync(kFull, (mine & (mine - 1u)) != 0u)) {
      const bool cand = hi == mhi;
      const unsigned l0 = __reduce_min_sync(kFull, (g0 && cand) ? lo : 0xffffffffu);
      const unsigned l1 = __reduce_min_sync(kFull, (!g0 && cand) ? lo : 0xffffffffu);
      const unsigned mlo = g0 ? l0 : l1;
      mine = (__ballot_sync(kFull, cand && lo == mlo) >> gb) & 0xffffu;
    }
    return __ffs(mine) - 1;
  } else {
    // xor butterfly (a redux.sync on the group's own lane mask was slower
    // here: 0.121 against 0.104 ms per iteration at n = 12)
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

// Called by group_lap once the column reduction has read the staged raw tile
// (all lanes, after a __syncwarp): the caller may then reuse the raw buffer.
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// Solve one LAP per group of G lanes (32/G LAPs per warp) in lockstep: every
// intrinsic is executed by all 32 lanes with the full mask and all loops are
// warp-uniform (they run while any group still has work; idle groups only
// predicate their updates), so the LAPs of one warp share every instruction.
// Group lane gl = lane % G holds row gl and column gl of its LAP.  `cs` is the
// group's m x m tile (row stride ld) in shared memory, `scr` G ints of group
// scratch, m the group's LAP size (0 = no LAP, 1 <= m <= G otherwise).  The
// arithmetic is identical for every G.
// PRE: the caller does not need the tile afterwards, so the canonical pass may
// replace it by its reduced costs first (uvs: 64 values of group staging).
// A: ArithF64 or ArithFx (the tile and u0 already on the grid).
// raw (fixed point only, nullable): the group's tile as m*m doubles, row-major
// and unconverted, in shared memory; the column reduction then converts each
// entry onto the grid 2^L as it reads it (lanes = columns) and stores it into
// cs, and calls hook() once raw is no longer needed.  Without raw, cs already
// holds the converted tile.
// RR (exact form only): a cold start reduces the rows first, u_r = the row's
// minimum, as the classical Hungarian method does, before the column
// reduction: fewer searches are left after the greedy matching, and the
// canonical result does not depend on the start.
template <int G, bool PRE, typename A, bool RR = false, typename Hook = NoHook>
__device__ __forceinline__ WarpLapResult<typename A::T> group_lap(typename A::T* __restrict__ cs, int ld, int m,
                                                                  int lane, bool warm, typename A::T u0,
                                                                  int dual_mode, int* scr, typename A::T* uvs,
                                                                  const double* raw = nullptr, int L = 0,
                                                                  const Hook& hook = Hook()) {
  using T = typename A::T;
  const int gl = lane & (G - 1);
  const int gb = lane - gl;
  const bool cv = gl < m;
  const int M = (G == 32) ? m : (int)__reduce_max_sync(kFull, (unsigned)m);
  WarpLapResult<T> R;
  T u = (cv && warm) ? u0 : T(0);
  T v = T(0);
  int naug = 0, nrelax = 0;

  // column reduction with the argmin row (fixed point: the row duals are
  // broadcast from shared memory, one load instead of two shuffles per row;
  // uvs holds the group's row duals until the canonical pass)
  unsigned long long bestk = ~0ull;
  int arg = -1;
  // exact form: the running minimum starts above every |x| < 2^58, so the first
  // row always takes it (the same result as testing arg < 0)
  T vmin = A::kExact ? T(0x7fffffffffffffffll) : T(0);
  if constexpr (A::kExact && RR) {
    // warp-uniform (the launches that take RR start every LAP cold)
    if (!__any_sync(kFull, warm)) {
      if (raw) {  // the tile onto the grid first (lanes = columns)
        for (int r = 0; r < M; ++r)
          if (cv && r < m) cs[r * ld + gl] = fx_floor_entry(raw[r * m + gl], L);
        __syncwarp();
        hook();
        raw = nullptr;
      }
      T mn = T(0x7fffffffffffffffll);  // above every entry (|x| < 2^58)
      for (int c = 0; c < M; ++c)
        if (cv && c < m) {
          const T x = cs[gl * ld + c];  // lane = row (odd row stride: no bank conflicts)
          mn = x < mn ? x : mn;
        }
      u = cv ? mn : T(0);
      warm = true;  // the column reduction below subtracts these row duals
    }
  }
  if constexpr (A::kExact) {
    uvs[gl] = u;
    __syncwarp();
  }
  for (int r = 0; r < M; ++r) {
    T ur;
    if constexpr (A::kExact) ur = warm ? uvs[r] : T(0);
    else ur = __shfl_sync(kFull, u, gb + r);
    if (cv && r < m) {
      T c;
      if constexpr (A::kExact) {
        if (raw) {
          c = fx_floor_entry(raw[r * m + gl], L);
          cs[r * ld + gl] = c;
        } else {
          c = cs[r * ld + gl];
        }
      } else {
        c = cs[r * ld + gl];
      }
      const T x = warm ? A::sub(c, ur) : c;  // c - 0 == c exactly
      if constexpr (A::kExact) {
        if (x < vmin) {
          arg = r;
          vmin = x;
        }
      } else if (arg < 0 || A::key(x) < bestk) {
        bestk = A::key(x);
        arg = r;
        v = x;
      }
    }
  }
  if constexpr (A::kExact) {
    if (cv) v = vmin;
  }
  if constexpr (A::kExact) {
    if (raw) {
      __syncwarp();  // every lane's reads of raw are done
      hook();
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

  // at G = 32 the warp is one group, so every loop condition below is
  // warp-uniform and needs no vote
  unsigned freerows = group_bits<G>(__ballot_sync(kFull, cv && r2c < 0), gb);
  while (G == 32 ? freerows != 0 : __any_sync(kFull, freerows != 0)) {
    const bool act = freerows != 0;  // this group runs a search in this pass
    const int i = act ? __ffs(freerows) - 1 : 0;
    if (act) {
      freerows &= freerows - 1;
      ++naug;
      nrelax += m;
    }
    T ui;
    if constexpr (A::kExact) ui = uvs[i];
    else ui = __shfl_sync(kFull, u, gb + i);
    T d = (act && cv) ? A::sub(A::sub(cs[i * ld + gl], ui), v) : T(0);
    unsigned long long dk = A::key(d);  // cached key of d (rounded form only)
    int pred = i;
    bool scanned = !(act && cv);
    bool searching = act;
    int sink = 0;
    T dlast = T(0);
    while (G == 32 ? searching : __any_sync(kFull, searching)) {
      const int c = group_argmin<G>(scanned ? ~0ull : (A::kExact ? A::key(d) : dk), gb);
      const T dm = __shfl_sync(kFull, d, gb + c);
      if (searching && gl == c) scanned = true;
      // the matching does not change during a search, so column c is free
      // exactly when it has no matched row
      const int r0 = __shfl_sync(kFull, c2r, gb + c);
      const bool found = searching && r0 < 0;
      if (found) {
        sink = c;
        dlast = dm;
      }
      const bool relaxing = searching && !found;
      const int r = r0 < 0 ? 0 : r0;
      T ur;
      if constexpr (A::kExact) ur = uvs[RLT2_IDX(r, m > 0 ? m : 1)];
      else ur = __shfl_sync(kFull, u, gb + r);
      if (relaxing && !scanned) {
        const T nd = A::add(dm, A::sub(A::sub(cs[RLT2_IDX(r, m) * ld + gl], ur), v));
        if (A::kExact ? nd < d : A::key(nd) < dk) {
          d = nd;
          if constexpr (!A::kExact) dk = A::key(nd);
          pred = r;
        }
      }
      searching = relaxing;
    }
    // every step scanned one column, the last one the sink: the relaxing
    // steps are the scanned columns but one, and the k-th of them relaxed the
    // m - k columns still unscanned
    const int step = __popc(group_bits<G>(__ballot_sync(kFull, act && cv && scanned), gb)) - 1;
    if (act) nrelax += step * m - (step * (step + 1)) / 2;
    if (act && cv && scanned) v = A::add(v, A::sub(d, dlast));
    // augment back to row i (groups walk their own chains in lockstep)
    bool walking = act;
    int col = sink;
    while (G == 32 ? walking : __any_sync(kFull, walking)) {
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
    const T vm = __shfl_sync(kFull, v, gb + mc);
    if (act && cv && r2c >= 0) u = A::sub(cs[gl * ld + RLT2_IDX(r2c, m)], vm);
    if constexpr (A::kExact) {
      uvs[gl] = u;
      __syncwarp();
    }
  }

  // optimum: pairwise tree over P = next power of two >= m rows (empty rows add
  // nothing), lane i adding lane i + h for h = P/2, ..., 1
  const T xr = cv ? cs[gl * ld + RLT2_IDX(r2c, m)] : T(0);
  T val;
  if constexpr (G == 32 && A::kExact) {
    // exact sums do not depend on the order: the 64-bit entries as two
    // non-negative 26-bit limbs and a signed top part, each summed over the
    // warp by one 32-bit reduction (32 limbs < 2^31, no overflow)
    const unsigned long long ux = (unsigned long long)xr;
    const int l0 = (int)(ux & 0x3ffffffull), l1 = (int)((ux >> 26) & 0x3ffffffull);
    const int l2 = (int)(xr >> 52);
    const long long s0 = __reduce_add_sync(kFull, l0), s1 = __reduce_add_sync(kFull, l1);
    const long long s2 = __reduce_add_sync(kFull, l2);
    val = (T)(s2 * (1ll << 52) + s1 * (1ll << 26) + s0);
  } else {
    int P = 1;
    while (P < m) P <<= 1;
    const int PM = (G == 32) ? P : (int)__reduce_max_sync(kFull, (unsigned)P);
    val = xr;
    for (int h = PM >> 1; h >= 1; h >>= 1) {
      const T o = __shfl_xor_sync(kFull, val, h);
      if (h < P) val = A::add(val, o);
    }
    val = __shfl_sync(kFull, val, gb);
  }

  if (dual_mode != 0) {
    // canonical duals: shortest paths from row 0 on reduced weights
    // pi(r, sigma(r')) = (c_{r,sigma(r')} - u_r) - v_{sigma(r')} >= 0
    const int s0 = __shfl_sync(kFull, r2c, gb);
    // exact form: a lane forms only the reduced costs of its own row that the
    // pass reads (two integer subtractions each, with the column duals
    // broadcast from shared memory) instead of the whole reduced tile first
    constexpr bool kRed = PRE && !A::kExact;  // the reduced tile is formed first
    if constexpr (A::kExact) {
      uvs[32 + gl] = v;
      __syncwarp();
    } else if constexpr (PRE) {
      // an FP64 instruction costs the same with few lanes active, so the group's
      // lanes take the m*m entries in row-major turns (every lane busy); (r, c)
      // of entry gl + k*G advance without a division per entry
      uvs[gl] = u;
      uvs[32 + gl] = v;
      __syncwarp();
      if (m > 0) {
        const int qg = G / m, rg = G - qg * m;
        int r = gl / m, c = gl - r * m;
        for (; r < m; r += qg) {
          cs[r * ld + c] = A::sub(A::sub(cs[r * ld + c], uvs[r]), uvs[32 + c]);
          c += rg;
          if (c >= m) {
            c -= m;
            ++r;
          }
        }
      }
      __syncwarp();
    }
    T vs0 = T(0);
    if constexpr (A::kExact) vs0 = uvs[32 + RLT2_IDX(s0 < 0 ? 0 : s0, m > 0 ? m : 1)];
    else vs0 = __shfl_sync(kFull, v, gb + (s0 < 0 ? 0 : s0));
    T dist = T(0);
    if (cv && gl != 0) {
      if constexpr (kRed) dist = cs[gl * ld + RLT2_IDX(s0, m)];
      else dist = A::sub(A::sub(cs[gl * ld + RLT2_IDX(s0, m)], u), vs0);
    }
    bool done = !cv || gl == 0;
    unsigned long long dk = A::key(dist);  // cached key of dist (rounded form only)
    for (int it = 0; it < M - 2; ++it) {
      const bool stepping = it < m - 2;
      const int rs = group_argmin<G>(done ? ~0ull : (A::kExact ? A::key(dist) : dk), gb);
      const T dr = __shfl_sync(kFull, dist, gb + rs);
      if (stepping && gl == rs) done = true;
      const int s = __shfl_sync(kFull, r2c, gb + rs);
      T vs = T(0);
      if constexpr (A::kExact) vs = uvs[32 + RLT2_IDX(s < 0 ? 0 : s, m > 0 ? m : 1)];
      else if constexpr (!kRed) vs = __shfl_sync(kFull, v, gb + (s < 0 ? 0 : s));
      if (stepping && !done) {
        T w;
        if constexpr (kRed) w = cs[gl * ld + RLT2_IDX(s, m)];
        else w = A::sub(A::sub(cs[gl * ld + RLT2_IDX(s, m)], u), vs);
        const T nd = A::add(dr, w);
        if (A::kExact ? nd < dist : A::key(nd) < dk) {
          dist = nd;
          if constexpr (!A::kExact) dk = A::key(nd);
        }
      }
    }
    const T u0r = __shfl_sync(kFull, u, gb);
    const T ucan = cv ? (m > 1 ? A::add(dist, A::sub(u, u0r)) : T(0)) : T(0);
    // v_c = c_{sigma^-1(c), c} - u_{sigma^-1(c)}, from the matched row's own entry
    const T wrow = A::sub(xr, ucan);
    const int rr = cv ? c2r : 0;
    const T vcan = __shfl_sync(kFull, wrow, gb + rr);
    u = ucan;
    v = cv ? vcan : T(0);
    if constexpr (A::kExact) __syncwarp();  // the reads of uvs are done before a caller reuses it
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

// ---- launch helpers shared by the LAP kernels ------------------------------
constexpr int kMaxWarpsPerBlock = 8;

__host__ __device__ inline int tile_ld(int m) { return m | 1; }  // odd stride: conflict-free rows and columns

// Shared memory per warp: 32/G tiles, u/v staging (64 doubles) and 32 ints.
__host__ __device__ inline size_t warp_smem_bytes(int m, int G) {
  return (size_t)(32 / G) * m * tile_ld(m) * sizeof(double) + 64 * sizeof(double) + 32 * sizeof(int);
}
// The prefetching form adds, per group, the next tile (m*m doubles, as stored)
// and its start duals (m doubles), rounded to 16 bytes.
__host__ __device__ inline size_t raw_group_doubles(int m) { return ((size_t)m * m + m + 1) & ~size_t(1); }
__host__ __device__ inline size_t warp_smem_bytes_async(int m, int G) {
  return warp_smem_bytes(m, G) + (size_t)(32 / G) * raw_group_doubles(m) * sizeof(double);
}

// Stages one group's tile (plus an optional addend) into shared memory, the
// group's G lanes reading a contiguous m*m run (coalesced).  FX: the tile is
// rounded down onto the group's fixed-point grid and the grid exponent L is
// returned (0 for FP64).  All 32 lanes call it; src == nullptr for a group
// without a LAP.  CG: load through L2 only (the tile was written by other SMs
// during the same launch, so a line in this SM's L1 may be stale).
// The lane's entries e = gl, gl + G, ... < mm of src (+ add, rounded), U
// of them loaded before any is used (U > 1 for latency-bound launches of few
// LAPs, where one warp's serial loads would be its time), each passed to f(e, x).
template <int G, bool CG, int U, typename F>
__device__ __forceinline__ void for_tile_entries(int mm, int gl, const double* src, const double* add, F&& f) {
  for (int e0 = gl; e0 < mm; e0 += G * U) {
    double x[U], y[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int e = e0 + k * G;
      x[k] = e < mm ? (CG ? __ldcg(src + e) : __ldcs(src + e)) : 0.0;
      y[k] = (add && e < mm) ? (CG ? __ldcg(add + e) : __ldcs(add + e)) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int e = e0 + k * G;
      if (e < mm) f(e, add ? __dadd_rn(x[k], y[k]) : x[k]);
    }
  }
}

template <int G, bool FX, bool CG = false, int U = 1>
__device__ __forceinline__ int stage_tile(typename std::conditional<FX, long long, double>::type* tile, int ld,
                                          int m, int gl, const double* src, const double* add) {
  const int mm = m * m;
  if constexpr (!FX) {
    if (src)
      for_tile_entries<G, CG, U>(mm, gl, src, add, [&](int e, double x) {
        const int r = e / m, c = e - r * m;
        tile[r * ld + c] = x;
      });
    return 0;
  } else {
    unsigned eb = 0;
    if (src)
      for_tile_entries<G, CG, U>(mm, gl, src, add, [&](int e, double x) {
        const int r = e / m, c = e - r * m;
        tile[r * ld + c] = __double_as_longlong(x);  // bits; converted below once the grid is known
        eb = max(eb, fx_expfield(x));
      });
    if constexpr (G == 32) {
      eb = __reduce_max_sync(kFull, eb);
    } else {
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) eb = max(eb, __shfl_xor_sync(kFull, eb, off));
    }
    const int L = fx_grid(eb);
    if (src) {
      for (int e = gl; e < mm; e += G) {  // the entries this lane wrote
        const int r = e / m, c = e - r * m;
        tile[r * ld + c] = fx_floor(__longlong_as_double(tile[r * ld + c]), L, kFxEntryBits);
      }
    }
    return L;
  }
}

template <bool FX, typename T>
__device__ __forceinline__ double out_value(T x, int L) {
  if constexpr (FX) return fx_to_double(x, L);
  else return x;
}

template <bool FX>
__device__ __forceinline__ typename std::conditional<FX, long long, double>::type start_dual(double u0, int L) {
  if constexpr (FX) return fx_floor(u0, L, kFxStartBits);
  else return u0;
}

}  // namespace rlt2
