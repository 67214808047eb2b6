"""Seeded synthetic QAP instances (flow F, distance D, fixed cost B).

This module holds only input generation: it contains none of the bound's
arithmetic, so both the CUDA path and the CPU oracle draw their inputs from it.

The paper evaluates on QAPLIB's Nugent instances (Manhattan distances on a grid,
sparse small-integer flows) and Taillard-a instances (dense uniform matrices),
Section 5.  Those files are not shipped; the recipes below produce instances of
the same shapes and value distributions:

* PRNG: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then two
  xor-shift-multiply rounds and a final xor-shift.
* Symmetric matrix with zero diagonal: for i < j in row-major order draw
  ``v = next() % (hi + 1)`` then ``keep = (next() >> 11) * 2**-53 < density``;
  ``M[i, j] = M[j, i] = v if keep else 0``.
* Grid distances: cell c sits at (c // cols, c % cols); d = |drow| + |dcol|.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (64-bit state, 64-bit output)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def below(self, k: int) -> int:
        return self.next() % k


def symmetric_matrix(rng: SplitMix64, n: int, hi: int, density: float) -> np.ndarray:
    m = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        for j in range(i + 1, n):
            v = rng.below(hi + 1)
            keep = rng.uniform() < density
            m[i, j] = m[j, i] = float(v) if keep else 0.0
    return m


def grid_distance(rows: int, cols: int) -> np.ndarray:
    n = rows * cols
    d = np.zeros((n, n), dtype=np.float64)
    for a in range(n):
        ra, ca = divmod(a, cols)
        for b in range(n):
            rb, cb = divmod(b, cols)
            d[a, b] = abs(ra - rb) + abs(ca - cb)
    return d


@dataclass
class Instance:
    name: str
    n: int
    F: np.ndarray
    D: np.ndarray
    B: np.ndarray
    iterations: int
    partials: Optional[np.ndarray] = None  # (n_nodes, n) int32, -1 = free facility
    recipe: str = ""
    extra: dict = field(default_factory=dict)


def grid_instance(name, rows, cols, hi, density, seed, iterations) -> Instance:
    n = rows * cols
    rng = SplitMix64(seed)
    F = symmetric_matrix(rng, n, hi, density)
    D = grid_distance(rows, cols)
    return Instance(name, n, F, D, np.zeros((n, n)), iterations,
                    recipe=f"D=Manhattan {rows}x{cols} grid; F sym 0..{hi} density {density}; seed {seed}; B=0")


def dense_instance(name, n, hi, seed, iterations) -> Instance:
    rng = SplitMix64(seed)
    F = symmetric_matrix(rng, n, hi, 1.0)
    D = symmetric_matrix(rng, n, hi, 1.0)
    return Instance(name, n, F, D, np.zeros((n, n)), iterations,
                    recipe=f"F,D sym dense uniform 0..{hi} (D drawn after F); seed {seed}; B=0")


def random_partials(n: int, n_nodes: int, depth_lo: int, depth_hi: int, seed: int) -> np.ndarray:
    """Branch-and-bound nodes: depth l uniform in [depth_lo, depth_hi]; the first l
    facilities of a random order are fixed to random distinct locations."""
    rng = SplitMix64(seed)
    out = -np.ones((n_nodes, n), dtype=np.int32)
    for t in range(n_nodes):
        depth = depth_lo + rng.below(depth_hi - depth_lo + 1)
        fac = list(range(n))
        loc = list(range(n))
        for arr in (fac, loc):
            for i in range(n - 1, 0, -1):
                j = rng.below(i + 1)
                arr[i], arr[j] = arr[j], arr[i]
        for a in range(depth):
            out[t, fac[a]] = loc[a]
    return out


def config(idx: int) -> Instance:
    """The five workloads: 1) n=8 grid 2x4, 2) n=12 grid 3x4, 3) n=20 dense
    uniform 0..99, 4) n=22 grid 2x11 with 64 nodes at depths 4..8, 5) n=30 grid 5x6."""
    if idx == 1:
        return grid_instance("n8_grid2x4", 2, 4, 9, 0.5, 0, 50)
    if idx == 2:
        return grid_instance("n12_grid3x4", 3, 4, 9, 0.5, 1, 200)
    if idx == 3:
        return dense_instance("n20_dense99", 20, 99, 2, 300)
    if idx == 4:
        inst = grid_instance("n22_grid2x11_nodes64", 2, 11, 9, 0.6, 3, 100)
        inst.partials = random_partials(22, 64, 4, 8, 3 + 1)
        inst.recipe += "; 64 nodes, depth uniform 4..8, SplitMix64 seed 4 (shuffle facilities, shuffle locations)"
        return inst
    if idx == 5:
        return grid_instance("n30_grid5x6", 5, 6, 9, 0.5, 4, 100)
    raise ValueError(idx)


def random_instance(n: int, seed: int, hi: int = 9, density: float = 0.7,
                    with_b: bool = False, asymmetric: bool = False) -> Instance:
    """Small random instance for tests (optionally with B and asymmetric F)."""
    rng = SplitMix64(seed)
    F = symmetric_matrix(rng, n, hi, density)
    D = symmetric_matrix(rng, n, hi, 1.0)
    if asymmetric:
        for i in range(n):
            for j in range(n):
                if i != j and rng.uniform() < 0.3:
                    F[i, j] = float(rng.below(hi + 1))
        for i in range(n):
            F[i, i] = float(rng.below(3))
            D[i, i] = float(rng.below(3))
    B = np.zeros((n, n))
    if with_b:
        for i in range(n):
            for p in range(n):
                B[i, p] = float(rng.below(hi + 1))
    return Instance(f"rand_n{n}_s{seed}", n, F, D, B, 10)


def sa_draws(n: int, count: int, seed: int, kappa_max: float = 0.25):
    """Random draws of the Type 4 (annealing) rule, passed to both sides as inputs.

    Per draw d (SplitMix64, in this order): a total ``k = kappa_max * U``, then
    2n weights ``w = U`` (facilities first, then locations), then ``u`` in
    (0, 1] as ``((next() >> 11) + 1) * 2**-53``.  The fractions are
    ``kf[d] = k * w[:n] / sum(w)``, ``kl[d] = k * w[n:] / sum(w)`` (their sum is
    at most kappa_max, as Section 5 draws them) and ``neglog_u[d] = -ln(u)``.
    Returns (kf[count, n], kl[count, n], neglog_u[count]) as float64."""
    import math
    rng = SplitMix64(seed)
    kf = np.zeros((count, n))
    kl = np.zeros((count, n))
    ng = np.zeros(count)
    for d in range(count):
        k = kappa_max * rng.uniform()
        w = np.array([rng.uniform() for _ in range(2 * n)])
        u = ((rng.next() >> 11) + 1) * (1.0 / (1 << 53))
        tot = float(w.sum())
        frac = (k / tot) * w if tot > 0 else np.zeros(2 * n)
        kf[d] = frac[:n]
        kl[d] = frac[n:]
        ng[d] = -math.log(u)
    return kf, kl, ng
