"""CPU oracle for RLT2 dual ascent -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package never imports the CUDA library: the two share nothing but the seeded
input generator (``paper_1710_03732_gb300.instances``), which holds none of
the method's arithmetic.

The C source ``rlt2_oracle.c`` is compiled with gcc (``-O2 -ffp-contract=off``,
OpenMP when available) into ``oracle/_build/liboracle.so`` on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rlt2_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_longlong)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2 -ffp-contract=off; OpenMP if it links)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.or_lap.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _ip, _ip, _lp]
        L.or_lap_canonical.argtypes = [ctypes.c_int, _dp, _ip, _dp, _dp]
        L.or_lap_brute.argtypes = [ctypes.c_int, _dp, _ip]
        L.or_lap_brute.restype = ctypes.c_double
        L.or_qap_cost.argtypes = [ctypes.c_int, _dp, _dp, _dp, _ip]
        L.or_qap_cost.restype = ctypes.c_double
        L.or_qap_brute.argtypes = [ctypes.c_int, _dp, _dp, _dp, _ip]
        L.or_qap_brute.restype = ctypes.c_double
        L.or_num_tiles.argtypes = [ctypes.c_int]
        L.or_num_tiles.restype = ctypes.c_longlong
        L.or_num_z.argtypes = [ctypes.c_int]
        L.or_num_z.restype = ctypes.c_longlong
        L.or_setup.argtypes = [ctypes.c_int, _dp, _dp, _dp, _ip, _ip, _dp, _dp, _dp, _dp]
        L.or_stage_z.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _lp, _lp, ctypes.c_int]
        L.or_stage_y.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _lp, _lp]
        L.or_stage_x.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _ip, _lp, _lp]
        L.or_reduced_xy.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_redistribute_z.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
        L.or_redistribute_y.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
        L.or_feasibility.argtypes = [ctypes.c_int, _ip, _dp, _dp, _dp, _dp, ctypes.c_double]
        L.or_iterate.argtypes = ([ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                  _dp, _dp, _dp, _dp, _dp, _ip, _dp, _dp, _lp, ctypes.c_int])
        L.or_redistribute_z_v.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
        L.or_redistribute_y_fast.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.or_move_x_fast.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
        L.or_phase2_z.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, ctypes.c_int]
        L.or_sa_schedule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
        L.or_sa_term.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
        L.or_sa_term.restype = ctypes.c_int
        L.or_iterate_v.argtypes = ([ctypes.c_int, _dp, _ip, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                    _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _ip, _dp, _dp, _ip, _lp,
                                    ctypes.c_int])
        L.or_stage_z_upper.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _lp, _lp]
        L.or_redistribute_half.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_redistribute_half_form.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_redistribute_z_form.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, _dp,
                                             _dp, ctypes.c_int]
        L.or_iterate_half.argtypes = ([ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                       _dp, _dp, _dp, _dp, _dp, _dp, _ip, _dp, _dp, _lp])
        L.or_child_state.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _dp,
                                     _dp, _dp, _dp]
        L.or_lagrangian_objective.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _ip]
        L.or_lagrangian_objective.restype = ctypes.c_double
        L.or_have_openmp.restype = ctypes.c_int
        _fp = ctypes.POINTER(ctypes.c_float)
        L.or_f32_trunc.argtypes = [ctypes.c_double]
        L.or_f32_trunc.restype = ctypes.c_float
        L.or_bf16_round.argtypes = [ctypes.c_float]
        L.or_bf16_round.restype = ctypes.c_float
        L.or_mlp_features.argtypes = [ctypes.c_int, _dp, _dp, _dp, _fp, _fp, _fp]
        L.or_mlp_forward.argtypes = [ctypes.c_int, ctypes.c_int, _fp, _fp, _fp, _fp, _fp, _fp, ctypes.c_double,
                                     ctypes.c_int, _dp, _dp, _dp]
        L.or_mlp_backward.argtypes = [ctypes.c_int, ctypes.c_int, _fp, _fp, _fp, ctypes.c_int, _dp, _dp, _dp, _dp,
                                      _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_mlp_backward.restype = ctypes.c_double
    return _lib


def _d(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_dp)


def _i(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_ip)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(lib().or_have_openmp())


# --------------------------------------------------------------------------
# LAP
# --------------------------------------------------------------------------
@dataclass
class LapResult:
    value: float
    u: np.ndarray
    v: np.ndarray
    row_to_col: np.ndarray
    n_aug: int
    n_relax: int


def lap(cost: np.ndarray, u0: Optional[np.ndarray] = None, canonical: bool = False) -> LapResult:
    c = _f64(cost)
    m = c.shape[0]
    u = np.zeros(m)
    v = np.zeros(m)
    r2c = np.zeros(m, dtype=np.int32)
    val = ctypes.c_double()
    aug = ctypes.c_int()
    rel = ctypes.c_longlong()
    u0c = None if u0 is None else _f64(u0)
    lib().or_lap(m, _d(c), _d(u0c), ctypes.byref(val), _d(u), _d(v), _i(r2c), ctypes.byref(aug), ctypes.byref(rel))
    if canonical:
        u, v = lap_canonical(c, r2c)
    return LapResult(val.value, u, v, r2c, aug.value, rel.value)


def lap_canonical(cost: np.ndarray, row_to_col: np.ndarray):
    c = _f64(cost)
    m = c.shape[0]
    r2c = np.ascontiguousarray(row_to_col, dtype=np.int32)
    u = np.zeros(m)
    v = np.zeros(m)
    lib().or_lap_canonical(m, _d(c), _i(r2c), _d(u), _d(v))
    return u, v


def lap_brute(cost: np.ndarray):
    c = _f64(cost)
    m = c.shape[0]
    perm = np.zeros(m, dtype=np.int32)
    val = lib().or_lap_brute(m, _d(c), _i(perm))
    return val, perm


def qap_cost(F, D, B, perm) -> float:
    F, D = _f64(F), _f64(D)
    B = None if B is None else _f64(B)
    p = np.ascontiguousarray(perm, dtype=np.int32)
    return lib().or_qap_cost(F.shape[0], _d(F), _d(D), _d(B), _i(p))


def qap_brute(F, D, B=None):
    F, D = _f64(F), _f64(D)
    B = None if B is None else _f64(B)
    n = F.shape[0]
    perm = np.zeros(n, dtype=np.int32)
    val = lib().or_qap_brute(n, _d(F), _d(D), _d(B), _i(perm))
    return val, perm


# --------------------------------------------------------------------------
# RLT2 state and one iteration
# --------------------------------------------------------------------------
def num_tiles(n: int) -> int:
    return n * n * (n - 1) * (n - 1)


def num_z(n: int) -> int:
    return num_tiles(n) * (n - 2) * (n - 2)


def params_array(kz=1.0, ky=0.5, kx=1.0, phi_y=0.5, phi_z: Sequence[float] = (0.2,) * 5) -> np.ndarray:
    return np.array([kz, ky, kx, phi_y] + list(phi_z), dtype=np.float64)


@dataclass
class State:
    n: int           # residual size
    const: float     # constant from the fixed facilities
    bprime: np.ndarray
    Chat: np.ndarray
    Dhat: np.ndarray


def setup(F, D, B=None, partial=None) -> State:
    F, D = _f64(F), _f64(D)
    n = F.shape[0]
    B = None if B is None else _f64(B)
    part = None if partial is None else np.ascontiguousarray(partial, dtype=np.int32)
    nr = n if part is None else int((part < 0).sum())
    bprime = np.zeros(nr * nr)
    Chat = np.zeros(max(num_tiles(nr), 1))
    Dhat = np.zeros(max(num_z(nr), 1)) if nr >= 3 else np.zeros(1)
    nres = ctypes.c_int()
    cst = ctypes.c_double()
    rc = lib().or_setup(n, _d(F), _d(D), _d(B), _i(part), ctypes.byref(nres), ctypes.byref(cst), _d(bprime),
                        _d(Chat), _d(Dhat))
    if rc != 0:
        raise ValueError("or_setup rejected the input")
    return State(nr, cst.value, bprime, Chat, Dhat)


@dataclass
class IterOut:
    lb: float
    Theta: np.ndarray
    xi: np.ndarray
    psi: np.ndarray
    Delta: np.ndarray
    gamma: np.ndarray
    delta: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    xperm: np.ndarray
    pix: np.ndarray
    piy: np.ndarray
    stats: np.ndarray  # [aug_z, relax_z, aug_y, relax_y, aug_x, relax_x]


def iterate(st: State, prm: np.ndarray, dual_mode: int = 1, u0z: Optional[np.ndarray] = None,
            threads: int = 1, u0y: Optional[np.ndarray] = None, u0x: Optional[np.ndarray] = None) -> IterOut:
    """One S1 iteration in place on st.Chat / st.Dhat; returns the bound and all duals
    (the bound is of the multipliers before this iteration's ascent step)."""
    n = st.n
    T = num_tiles(n)
    mz, my = n - 2, n - 1
    o = IterOut(0.0, np.zeros(T), np.zeros(T * mz), np.zeros(T * mz), np.zeros(n * n), np.zeros(n * n * my),
                np.zeros(n * n * my), np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.int32), np.zeros(n * n),
                np.zeros(T), np.zeros(6, dtype=np.int64))
    lb = ctypes.c_double()
    prm = _f64(prm)
    u0c = None if u0z is None else _f64(u0z)
    u0yc = None if u0y is None else _f64(u0y)
    u0xc = None if u0x is None else _f64(u0x)
    rc = lib().or_iterate(n, _d(prm), dual_mode, _d(st.bprime), _d(st.Chat), _d(st.Dhat), _d(u0c), _d(u0yc), _d(u0xc),
                          ctypes.byref(lb), _d(o.Theta), _d(o.xi), _d(o.psi), _d(o.Delta), _d(o.gamma),
                          _d(o.delta), _d(o.alpha), _d(o.beta), _i(o.xperm), _d(o.pix), _d(o.piy),
                          o.stats.ctypes.data_as(_lp), threads)
    if rc != 0:
        raise ValueError("or_iterate rejected the input")
    o.lb = lb.value
    return o


def stage_z(n, Dhat, dual_mode=1, u0=None, threads=1):
    T = num_tiles(n)
    m = n - 2
    Theta, xi, psi = np.zeros(T), np.zeros(T * m), np.zeros(T * m)
    aug, rel = ctypes.c_longlong(), ctypes.c_longlong()
    lib().or_stage_z(n, dual_mode, _d(_f64(Dhat)), _d(None if u0 is None else _f64(u0)), _d(Theta), _d(xi),
                     _d(psi), ctypes.byref(aug), ctypes.byref(rel), threads)
    return Theta, xi, psi, aug.value, rel.value


def redistribute_z(n, prm, Dhat, xi, psi, piy, pix, threads=1):
    """Returns a new D^ after the z move (input left untouched)."""
    out = _f64(Dhat).copy()
    lib().or_redistribute_z(n, _d(_f64(prm)), _d(out), _d(_f64(xi)), _d(_f64(psi)), _d(_f64(piy)), _d(_f64(pix)),
                            threads)
    return out


def redistribute_y(n, phi_y, Chat, piy):
    out = _f64(Chat).copy()
    lib().or_redistribute_y(n, float(phi_y), _d(out), _d(_f64(piy)))
    return out


def feasibility(n, xperm, piy, Dhat, xi, psi, tol=1e-9) -> bool:
    return bool(lib().or_feasibility(n, _i(np.ascontiguousarray(xperm, dtype=np.int32)), _d(_f64(piy)),
                                     _d(_f64(Dhat)), _d(_f64(xi)), _d(_f64(psi)), float(tol)))


def run(F, D, B=None, iters=10, prm=None, dual_mode=1, partial=None, threads=1, warm=False, variant=0,
        two_phase=False, sa=None, ub=None, sa_t0=0.04, sa_cool=0.99, sa_period=100, trace=None, p2tol=1e-9):
    """Run the dual ascent; returns (state, list of per-iteration bounds incl. const, last IterOut).

    variant 0 = S (slow), 1 = F (fast, incremental costs); two_phase adds the
    second Z phase; sa = (kf[count, n], kl[count, n], neglog_u[count]) are the
    Type 4 draws (annealing temperature sa_t0 * ub).  With warm, every LAP starts
    from the previous iteration's row duals (and the second Z phase from the
    first phase's).  trace (a list) receives per-iteration dicts (sa_on, stats).
    Plain S1 runs take the original single-iteration path."""
    st = setup(F, D, B, partial)
    prm = params_array() if prm is None else prm
    lbs = []
    out = None
    if variant == 0 and not two_phase and sa is None:
        for _ in range(iters):
            w = warm and out is not None
            out = iterate(st, prm, dual_mode, u0z=out.xi.copy() if w else None, threads=threads,
                          u0y=out.gamma.copy() if w else None, u0x=out.alpha.copy() if w else None)
            lbs.append(st.const + out.lb)
            if trace is not None:
                trace.append({"sa_on": 0, "stats": out.stats.copy()})
        return st, lbs, out
    n = st.n
    K = thr = None
    if sa is not None:
        kf, kl, ng = (_f64(a) for a in sa)
        kf = kf.reshape(-1, n)
        kl = kl.reshape(-1, n)
        ng = ng.reshape(-1)
        if ub is None or ub <= 0:
            raise ValueError("the Type 4 rule needs a known upper bound (ub > 0)")
        K, thr = sa_schedule(n, kf, kl, ng, ub, sa_t0, sa_cool, sa_period)
    bx = st.bprime.copy()
    base = st.const
    for it in range(iters):
        w = warm and out is not None
        draw = None
        if sa is not None and it < len(K):
            draw = (K[it], thr[it], kf[it], kl[it])
        out, lb, on = iterate_v(st, bx, prm, base, dual_mode=dual_mode, variant=variant, two_phase=two_phase,
                                warm2=warm, u0z=out.xi.copy() if w else None,
                                u0y=out.gamma.copy() if w else None, u0x=out.alpha.copy() if w else None,
                                draw=draw, threads=threads, p2tol=p2tol)
        lbs.append(lb)
        if variant == 1:
            base = lb
        if trace is not None:
            trace.append({"sa_on": on, "stats": out.stats.copy()})
    return st, lbs, out


def iterate_v(st: State, bx: np.ndarray, prm, lb_base: float, dual_mode=1, variant=0, two_phase=False, warm2=False,
              u0z=None, u0y=None, u0x=None, draw=None, threads=1, p2tol=1e-9):
    """One iteration of a Section 3.4 variant in place on st.Chat, st.Dhat and bx.
    Returns (IterOut, bound, Type 4 accepted)."""
    n = st.n
    T = num_tiles(n)
    mz, my = n - 2, n - 1
    o = IterOut(0.0, np.zeros(T), np.zeros(T * mz), np.zeros(T * mz), np.zeros(n * n), np.zeros(n * n * my),
                np.zeros(n * n * my), np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.int32), np.zeros(n * n),
                np.zeros(T), np.zeros(6, dtype=np.int64))
    opt = np.array([dual_mode, variant, int(bool(two_phase)), int(bool(warm2))], dtype=np.int32)
    lb = ctypes.c_double()
    on = ctypes.c_int()
    dr = kf = kl = None
    if draw is not None:
        dr = np.array([draw[0], draw[1]], dtype=np.float64)
        kf, kl = _f64(draw[2]), _f64(draw[3])
    rc = lib().or_iterate_v(n, _d(_f64(prm)), _i(opt), float(p2tol), float(lb_base), _d(bx), _d(st.Chat), _d(st.Dhat),
                            _d(None if u0z is None else _f64(u0z)), _d(None if u0y is None else _f64(u0y)),
                            _d(None if u0x is None else _f64(u0x)), _d(dr), _d(kf), _d(kl), ctypes.byref(lb),
                            _d(o.Theta), _d(o.xi), _d(o.psi), _d(o.Delta), _d(o.gamma), _d(o.delta), _d(o.alpha),
                            _d(o.beta), _i(o.xperm), _d(o.pix), _d(o.piy), ctypes.byref(on),
                            o.stats.ctypes.data_as(_lp), threads)
    if rc != 0:
        raise ValueError("or_iterate_v rejected the input")
    o.lb = lb.value
    return o, lb.value, int(on.value)


HALF_PRM = (2.0 / 3.0, 1.0, 1.0, 0.5)  # kz, ky, kx, phi_y of the half-Z scheme (Section 5)


def iterate_half(st: State, prm=HALF_PRM, dual_mode: int = 1, u0z=None, u0y=None, u0x=None) -> IterOut:
    """One iteration of the half-Z scheme in place on st.Chat / st.Dhat."""
    n = st.n
    T = num_tiles(n)
    mz, my = n - 2, n - 1
    o = IterOut(0.0, np.zeros(T), np.zeros(T * mz), np.zeros(T * mz), np.zeros(n * n), np.zeros(n * n * my),
                np.zeros(n * n * my), np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.int32), np.zeros(n * n),
                np.zeros(T), np.zeros(6, dtype=np.int64))
    lb = ctypes.c_double()
    rc = lib().or_iterate_half(n, _d(_f64(prm)), dual_mode, _d(st.bprime), _d(st.Chat), _d(st.Dhat),
                               _d(None if u0z is None else _f64(u0z)), _d(None if u0y is None else _f64(u0y)),
                               _d(None if u0x is None else _f64(u0x)), ctypes.byref(lb), _d(o.Theta), _d(o.xi),
                               _d(o.psi), _d(o.Delta), _d(o.gamma), _d(o.delta), _d(o.alpha), _d(o.beta),
                               _i(o.xperm), _d(o.pix), _d(o.piy), o.stats.ctypes.data_as(_lp))
    if rc != 0:
        raise ValueError("or_iterate_half rejected the input")
    o.lb = lb.value
    return o


def run_half(F, D, B=None, iters=10, prm=HALF_PRM, dual_mode=1, partial=None, warm=False):
    """Half-Z scheme run; returns (state, bounds incl. const, last IterOut)."""
    st = setup(F, D, B, partial)
    lbs, out = [], None
    for _ in range(iters):
        w = warm and out is not None
        out = iterate_half(st, prm, dual_mode, u0z=out.xi.copy() if w else None,
                           u0y=out.gamma.copy() if w else None, u0x=out.alpha.copy() if w else None)
        lbs.append(st.const + out.lb)
    return st, lbs, out


def sa_schedule(n, kf, kl, neglog_u, ub, t0=0.04, cool=0.99, period=100):
    """(K[d], thr[d]) of the Type 4 annealing schedule (Section 5)."""
    kf = _f64(kf).reshape(-1, n)
    kl = _f64(kl).reshape(-1, n)
    ng = _f64(neglog_u).reshape(-1)
    cnt = ng.shape[0]
    K, thr = np.zeros(cnt), np.zeros(cnt)
    lib().or_sa_schedule(n, cnt, float(ub), float(t0), float(cool), int(period), _d(kf), _d(kl), _d(ng), _d(K),
                         _d(thr))
    return K, thr


def sa_term(n, nu, K, thr, kf, kl):
    """Type 4 amounts per (i, p) of one draw, or None if the draw is rejected."""
    out = np.zeros(n * n)
    ok = lib().or_sa_term(n, float(nu), float(K), float(thr), _d(_f64(kf)), _d(_f64(kl)), _d(out))
    return out if ok else None


def redistribute_z_v(n, prm, Dhat, xi, psi, piy, pix, variant=0, sa=None, threads=1):
    out = _f64(Dhat).copy()
    lib().or_redistribute_z_v(n, _d(_f64(prm)), variant, _d(None if sa is None else _f64(sa)), _d(out),
                              _d(_f64(xi)), _d(_f64(psi)), _d(_f64(piy)), _d(_f64(pix)), threads)
    return out


def redistribute_z_form(n, prm, Dhat, xi, psi, piy, pix, form, variant=0, sa=None, threads=1):
    """The z move with the branch chosen by form: 0 as the iteration picks it
    (regrouped where phi are equal), 1 the general branch (Eq. 2.20 term by term)."""
    out = _f64(Dhat).copy()
    lib().or_redistribute_z_form(n, _d(_f64(prm)), variant, _d(None if sa is None else _f64(sa)), int(form), _d(out),
                                 _d(_f64(xi)), _d(_f64(psi)), _d(_f64(piy)), _d(_f64(pix)), threads)
    return out


def redistribute_half_form(n, prm, Dhat, Chat, xi, psi, piy, pix, form):
    """The half-Z scheme's move (z and y) with form 0 (regrouped member update)
    or 1 (the plain sum); returns (D^', C^')."""
    D, C = _f64(Dhat).copy(), _f64(Chat).copy()
    lib().or_redistribute_half_form(n, _d(_f64(prm)), int(form), _d(D), _d(C), _d(_f64(xi)), _d(_f64(psi)),
                                    _d(_f64(piy)), _d(_f64(pix)))
    return D, C


def phase2_z(n, Dhat, xi, psi, tol=1e-9, threads=1):
    """Returns a new D^ after the second-phase move of the two-phase Z solve."""
    out = _f64(Dhat).copy()
    lib().or_phase2_z(n, float(tol), _d(out), _d(_f64(xi)), _d(_f64(psi)), threads)
    return out


# index helpers used by tests
def tile_index(n, i, p, j, q):
    jj = j - (j > i)
    qq = q - (q > p)
    return ((i * n + p) * (n - 1) + jj) * (n - 1) + qq


def z_index(n, i, j, k, p, q, r):
    m = n - 2
    kk = k - (k > i) - (k > j)
    rr = r - (r > p) - (r > q)
    return tile_index(n, i, p, j, q) * m * m + kk * m + rr


# --------------------------------------------------------------------------
# learned warm start: features and FP64 reference MLP
# --------------------------------------------------------------------------
MLP_IN = 34


def _f(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def f32_trunc(x: float) -> float:
    return float(lib().or_f32_trunc(float(x)))


def bf16_round(x: float) -> float:
    return float(lib().or_bf16_round(float(x)))


def mlp_features(tile, prev_u=None, target_u=None):
    """Row features (m x 34, float32), scaled targets (m, float32) and the tile scale."""
    c = _f64(tile)
    m = c.shape[0]
    feat = np.zeros((m, MLP_IN), dtype=np.float32)
    tgt = np.zeros(m, dtype=np.float32)
    sc = ctypes.c_float()
    pu = None if prev_u is None else _f64(prev_u)
    tu = None if target_u is None else _f64(target_u)
    lib().or_mlp_features(m, _d(c), _d(pu), _d(tu), _f(feat), _f(tgt), ctypes.byref(sc))
    return feat, tgt, sc.value


def mlp_forward(X, W1, b1, W2, b2, w3, b3, bf16_acts=True):
    X = np.ascontiguousarray(X, dtype=np.float32)
    N, H = X.shape[0], W1.shape[1]
    out = np.zeros(N)
    h1 = np.zeros((N, H))
    h2 = np.zeros((N, H))
    args = [np.ascontiguousarray(a, dtype=np.float32) for a in (W1, b1, W2, b2, w3)]
    lib().or_mlp_forward(N, H, _f(X), *(_f(a) for a in args), float(b3), int(bf16_acts), _d(out), _d(h1), _d(h2))
    return out, h1, h2


def mlp_grads(X, W1, b1, W2, b2, w3, b3, t, bf16_acts=True):
    """Loss and FP64 gradients (gW1, gb1, gW2, gb2, gw3, gb3)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    N, H = X.shape[0], W1.shape[1]
    out, h1, h2 = mlp_forward(X, W1, b1, W2, b2, w3, b3, bf16_acts)
    g = [np.zeros((MLP_IN, H)), np.zeros(H), np.zeros((H, H)), np.zeros(H), np.zeros(H)]
    gb3 = ctypes.c_double()
    W2c = np.ascontiguousarray(W2, dtype=np.float32)
    w3c = np.ascontiguousarray(w3, dtype=np.float32)
    loss = lib().or_mlp_backward(N, H, _f(X), _f(W2c), _f(w3c), int(bf16_acts), _d(out), _d(h1), _d(h2),
                                 _d(_f64(t)), *(_d(a) for a in g), ctypes.byref(gb3))
    return loss, g[0], g[1], g[2], g[3], g[4], gb3.value


# --------------------------------------------------------------------------
# branch and bound: parent -> child multiplier warm start (Section 4)
# --------------------------------------------------------------------------
def child_state(st: State, f: int, l: int) -> State:
    """Child of `st` (residual indices) with facility f fixed at location l,
    keeping the parent's multiplier-adjusted costs."""
    n = st.n
    nc = n - 1
    bc = np.zeros(nc * nc)
    Cc = np.zeros(max(num_tiles(nc), 1))
    Dc = np.zeros(max(num_z(nc), 1)) if nc >= 3 else np.zeros(1)
    cst = ctypes.c_double()
    lib().or_child_state(n, f, l, _d(st.bprime), _d(st.Chat), _d(st.Dhat), float(st.const), _d(bc), _d(Cc), _d(Dc),
                         ctypes.byref(cst))
    return State(nc, cst.value, bc, Cc, Dc)


def lagrangian_objective(st: State, perm) -> float:
    s = np.ascontiguousarray(perm, dtype=np.int32)
    return float(lib().or_lagrangian_objective(st.n, _d(st.bprime), _d(st.Chat), _d(st.Dhat), float(st.const),
                                               _i(s)))
