"""Thin ctypes binding of the C ABI in include/rlt2.h (argument marshalling only).

Every function below has the name of the C entry point it calls and does no
arithmetic of the method: all of it runs in the CUDA library.  Device buffers
are torch CUDA tensors (PyTorch supplies memory and streams); host buffers are
numpy arrays.  If the library is missing the import of a function fails loudly:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librlt2.so")

RLT2_OK, RLT2_EINVAL, RLT2_ENOMEM, RLT2_ECUDA, RLT2_ETIMEOUT, RLT2_EADMIT = range(6)


class rlt2_params(ctypes.Structure):
    _fields_ = [("kz", ctypes.c_double), ("ky", ctypes.c_double), ("kx", ctypes.c_double),
                ("phi_y", ctypes.c_double), ("phi_z", ctypes.c_double * 5), ("dual_mode", ctypes.c_int),
                ("warm", ctypes.c_int), ("min_gap", ctypes.c_double), ("ub", ctypes.c_double),
                ("feas_tol", ctypes.c_double), ("stall_window", ctypes.c_int), ("stall_tol", ctypes.c_double),
                ("variant", ctypes.c_int), ("two_phase", ctypes.c_int), ("phase2_tol", ctypes.c_double),
                ("sa_t0", ctypes.c_double), ("sa_cool", ctypes.c_double), ("sa_period", ctypes.c_int),
                ("half_z", ctypes.c_int), ("pipeline", ctypes.c_int)]


class rlt2_bnb_options(ctypes.Structure):
    _fields_ = [("order_rule", ctypes.c_int), ("iters_root", ctypes.c_int), ("iters_node", ctypes.c_int),
                ("warm_depth", ctypes.c_int), ("max_states", ctypes.c_int), ("max_nodes", ctypes.c_longlong),
                ("time_limit_s", ctypes.c_double), ("ub0", ctypes.c_double), ("abs_tol", ctypes.c_double),
                ("max_state_bytes", ctypes.c_double), ("batch_children", ctypes.c_int)]


class Rlt2Error(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p

EXPORTS = ["rlt2_params_default", "rlt2_create", "rlt2_iterate", "rlt2_iterate_async", "rlt2_bound", "rlt2_duals",
           "rlt2_reduced_costs", "rlt2_export_state", "rlt2_import_state", "rlt2_stats", "rlt2_sizes",
           "rlt2_set_timing", "rlt2_kernel_times", "rlt2_destroy", "rlt2_lap_batched", "rlt2_bound_nodes",
           "rlt2_iterate_noalloc", "rlt2_mlp_create", "rlt2_mlp_destroy", "rlt2_mlp_get_weights",
           "rlt2_mlp_set_weights", "rlt2_mlp_add_samples", "rlt2_mlp_samples", "rlt2_mlp_clear_samples",
           "rlt2_mlp_grad", "rlt2_mlp_fit", "rlt2_mlp_set_gate", "rlt2_mlp_predict", "rlt2_set_mlp",
           "rlt2_export_xstate", "rlt2_import_xstate", "rlt2_set_sa", "rlt2_create_child", "rlt2_bnb_options_default",
           "rlt2_bnb_solve", "rlt2_mlp_check_wait_timeout", "rlt2_mlp_check_gemm_wait_timeout",
           "rlt2_pipeline_check_wait_timeout",
           "rlt2_debug_bounds_violations", "rlt2_probe_rates", "rlt2_fp64_add_emulated", "rlt2_node_tuning", "rlt2_iterate_many",
           "rlt2_strerror",
           "rlt2_last_error"]


def lib():
    """Load librlt2.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    L.rlt2_params_default.argtypes = [ctypes.POINTER(rlt2_params)]
    L.rlt2_params_default.restype = None
    L.rlt2_create.argtypes = [ctypes.c_int, _dp, _dp, _dp, _ip, ctypes.POINTER(rlt2_params), _vp,
                              ctypes.POINTER(_vp)]
    L.rlt2_iterate.argtypes = [_vp, ctypes.c_int, _dp, _ip]
    L.rlt2_iterate_async.argtypes = [_vp, ctypes.c_int]
    L.rlt2_bound.argtypes = [_vp, _dp, _dp, _dp, _ip, _ip, _ip]
    L.rlt2_duals.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int]
    L.rlt2_reduced_costs.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int]
    L.rlt2_export_state.argtypes = [_vp, _vp, _vp, ctypes.c_int]
    L.rlt2_import_state.argtypes = [_vp, _vp, _vp, ctypes.c_int]
    L.rlt2_export_xstate.argtypes = [_vp, _dp, _dp]
    L.rlt2_import_xstate.argtypes = [_vp, _dp, ctypes.c_double]
    L.rlt2_set_sa.argtypes = [_vp, ctypes.c_int, _dp, _dp, _dp]
    L.rlt2_create_child.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(rlt2_params), ctypes.POINTER(_vp)]
    L.rlt2_bnb_options_default.argtypes = [ctypes.POINTER(rlt2_bnb_options)]
    L.rlt2_bnb_options_default.restype = None
    L.rlt2_bnb_solve.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.POINTER(rlt2_params),
                                 ctypes.POINTER(rlt2_bnb_options), _dp, _ip, _dp, ctypes.POINTER(ctypes.c_longlong), _vp]
    L.rlt2_stats.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong)]
    L.rlt2_sizes.argtypes = [_vp, _ip, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), _dp]
    L.rlt2_set_timing.argtypes = [_vp, ctypes.c_int]
    L.rlt2_kernel_times.argtypes = [_vp, _dp, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
    L.rlt2_destroy.argtypes = [_vp]
    L.rlt2_lap_batched.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]
    L.rlt2_bound_nodes.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, _ip, ctypes.POINTER(rlt2_params), _vp,
                                   ctypes.c_int, ctypes.c_size_t, _dp, _dp, _ip, ctypes.POINTER(ctypes.c_longlong), _vp]
    L.rlt2_iterate_noalloc.argtypes = [ctypes.c_int, _vp, _vp, _vp, ctypes.POINTER(rlt2_params), ctypes.c_int, _vp,
                                       _vp]
    _fp = ctypes.POINTER(ctypes.c_float)
    L.rlt2_mlp_create.argtypes = [ctypes.c_int, ctypes.c_ulonglong, _vp, ctypes.POINTER(_vp)]
    L.rlt2_mlp_destroy.argtypes = [_vp]
    L.rlt2_mlp_get_weights.argtypes = [_vp, _fp, _fp, _fp, _fp, _fp, _fp]
    L.rlt2_mlp_set_weights.argtypes = [_vp, _fp, _fp, _fp, _fp, _fp, _fp]
    L.rlt2_mlp_add_samples.argtypes = [_vp, ctypes.c_longlong, ctypes.c_int, _vp, _vp, _vp]
    L.rlt2_mlp_samples.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong), _vp, _fp]
    L.rlt2_mlp_clear_samples.argtypes = [_vp]
    L.rlt2_mlp_grad.argtypes = [_vp, ctypes.c_longlong, _dp, _fp, _fp, _fp, _fp, _fp, _fp]
    L.rlt2_mlp_fit.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_ulonglong,
                               _dp]
    L.rlt2_mlp_predict.argtypes = [_vp, ctypes.c_longlong, ctypes.c_int, _vp, _vp, _vp]
    L.rlt2_mlp_set_gate.argtypes = [_vp, ctypes.c_double]
    L.rlt2_mlp_check_wait_timeout.argtypes = [_vp]
    L.rlt2_mlp_check_gemm_wait_timeout.argtypes = [_vp]
    L.rlt2_pipeline_check_wait_timeout.argtypes = [_vp]
    L.rlt2_probe_rates.argtypes = [_dp, _dp, _vp]
    L.rlt2_node_tuning.argtypes = [ctypes.c_int, _ip, _ip, _ip, _dp, _ip]
    L.rlt2_iterate_many.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, _ip]
    L.rlt2_fp64_add_emulated.argtypes = [ctypes.c_longlong, _vp, _vp, _vp, _vp, _vp]
    L.rlt2_set_mlp.argtypes = [_vp, _vp]
    L.rlt2_strerror.argtypes = [ctypes.c_int]
    L.rlt2_strerror.restype = ctypes.c_char_p
    L.rlt2_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("rlt2_params_default", "rlt2_bnb_options_default", "rlt2_strerror", "rlt2_last_error",
                        "rlt2_debug_bounds_violations"):
            getattr(L, name).restype = ctypes.c_int
    L.rlt2_debug_bounds_violations.argtypes = []
    L.rlt2_debug_bounds_violations.restype = ctypes.c_longlong
    _lib = L
    return L


def _check(status: int, where: str):
    if status != RLT2_OK:
        L = lib()
        raise Rlt2Error(status, where, f"{L.rlt2_strerror(status).decode()}: {L.rlt2_last_error().decode()}")


def _host_d(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _ptr(buf) -> Optional[int]:
    """Pointer of a torch tensor (device) or numpy array (host), None for None."""
    if buf is None:
        return None
    if isinstance(buf, np.ndarray):
        assert buf.flags.c_contiguous
        return buf.ctypes.data
    assert buf.is_contiguous()
    return buf.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is not None:
        return int(stream)
    import torch
    return int(torch.cuda.current_stream().cuda_stream) or None


def params(kz=1.0, ky=0.5, kx=1.0, phi_y=0.5, phi_z=(0.2,) * 5, dual_mode=1, warm=0, min_gap=0.0, ub=0.0,
           feas_tol=1e-9, stall_window=0, stall_tol=0.0002, variant=0, two_phase=0, phase2_tol=1e-9, sa_t0=0.04,
           sa_cool=0.99, sa_period=100, half_z=0, pipeline=0) -> rlt2_params:
    """Parameters (dual_mode 0 = raw FP64 Hungarian duals, 1 = canonical duals in exact
    fixed point, 2 = canonical duals in FP64; variant 0 = S, 1 = F; two_phase;
    annealing schedule of the Type 4 rule; half_z = the half-Z-LAP scheme, see
    half_z_params; pipeline = the z move and the next Z-LAPs in one launch)."""
    p = rlt2_params()
    lib().rlt2_params_default(ctypes.byref(p))
    p.kz, p.ky, p.kx, p.phi_y = kz, ky, kx, phi_y
    for i, x in enumerate(phi_z):
        p.phi_z[i] = x
    p.dual_mode, p.warm, p.min_gap, p.ub, p.feas_tol = dual_mode, warm, min_gap, ub, feas_tol
    p.stall_window, p.stall_tol = stall_window, stall_tol
    p.variant, p.two_phase, p.phase2_tol = int(variant), int(two_phase), phase2_tol
    p.sa_t0, p.sa_cool, p.sa_period = sa_t0, sa_cool, int(sa_period)
    p.half_z = int(half_z)
    p.pipeline = int(pipeline)
    return p


def half_z_params(**kw) -> rlt2_params:
    """The half-Z-LAP scheme with the paper's values (Section 5): kz = 2/3 for the
    upper members, ky = kx = 1, phi_y = 1/2."""
    d = dict(kz=2.0 / 3.0, ky=1.0, kx=1.0, phi_y=0.5, half_z=1)
    d.update(kw)
    return params(**d)


# ------------------------------------------------------------ C entry points --
def rlt2_create(F: np.ndarray, D: np.ndarray, B: Optional[np.ndarray] = None, partial: Optional[np.ndarray] = None,
                prm: Optional[rlt2_params] = None, stream=None) -> int:
    F = np.ascontiguousarray(F, dtype=np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    B = None if B is None else np.ascontiguousarray(B, dtype=np.float64)
    part = None if partial is None else np.ascontiguousarray(partial, dtype=np.int32)
    out = _vp()
    st = lib().rlt2_create(F.shape[0], _host_d(F), _host_d(D), _host_d(B),
                           None if part is None else part.ctypes.data_as(_ip),
                           None if prm is None else ctypes.byref(prm), _stream(stream), ctypes.byref(out))
    _check(st, "rlt2_create")
    return out.value


def rlt2_iterate(ctx: int, iters: int):
    """Returns (bounds per iteration as numpy, iterations performed)."""
    hist = np.empty(iters, dtype=np.float64)
    done = ctypes.c_int()
    _check(lib().rlt2_iterate(ctx, iters, _host_d(hist), ctypes.byref(done)), "rlt2_iterate")
    return hist, done.value


def rlt2_iterate_async(ctx: int, iters: int):
    _check(lib().rlt2_iterate_async(ctx, iters), "rlt2_iterate_async")


def rlt2_bound(ctx: int, n_full: int):
    lb, best, ub = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    perm = np.zeros(n_full, dtype=np.int32)
    ub_perm = np.zeros(n_full, dtype=np.int32)
    it = ctypes.c_int()
    _check(lib().rlt2_bound(ctx, ctypes.byref(lb), ctypes.byref(best), ctypes.byref(ub), perm.ctypes.data_as(_ip),
                            ub_perm.ctypes.data_as(_ip), ctypes.byref(it)), "rlt2_bound")
    return lb.value, best.value, ub.value, perm, ub_perm, it.value


def rlt2_duals(ctx: int, alpha=None, beta=None, gamma=None, delta=None, xi=None, psi=None, on_device=0):
    _check(lib().rlt2_duals(ctx, _ptr(alpha), _ptr(beta), _ptr(gamma), _ptr(delta), _ptr(xi), _ptr(psi), on_device),
           "rlt2_duals")


def rlt2_reduced_costs(ctx: int, pi_x=None, pi_y=None, pi_z=None, on_device=0):
    _check(lib().rlt2_reduced_costs(ctx, _ptr(pi_x), _ptr(pi_y), _ptr(pi_z), on_device), "rlt2_reduced_costs")


def rlt2_export_state(ctx: int, Dhat=None, Chat=None, on_device=0):
    _check(lib().rlt2_export_state(ctx, _ptr(Dhat), _ptr(Chat), on_device), "rlt2_export_state")


def rlt2_import_state(ctx: int, Dhat=None, Chat=None, on_device=0):
    _check(lib().rlt2_import_state(ctx, _ptr(Dhat), _ptr(Chat), on_device), "rlt2_import_state")


def rlt2_stats(ctx: int) -> np.ndarray:
    out = (ctypes.c_longlong * 8)()
    _check(lib().rlt2_stats(ctx, out), "rlt2_stats")
    return np.array(list(out), dtype=np.int64)


def rlt2_sizes(ctx: int):
    nr, T, E, cst = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
    _check(lib().rlt2_sizes(ctx, ctypes.byref(nr), ctypes.byref(T), ctypes.byref(E), ctypes.byref(cst)), "rlt2_sizes")
    return nr.value, T.value, E.value, cst.value


def rlt2_set_timing(ctx: int, on: bool):
    _check(lib().rlt2_set_timing(ctx, int(bool(on))), "rlt2_set_timing")


KERNEL_KINDS = ["move_y", "move_z", "lap_z", "lap_y", "lap_x", "finalize", "phase2_move", "lap_z2"]


def rlt2_kernel_times(ctx: int):
    k = len(KERNEL_KINDS)
    ms = (ctypes.c_double * k)()
    cnt = (ctypes.c_longlong * k)()
    _check(lib().rlt2_kernel_times(ctx, ms, cnt, k), "rlt2_kernel_times")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}


def rlt2_export_xstate(ctx: int, n: int):
    bx = np.empty(n * n)
    base = ctypes.c_double()
    _check(lib().rlt2_export_xstate(ctx, _host_d(bx), ctypes.byref(base)), "rlt2_export_xstate")
    return bx, base.value


def rlt2_import_xstate(ctx: int, bx, lb_base: float):
    bx = np.ascontiguousarray(bx, dtype=np.float64)
    _check(lib().rlt2_import_xstate(ctx, _host_d(bx), float(lb_base)), "rlt2_import_xstate")


def rlt2_set_sa(ctx: int, kappa_fac, kappa_loc, neglog_u):
    kf = np.ascontiguousarray(kappa_fac, dtype=np.float64).reshape(-1)
    kl = np.ascontiguousarray(kappa_loc, dtype=np.float64).reshape(-1)
    ng = np.ascontiguousarray(neglog_u, dtype=np.float64).reshape(-1)
    count = int(ng.shape[0])
    _check(lib().rlt2_set_sa(ctx, count, _host_d(kf) if count else None, _host_d(kl) if count else None,
                             _host_d(ng) if count else None), "rlt2_set_sa")


def rlt2_create_child(ctx: int, facility: int, location: int, prm: Optional[rlt2_params] = None) -> int:
    out = _vp()
    _check(lib().rlt2_create_child(ctx, int(facility), int(location), None if prm is None else ctypes.byref(prm),
                                   ctypes.byref(out)), "rlt2_create_child")
    return out.value


def bnb_options(**kw) -> rlt2_bnb_options:
    o = rlt2_bnb_options()
    lib().rlt2_bnb_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def rlt2_bnb_solve(F, D, B=None, prm: Optional[rlt2_params] = None, opts: Optional[rlt2_bnb_options] = None,
                   stream=None):
    """Branch and bound to optimality; returns (best value, permutation, root bound,
    stats {bounded, branched, enumerated, iterations, max_depth, proven, warm, cold})."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    B = None if B is None else np.ascontiguousarray(B, dtype=np.float64)
    n = F.shape[0]
    best, rlb = ctypes.c_double(), ctypes.c_double()
    perm = np.zeros(n, dtype=np.int32)
    st = (ctypes.c_longlong * 8)()
    _check(lib().rlt2_bnb_solve(n, _host_d(F), _host_d(D), _host_d(B), None if prm is None else ctypes.byref(prm),
                                None if opts is None else ctypes.byref(opts), ctypes.byref(best),
                                perm.ctypes.data_as(_ip), ctypes.byref(rlb), st, _stream(stream)), "rlt2_bnb_solve")
    keys = ["bounded", "branched", "enumerated", "iterations", "max_depth", "proven", "warm", "cold"]
    return best.value, perm, rlb.value, dict(zip(keys, list(st)))


def rlt2_debug_bounds_violations() -> int:
    """Indices the bounds-checked library caught out of range (-1: normal build)."""
    return int(lib().rlt2_debug_bounds_violations())


def rlt2_pipeline_check_wait_timeout(ctx: int) -> int:
    """Runs the pipelined launch's failure-detection check on ctx; returns the
    status (RLT2_ETIMEOUT is the expected outcome) without raising for it."""
    st = lib().rlt2_pipeline_check_wait_timeout(ctx)
    if st not in (RLT2_OK, RLT2_ETIMEOUT):
        _check(st, "rlt2_pipeline_check_wait_timeout")
    return st


def rlt2_probe_rates(stream=None) -> dict:
    """Measured lane-operation rates of the current device (G ops/s) and its
    rated SM clock (GHz)."""
    r = np.zeros(5)
    clk = ctypes.c_double()
    _check(lib().rlt2_probe_rates(_host_d(r), ctypes.byref(clk), _stream(stream)), "rlt2_probe_rates")
    return {"dadd": r[0], "dfma": r[1], "iadd64": r[2], "iadd32": r[3], "emu_add": r[4], "sm_clock_ghz": clk.value}


def rlt2_fp64_add_emulated(a, b, total, diff, stream=None):
    """a + b and a - b by the integer-pipe binary64 addition (CUDA float64 tensors)."""
    _check(lib().rlt2_fp64_add_emulated(int(a.numel()), _ptr(a), _ptr(b), _ptr(total), _ptr(diff), _stream(stream)),
           "rlt2_fp64_add_emulated")


def rlt2_iterate_many(ctxs, iters: int) -> np.ndarray:
    """Iterates several contexts (Context objects or handles) in lockstep
    batched launches; returns the iterations each ran."""
    handles = [c.ctx if isinstance(c, Context) else c for c in ctxs]
    arr = (_vp * len(handles))(*handles)
    done = np.zeros(len(handles), dtype=np.int32)
    _check(lib().rlt2_iterate_many(arr, len(handles), iters, done.ctypes.data_as(_ip)), "rlt2_iterate_many")
    return done


def rlt2_node_tuning() -> list:
    """The batched nodes' per-size Z-stage launch shapes tuned so far:
    [{"m", "lanes_per_lap", "warps_per_block", "ms"}, ...] sorted by size."""
    cap = 64
    m, g, w = (np.zeros(cap, dtype=np.int32) for _ in range(3))
    ms = np.zeros(cap)
    cnt = ctypes.c_int()
    _check(lib().rlt2_node_tuning(cap, m.ctypes.data_as(_ip), g.ctypes.data_as(_ip), w.ctypes.data_as(_ip),
                                  _host_d(ms), ctypes.byref(cnt)), "rlt2_node_tuning")
    k = min(cnt.value, cap)
    return [{"m": int(m[i]), "lanes_per_lap": int(g[i]), "warps_per_block": int(w[i]), "ms": float(ms[i])}
            for i in range(k)]


def rlt2_destroy(ctx: int):
    _check(lib().rlt2_destroy(ctx), "rlt2_destroy")


def rlt2_lap_batched(cost, value, u0=None, u=None, v=None, row_to_col=None, n_aug=None, dual_mode=1, stream=None):
    """cost: CUDA tensor (batch, m, m) float64; outputs are CUDA tensors of matching batch."""
    batch, m = int(cost.shape[0]), int(cost.shape[1])
    _check(lib().rlt2_lap_batched(batch, m, _ptr(cost), _ptr(u0), _ptr(value), _ptr(u), _ptr(v), _ptr(row_to_col),
                                  _ptr(n_aug), dual_mode, _stream(stream)), "rlt2_lap_batched")


def rlt2_bound_nodes(F, D, partials, iters: int, B=None, prm: Optional[rlt2_params] = None, mem_budget: int = 0,
                     stream=None, mlp=None):
    """Bound every node (row of `partials`); returns (best bounds, bound history
    [n_nodes, iters], iterations per node, stats {waves, z_aug, z_relax, group, wpb})."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    B = None if B is None else np.ascontiguousarray(B, dtype=np.float64)
    part = np.ascontiguousarray(partials, dtype=np.int32)
    nn, n = part.shape
    lb = np.empty(nn)
    hist = np.empty((nn, iters))
    its = np.zeros(nn, dtype=np.int32)
    st = (ctypes.c_longlong * 5)()
    _check(lib().rlt2_bound_nodes(n, _host_d(F), _host_d(D), _host_d(B), nn, part.ctypes.data_as(_ip),
                                  None if prm is None else ctypes.byref(prm), None if mlp is None else mlp.ptr, iters,
                                  mem_budget, _host_d(lb),
                                  _host_d(hist), its.ctypes.data_as(_ip), st, _stream(stream)), "rlt2_bound_nodes")
    stats = dict(zip(["waves", "z_aug", "z_relax", "group", "wpb"], list(st)))
    return lb, hist, its, stats


def rlt2_iterate_noalloc(F, D, lb_hist, B=None, prm: Optional[rlt2_params] = None, stream=None):
    """Dual ascent with no device allocation (n <= 10).  F, D, B, lb_hist: CUDA
    float64 tensors; the number of iterations is len(lb_hist).  Asynchronous."""
    n = int(F.shape[0])
    _check(lib().rlt2_iterate_noalloc(n, _ptr(F), _ptr(D), _ptr(B), None if prm is None else ctypes.byref(prm),
                                      int(lb_hist.shape[0]), _ptr(lb_hist), _stream(stream)), "rlt2_iterate_noalloc")


def _fptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Mlp:
    """Owns one rlt2_mlp (learned warm start network)."""

    IN = 34

    def __init__(self, hidden=256, seed=1, stream=None):
        self.H = hidden
        out = _vp()
        _check(lib().rlt2_mlp_create(hidden, seed, _stream(stream), ctypes.byref(out)), "rlt2_mlp_create")
        self.ptr = out.value

    def get_weights(self):
        H = self.H
        W1, b1 = np.zeros((self.IN, H), np.float32), np.zeros(H, np.float32)
        W2, b2 = np.zeros((H, H), np.float32), np.zeros(H, np.float32)
        w3, b3 = np.zeros(H, np.float32), np.zeros(1, np.float32)
        _check(lib().rlt2_mlp_get_weights(self.ptr, _fptr(W1), _fptr(b1), _fptr(W2), _fptr(b2), _fptr(w3), _fptr(b3)),
               "rlt2_mlp_get_weights")
        return W1, b1, W2, b2, w3, float(b3[0])

    def set_weights(self, W1, b1, W2, b2, w3, b3):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (W1, b1, W2, b2, w3)]
        b3a = np.array([b3], dtype=np.float32)
        _check(lib().rlt2_mlp_set_weights(self.ptr, *(_fptr(a) for a in arrs), _fptr(b3a)), "rlt2_mlp_set_weights")

    def add_samples(self, tiles, target_u, prev_u=None):
        """tiles: CUDA float64 (ntiles, m, m); target_u / prev_u: CUDA float64 (ntiles, m)."""
        nt, m = int(tiles.shape[0]), int(tiles.shape[1])
        _check(lib().rlt2_mlp_add_samples(self.ptr, nt, m, _ptr(tiles), _ptr(prev_u), _ptr(target_u)),
               "rlt2_mlp_add_samples")

    def samples(self):
        rows = ctypes.c_longlong()
        _check(lib().rlt2_mlp_samples(self.ptr, ctypes.byref(rows), None, None), "rlt2_mlp_samples")
        X = np.zeros((rows.value, 64), dtype=np.uint16)
        T = np.zeros(rows.value, dtype=np.float32)
        _check(lib().rlt2_mlp_samples(self.ptr, ctypes.byref(rows), X.ctypes.data, _fptr(T)), "rlt2_mlp_samples")
        Xf = (X.astype(np.uint32) << 16).view(np.float32)
        return Xf[:, :self.IN].copy(), T

    def clear_samples(self):
        _check(lib().rlt2_mlp_clear_samples(self.ptr), "rlt2_mlp_clear_samples")

    def grad(self, rows):
        H = self.H
        g = [np.zeros((self.IN, H), np.float32), np.zeros(H, np.float32), np.zeros((H, H), np.float32),
             np.zeros(H, np.float32), np.zeros(H, np.float32), np.zeros(1, np.float32)]
        loss = ctypes.c_double()
        _check(lib().rlt2_mlp_grad(self.ptr, rows, ctypes.byref(loss), *(_fptr(a) for a in g)), "rlt2_mlp_grad")
        return loss.value, g[0], g[1], g[2], g[3], g[4], float(g[5][0])

    def fit(self, steps, batch_rows=8192, lr=1e-3, weight_decay=1e-4, seed=0):
        hist = np.zeros(steps)
        _check(lib().rlt2_mlp_fit(self.ptr, steps, batch_rows, lr, weight_decay, seed, _host_d(hist)), "rlt2_mlp_fit")
        return hist

    def set_gate(self, gate: float):
        _check(lib().rlt2_mlp_set_gate(self.ptr, float(gate)), "rlt2_mlp_set_gate")

    def predict(self, tiles, u0, prev_u=None):
        nt, m = int(tiles.shape[0]), int(tiles.shape[1])
        _check(lib().rlt2_mlp_predict(self.ptr, nt, m, _ptr(tiles), _ptr(prev_u), _ptr(u0)), "rlt2_mlp_predict")

    def save(self, path):
        W1, b1, W2, b2, w3, b3 = self.get_weights()
        np.savez(path, W1=W1, b1=b1, W2=W2, b2=b2, w3=w3, b3=np.float32(b3))

    def load(self, path):
        d = np.load(path)
        self.set_weights(d["W1"], d["b1"], d["W2"], d["b2"], d["w3"], float(d["b3"]))

    def close(self):
        if self.ptr:
            _check(lib().rlt2_mlp_destroy(self.ptr), "rlt2_mlp_destroy")
            self.ptr = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rlt2_set_mlp(ctx: int, mlp: Optional["Mlp"]):
    _check(lib().rlt2_set_mlp(ctx, mlp.ptr if mlp is not None else None), "rlt2_set_mlp")


# ------------------------------------------------------------ convenience ----
class Context:
    """Owns one rlt2_ctx: ``Context(F, D).iterate(300)``."""

    def __init__(self, F, D, B=None, partial=None, prm: Optional[rlt2_params] = None, stream=None):
        self.n_full = int(np.asarray(F).shape[0])
        self.ctx = rlt2_create(F, D, B, partial, prm, stream)
        self.n, self.T, self.E, self.const = rlt2_sizes(self.ctx)

    def iterate(self, iters: int):
        return rlt2_iterate(self.ctx, iters)

    def iterate_async(self, iters: int):
        rlt2_iterate_async(self.ctx, iters)

    def bound(self):
        return rlt2_bound(self.ctx, self.n_full)

    def duals(self):
        n, T, m = self.n, self.T, self.n - 2
        out = dict(alpha=np.empty(n), beta=np.empty(n), gamma=np.empty(n * n * (n - 1)),
                   delta=np.empty(n * n * (n - 1)), xi=np.empty(T * m), psi=np.empty(T * m))
        rlt2_duals(self.ctx, **out)
        return out

    def reduced_costs(self, with_z=True):
        out = dict(pi_x=np.empty(self.n * self.n), pi_y=np.empty(self.T),
                   pi_z=np.empty(self.E) if with_z else None)
        rlt2_reduced_costs(self.ctx, **out)
        return out

    def export_state(self):
        D, C = np.empty(self.E), np.empty(self.T)
        rlt2_export_state(self.ctx, D, C)
        return D, C

    def import_state(self, Dhat, Chat):
        rlt2_import_state(self.ctx, np.ascontiguousarray(Dhat, dtype=np.float64),
                          np.ascontiguousarray(Chat, dtype=np.float64))

    def child(self, facility: int, location: int, prm: Optional[rlt2_params] = None) -> "Context":
        """Branch-and-bound child starting from this context's multipliers."""
        c = Context.__new__(Context)
        c.n_full = self.n_full
        c.ctx = rlt2_create_child(self.ctx, facility, location, prm)
        c.n, c.T, c.E, c.const = rlt2_sizes(c.ctx)
        return c

    def export_xstate(self):
        """(incremental x costs, bound base) of an F-variant checkpoint."""
        return rlt2_export_xstate(self.ctx, self.n)

    def import_xstate(self, bx, lb_base):
        rlt2_import_xstate(self.ctx, bx, lb_base)

    def set_sa(self, kappa_fac, kappa_loc, neglog_u):
        """Type 4 draws (count x n, count x n, count); count = 0 switches the rule off."""
        rlt2_set_sa(self.ctx, kappa_fac, kappa_loc, neglog_u)

    def stats(self):
        return rlt2_stats(self.ctx)

    def set_mlp(self, mlp):
        self._mlp = mlp  # keep the network alive while attached
        rlt2_set_mlp(self.ctx, mlp)

    def set_timing(self, on=True):
        rlt2_set_timing(self.ctx, on)

    def kernel_times(self):
        return rlt2_kernel_times(self.ctx)

    def close(self):
        if self.ctx:
            rlt2_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
