"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/rlt2.h declares, and rejects invalid arguments before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1710_03732_gb300 import build as B
from paper_1710_03732_gb300 import rlt2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return rlt2.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rlt2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rlt2_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_expected_api():
    names = declared_functions()
    for must in ("rlt2_create", "rlt2_iterate", "rlt2_bound", "rlt2_duals", "rlt2_reduced_costs",
                 "rlt2_export_state", "rlt2_import_state", "rlt2_lap_batched", "rlt2_destroy", "rlt2_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_names_match_header():
    assert set(declared_functions()) == set(rlt2.EXPORTS)


def test_params_default(L):
    p = rlt2.rlt2_params()
    L.rlt2_params_default(ctypes.byref(p))
    assert (p.kz, p.ky, p.kx, p.phi_y, p.dual_mode, p.warm) == (1.0, 0.5, 1.0, 0.5, 1, 0)
    assert (p.stall_window, p.stall_tol, p.feas_tol) == (0, 0.0002, 1e-9)
    assert abs(sum(p.phi_z) - 1.0) < 1e-15


def _create(L, n, F, D, B=None, partial=None, prm=None):
    out = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    return L.rlt2_create(n, None if F is None else F.ctypes.data_as(dp), None if D is None else D.ctypes.data_as(dp),
                         None if B is None else B.ctypes.data_as(dp),
                         None if partial is None else partial.ctypes.data_as(ip),
                         None if prm is None else ctypes.byref(prm), None, ctypes.byref(out))


def test_create_rejects_bad_input(L):
    F = np.ones((5, 5))
    D = np.ones((5, 5))
    assert _create(L, 2, F, D) == rlt2.RLT2_EINVAL              # n < 3
    assert _create(L, 5, None, D) == rlt2.RLT2_EINVAL            # NULL F
    Fn = F.copy()
    Fn[1, 2] = np.nan
    assert _create(L, 5, Fn, D) == rlt2.RLT2_EINVAL              # non-finite
    Dn = D.copy()
    Dn[0, 0] = np.inf
    assert _create(L, 5, F, Dn) == rlt2.RLT2_EINVAL
    bad = np.array([1, 1, -1, -1, -1], dtype=np.int32)           # not injective
    assert _create(L, 5, F, D, partial=bad) == rlt2.RLT2_EINVAL
    bad = np.array([7, -1, -1, -1, -1], dtype=np.int32)          # out of range
    assert _create(L, 5, F, D, partial=bad) == rlt2.RLT2_EINVAL
    bad = np.array([0, 1, 2, -1, -1], dtype=np.int32)            # residual size 2 < 3
    assert _create(L, 5, F, D, partial=bad) == rlt2.RLT2_EINVAL
    big = np.ones((40, 40))
    assert _create(L, 40, big, big) == rlt2.RLT2_EINVAL          # residual 40 > 32


@pytest.mark.parametrize("field,value", [("kz", 1.5), ("ky", -0.1), ("phi_y", 0.8), ("dual_mode", 3),
                                         ("warm", 7), ("phi_sum", 0.9), ("stall_window", 64),
                                         ("stall_window", -1)])
def test_create_rejects_bad_params(L, field, value):
    p = rlt2.rlt2_params()
    L.rlt2_params_default(ctypes.byref(p))
    if field == "phi_sum":
        p.phi_z[0] = 0.1
    else:
        setattr(p, field, value)
    F = np.ones((5, 5))
    assert _create(L, 5, F, F, prm=p) == rlt2.RLT2_EINVAL


def test_lap_batched_rejects_bad_sizes(L):
    assert L.rlt2_lap_batched(4, 33, None, None, None, None, None, None, None, 1, None) == rlt2.RLT2_EINVAL
    assert L.rlt2_lap_batched(4, 0, None, None, None, None, None, None, None, 1, None) == rlt2.RLT2_EINVAL
    assert L.rlt2_lap_batched(4, 5, None, None, None, None, None, None, None, 1, None) == rlt2.RLT2_EINVAL
    assert L.rlt2_lap_batched(0, 5, None, None, None, None, None, None, None, 1, None) == rlt2.RLT2_OK


def test_strerror(L):
    assert L.rlt2_strerror(rlt2.RLT2_EINVAL) == b"invalid argument"
    assert L.rlt2_destroy(None) == rlt2.RLT2_OK


def test_bound_nodes_rejects_bad_input(L):
    n = 6
    F = np.ones((n, n))
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lb = np.zeros(2)

    def call(parts, iters=5):
        parts = np.ascontiguousarray(parts, dtype=np.int32)
        return L.rlt2_bound_nodes(n, F.ctypes.data_as(dp), F.ctypes.data_as(dp), None, parts.shape[0],
                                  parts.ctypes.data_as(ip), None, None, iters, 0, lb.ctypes.data_as(dp), None, None,
                                  None, None)
    ok = -np.ones((2, n))
    assert call(ok, iters=0) == rlt2.RLT2_EINVAL
    bad = ok.copy()
    bad[1, :2] = [3, 3]                          # not injective
    assert call(bad) == rlt2.RLT2_EINVAL
    bad = ok.copy()
    bad[0, :4] = [0, 1, 2, 3]                    # residual size 2
    assert call(bad) == rlt2.RLT2_EINVAL
