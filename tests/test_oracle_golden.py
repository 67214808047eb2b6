"""The oracle reproduces its stored trajectories (written by tests/golden/make_golden.py)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1710_03732_gb300 import instances as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PRM = O.params_array(kz=1.0, ky=0.5, kx=1.0, phi_y=0.5, phi_z=(0.2,) * 5)


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return np.array([float(x) for x in f if not x.startswith("#")])


@pytest.mark.parametrize("name,cfg,iters,mode", [
    ("lb_n8_grid2x4_canonical.txt", 1, 50, 1),
    ("lb_n8_grid2x4_raw.txt", 1, 50, 0),
    ("lb_n12_grid3x4_canonical.txt", 2, 200, 1),
    ("lb_n12_grid3x4_raw.txt", 2, 200, 0),
])
def test_oracle_matches_golden(name, cfg, iters, mode):
    inst = I.config(cfg)
    ref = load(name)
    assert len(ref) == iters
    _, lbs, _ = O.run(inst.F, inst.D, inst.B, iters=iters, prm=PRM, dual_mode=mode, threads=O.max_threads() or 1)
    assert np.array_equal(np.array(lbs), ref)


def test_golden_trajectories_monotone_and_valid():
    inst = I.config(1)
    opt, _ = O.qap_brute(inst.F, inst.D, inst.B)
    for name in ("lb_n8_grid2x4_canonical.txt", "lb_n8_grid2x4_raw.txt"):
        lb = load(name)
        assert np.all(np.diff(lb) >= -1e-9 * np.abs(lb[:-1]))
        assert lb.max() <= opt + 1e-9
