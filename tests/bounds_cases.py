"""Cases run against the bounds-checked library (-DRLT2_BOUNDS_CHECK) in a child
process of test_gpu_bounds.py: every entry point on small problems, results
compared with the oracle, then the number of out-of-range kernel indices the
library counted.  Prints one JSON line; exits non-zero on a mismatch.

    python tests/bounds_cases.py <path of librlt2_check.so>
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1710_03732_gb300 import instances as I  # noqa: E402
from paper_1710_03732_gb300 import rlt2 as R  # noqa: E402


def raw_run(inst, iters, partial=None, **kw):
    prm = R.params(dual_mode=0, feas_tol=0.0, **kw)
    with R.Context(inst.F, inst.D, inst.B, partial=partial, prm=prm) as ctx:
        lbs, done = ctx.iterate(iters)
        D, _ = ctx.export_state()
    return lbs, done, D


def oracle_raw(inst, iters, partial=None, threads=1):
    st = O.setup(inst.F, inst.D, inst.B, partial)
    ref, before = [], None
    for it in range(iters):
        if it == iters - 1:
            before = st.Dhat.copy()
        out = O.iterate(st, O.params_array(), 0, threads=threads)
        ref.append(st.const + out.lb)
    return np.array(ref), before


def main():
    R.LIB_PATH = sys.argv[1]
    import torch
    checks = []

    def check(name, ok):
        checks.append((name, bool(ok)))

    # the S1 ascent, raw duals, n = 4..8 and a partial node: bit-exact with the oracle
    for n, seed in ((4, 1), (5, 2), (6, 3), (7, 4), (8, 5)):
        inst = I.random_instance(n, seed, with_b=True, asymmetric=(n % 2 == 1))
        lbs, done, D = raw_run(inst, 6)
        ref, Dref = oracle_raw(inst, 6)
        check(f"raw n={n}", done == 6 and np.array_equal(lbs, ref) and np.array_equal(D, Dref))
    inst = I.random_instance(9, 6, with_b=True)
    part = -np.ones(9, dtype=np.int32)
    part[[2, 6]] = [4, 0]
    lbs, _, D = raw_run(inst, 5, part)
    ref, Dref = oracle_raw(inst, 5, part)
    check("raw partial n=9", np.array_equal(lbs, ref) and np.array_equal(D, Dref))
    # canonical duals in fixed point
    inst = I.config(1)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, warm=1)) as ctx:
        lbs, _ = ctx.iterate(20)
    _, ref, _ = O.run(inst.F, inst.D, inst.B, iters=20, dual_mode=1)
    check("canonical n=8", np.max(np.abs(lbs - np.array(ref)) / np.abs(ref)) <= 1e-6)
    # variants: F with two phases and Type 4, the half-Z scheme, the pipelined launch
    inst = I.random_instance(7, 31, with_b=True, asymmetric=True)
    draws = I.sa_draws(7, 10, 3)
    prm = R.params(dual_mode=0, feas_tol=0.0, warm=1, variant=1, two_phase=1, ub=400.0, sa_t0=0.05)
    with R.Context(inst.F, inst.D, inst.B, prm=prm) as ctx:
        ctx.set_sa(*draws)
        lbs, _ = ctx.iterate(10)
    _, ref, _ = O.run(inst.F, inst.D, inst.B, iters=10, dual_mode=0, warm=True, variant=1, two_phase=True, sa=draws,
                      ub=400.0, sa_t0=0.05)
    check("F2 + Type 4", np.array_equal(lbs, np.array(ref)))
    inst = I.config(1)
    with R.Context(inst.F, inst.D, inst.B, prm=R.half_z_params(dual_mode=0, feas_tol=0.0)) as ctx:
        lbs, _ = ctx.iterate(10)
    _, ref, _ = O.run_half(inst.F, inst.D, inst.B, iters=10, dual_mode=0)
    check("half-Z", np.array_equal(lbs, np.array(ref)))
    inst = I.random_instance(7, 3, with_b=True)
    a = raw_run(inst, 8, pipeline=1)
    b = raw_run(inst, 8, pipeline=0)
    check("pipelined", np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2]))
    # n = 22: the banded class order of the z move
    inst = I.random_instance(22, 17, with_b=True)
    lbs, _, D = raw_run(inst, 2)
    ref, Dref = oracle_raw(inst, 2, threads=O.max_threads() or 1)
    check("raw n=22", np.array_equal(lbs, ref) and np.array_equal(D, Dref))
    # batched nodes, the batched LAP entry point, branch and bound
    inst = I.random_instance(9, 2, with_b=True, asymmetric=True)
    parts = -np.ones((4, 9), dtype=np.int32)
    parts[1, 0] = 3
    parts[2, [1, 4]] = [0, 7]
    parts[3, [0, 2, 5]] = [8, 1, 2]
    _, hist, _, _ = R.rlt2_bound_nodes(inst.F, inst.D, parts, 8, B=inst.B, prm=R.params(dual_mode=0, feas_tol=0.0))
    ok = True
    for k in range(4):
        _, ref, _ = O.run(inst.F, inst.D, inst.B, iters=8, dual_mode=0, partial=parts[k])
        ok = ok and np.array_equal(hist[k], np.array(ref))
    check("nodes", ok)
    rng = np.random.default_rng(4)
    ok = True
    for m in (1, 3, 8, 9, 16, 17, 32):
        c = rng.normal(size=(37, m, m))
        val = torch.empty(37, dtype=torch.float64, device="cuda")
        R.rlt2_lap_batched(torch.from_numpy(c).cuda(), val, dual_mode=0)
        v = val.cpu().numpy()
        ok = ok and all(v[b] == O.lap(c[b]).value for b in range(37))
    check("lap_batched", ok)
    inst = I.config(1)
    best, perm, _, st = R.rlt2_bnb_solve(inst.F, inst.D, inst.B, prm=R.params(warm=1, stall_window=25),
                                         opts=R.bnb_options(iters_root=60, iters_node=30))
    check("branch and bound", best == O.qap_brute(inst.F, inst.D, inst.B)[0] and st["proven"] == 1)

    torch.cuda.synchronize()
    violations = R.rlt2_debug_bounds_violations()
    print(json.dumps({"violations": violations, "checks": checks}))
    return 0 if all(ok for _, ok in checks) else 1


if __name__ == "__main__":
    sys.exit(main())
