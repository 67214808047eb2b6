"""Branch and bound on the GPU (Section 4): the parent -> child warm start
against the oracle, and rlt2_bnb_solve against brute-force optima."""
import numpy as np
import pytest

import oracle as O
from paper_1710_03732_gb300 import instances as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1710_03732_gb300 import build, rlt2
    build.build()
    rlt2.lib()
    return rlt2


def _snapshot(ctx):
    """The parent's costs of its last solve as an oracle State."""
    D, C = ctx.export_state()
    b, base = ctx.export_xstate()
    return O.State(ctx.n, base, b, C, D)


@pytest.mark.parametrize("mode", [0, 1])
def test_child_state_and_trajectory_bit_exact(R, mode):
    """The child built on the device from the parent's multiplier-adjusted costs
    equals the oracle's derivation bit for bit, and (raw duals) so does its
    ascent; its upper bound is the QAP value of its permutation."""
    inst = I.random_instance(8, 61, with_b=True, asymmetric=True)
    prm = R.params(dual_mode=mode, feas_tol=0.0)
    part = -np.ones(8, dtype=np.int32)
    part[5] = 1
    with R.Context(inst.F, inst.D, inst.B, partial=part, prm=prm) as parent:
        parent.iterate(7)
        snap = _snapshot(parent)
        fac, loc = 2, 6  # original indices; residual indices below
        free_f = [a for a in range(8) if part[a] < 0]
        free_l = [q for q in range(8) if q not in set(part[part >= 0])]
        ref = O.child_state(snap, free_f.index(fac), free_l.index(loc))
        with parent.child(fac, loc) as ch:
            D, C = ch.export_state()
            b, base = ch.export_xstate()
            assert ch.n == 6 and ch.const == ref.const and base == ref.const
            assert np.array_equal(b, ref.bprime)
            assert np.array_equal(C, ref.Chat) and np.array_equal(D, ref.Dhat)
            lbs, _ = ch.iterate(6)
            _, _, ub, _, ub_perm, _ = ch.bound()
        assert ub_perm[fac] == loc and ub_perm[5] == 1
        assert ub == O.qap_cost(inst.F, inst.D, inst.B, ub_perm)
    if mode == 0:
        want = []
        for _ in range(6):
            out = O.iterate(ref, O.params_array(), 0)
            want.append(ref.const + out.lb)
        assert np.array_equal(lbs, np.array(want))


def _opt(inst):
    v, p = O.qap_brute(inst.F, inst.D, inst.B)
    return v


@pytest.mark.parametrize("rule", [1, 2, 3])
@pytest.mark.parametrize("warm_depth", [-1, 64])
def test_bnb_exact_on_small_instances(R, rule, warm_depth):
    """The optimum of n = 8 and n = 9 instances (brute force over n!), with the
    permutation's value equal to it and the search proven complete."""
    for inst in (I.config(1), I.random_instance(8, 62, with_b=True, asymmetric=True),
                 I.random_instance(9, 63, with_b=True)):
        opts = R.bnb_options(order_rule=rule, warm_depth=warm_depth, iters_root=60, iters_node=30)
        best, perm, rlb, st = R.rlt2_bnb_solve(inst.F, inst.D, inst.B, prm=R.params(warm=1, stall_window=25),
                                               opts=opts)
        opt = _opt(inst)
        assert best == opt, (inst.name, best, opt, st)
        assert O.qap_cost(inst.F, inst.D, inst.B, perm) == opt
        assert sorted(perm) == list(range(inst.n))
        assert st["proven"] == 1
        assert rlb <= opt + 1e-9 * abs(opt)
        if warm_depth < 0:
            assert st["warm"] == 0


def test_bnb_short_ascents_branch_and_still_solve(R):
    """With two ascent iterations per node the bounds stay weak, so the tree
    branches deep; the optimum is still found and proven."""
    inst = I.random_instance(9, 64, with_b=True, asymmetric=True)
    opts = R.bnb_options(iters_root=2, iters_node=2)
    best, perm, rlb, st = R.rlt2_bnb_solve(inst.F, inst.D, inst.B, prm=R.params(), opts=opts)
    assert best == _opt(inst) and st["proven"] == 1
    assert st["branched"] > 1 and st["max_depth"] >= 2


def test_bnb_node_limit_is_not_proven(R):
    inst = I.random_instance(9, 65, with_b=True, asymmetric=True)
    opts = R.bnb_options(iters_root=2, iters_node=2, max_nodes=3)
    best, perm, rlb, st = R.rlt2_bnb_solve(inst.F, inst.D, inst.B, prm=R.params(), opts=opts)
    opt = _opt(inst)
    assert best >= opt and O.qap_cost(inst.F, inst.D, inst.B, perm) == best
    if st["bounded"] >= 3 and best > opt:
        assert st["proven"] == 0


def test_child_rejections(R):
    inst = I.config(1)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params()) as ctx:
        ctx.iterate(2)
        with pytest.raises(R.Rlt2Error):
            ctx.child(0, 8)  # no such location
        with ctx.child(0, 3) as ch:
            with pytest.raises(R.Rlt2Error):
                ch.child(0, 4)  # facility 0 is fixed already
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(variant=1)) as ctx:
        ctx.iterate(2)
        with pytest.raises(R.Rlt2Error):
            ctx.child(0, 3)


def test_bnb_with_half_z_scheme(R):
    """Children of a half-Z-scheme parent inherit its multipliers (the lower-order
    z stay 0 under the renumbering, which keeps the index order); the search
    still returns the brute-force optimum."""
    for inst in (I.config(1), I.random_instance(9, 66, with_b=True, asymmetric=True)):
        opts = R.bnb_options(iters_root=40, iters_node=20)
        best, perm, rlb, st = R.rlt2_bnb_solve(inst.F, inst.D, inst.B, prm=R.half_z_params(warm=1), opts=opts)
        assert best == _opt(inst) and st["proven"] == 1
