"""Batched branch-and-bound node bounding (rlt2_bound_nodes) on the GPU."""
import itertools

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


def _nodes(n, depths, seed):
    rng = np.random.default_rng(seed)
    out = -np.ones((len(depths), n), dtype=np.int32)
    for k, d in enumerate(depths):
        fac = rng.permutation(n)[:d]
        loc = rng.permutation(n)[:d]
        out[k, fac] = loc
    return out


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_nodes_bit_identical_to_single_contexts(R, mode):
    """Each node of the batch follows exactly the trajectory of its own context
    (same kernels, same arithmetic; the batch only changes the launch shape)."""
    inst = I.random_instance(12, 4, with_b=True)
    parts = _nodes(12, [0, 1, 2, 3, 4, 5, 6, 7, 9], 1)
    iters = 14
    prm = R.params(dual_mode=mode, feas_tol=0.0, warm=1)
    lb, hist, its, stats = R.rlt2_bound_nodes(inst.F, inst.D, parts, iters, B=inst.B, prm=prm)
    assert (its == iters).all() and stats["waves"] == 1
    for k in range(len(parts)):
        with R.Context(inst.F, inst.D, inst.B, partial=parts[k], prm=prm) as ctx:
            ref, _ = ctx.iterate(iters)
        assert np.array_equal(hist[k], ref), k
        assert lb[k] == ref.max()


def test_nodes_match_oracle(R):
    inst = I.random_instance(9, 2, with_b=True, asymmetric=True)
    parts = _nodes(9, [0, 2, 4, 6], 3)
    iters = 10
    for mode in (0, 1):
        _, hist, _, _ = R.rlt2_bound_nodes(inst.F, inst.D, parts, iters, B=inst.B,
                                           prm=R.params(dual_mode=mode, feas_tol=0.0))
        for k in range(len(parts)):
            _, ref, _ = O.run(inst.F, inst.D, inst.B, iters=iters, dual_mode=mode, partial=parts[k])
            ref = np.array(ref)
            if mode == 0:
                assert np.array_equal(hist[k], ref)
            else:
                assert np.max(np.abs(hist[k] - ref) / np.maximum(1, np.abs(ref))) <= 1e-6


def test_node_bounds_below_best_completion(R):
    """Weak duality per node: each node's bound is at most the best QAP value among
    the completions of its partial assignment (brute force)."""
    inst = I.random_instance(8, 6, with_b=True)
    parts = _nodes(8, [1, 2, 3, 3, 4], 7)
    lb, hist, _, _ = R.rlt2_bound_nodes(inst.F, inst.D, parts, 30, B=inst.B)
    for k, part in enumerate(parts):
        free_f = [i for i in range(8) if part[i] < 0]
        free_l = [p for p in range(8) if p not in part]
        best = np.inf
        for sig in itertools.permutations(free_l):
            full = part.copy()
            full[free_f] = sig
            best = min(best, O.qap_cost(inst.F, inst.D, inst.B, full))
        h = hist[k][~np.isnan(hist[k])]
        assert lb[k] <= best + 1e-9 and np.all(np.diff(h) >= -1e-9 * np.abs(h[:-1]))


def test_memory_admission_waves(R):
    """A budget that holds only a few arenas splits the batch into waves with the
    same results; a budget below one node's arena is refused with EADMIT."""
    inst = I.random_instance(12, 4, with_b=True)
    parts = _nodes(12, [0, 2, 2, 3, 5, 6], 9)
    iters = 8
    prm = R.params(feas_tol=0.0)
    lb1, h1, _, s1 = R.rlt2_bound_nodes(inst.F, inst.D, parts, iters, B=inst.B, prm=prm)
    lb2, h2, _, s2 = R.rlt2_bound_nodes(inst.F, inst.D, parts, iters, B=inst.B, prm=prm, mem_budget=20 << 20)
    assert s1["waves"] == 1 and s2["waves"] > 1
    assert np.array_equal(h1, h2) and np.array_equal(lb1, lb2)
    with pytest.raises(R.Rlt2Error) as e:
        R.rlt2_bound_nodes(inst.F, inst.D, parts, iters, B=inst.B, prm=prm, mem_budget=1 << 20)
    assert e.value.status == R.RLT2_EADMIT


def test_config4_batched_nodes(R):
    """n = 22, Manhattan 2x11 grid, 64 nodes at depths 4..8 (residual 14..18): one
    wave, autotuned Z-stage shape, bounds monotone, sampled nodes identical to
    their own contexts."""
    inst = I.config(4)
    parts = inst.partials
    iters = 12
    prm = R.params(feas_tol=0.0, warm=1)
    lb, hist, its, stats = R.rlt2_bound_nodes(inst.F, inst.D, parts, iters, B=inst.B, prm=prm)
    assert stats["waves"] == 1 and (its == iters).all()
    assert stats["group"] in (16, 32) and stats["wpb"] in (4, 8)
    # every Z-LAP size present has its own tuned shape (lanes >= size)
    table = {e["m"]: e for e in R.rlt2_node_tuning()}
    for mz in {int((parts[k] < 0).sum()) - 2 for k in range(len(parts))}:
        assert mz in table and table[mz]["lanes_per_lap"] >= mz and table[mz]["warps_per_block"] in (4, 8)
    assert np.all(np.diff(hist, axis=1) >= -1e-9 * np.abs(hist[:, :-1]))
    for k in (0, 17, 63):
        with R.Context(inst.F, inst.D, inst.B, partial=parts[k], prm=prm) as ctx:
            ref, _ = ctx.iterate(iters)
        assert np.array_equal(hist[k], ref)


@pytest.mark.parametrize("mode", [0, 1])
def test_iterate_many_equals_single_contexts(R, mode):
    """rlt2_iterate_many runs several contexts (different residual sizes, one
    already advanced, another a child derived from a parent) in lockstep
    batched launches; each ends exactly where rlt2_iterate alone takes it:
    bounds, multiplier-adjusted costs and duals bit for bit."""
    inst = I.random_instance(12, 4, with_b=True)
    parts = _nodes(12, [1, 2, 3, 5, 7], 3)
    prm = R.params(dual_mode=mode, feas_tol=0.0, warm=1)

    def make():
        cs = [R.Context(inst.F, inst.D, inst.B, partial=p, prm=prm) for p in parts]
        cs[0].iterate(3)
        root = R.Context(inst.F, inst.D, inst.B, prm=prm)
        root.iterate(4)
        cs.append(root.child(facility=2, location=5))
        root.close()
        return cs

    many = make()
    done = R.rlt2_iterate_many(many, 9)
    assert (done == 9).all()
    single = make()
    for c in single:
        _, d = c.iterate(9)
        assert d == 9
    for a, b in zip(many, single):
        assert a.bound()[:3] == b.bound()[:3]
        Da, Ca = a.export_state()
        Db, Cb = b.export_state()
        assert np.array_equal(Da, Db) and np.array_equal(Ca, Cb)
        for k in ("xi", "psi", "gamma", "alpha"):
            assert np.array_equal(a.duals()[k], b.duals()[k]), k
        # and the next iterations continue identically on the single path
        ha, _ = a.iterate(2)
        hb, _ = b.iterate(2)
        assert np.array_equal(ha, hb)
    for c in many + single:
        c.close()


def test_iterate_many_stops_each_context_on_its_own(R):
    """Contexts with a known upper bound stop on the min-gap rule at their own
    iteration; the batch reports each one's count, equal to rlt2_iterate's, and
    ends once all have stopped."""
    inst = I.config(1)
    opt, _ = O.qap_brute(inst.F, inst.D, inst.B)
    parts = _nodes(8, [0, 1, 2, 3], 11)
    prm = R.params(feas_tol=0.0, warm=1, ub=float(opt) * 1.02, min_gap=0.03)
    many = [R.Context(inst.F, inst.D, inst.B, partial=p, prm=prm) for p in parts]
    done = R.rlt2_iterate_many(many, 400)
    for k, p in enumerate(parts):
        with R.Context(inst.F, inst.D, inst.B, partial=p, prm=prm) as c:
            _, d = c.iterate(400)
            ref_best = c.bound()[1]
        assert done[k] == d and many[k].bound()[1] == ref_best
    assert done.max() < 400 and len(set(done.tolist())) > 1
    for c in many:
        c.close()


def test_iterate_many_rejects_mixed_parameters(R):
    inst = I.config(1)
    a = R.Context(inst.F, inst.D, inst.B, prm=R.params(warm=1))
    b = R.Context(inst.F, inst.D, inst.B, prm=R.params(warm=0))
    with pytest.raises(R.Rlt2Error) as e:
        R.rlt2_iterate_many([a, b], 3)
    assert e.value.status == R.RLT2_EINVAL
    with pytest.raises(R.Rlt2Error):
        R.rlt2_iterate_many([a, a], 3)
    a.close()
    b.close()


@pytest.mark.parametrize("variant,two_phase", [(1, 0), (0, 1), (1, 1)])
def test_iterate_many_runs_the_variants(R, variant, two_phase):
    """The F variant and the two-phase Z solve through the batched engine:
    raw duals, each context bit for bit where rlt2_iterate takes it."""
    inst = I.random_instance(10, 23, with_b=True, asymmetric=True)
    parts = _nodes(10, [0, 1, 2, 4], 5)
    prm = R.params(dual_mode=0, feas_tol=0.0, warm=1, variant=variant, two_phase=two_phase)
    many = [R.Context(inst.F, inst.D, inst.B, partial=p, prm=prm) for p in parts]
    done = R.rlt2_iterate_many(many, 7)
    assert (done == 7).all()
    for k, p in enumerate(parts):
        with R.Context(inst.F, inst.D, inst.B, partial=p, prm=prm) as c:
            ref, _ = c.iterate(7)
            Dr, Cr = c.export_state()
            ref_best = c.bound()[1]
        D, C = many[k].export_state()
        assert np.array_equal(D, Dr) and np.array_equal(C, Cr)
        assert many[k].bound()[1] == ref_best
    for c in many:
        c.close()
