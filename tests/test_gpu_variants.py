"""GPU parity of the Section 3.4 variants against the CPU oracle: F (incremental
costs), the two-phase Z solve and the Type 4 rule with annealing.

Raw duals: bound trajectories, duals, reduced costs, C^, the x costs and the
bound base equal the oracle's bit for bit (same operation order on both sides).
Canonical duals: bounds within 1e-6 relative.  The Type 4 draws are inputs
(``instances.sa_draws``), identical on both sides.
"""
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


COMBOS = {
    "F1": dict(variant=1, two_phase=0, sa=False),
    "S2": dict(variant=0, two_phase=1, sa=False),
    "F2": dict(variant=1, two_phase=1, sa=False),
    "S1SA": dict(variant=0, two_phase=0, sa=True),
    "F2SA": dict(variant=1, two_phase=1, sa=True),
}
UB, T0 = 400.0, 0.05  # temperature T0 * UB accepts some draws and rejects others


def _oracle(inst, iters, mode, variant, two_phase, sa, warm, partial=None, draws=None):
    """Oracle trajectory plus everything the GPU holds after its last solve."""
    st = O.setup(inst.F, inst.D, inst.B, partial)
    n = st.n
    prm = O.params_array()
    bx = st.bprime.copy()
    base = st.const
    K = thr = None
    if sa:
        kf, kl, ng = draws
        K, thr = O.sa_schedule(n, kf, kl, ng, UB, T0, 0.99, 100)
    lbs, acc, out = [], [], None
    for it in range(iters):
        C_before, bx_before, base_before = st.Chat.copy(), bx.copy(), base
        w = warm and out is not None
        draw = (K[it], thr[it], kf[it], kl[it]) if sa and it < len(K) else None
        out, lb, on = O.iterate_v(st, bx, prm, base, dual_mode=mode, variant=variant, two_phase=two_phase,
                                  warm2=warm, u0z=out.xi.copy() if w else None,
                                  u0y=out.gamma.copy() if w else None, u0x=out.alpha.copy() if w else None,
                                  draw=draw)
        lbs.append(lb)
        acc.append(on)
        if variant == 1:
            base = lb
    return np.array(lbs), acc, out, C_before, bx_before, base_before


def _gpu(R, inst, iters, mode, variant, two_phase, sa, warm, partial=None, draws=None):
    prm = R.params(dual_mode=mode, feas_tol=0.0, warm=int(warm), variant=variant, two_phase=two_phase, ub=UB,
                   sa_t0=T0)
    with R.Context(inst.F, inst.D, inst.B, partial=partial, prm=prm) as ctx:
        if sa:
            ctx.set_sa(*draws)
        lbs, done = ctx.iterate(iters)
        _, C = ctx.export_state()
        bx, base = ctx.export_xstate()
        duals = ctx.duals()
        red = ctx.reduced_costs(with_z=False)
    return lbs, done, C, bx, base, duals, red


@pytest.mark.parametrize("name", list(COMBOS))
@pytest.mark.parametrize("which", ["cfg1", "asymB", "partial"])
@pytest.mark.parametrize("warm", [False, True])
def test_raw_bit_exact(R, name, which, warm):
    c = COMBOS[name]
    partial = None
    if which == "cfg1":
        inst, iters = I.config(1), 14
    elif which == "asymB":
        inst, iters = I.random_instance(7, 31, with_b=True, asymmetric=True), 12
    else:
        inst, iters = I.random_instance(9, 32, with_b=True), 10
        partial = -np.ones(9, dtype=np.int32)
        partial[[3, 7]] = [1, 5]
    n = inst.n - (0 if partial is None else int((partial >= 0).sum()))
    draws = I.sa_draws(n, iters, 40 + len(which)) if c["sa"] else None
    lbs, done, C, bx, base, duals, red = _gpu(R, inst, iters, 0, c["variant"], c["two_phase"], c["sa"], warm,
                                             partial, draws)
    ref, acc, out, C_ref, bx_ref, base_ref = _oracle(inst, iters, 0, c["variant"], c["two_phase"], c["sa"], warm,
                                                     partial, draws)
    assert done == iters
    assert np.array_equal(lbs, ref), (lbs, ref)
    if c["sa"]:
        assert 0 < sum(acc[:-1]) < iters - 1  # draws both accepted and rejected
    assert np.array_equal(C, C_ref)
    assert np.array_equal(bx, bx_ref)
    if c["variant"] == 1:
        assert base == base_ref
    assert np.array_equal(duals["xi"], out.xi) and np.array_equal(duals["psi"], out.psi)
    assert np.array_equal(duals["gamma"], out.gamma) and np.array_equal(duals["alpha"], out.alpha)
    assert np.array_equal(red["pi_y"], out.piy) and np.array_equal(red["pi_x"], out.pix)


def test_two_phase_state_bit_exact(R):
    """The GPU's D^ after a two-phase iteration is the oracle's D^ after the
    second-phase move of that iteration (the ascent step is still pending)."""
    inst = I.random_instance(7, 33, with_b=True)
    iters = 6
    prm = R.params(dual_mode=0, feas_tol=0.0, two_phase=1)
    with R.Context(inst.F, inst.D, inst.B, prm=prm) as ctx:
        ctx.iterate(iters)
        D, _ = ctx.export_state()
    st = O.setup(inst.F, inst.D, inst.B)
    bx = st.bprime.copy()
    for _ in range(iters - 1):
        O.iterate_v(st, bx, O.params_array(), st.const, dual_mode=0, two_phase=True)
    _, xi, psi, _, _ = O.stage_z(st.n, st.Dhat, dual_mode=0)
    D_ref = O.phase2_z(st.n, st.Dhat, xi, psi)
    assert np.array_equal(D, D_ref)


@pytest.mark.parametrize("name", ["F1", "S2", "F2SA"])
def test_canonical_close(R, name):
    """Canonical duals on the n = 12 grid workload, warm-started: bounds within 1e-6."""
    c = COMBOS[name]
    inst = I.config(2)
    iters = 30
    draws = I.sa_draws(inst.n, iters, 50) if c["sa"] else None
    lbs, done, *_ = _gpu(R, inst, iters, 1, c["variant"], c["two_phase"], c["sa"], True, None, draws)
    st, ref, _ = O.run(inst.F, inst.D, inst.B, iters=iters, dual_mode=1, warm=True, variant=c["variant"],
                       two_phase=bool(c["two_phase"]), sa=draws, ub=UB, sa_t0=T0, threads=8)
    ref = np.array(ref)
    assert done == iters
    assert np.max(np.abs(lbs - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-6


def test_fast_equals_slow_on_gpu(R):
    """F and S reach the same bounds (exact split of Eq. 3.6), here on the GPU."""
    inst = I.config(2)
    out = {}
    for variant in (0, 1):
        prm = R.params(feas_tol=0.0, variant=variant, warm=1)
        with R.Context(inst.F, inst.D, inst.B, prm=prm) as ctx:
            out[variant], _ = ctx.iterate(40)
    assert np.max(np.abs(out[1] - out[0]) / np.maximum(1.0, np.abs(out[0]))) <= 1e-9


def test_fast_checkpoint_resume(R):
    """F-variant checkpoint: D^, C^, the x costs and the bound base moved to a
    fresh context continue the run exactly (raw duals, cold starts)."""
    inst = I.random_instance(8, 34, with_b=True, asymmetric=True)
    prm = R.params(dual_mode=0, feas_tol=0.0, variant=1)
    with R.Context(inst.F, inst.D, inst.B, prm=prm) as a:
        first, _ = a.iterate(7)
        D, C = a.export_state()
        bx, base = a.export_xstate()
        rest, _ = a.iterate(6)
    with R.Context(inst.F, inst.D, inst.B, prm=prm) as b:
        b.import_state(D, C)
        b.import_xstate(bx, base)
        again, _ = b.iterate(7)
    assert again[0] == first[-1]
    assert np.array_equal(again[1:], rest)


def test_type4_needs_upper_bound(R):
    inst = I.config(1)
    kf, kl, ng = I.sa_draws(inst.n, 4, 1)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(ub=0.0)) as ctx:
        with pytest.raises(R.Rlt2Error):
            ctx.set_sa(kf, kl, ng)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(ub=100.0)) as ctx:
        with pytest.raises(R.Rlt2Error):
            ctx.set_sa(kf + 1.5, kl, ng)  # fractions above 1
        ctx.set_sa(kf, kl, ng)
        ctx.iterate(3)
        ctx.set_sa(np.zeros((0, inst.n)), np.zeros((0, inst.n)), np.zeros(0))  # off again
        lbs, done = ctx.iterate(2)
        assert done == 2


def test_kernel_times_two_phase(R):
    inst = I.config(2)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(two_phase=1, variant=1)) as ctx:
        ctx.set_timing(True)
        ctx.iterate(5)
        kt = ctx.kernel_times()
    assert kt["phase2_move"][1] == 5 and kt["lap_z2"][1] == 5
    assert kt["lap_z2"][0] > 0.0


@pytest.mark.parametrize("mode", [0, 1])
def test_nodes_variants_match_single_contexts(R, mode):
    """Batched nodes run F and the two-phase Z solve with the same arithmetic as
    single contexts."""
    inst = I.random_instance(11, 35, with_b=True)
    rng = np.random.default_rng(2)
    parts = -np.ones((5, 11), dtype=np.int32)
    for k, d in enumerate([0, 1, 2, 4, 5]):
        parts[k, rng.permutation(11)[:d]] = rng.permutation(11)[:d]
    iters = 9
    prm = R.params(dual_mode=mode, feas_tol=0.0, warm=1, variant=1, two_phase=1)
    lb, hist, its, _ = R.rlt2_bound_nodes(inst.F, inst.D, parts, iters, B=inst.B, prm=prm)
    assert (its == iters).all()
    for k in range(len(parts)):
        with R.Context(inst.F, inst.D, inst.B, partial=parts[k], prm=prm) as ctx:
            ref, _ = ctx.iterate(iters)
        assert np.array_equal(hist[k], ref), k


# ----------------------------------------------------------- half-Z scheme ----
@pytest.mark.parametrize("which", ["cfg1", "asymB", "partial"])
@pytest.mark.parametrize("warm", [False, True])
def test_half_raw_bit_exact(R, which, warm):
    """Half-Z scheme (only the Z-LAPs with i < j solved): bounds, D^ and C^ of the
    last solve, duals and reduced costs equal the oracle's bit for bit; the
    lower-order z stay exactly 0."""
    partial = None
    if which == "cfg1":
        inst, iters = I.config(1), 14
    elif which == "asymB":
        inst, iters = I.random_instance(7, 43, with_b=True, asymmetric=True), 12
    else:
        inst, iters = I.random_instance(9, 44, with_b=True), 10
        partial = -np.ones(9, dtype=np.int32)
        partial[[0, 8]] = [4, 7]
    prm = R.half_z_params(dual_mode=0, feas_tol=0.0, warm=int(warm))
    with R.Context(inst.F, inst.D, inst.B, partial=partial, prm=prm) as ctx:
        lbs, done = ctx.iterate(iters)
        D, C = ctx.export_state()
        duals = ctx.duals()
        red = ctx.reduced_costs()
    st = O.setup(inst.F, inst.D, inst.B, partial)
    ref, out = [], None
    for _ in range(iters):
        before = (st.Dhat.copy(), st.Chat.copy())
        w = warm and out is not None
        out = O.iterate_half(st, dual_mode=0, u0z=out.xi.copy() if w else None,
                             u0y=out.gamma.copy() if w else None, u0x=out.alpha.copy() if w else None)
        ref.append(st.const + out.lb)
    assert done == iters
    assert np.array_equal(lbs, np.array(ref))
    assert np.array_equal(D, before[0]) and np.array_equal(C, before[1])
    assert np.array_equal(duals["xi"], out.xi) and np.array_equal(duals["psi"], out.psi)
    assert np.array_equal(duals["gamma"], out.gamma) and np.array_equal(duals["alpha"], out.alpha)
    assert np.array_equal(red["pi_y"], out.piy) and np.array_equal(red["pi_x"], out.pix)
    n, m = st.n, st.n - 2
    for i in range(n):
        for j in range(i):
            t = O.tile_index(n, i, 0 if i != 0 else 1, j, 1 if i != 0 else 0)
            assert np.all(D[t * m * m:(t + 1) * m * m] == 0.0)


def test_half_canonical_close_and_half_the_work(R):
    """n = 12 grid, canonical duals, warm starts: bounds within 1e-6 of the oracle;
    the Z stage runs half the LAPs of the full scheme."""
    inst = I.config(2)
    iters = 25
    with R.Context(inst.F, inst.D, inst.B, prm=R.half_z_params(feas_tol=0.0, warm=1)) as ctx:
        lbs, done = ctx.iterate(iters)
    _, ref, _ = O.run_half(inst.F, inst.D, inst.B, iters=iters, warm=True)
    ref = np.array(ref)
    assert done == iters
    assert np.max(np.abs(lbs - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-6
    assert np.all(np.diff(lbs) >= -1e-9 * np.abs(lbs[:-1]))


def test_half_rejections(R):
    inst = I.config(1)
    with pytest.raises(R.Rlt2Error):
        R.Context(inst.F, inst.D, inst.B, prm=R.half_z_params(variant=1))
    with pytest.raises(R.Rlt2Error):
        R.Context(inst.F, inst.D, inst.B, prm=R.half_z_params(two_phase=1))
    with R.Context(inst.F, inst.D, inst.B, prm=R.half_z_params(ub=100.0)) as ctx:
        kf, kl, ng = I.sa_draws(inst.n, 3, 2)
        with pytest.raises(R.Rlt2Error):
            ctx.set_sa(kf, kl, ng)
    parts = -np.ones((2, 8), dtype=np.int32)
    with pytest.raises(R.Rlt2Error):
        R.rlt2_bound_nodes(inst.F, inst.D, parts, 3, prm=R.half_z_params())
