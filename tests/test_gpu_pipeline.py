"""The pipelined z move + Z-LAP launch (rlt2_params.pipeline = 1) against the
two-launch sequence (pipeline = 0, the default): every LAP sees the same costs
and start duals, so bounds, multiplier-adjusted costs and duals agree bit for
bit, for every dual mode, start and Section 3.4 variant, at every residual
size class (LAPs of 8, 16 and 32 lanes)."""
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


def _run(R, inst, iters, partial=None, **kw):
    with R.Context(inst.F, inst.D, inst.B, partial=partial, prm=R.params(feas_tol=0.0, **kw)) as ctx:
        lbs, done = ctx.iterate(iters)
        D, C = ctx.export_state()
        du = ctx.duals()
        st = ctx.stats()
    return lbs, done, D, C, du, st


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("warm", [0, 1])
@pytest.mark.parametrize("case", ["n3", "n7", "n10_partial", "n12_grid", "n19"])
def test_pipeline_equals_two_launches(R, mode, warm, case):
    partial = None
    if case == "n3":
        inst, iters = I.random_instance(3, 1, with_b=True), 6
    elif case == "n7":
        inst, iters = I.random_instance(7, 3, with_b=True, asymmetric=True), 12
    elif case == "n10_partial":
        inst, iters = I.random_instance(12, 5, with_b=True), 10
        partial = -np.ones(12, dtype=np.int32)
        partial[[1, 7]] = [3, 0]
    elif case == "n12_grid":
        inst, iters = I.config(2), 15
    else:
        inst, iters = I.random_instance(19, 8, with_b=True), 4
    a = _run(R, inst, iters, partial, dual_mode=mode, warm=warm, pipeline=1)
    b = _run(R, inst, iters, partial, dual_mode=mode, warm=warm, pipeline=0)
    assert a[1] == b[1] == iters
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    for k in ("xi", "psi", "gamma", "delta", "alpha", "beta"):
        assert np.array_equal(a[4][k], b[4][k]), k
    assert np.array_equal(a[5], b[5])  # iterations, augmentations and relaxations too


@pytest.mark.parametrize("variant,two_phase", [(1, 0), (0, 1), (1, 1)])
def test_pipeline_variants_and_annealing(R, variant, two_phase):
    """F, the two-phase Z solve and the Type 4 rule run through the pipelined
    launch; raw duals keep them bit-exact with the oracle."""
    inst = I.random_instance(8, 21, with_b=True, asymmetric=True)
    iters = 10
    draws = I.sa_draws(inst.n, iters, 3)
    out = []
    for pipe in (1, 0):
        prm = R.params(dual_mode=0, feas_tol=0.0, warm=1, variant=variant, two_phase=two_phase, ub=400.0,
                       sa_t0=0.05, pipeline=pipe)
        with R.Context(inst.F, inst.D, inst.B, prm=prm) as ctx:
            ctx.set_sa(*draws)
            lbs, _ = ctx.iterate(iters)
            out.append((lbs, ctx.export_state()[0]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    _, ref, _ = O.run(inst.F, inst.D, inst.B, iters=iters, dual_mode=0, warm=True, variant=variant,
                      two_phase=bool(two_phase), sa=draws, ub=400.0, sa_t0=0.05)
    assert np.array_equal(out[0][0], np.array(ref))


def test_pipeline_graph_replay_and_stops(R):
    """Past the direct-launch iterations the pipelined launch is replayed from
    the CUDA graph (its queue and counters reset themselves every launch); a
    device-side stop makes it a no-op like the other kernels."""
    inst = I.config(1)
    prm = R.params(dual_mode=0, feas_tol=0.0, warm=1, pipeline=1)
    with R.Context(inst.F, inst.D, inst.B, prm=prm) as ctx:
        one, _ = ctx.iterate(150)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(dual_mode=0, feas_tol=0.0, warm=1, pipeline=0)) as ctx:
        two, _ = ctx.iterate(150)
    assert np.array_equal(one, two)
    # the feasibility stop of Algorithm 1 on an instance it closes at once
    F = np.zeros((6, 6))
    D = np.abs(np.subtract.outer(np.arange(6.0), np.arange(6.0)))
    B = np.random.default_rng(3).integers(0, 9, (6, 6)).astype(float)
    with R.Context(F, D, B, prm=R.params(warm=1, pipeline=1)) as ctx:
        lbs, done = ctx.iterate(40)
        assert done == 1 and ctx.stats()[7] == 1
        assert lbs[0] == O.qap_brute(F, D, B)[0]


def test_pipeline_kernel_times(R):
    """With the pipeline the z move runs inside the Z-stage launch: the move kind
    records no launches and the Z-stage kind one per iteration."""
    inst = I.config(2)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(warm=1, pipeline=1)) as ctx:
        ctx.set_timing(True)
        ctx.iterate(5)
        kt = ctx.kernel_times()
    assert kt["move_z"][1] == 0 and kt["lap_z"][1] == 5 and kt["lap_z"][0] > 0.0
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(warm=1, pipeline=0)) as ctx:
        ctx.set_timing(True)
        ctx.iterate(5)
        kt = ctx.kernel_times()
    assert kt["move_z"][1] == 5 and kt["lap_z"][1] == 5


def test_pipeline_parameter_checked(R):
    inst = I.config(1)
    with pytest.raises(R.Rlt2Error):
        R.Context(inst.F, inst.D, inst.B, prm=R.params(pipeline=2))


def test_pipeline_wait_times_out_without_a_fault(R):
    """Failure detection of the pipelined launch: in its check form the LAP
    warps wait for pair counts the move never reaches, with the polls capped
    low; the wait gives up, the step reports RLT2_ETIMEOUT through the host,
    the launch ends, and the same device then runs a fresh pipelined ascent
    with the two-launch sequence's results."""
    inst = I.config(2)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, warm=1, pipeline=1)) as ctx:
        with pytest.raises(R.Rlt2Error) as e:  # no move pending before the first solve
            R._check(R.lib().rlt2_pipeline_check_wait_timeout(ctx.ctx), "check")
        assert e.value.status == R.RLT2_EINVAL
        _, done = ctx.iterate(3)
        assert done == 3
        assert R.rlt2_pipeline_check_wait_timeout(ctx.ctx) == R.RLT2_ETIMEOUT
        assert "gave up" in R.lib().rlt2_last_error().decode()
        with pytest.raises(R.Rlt2Error) as e:  # the context is stopped and keeps reporting it
            ctx.iterate(2)
        assert e.value.status == R.RLT2_ETIMEOUT
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, warm=1, pipeline=0)) as ctx:
        with pytest.raises(R.Rlt2Error) as e:
            R._check(R.lib().rlt2_pipeline_check_wait_timeout(ctx.ctx), "check")
        assert e.value.status == R.RLT2_EINVAL
    a = _run(R, inst, 12, None, warm=1, pipeline=1)
    b = _run(R, inst, 12, None, warm=1, pipeline=0)
    assert a[1] == b[1] == 12 and np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
