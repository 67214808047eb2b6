"""The no-allocation entry point (rlt2_iterate_noalloc) against the context path.

rlt2_iterate_noalloc serves callers that cannot call cudaMalloc (a framework that
owns the device memory pool, loops that must avoid the allocator's implicit
synchronisation, deployments that forbid allocation after start-up): it keeps all
working memory in one fixed device array inside the library.  This file runs
last so that a failure here stops a -x run only after every other test ran; it
passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_1710_03732_gb300 import instances as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1710_03732_gb300 import build, rlt2
    build.build()
    rlt2.lib()
    return rlt2


def _context_bounds(R, inst, iters, prm):
    with R.Context(inst.F, inst.D, inst.B, prm=prm) as ctx:
        lbs, done = ctx.iterate(iters)
    return lbs, done


def _noalloc_bounds(R, inst, iters, prm):
    F = torch.from_numpy(inst.F).cuda()
    D = torch.from_numpy(inst.D).cuda()
    B = torch.from_numpy(inst.B).cuda()
    out = torch.empty(iters, dtype=torch.float64, device="cuda")
    R.rlt2_iterate_noalloc(F, D, out, B=B, prm=prm)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_context_path_twice_in_a_row(R):
    """Two calls in a row on different problems share the fixed array; each must
    give the same bound trajectory as rlt2_create + rlt2_iterate (within the
    1e-6 relative trajectory tolerance; observed identical)."""
    cases = [(I.config(1), 30, R.params(feas_tol=0.0)),                              # n = 8, canonical duals
             (I.random_instance(10, 7, with_b=True), 12, R.params(dual_mode=0, feas_tol=0.0, warm=1))]  # n = 10
    for inst, iters, prm in cases:
        ref, done = _context_bounds(R, inst, iters, prm)
        assert done == iters
        got = _noalloc_bounds(R, inst, iters, prm)
        rel = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
        assert rel.max() <= 1e-6, rel.max()
    # and the first problem again after the second one left its contents behind
    inst, iters, prm = cases[0]
    ref, _ = _context_bounds(R, inst, iters, prm)
    got = _noalloc_bounds(R, inst, iters, prm)
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-6


def test_noalloc_rejects_sizes_beyond_the_workspace(R):
    inst = I.random_instance(11, 1)
    with pytest.raises(R.Rlt2Error) as e:
        _noalloc_bounds(R, inst, 3, None)
    assert e.value.status == R.RLT2_EINVAL and "n must be in [3, 10]" in str(e.value)


@pytest.mark.parametrize("variant,two_phase", [(1, 0), (0, 1), (1, 1)])
def test_noalloc_runs_the_variants(R, variant, two_phase):
    """The fixed array also holds the F variant's x costs; the F variant and the
    two-phase Z solve give the context path's trajectory (raw duals: identical)."""
    inst = I.random_instance(9, 17, with_b=True, asymmetric=True)
    prm = R.params(dual_mode=0, feas_tol=0.0, warm=1, variant=variant, two_phase=two_phase)
    ref, done = _context_bounds(R, inst, 15, prm)
    assert done == 15
    got = _noalloc_bounds(R, inst, 15, prm)
    assert np.array_equal(got, ref)


def test_noalloc_rejects_the_half_z_scheme(R):
    inst = I.config(1)
    F = torch.from_numpy(inst.F).cuda()
    D = torch.from_numpy(inst.D).cuda()
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(R.Rlt2Error):
        R.rlt2_iterate_noalloc(F, D, out, prm=R.half_z_params())


def test_noalloc_rejects_the_learned_start(R):
    """warm = 2 needs a network set on a context; the no-allocation path has
    none, so it must refuse instead of running a cold start."""
    inst = I.config(1)
    F = torch.from_numpy(inst.F).cuda()
    D = torch.from_numpy(inst.D).cuda()
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(R.Rlt2Error) as e:
        R.rlt2_iterate_noalloc(F, D, out, prm=R.params(warm=2))
    assert e.value.status == R.RLT2_EINVAL and "learned start" in str(e.value)
