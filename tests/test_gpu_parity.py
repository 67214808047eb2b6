"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: LAP optima within 1e-9 relative; every dual feasible (reduced costs
>= -1e-9 relative); raw-mode Hungarian duals, assignments and the whole raw
dual-ascent trajectory and state bit-identical (same operation order, lowest-
index ties); canonical-mode bound trajectories within 1e-6 relative.  Canonical
duals come in two arithmetic forms: exact 64-bit fixed point on a per-tile grid
of 2^-48 of the tile's magnitude bound (dual_mode 1, the default) and FP64
(dual_mode 2); both are held to the same tolerances against the FP64 oracle.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1710_03732_gb300 import instances as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PRM = dict(kz=1.0, ky=0.5, kx=1.0, phi_y=0.5, phi_z=(0.2,) * 5)


@pytest.fixture(scope="module")
def R():
    from paper_1710_03732_gb300 import build, rlt2
    build.build()
    rlt2.lib()
    return rlt2


def _prm(R, mode, **kw):
    """Device parameters; feas_tol = 0 disables the early stop so runs have full length."""
    d = dict(PRM)
    d.update(kw)
    return R.params(dual_mode=mode, feas_tol=0.0, **d)


def _oprm(**kw):
    d = dict(PRM)
    d.update(kw)
    return O.params_array(**d)


def _rand_costs(rng, batch, m, kind):
    if kind == "int":
        return rng.integers(-3, 4, (batch, m, m)).astype(np.float64)
    if kind == "zero":
        return np.zeros((batch, m, m))
    if kind == "big":
        return rng.normal(size=(batch, m, m)) * 1e6
    return rng.normal(size=(batch, m, m)) * 10


# ------------------------------------------------------------------ LAP ----
@pytest.mark.parametrize("m", [1, 2, 3, 5, 7, 12, 18, 19, 28, 31, 32])
@pytest.mark.parametrize("kind", ["real", "int", "zero"])
def test_lap_batched_raw_bit_exact(R, m, kind):
    """Raw mode follows the oracle's Hungarian step for step: identical values,
    duals, assignments and augmentation counts; batch spans several blocks and a
    ragged tail."""
    rng = np.random.default_rng(m * 7 + len(kind))
    batch = 8 * 8 * 3 + 5
    c = _rand_costs(rng, batch, m, kind)
    dc = torch.from_numpy(c).cuda()
    val = torch.empty(batch, dtype=torch.float64, device="cuda")
    u = torch.empty(batch, m, dtype=torch.float64, device="cuda")
    v = torch.empty_like(u)
    r2c = torch.empty(batch, m, dtype=torch.int32, device="cuda")
    naug = torch.empty(batch, dtype=torch.int32, device="cuda")
    R.rlt2_lap_batched(dc, val, u=u, v=v, row_to_col=r2c, n_aug=naug, dual_mode=0)
    torch.cuda.synchronize()
    val, u, v, r2c, naug = (x.cpu().numpy() for x in (val, u, v, r2c, naug))
    for b in range(batch):
        o = O.lap(c[b])
        assert val[b] == o.value
        assert np.array_equal(u[b], o.u) and np.array_equal(v[b], o.v)
        assert np.array_equal(r2c[b], o.row_to_col)
        assert naug[b] == o.n_aug


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("m", [1, 2, 4, 9, 18, 28, 32])
def test_lap_batched_canonical(R, m, mode):
    rng = np.random.default_rng(100 + m)
    batch = 300
    c = np.concatenate([_rand_costs(rng, batch // 3, m, "real"), _rand_costs(rng, batch // 3, m, "int"),
                        _rand_costs(rng, batch - 2 * (batch // 3), m, "big")])
    dc = torch.from_numpy(c).cuda()
    val = torch.empty(batch, dtype=torch.float64, device="cuda")
    u = torch.empty(batch, m, dtype=torch.float64, device="cuda")
    v = torch.empty_like(u)
    R.rlt2_lap_batched(dc, val, u=u, v=v, dual_mode=mode)
    torch.cuda.synchronize()
    val, u, v = val.cpu().numpy(), u.cpu().numpy(), v.cpu().numpy()
    for b in range(batch):
        o = O.lap(c[b], canonical=True)
        scale = max(1.0, np.abs(c[b]).max())
        assert abs(val[b] - o.value) <= 1e-9 * max(1.0, abs(o.value))
        red = c[b] - u[b][:, None] - v[b][None, :]
        assert red.min() >= -1e-9 * scale
        assert abs(u[b].sum() + v[b].sum() - o.value) <= 1e-9 * scale * m
        assert np.allclose(u[b], o.u, rtol=0, atol=1e-9 * scale)
        assert np.allclose(v[b], o.v, rtol=0, atol=1e-9 * scale)


def _fixed_point_solve(R, c, u0=None):
    batch, m = c.shape[0], c.shape[1]
    val = torch.empty(batch, dtype=torch.float64, device="cuda")
    u = torch.empty(batch, m, dtype=torch.float64, device="cuda")
    v = torch.empty_like(u)
    R.rlt2_lap_batched(torch.from_numpy(c).cuda(), val, u0=None if u0 is None else torch.from_numpy(u0).cuda(),
                       u=u, v=v, dual_mode=1)
    torch.cuda.synchronize()
    return val.cpu().numpy(), u.cpu().numpy(), v.cpu().numpy()


@pytest.mark.parametrize("m", [3, 7, 18, 28])
def test_lap_fixed_point_start_independent(R, m):
    """The fixed-point canonical duals are exact for the tile rounded onto its
    grid, so every start (cold, good, poor, absurdly large) returns the same
    value and duals bit for bit, and the duals are feasible for the given tile."""
    rng = np.random.default_rng(300 + m)
    batch = 200
    c = rng.normal(size=(batch, m, m)) * 100.0
    c[: batch // 4] = np.round(c[: batch // 4])
    cold = _fixed_point_solve(R, c)
    good = np.array([O.lap(c[b], canonical=True).u for b in range(batch)]) + rng.normal(size=(batch, m)) * 1e-3
    starts = [good, rng.normal(size=(batch, m)) * 500.0, np.full((batch, m), 1e200),
              np.where(rng.random((batch, m)) < 0.5, -1e300, 1e-300)]
    for u0 in starts:
        warm = _fixed_point_solve(R, c, u0)
        for a, b in zip(cold, warm):
            assert np.array_equal(a, b)
    val, u, v = cold
    for b in range(batch):
        scale = np.abs(c[b]).max()
        assert (c[b] - u[b][:, None] - v[b][None, :]).min() >= -1e-14 * scale * m
        assert abs(val[b] - O.lap(c[b]).value) <= 1e-13 * scale * m


@pytest.mark.parametrize("kind", ["tiny", "huge", "mixed", "zero_rows", "subnormal"])
def test_lap_fixed_point_scales(R, kind):
    """Tiles at the ends of the double range and with entries of very different
    magnitude: the fixed-point solve stays within the FP64 oracle's tolerance."""
    rng = np.random.default_rng({"tiny": 1, "huge": 2, "mixed": 3, "zero_rows": 4, "subnormal": 5}[kind])
    batch, m = 64, 18
    c = rng.normal(size=(batch, m, m))
    if kind == "tiny":
        c *= 1e-300
    elif kind == "huge":
        c *= 1e300
    elif kind == "mixed":
        c *= 10.0 ** rng.integers(-12, 12, (batch, m, m))
    elif kind == "zero_rows":
        c[:, ::3, :] = 0.0
    else:
        c *= 1e-310
    val, u, v = _fixed_point_solve(R, c)
    for b in range(batch):
        o = O.lap(c[b], canonical=True)
        scale = np.abs(c[b]).max()
        assert abs(val[b] - o.value) <= 1e-9 * max(scale, abs(o.value)) + 1e-320
        assert np.allclose(u[b], o.u, rtol=0, atol=1e-9 * scale + 1e-320)
        assert np.allclose(v[b], o.v, rtol=0, atol=1e-9 * scale + 1e-320)


def test_lap_fixed_point_wide_range_small_optimum(R):
    """Tiles with a 1e12 dynamic range whose optimum is near 0: a permutation of
    entries of size ~1 in a tile of entries up to 1e12.  The fixed-point grid
    of such a tile is 2^L with L = E - 48 (2^E the first power of two above its
    largest entry, here 2^-8), so the exact optimum of the rounded tile differs
    from the FP64 optimum by less than m * 2^L; against the optimum itself that
    is a relative error of up to ~1e-3 (recorded here, not hidden behind the
    tile-scale tolerance).  Duals stay feasible for the given tile."""
    rng = np.random.default_rng(77)
    batch, m = 64, 18
    c = rng.uniform(1e11, 1e12, size=(batch, m, m))
    for b in range(batch):
        perm = rng.permutation(m)
        c[b, np.arange(m), perm] = rng.uniform(0.0, 2.0, m)
    val, u, v = _fixed_point_solve(R, c)
    worst = 0.0
    for b in range(batch):
        o = O.lap(c[b], canonical=True)
        E = int(np.floor(np.log2(np.abs(c[b]).max()))) + 1
        grid = 2.0 ** (E - 48)
        assert abs(val[b] - o.value) <= m * grid
        worst = max(worst, abs(val[b] - o.value) / abs(o.value))
        assert (c[b] - u[b][:, None] - v[b][None, :]).min() >= -1e-14 * np.abs(c[b]).max() * m
    # the recorded figure: relative error against the optimum itself
    assert worst < 5e-3
    print(f"fixed point, 1e12 dynamic range, optimum ~{np.mean(val):.2f}: worst relative error {worst:.2e}")


def test_lap_batched_warm_start(R):
    rng = np.random.default_rng(5)
    batch, m = 500, 18
    c = rng.normal(size=(batch, m, m))
    u0 = rng.normal(size=(batch, m))
    val = torch.empty(batch, dtype=torch.float64, device="cuda")
    u = torch.empty(batch, m, dtype=torch.float64, device="cuda")
    v = torch.empty_like(u)
    R.rlt2_lap_batched(torch.from_numpy(c).cuda(), val, u0=torch.from_numpy(u0).cuda(), u=u, v=v, dual_mode=0)
    torch.cuda.synchronize()
    val, u, v = val.cpu().numpy(), u.cpu().numpy(), v.cpu().numpy()
    for b in range(batch):
        o = O.lap(c[b], u0=u0[b])
        assert val[b] == o.value and np.array_equal(u[b], o.u) and np.array_equal(v[b], o.v)


def test_lap_batched_brute_force(R):
    rng = np.random.default_rng(8)
    for m in range(1, 8):
        c = rng.integers(0, 9, (64, m, m)).astype(np.float64)
        val = torch.empty(64, dtype=torch.float64, device="cuda")
        R.rlt2_lap_batched(torch.from_numpy(c).cuda(), val, dual_mode=1)
        torch.cuda.synchronize()
        for b in range(64):
            assert val[b].item() == O.lap_brute(c[b])[0]


# ------------------------------------------------------------ dual ascent ----
def _gpu_run(R, inst, iters, mode, partial=None, **kw):
    with R.Context(inst.F, inst.D, inst.B, partial=partial, prm=_prm(R, mode, **kw)) as ctx:
        lbs, done = ctx.iterate(iters)
        D, C = ctx.export_state()
        duals = ctx.duals()
        red = ctx.reduced_costs()
        st = ctx.stats()
        bound = ctx.bound()
    return lbs, done, D, C, duals, red, st, bound


@pytest.mark.parametrize("which", ["cfg1", "randB", "asym", "partial", "n3", "PX"])
def test_raw_trajectory_and_state_bit_exact(R, which):
    """Raw duals: GPU bounds, duals, reduced costs and the multiplier-adjusted
    state after k iterations equal the oracle's bit for bit."""
    partial = None
    okw = {}
    if which == "cfg1":
        inst, iters = I.config(1), 12
    elif which == "randB":
        inst, iters = I.random_instance(7, 3, with_b=True), 10
    elif which == "asym":
        inst, iters = I.random_instance(7, 4, with_b=True, asymmetric=True), 10
    elif which == "partial":
        inst, iters = I.random_instance(9, 5, with_b=True), 8
        partial = -np.ones(9, dtype=np.int32)
        partial[[2, 6]] = [4, 0]
    elif which == "n3":
        inst, iters = I.random_instance(3, 1, with_b=True), 6
    else:
        inst, iters = I.random_instance(6, 9, with_b=True), 10
        okw = dict(kz=0.8, ky=0.6, kx=0.9, phi_y=0.3, phi_z=(0.1, 0.3, 0.15, 0.25, 0.2))
    lbs, done, D, C, duals, red, st, _ = _gpu_run(R, inst, iters, 0, partial=partial, **okw)
    assert done == iters
    ost = O.setup(inst.F, inst.D, inst.B, partial)
    ref = []
    for it in range(iters):
        before = O.State(ost.n, ost.const, ost.bprime, ost.Chat.copy(), ost.Dhat.copy())
        out = O.iterate(ost, _oprm(**okw), 0)  # solve, then the ascent step in place
        ref.append(ost.const + out.lb)
    ost = before  # the GPU holds the state of its last solve (its ascent step is still pending)
    assert np.array_equal(lbs, np.array(ref)), (lbs, ref)
    # state of the last solve (before its ascent step), duals and reduced costs
    assert np.array_equal(D, ost.Dhat) and np.array_equal(C, ost.Chat)
    assert np.array_equal(duals["xi"], out.xi) and np.array_equal(duals["psi"], out.psi)
    assert np.array_equal(duals["gamma"], out.gamma) and np.array_equal(duals["alpha"], out.alpha)
    assert np.array_equal(red["pi_y"], out.piy) and np.array_equal(red["pi_x"], out.pix)
    n = ost.n
    m = n - 2
    T = O.num_tiles(n)
    piz = (ost.Dhat.reshape(T, m, m) - out.xi.reshape(T, m, 1)) - out.psi.reshape(T, 1, m)
    assert np.array_equal(red["pi_z"], piz.ravel())


def _golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return np.array([float(x) for x in f if not x.startswith("#")])


@pytest.mark.parametrize("name,cfg,iters,mode", [
    ("lb_n8_grid2x4_canonical.txt", 1, 50, 1),
    ("lb_n8_grid2x4_canonical.txt", 1, 50, 2),
    ("lb_n8_grid2x4_raw.txt", 1, 50, 0),
    ("lb_n12_grid3x4_canonical.txt", 2, 200, 1),
    ("lb_n12_grid3x4_canonical.txt", 2, 200, 2),
    ("lb_n12_grid3x4_raw.txt", 2, 200, 0),
])
def test_trajectory_matches_golden(R, name, cfg, iters, mode):
    """Configs n=8 (50 iterations) and n=12 (200 iterations): bounds within 1e-6
    relative of the stored oracle trajectory; raw mode bit-identical."""
    inst = I.config(cfg)
    ref = _golden(name)
    with R.Context(inst.F, inst.D, inst.B, prm=_prm(R, mode)) as ctx:
        lbs, done = ctx.iterate(iters)
    assert done == iters
    rel = np.abs(lbs - ref) / np.maximum(1.0, np.abs(ref))
    assert rel.max() <= 1e-6, rel.max()
    if mode == 0:
        assert np.array_equal(lbs, ref)
    assert np.all(np.diff(lbs) >= -1e-9 * np.abs(lbs[:-1]))


def test_config1_bound_below_brute_force_optimum(R):
    inst = I.config(1)
    opt, _ = O.qap_brute(inst.F, inst.D, inst.B)
    for mode in (0, 1):
        with R.Context(inst.F, inst.D, inst.B, prm=_prm(R, mode)) as ctx:
            lbs, _ = ctx.iterate(50)
            lb, best, ub, perm, ub_perm, its = ctx.bound()
        assert lbs.max() <= opt * (1 + 1e-12) + 1e-9
        assert ub >= opt - 1e-9 and abs(O.qap_cost(inst.F, inst.D, inst.B, ub_perm) - ub) < 1e-9
        assert O.qap_cost(inst.F, inst.D, inst.B, perm) >= ub - 1e-9 and lb == lbs[-1]
        assert best == lbs.max() and its == 50


def test_canonical_state_close_to_oracle(R):
    """Canonical duals: after 20 iterations at n=8 the GPU's D^, C^ and duals agree
    with the oracle's within a tolerance scaled to the data."""
    inst = I.config(1)
    iters = 20
    lbs, _, D, C, duals, _, _, _ = _gpu_run(R, inst, iters, 1)
    ost = O.setup(inst.F, inst.D, inst.B)
    for it in range(iters - 1):
        O.iterate(ost, _oprm(), 1)
    out = O.iterate(O.State(ost.n, ost.const, ost.bprime, ost.Chat.copy(), ost.Dhat.copy()), _oprm(), 1)
    scale = np.abs(ost.Dhat).max() + np.abs(ost.Chat).max()
    assert np.abs(D - ost.Dhat).max() <= 1e-9 * scale
    assert np.abs(C - ost.Chat).max() <= 1e-9 * scale
    assert np.abs(duals["xi"] - out.xi).max() <= 1e-9 * scale
    assert abs(lbs[-1] - (ost.const + out.lb)) <= 1e-9 * abs(out.lb)


def test_zero_sum_invariants_on_gpu(R):
    inst = I.random_instance(7, 2, with_b=True)
    n = 7
    _, _, D, C, _, _, _, _ = _gpu_run(R, inst, 15, 1)
    st0 = O.setup(inst.F, inst.D, inst.B)
    import itertools
    scale = np.abs(D).max() + 1
    for i, j, k in itertools.combinations(range(n), 3):
        for p, q, r in itertools.permutations(range(n), 3):
            mem = [((i, j, k), (p, q, r)), ((i, k, j), (p, r, q)), ((j, i, k), (q, p, r)),
                   ((j, k, i), (q, r, p)), ((k, i, j), (r, p, q)), ((k, j, i), (r, q, p))]
            assert abs(sum(D[O.z_index(n, *f, *l)] for f, l in mem)) <= 1e-12 * scale * 6
    for i in range(n):
        for j in range(n):
            for p in range(n):
                for q in range(n):
                    if i != j and p != q:
                        a, b = O.tile_index(n, i, p, j, q), O.tile_index(n, j, q, i, p)
                        assert abs((C[a] + C[b]) - (st0.Chat[a] + st0.Chat[b])) <= 1e-9 * (abs(st0.Chat[a]) + 1)


def test_feasibility_stop_gives_optimum(R):
    """F = 0: all y/z slacks vanish, the feasibility check stops the ascent after one
    iteration and the bound is the optimum."""
    inst = I.random_instance(7, 2, with_b=True)
    F = np.zeros_like(inst.F)
    opt, _ = O.qap_brute(F, inst.D, inst.B)
    with R.Context(F, inst.D, inst.B, prm=R.params(feas_tol=1e-9)) as ctx:
        lbs, done = ctx.iterate(10)
        st = ctx.stats()
    assert done == 1 and st[7] == 1
    assert abs(lbs[0] - opt) < 1e-9 and np.isnan(lbs[1:]).all()


def test_import_state_resync(R):
    """Checkpoint/restore: importing the oracle's state at iteration k makes the next
    GPU solve reproduce the oracle's bound at k (canonical duals)."""
    inst = I.config(2)
    ost = O.setup(inst.F, inst.D, inst.B)
    for _ in range(30):
        O.iterate(ost, _oprm(), 1)
    out = O.iterate(O.State(ost.n, ost.const, ost.bprime, ost.Chat.copy(), ost.Dhat.copy()), _oprm(), 1)
    with R.Context(inst.F, inst.D, inst.B, prm=_prm(R, 1)) as ctx:
        ctx.iterate(3)
        ctx.import_state(ost.Dhat, ost.Chat)
        lbs, _ = ctx.iterate(1)
    assert abs(lbs[0] - out.lb) <= 1e-9 * abs(out.lb)


def test_raw_bit_exact_n22_banded_move(R):
    """From n = 22 on the z move hands its classes to a warp's lanes in bands of
    8 q x 4 r instead of along r; every class is still moved by one thread with
    the oracle's arithmetic, so raw-duals bounds and the moved state stay
    bit-identical to the oracle (two iterations: the second applies the first
    ascent step to all 85 M z entries)."""
    inst = I.random_instance(22, 17, with_b=True, asymmetric=True)
    iters = 2
    with R.Context(inst.F, inst.D, inst.B, prm=_prm(R, 0)) as ctx:
        lbs, done = ctx.iterate(iters)
        D, C = ctx.export_state()
    assert done == iters
    ost = O.setup(inst.F, inst.D, inst.B)
    ref = []
    for it in range(iters):
        before = O.State(ost.n, ost.const, ost.bprime, ost.Chat.copy(), ost.Dhat.copy()) if it == iters - 1 else None
        out = O.iterate(ost, _oprm(), 0, threads=O.max_threads() or 1)
        ref.append(ost.const + out.lb)
    assert np.array_equal(lbs, np.array(ref)), (lbs, ref)
    assert np.array_equal(D, before.Dhat) and np.array_equal(C, before.Chat)


# ------------------------------------------------------- full-size sampled ----
def test_n20_full_size_sampled(R):
    """n = 20 dense uniform 0..99 (144,400 Z-LAPs of size 18 per iteration), in the
    launch configuration the benchmark uses: the first bound equals the
    Gilmore-Lawler closed form, the next ones match the oracle within 1e-6, and
    sampled Z-LAPs of the GPU's state are re-solved by the oracle LAP."""
    from scipy.optimize import linear_sum_assignment
    inst = I.config(3)
    n = 20
    F, Dm = inst.F, inst.D
    L = np.zeros((n, n))
    for i in range(n):
        for p in range(n):
            L[i, p] = F[i, i] * Dm[p, p] + float(np.dot(np.sort(np.delete(F[i], i)), np.sort(np.delete(Dm[p], p))[::-1]))
    r, c = linear_sum_assignment(L)
    gl = L[r, c].sum()
    iters = 3
    with R.Context(inst.F, inst.D, inst.B, prm=_prm(R, 1)) as ctx:
        lbs, _ = ctx.iterate(iters)
        D, C = ctx.export_state()
        duals = ctx.duals()
    assert abs(lbs[0] - gl) <= 1e-9 * gl
    _, ref, _ = O.run(inst.F, inst.D, inst.B, iters=iters, dual_mode=1, threads=O.max_threads() or 1)
    assert np.max(np.abs(lbs - np.array(ref)) / np.abs(ref)) <= 1e-6
    m = n - 2
    T = O.num_tiles(n)
    rng = np.random.default_rng(0)
    for t in rng.choice(T, 200, replace=False):
        tile = D[t * m * m:(t + 1) * m * m].reshape(m, m)
        o = O.lap(tile, canonical=True)
        xi, psi = duals["xi"][t * m:(t + 1) * m], duals["psi"][t * m:(t + 1) * m]
        scale = max(1.0, np.abs(tile).max())
        assert abs(xi.sum() + psi.sum() - o.value) <= 1e-9 * scale * m
        assert (tile - xi[:, None] - psi[None, :]).min() >= -1e-9 * scale
        assert np.allclose(xi, o.u, atol=1e-9 * scale) and np.allclose(psi, o.v, atol=1e-9 * scale)


def test_stall_and_gap_stops(R):
    """Early termination (Section 5): the ascent stops once the best bound gains less
    than stall_tol*|UB| over stall_window iterations; min_gap stops on the gap."""
    inst = I.config(2)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0)) as ctx:
        full, _ = ctx.iterate(200)
        _, _, ub, _, _, _ = ctx.bound()
    W, tol = 10, 0.0005
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, stall_window=W, stall_tol=tol)) as ctx:
        lbs, done = ctx.iterate(200)
        st = ctx.stats()
        _, _, ub2, _, _, _ = ctx.bound()
    assert st[7] == 3 and W < done < 200
    assert np.array_equal(lbs[:done], full[:done])       # same trajectory up to the stop
    best = np.maximum.accumulate(full)
    k = done - 1
    assert best[k] - best[k - W] < tol * ub2             # the rule fired at k ...
    assert all(best[j] - best[j - W] >= tol * ub2 for j in range(W, k))   # ... and not before (same UB seen)
    gap_stop = (ub - best[60]) / ub * (1 + 1e-9)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, min_gap=gap_stop, ub=ub)) as ctx:
        _, done = ctx.iterate(200)
        assert ctx.stats()[7] == 2 and done <= 61


@pytest.mark.parametrize("K", [60, 101, 150])
def test_gap_stop_inside_graph_replays(R, K):
    """The min_gap stop lands on the same iteration whether it fires among the
    first 64 iterations (launched kernel by kernel) or inside a replay of the
    eight-iteration graph (the device flag makes the rest of that replay a no-op)."""
    inst = I.config(2)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0)) as ctx:
        full, _ = ctx.iterate(200)
        _, _, ub, _, _, _ = ctx.bound()
    best = np.maximum.accumulate(full)
    gap_stop = (ub - best[K]) / ub * (1 + 1e-9)
    first = int(np.argmax((ub - best) / ub < gap_stop))
    assert (first >= 64) == (K >= 64)  # the two launch paths are both exercised
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, min_gap=gap_stop, ub=ub)) as ctx:
        lbs, done = ctx.iterate(200)
        assert ctx.stats()[7] == 2 and done == first + 1
        assert np.array_equal(lbs[:done], full[:done])
        assert ctx.bound()[5] == done  # no iteration counted after the stop


def test_n30_full_size_sampled(R):
    """n = 30, Manhattan 5x6 grid (756,900 Z-LAPs of size 28, 4.75 GB z array): the
    first bound equals the Gilmore-Lawler closed form, the second matches the
    oracle within 1e-6, sampled Z-LAPs re-solved by the oracle LAP."""
    from scipy.optimize import linear_sum_assignment
    inst = I.config(5)
    n = 30
    F, Dm = inst.F, inst.D
    L = np.zeros((n, n))
    for i in range(n):
        for p in range(n):
            L[i, p] = F[i, i] * Dm[p, p] + float(np.dot(np.sort(np.delete(F[i], i)), np.sort(np.delete(Dm[p], p))[::-1]))
    r, c = linear_sum_assignment(L)
    gl = L[r, c].sum()
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, warm=1)) as ctx:
        lbs, _ = ctx.iterate(2)
        m = n - 2
        T = ctx.T
        rng = np.random.default_rng(3)
        pick = rng.choice(T, 60, replace=False)
        D, _ = ctx.export_state()
        tiles = {int(t): D[t * m * m:(t + 1) * m * m].reshape(m, m).copy() for t in pick}
        del D
        duals = ctx.duals()
    assert abs(lbs[0] - gl) <= 1e-9 * gl
    _, ref, _ = O.run(inst.F, inst.D, inst.B, iters=2, dual_mode=1, threads=O.max_threads() or 1)
    assert np.max(np.abs(lbs - np.array(ref)) / np.abs(ref)) <= 1e-6
    for t, tile in tiles.items():
        o = O.lap(tile, canonical=True)
        xi, psi = duals["xi"][t * m:(t + 1) * m], duals["psi"][t * m:(t + 1) * m]
        scale = max(1.0, np.abs(tile).max())
        assert abs(xi.sum() + psi.sum() - o.value) <= 1e-9 * scale * m
        assert (tile - xi[:, None] - psi[None, :]).min() >= -1e-9 * scale
        assert np.allclose(xi, o.u, atol=1e-9 * scale) and np.allclose(psi, o.v, atol=1e-9 * scale)


@pytest.mark.parametrize("which", ["cfg1", "randB", "partial"])
def test_warm_start_raw_bit_exact_and_canonical_equal(R, which):
    """warm = 1 starts every Z, Y and X LAP from its previous row duals.  Raw
    duals: the trajectory equals the oracle's warm run bit for bit.  Canonical
    duals: the bounds equal those of the cold run (the start does not matter),
    bit for bit, and so does the whole state, in fixed point."""
    partial = None
    if which == "cfg1":
        inst, iters = I.config(1), 25
    elif which == "randB":
        inst, iters = I.random_instance(8, 12, with_b=True, asymmetric=True), 20
    else:
        inst, iters = I.random_instance(10, 13, with_b=True), 15
        partial = -np.ones(10, dtype=np.int32)
        partial[[0, 5]] = [3, 8]
    with R.Context(inst.F, inst.D, inst.B, partial=partial, prm=_prm(R, 0, warm=1)) as ctx:
        raw, _ = ctx.iterate(iters)
    _, ref, _ = O.run(inst.F, inst.D, inst.B, iters=iters, dual_mode=0, partial=partial, warm=True, prm=_oprm())
    assert np.array_equal(raw, np.array(ref))
    for mode in (1, 2):
        out = {}
        for warm in (0, 1):
            with R.Context(inst.F, inst.D, inst.B, partial=partial, prm=_prm(R, mode, warm=warm)) as ctx:
                out[warm], _ = ctx.iterate(iters)
                out[warm, "D"] = ctx.export_state()[0]
        if mode == 1:  # exact arithmetic: the start cannot change anything
            assert np.array_equal(out[1], out[0]) and np.array_equal(out[1, "D"], out[0, "D"])
        assert np.max(np.abs(out[1] - out[0]) / np.maximum(1.0, np.abs(out[0]))) <= 1e-9


def test_max_residual_size_n32_sampled(R):
    """The largest residual size a context takes (n = 32: 984,064 Z-LAPs of size 30,
    a 7.1 GB z array, 30 of 32 lanes per LAP): the first bound equals the
    Gilmore-Lawler closed form; after three iterations the bound has not
    decreased and sampled Z tiles (copied from the device state) re-solved by
    the oracle's LAP give the GPU's optimum and canonical duals."""
    from scipy.optimize import linear_sum_assignment
    inst = I.grid_instance("n32_grid4x8", 4, 8, 9, 0.5, 5, 3)
    n, m = 32, 30
    F, Dm = inst.F, inst.D
    L = np.zeros((n, n))
    for i in range(n):
        for p in range(n):
            L[i, p] = F[i, i] * Dm[p, p] + float(np.dot(np.sort(np.delete(F[i], i)), np.sort(np.delete(Dm[p], p))[::-1]))
    r, c = linear_sum_assignment(L)
    gl = L[r, c].sum()
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, warm=1)) as ctx:
        lbs, done = ctx.iterate(3)
        T, E = ctx.T, ctx.E
        assert T == 984064 and E == T * m * m
        D = torch.empty(E, dtype=torch.float64, device="cuda")
        R.rlt2_export_state(ctx.ctx, D, None, on_device=1)
        torch.cuda.synchronize()
        rng = np.random.default_rng(4)
        pick = [int(t) for t in rng.choice(T, 40, replace=False)] + [0, T - 1]
        tiles = {t: D[t * m * m:(t + 1) * m * m].view(m, m).cpu().numpy().copy() for t in pick}
        del D
        torch.cuda.empty_cache()
        duals = ctx.duals()
    assert done == 3
    assert abs(lbs[0] - gl) <= 1e-9 * gl
    assert np.all(np.diff(lbs) >= -1e-9 * np.abs(lbs[:-1]))
    for t, tile in tiles.items():
        o = O.lap(tile, canonical=True)
        xi, psi = duals["xi"][t * m:(t + 1) * m], duals["psi"][t * m:(t + 1) * m]
        scale = max(1.0, np.abs(tile).max())
        assert abs(xi.sum() + psi.sum() - o.value) <= 1e-9 * scale * m
        assert np.allclose(xi, o.u, atol=1e-9 * scale) and np.allclose(psi, o.v, atol=1e-9 * scale)


@pytest.mark.parametrize("mode", [0, 1])
def test_direct_launches_and_graph_replay_agree(R, mode):
    """A context launches its first 64 iterations kernel by kernel and later ones
    as CUDA-graph replays (of eight iterations, then of one); splitting a run
    over many calls, or running it in one call, gives the same trajectory bit
    for bit (raw duals; canonical duals in fixed point, whose Z stage takes its
    LAPs from a queue that the y-move launch resets every iteration)."""
    inst = I.random_instance(9, 81, with_b=True, asymmetric=True)
    prm = R.params(dual_mode=mode, feas_tol=0.0, warm=1)
    with R.Context(inst.F, inst.D, inst.B, prm=prm) as a:
        one, _ = a.iterate(90)
    parts = []
    with R.Context(inst.F, inst.D, inst.B, prm=prm) as b:
        for k in (5, 7, 20, 30, 28):
            h, _ = b.iterate(k)
            parts.append(h)
    assert np.array_equal(one, np.concatenate(parts))


def test_contexts_on_two_host_threads(R):
    """Separate contexts are independent: two host threads each create and run
    their own context (own stream) at the same time, and each gets exactly the
    trajectory of a run on its own (raw duals)."""
    import threading
    insts = [I.random_instance(9, 91, with_b=True), I.random_instance(10, 92, with_b=True, asymmetric=True)]
    prm = R.params(dual_mode=0, feas_tol=0.0, warm=1)
    ref = []
    for inst in insts:
        with R.Context(inst.F, inst.D, inst.B, prm=prm) as ctx:
            ref.append(ctx.iterate(80)[0])
    got = [None, None]

    def work(k):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            with R.Context(insts[k].F, insts[k].D, insts[k].B, prm=prm, stream=s.cuda_stream) as ctx:
                got[k] = ctx.iterate(80)[0]

    th = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for k in range(2):
        assert np.array_equal(got[k], ref[k])
