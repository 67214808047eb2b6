"""Learned warm start on the GPU: features, tensor-core forward/backward and the
exact-bound guarantee, against the CPU oracle's FP64 reference."""
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


def _tiles(rng, nt, m):
    kind = rng.integers(0, 3)
    if kind == 0:
        return rng.integers(0, 40, (nt, m, m)).astype(np.float64)
    return rng.normal(size=(nt, m, m)) * 10 ** rng.uniform(-2, 3)


def _bf(x):
    return np.array([O.bf16_round(float(v)) for v in np.ravel(x)], dtype=np.float32).reshape(np.shape(x))


@pytest.mark.parametrize("m", [1, 5, 12, 18, 28, 32])
def test_features_bit_identical(R, m):
    rng = np.random.default_rng(m)
    nt = 40
    tiles = _tiles(rng, nt, m)
    prev = rng.normal(size=(nt, m)) * 3
    tgt = rng.normal(size=(nt, m)) * 3
    mlp = R.Mlp(64, seed=1)
    mlp.add_samples(torch.from_numpy(tiles).cuda(), torch.from_numpy(tgt).cuda(), torch.from_numpy(prev).cuda())
    X, T = mlp.samples()
    assert X.shape == (nt * m, 34)
    for t in range(nt):
        f, tt, _ = O.mlp_features(tiles[t], prev_u=prev[t], target_u=tgt[t])
        assert np.array_equal(X[t * m:(t + 1) * m], _bf(f))
        assert np.array_equal(T[t * m:(t + 1) * m], tt)


def _random_weights(rng, H):
    W1 = _bf(rng.normal(size=(34, H)).astype(np.float32) * 0.3)
    W2 = _bf(rng.normal(size=(H, H)).astype(np.float32) / np.sqrt(H))
    return [W1, (rng.normal(size=H) * 0.1).astype(np.float32), W2, (rng.normal(size=H) * 0.1).astype(np.float32),
            (rng.normal(size=H) * 0.2).astype(np.float32), 0.07]


@pytest.mark.parametrize("H", [64, 256])
def test_forward_matches_oracle(R, H):
    rng = np.random.default_rng(H)
    m, nt = 18, 300
    tiles = _tiles(rng, nt, m)
    prev = rng.normal(size=(nt, m))
    net = _random_weights(rng, H)
    mlp = R.Mlp(H)
    mlp.set_weights(*net)
    u0 = torch.empty(nt, m, dtype=torch.float64, device="cuda")
    mlp.predict(torch.from_numpy(tiles).cuda(), u0, torch.from_numpy(prev).cuda())
    u0 = u0.cpu().numpy()
    for t in range(0, nt, 7):
        f, _, s = O.mlp_features(tiles[t], prev_u=prev[t])
        out, _, _ = O.mlp_forward(f, *net, bf16_acts=True)
        ref = prev[t] + (np.float32(out.astype(np.float32)) * np.float32(s)).astype(np.float64)
        assert np.allclose(u0[t], ref, rtol=2e-3, atol=2e-3 * abs(s)), (u0[t], ref)


@pytest.mark.parametrize("H", [64, 256, 320])
def test_gradients_match_oracle(R, H):
    """Tensor-core backward (BF16 activations, FP32 accumulation) vs the FP64
    oracle with the same BF16 rounding points: relative error <= 1e-2 per block.
    Widths up to 256 run the tcgen05 GEMMs, 320 the mma.sync ones."""
    rng = np.random.default_rng(10 + H)
    m, nt = 14, 150
    tiles = _tiles(rng, nt, m)
    prev = rng.normal(size=(nt, m))
    tgt = rng.normal(size=(nt, m))
    net = _random_weights(rng, H)
    mlp = R.Mlp(H)
    mlp.set_weights(*net)
    mlp.add_samples(torch.from_numpy(tiles).cuda(), torch.from_numpy(tgt).cuda(), torch.from_numpy(prev).cuda())
    X, T = mlp.samples()
    rows = X.shape[0]
    loss, *g = mlp.grad(rows)
    oloss, *og = O.mlp_grads(X, *net, T.astype(np.float64), bf16_acts=True)
    assert abs(loss - oloss) <= 1e-3 * abs(oloss)
    for name, a, b in zip(["W1", "b1", "W2", "b2", "w3", "b3"], g, og):
        a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert err <= 1e-2, (name, err)


def test_gradients_several_tiles_per_persistent_cta(R):
    """The tall products run on persistent CTAs (one per SM, two per 128-row
    tile at H = 256) that take several 128-row tiles each, alternating two TMEM
    accumulators and two staging tiles: 41,400 rows (324 tiles, the last
    ragged; four or more per CTA on a 152-SM GB300) against the FP64 oracle."""
    rng = np.random.default_rng(77)
    m, nt, H = 18, 2300, 256
    tiles = _tiles(rng, nt, m)
    prev = rng.normal(size=(nt, m))
    tgt = rng.normal(size=(nt, m))
    net = _random_weights(rng, H)
    mlp = R.Mlp(H)
    mlp.set_weights(*net)
    mlp.add_samples(torch.from_numpy(tiles).cuda(), torch.from_numpy(tgt).cuda(), torch.from_numpy(prev).cuda())
    X, T = mlp.samples()
    rows = X.shape[0]
    assert rows == nt * m and rows % 128 != 0 and rows // 128 >= 300
    loss, *g = mlp.grad(rows)
    oloss, *og = O.mlp_grads(X, *net, T.astype(np.float64), bf16_acts=True)
    assert abs(loss - oloss) <= 1e-3 * abs(oloss)
    for name, a, b in zip(["W1", "b1", "W2", "b2", "w3", "b3"], g, og):
        a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert err <= 1e-2, (name, err)
    mlp.close()


def test_training_reduces_loss_and_augmentations(R):
    """Train on (tile, canonical dual) pairs harvested from an n=12 ascent, then
    warm-start another n=12 ascent: bounds identical to the cold run (canonical
    duals), fewer augmenting searches than cold."""
    inst = I.config(2)
    n, m = 12, 10
    T = n * n * (n - 1) * (n - 1)
    mlp = R.Mlp(256, seed=3)
    with R.Context(inst.F, inst.D, prm=R.params(feas_tol=0.0)) as ctx:
        prev = None
        for it in range(12):
            ctx.iterate(1)
            D, _ = ctx.export_state()
            xi = ctx.duals()["xi"]
            if it >= 2:
                mlp.add_samples(torch.from_numpy(D.reshape(T, m, m)).cuda(), torch.from_numpy(xi.reshape(T, m)).cuda(),
                                torch.from_numpy(prev.reshape(T, m)).cuda())
            prev = xi.copy()
    hist = mlp.fit(300, batch_rows=8192, lr=2e-3)
    assert hist[-20:].mean() < 0.5 * hist[:5].mean()
    inst2 = I.grid_instance("n12b", 3, 4, 9, 0.5, 11, 40)
    res = {}
    for warm in (0, 2):
        with R.Context(inst2.F, inst2.D, prm=R.params(feas_tol=0.0, warm=warm)) as ctx:
            if warm == 2:
                ctx.set_mlp(mlp)
            lbs, _ = ctx.iterate(40)
            res[warm] = (lbs, ctx.stats())
    assert np.max(np.abs(res[2][0] - res[0][0]) / np.abs(res[0][0])) <= 1e-6
    assert res[2][1][1] < res[0][1][1]


def test_inference_wait_timeout_is_detected(R):
    """Failure detection without a fault: the tensor-core inference kernel is run
    with its MMA commit withheld, its bounded mbarrier wait runs out, the error
    is reported to the host and the device stays usable (a normal prediction
    afterwards still matches the oracle)."""
    mlp = R.Mlp(256)
    st = R.lib().rlt2_mlp_check_wait_timeout(mlp.ptr)
    assert st == R.RLT2_ETIMEOUT
    rng = np.random.default_rng(5)
    m, nt = 18, 40
    tiles = _tiles(rng, nt, m)
    prev = rng.normal(size=(nt, m))
    net = _random_weights(rng, 256)
    mlp.set_weights(*net)
    u0 = torch.empty(nt, m, dtype=torch.float64, device="cuda")
    mlp.predict(torch.from_numpy(tiles).cuda(), u0, torch.from_numpy(prev).cuda())
    u0 = u0.cpu().numpy()
    f, _, s = O.mlp_features(tiles[3], prev_u=prev[3])
    out, _, _ = O.mlp_forward(f, *net, bf16_acts=True)
    ref = prev[3] + (np.float32(out.astype(np.float32)) * np.float32(s)).astype(np.float64)
    assert np.allclose(u0[3], ref, rtol=2e-3, atol=2e-3 * abs(s))


def test_gemm_wait_timeout_is_detected(R):
    """Failure detection without a fault for the persistent training GEMM: its
    MMAs are withheld, the producer's and the epilogue's bounded waits run out,
    ETIMEOUT reaches the host, and the device stays usable (gradients on the
    next call still match the oracle)."""
    mlp = R.Mlp(256)
    st = R.lib().rlt2_mlp_check_gemm_wait_timeout(mlp.ptr)
    assert st == R.RLT2_ETIMEOUT
    rng = np.random.default_rng(21)
    m, nt = 14, 150
    tiles = _tiles(rng, nt, m)
    prev = rng.normal(size=(nt, m))
    tgt = rng.normal(size=(nt, m))
    net = _random_weights(rng, 256)
    mlp.set_weights(*net)
    mlp.add_samples(torch.from_numpy(tiles).cuda(), torch.from_numpy(tgt).cuda(), torch.from_numpy(prev).cuda())
    X, T = mlp.samples()
    loss, *g = mlp.grad(X.shape[0])
    oloss, *og = O.mlp_grads(X, *net, T.astype(np.float64), bf16_acts=True)
    assert abs(loss - oloss) <= 1e-3 * abs(oloss)
    for a, b in zip(g, og):
        a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        assert np.linalg.norm(a - b) <= 1e-2 * max(np.linalg.norm(b), 1e-30)
    mlp.close()


def test_trained_network_against_both_starts_on_held_out_grid(R):
    """The shipped network (weights/warmstart_h256.npz, trained on n = 20..25
    runs) on a held-out n = 22 grid (seed 99, never trained on), 12 iterations:
    bounds identical for the cold, previous-dual and learned starts (the exact
    Hungarian finishes every solve); the learned start needs fewer Z augmenting
    searches than the cold Hungarian but more than the previous-dual start (the
    method without the network): the network is a net loss against it."""
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1710_03732_gb300",
                        "weights", "warmstart_h256.npz")
    mlp = R.Mlp(256)
    mlp.load(path)
    inst = I.grid_instance("heldout_n22_2x11", 2, 11, 9, 0.5, 99, 0)
    res = {}
    for warm in (0, 1, 2):
        with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, warm=warm)) as ctx:
            if warm == 2:
                ctx.set_mlp(mlp)
            lbs, done = ctx.iterate(12)
            assert done == 12
            res[warm] = (lbs, int(ctx.stats()[1]))
    mlp.close()
    assert np.max(np.abs(res[2][0] - res[0][0]) / np.abs(res[0][0])) <= 1e-9
    assert np.array_equal(res[1][0], res[0][0])
    cold, prev, learned = res[0][1], res[1][1], res[2][1]
    assert learned < cold
    assert learned > prev
