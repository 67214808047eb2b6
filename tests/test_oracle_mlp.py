"""Pins for the oracle's learned-warm-start pieces: FP64 MLP gradients against
central finite differences, BF16 rounding against torch, feature invariances."""
import numpy as np
import pytest

import oracle as O


def _net(rng, H):
    W1 = rng.normal(size=(O.MLP_IN, H)).astype(np.float32) * 0.3
    W2 = rng.normal(size=(H, H)).astype(np.float32) * (1.0 / np.sqrt(H))
    b1 = rng.normal(size=H).astype(np.float32) * 0.1
    b2 = rng.normal(size=H).astype(np.float32) * 0.1
    w3 = rng.normal(size=H).astype(np.float32) * 0.3
    return [W1, b1, W2, b2, w3, 0.05]


@pytest.mark.parametrize("seed", [0, 1])
def test_mlp_gradients_match_finite_differences(seed):
    rng = np.random.default_rng(seed)
    H, N = 8, 6
    X = rng.normal(size=(N, O.MLP_IN)).astype(np.float32)
    t = rng.normal(size=N)
    net = _net(rng, H)
    loss, *g = O.mlp_grads(X, *net, t, bf16_acts=False)
    eps = 2.0 ** -12

    def L(params):
        out, _, _ = O.mlp_forward(X, *params, bf16_acts=False)
        return 0.5 * np.mean((out - t) ** 2)

    assert abs(loss - L(net)) < 1e-12
    for pi in range(5):
        arr = net[pi]
        for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(6)]:
            p = [a.copy() if isinstance(a, np.ndarray) else a for a in net]
            q = [a.copy() if isinstance(a, np.ndarray) else a for a in net]
            p[pi][idx] += np.float32(eps)
            q[pi][idx] -= np.float32(eps)
            h = float(p[pi][idx]) - float(q[pi][idx])
            fd = (L(p) - L(q)) / h
            assert abs(fd - g[pi][idx]) <= 1e-6 + 1e-4 * abs(fd), (pi, idx, fd, g[pi][idx])
    fd3 = (L(net[:5] + [net[5] + eps]) - L(net[:5] + [net[5] - eps])) / (2 * eps)
    assert abs(fd3 - g[5]) <= 1e-6 + 1e-4 * abs(fd3)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    xs = np.concatenate([rng.normal(size=2000) * 10 ** rng.uniform(-6, 6, 2000), [0.0, -0.0, 1.0, 1.00390625, 3.0]])
    xs = xs.astype(np.float32)
    ref = torch.from_numpy(xs).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([O.bf16_round(float(x)) for x in xs], dtype=np.float32)
    assert np.array_equal(got, ref)


def test_f32_trunc_truncates():
    rng = np.random.default_rng(3)
    xs = rng.normal(size=500) * 10 ** rng.uniform(-10, 10, 500)
    for x in xs:
        y = O.f32_trunc(x)
        assert abs(y) <= abs(x) and np.sign(y) == np.sign(x)
        assert abs(x) - abs(y) < np.spacing(np.float32(abs(y))) * 1.0000001
        assert O.f32_trunc(float(np.float32(y))) == y
    assert O.f32_trunc(1.5) == 1.5 and O.f32_trunc(-2.25) == -2.25


def test_features_invariances():
    """Column shifts do not change the features of an integer tile; column
    permutations and power-of-two scalings never do; rows are sorted in [0, 1]."""
    rng = np.random.default_rng(4)
    m = 9
    c = rng.integers(0, 50, (m, m)).astype(np.float64)
    u = rng.normal(size=m) * 5
    f0, t0, s0 = O.mlp_features(c, prev_u=u, target_u=u)
    assert np.all(np.diff(f0[:, :m], axis=1) >= 0) and f0[:, :m].min() == 0.0 and f0[:, :m].max() <= 1.0
    assert np.all(f0[:, m:32] == 0) and np.all(f0[:, 33] == m / 32)
    f1, _, _ = O.mlp_features(c + rng.integers(-20, 20, m)[None, :].astype(float), prev_u=u)
    assert np.array_equal(f0[:, :32], f1[:, :32])
    perm = rng.permutation(m)
    f2, _, _ = O.mlp_features(c[:, perm], prev_u=u)
    assert np.array_equal(f0, f2)
    f3, t3, s3 = O.mlp_features(c * 8.0, prev_u=u * 8.0, target_u=u * 8.0)
    assert np.array_equal(f0, f3) and np.array_equal(t0, t3) and s3 == 8 * s0
