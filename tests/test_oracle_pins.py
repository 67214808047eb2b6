"""Pins for the CPU oracle: each check ties the oracle to something other than
itself (brute force, a library routine, a closed form, an invariant the paper
proves, or a hand-computed example)."""
import itertools

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment, linprog

import oracle as O
from paper_1710_03732_gb300 import instances as I

P1 = O.params_array(kz=1.0, ky=0.5, kx=1.0, phi_y=0.5, phi_z=(0.2,) * 5)
P0 = O.params_array(kz=1.0, ky=1.0, kx=1.0, phi_y=0.0, phi_z=(0.2,) * 5)
PX = O.params_array(kz=0.8, ky=0.6, kx=0.9, phi_y=0.3, phi_z=(0.1, 0.3, 0.15, 0.25, 0.2))


def _reduced(c, u, v):
    return c - u[:, None] - v[None, :]


# ---------------------------------------------------------------- LAP ----
@pytest.mark.parametrize("seed", range(6))
def test_lap_vs_brute_force(seed):
    """Hungarian optimum = brute force over all m! assignments (m <= 7);
    duals feasible, complementary slack, and sum u + sum v = value."""
    rng = np.random.default_rng(seed)
    for trial in range(60):
        m = int(rng.integers(1, 8))
        if trial % 3 == 0:
            c = rng.integers(-4, 5, (m, m)).astype(float)  # many ties
        elif trial % 3 == 1:
            c = rng.normal(size=(m, m)) * 10
        else:
            c = np.zeros((m, m))  # fully degenerate
        r = O.lap(c)
        best, _ = O.lap_brute(c)
        scale = max(1.0, np.abs(c).max())
        assert abs(r.value - best) <= 1e-12 * scale * m
        red = _reduced(c, r.u, r.v)
        assert red.min() >= -1e-12 * scale
        assert sorted(r.row_to_col.tolist()) == list(range(m))
        for i in range(m):
            assert abs(red[i, r.row_to_col[i]]) <= 1e-12 * scale
        assert abs(r.u.sum() + r.v.sum() - best) <= 1e-11 * scale * m


def test_lap_vs_scipy_large():
    rng = np.random.default_rng(7)
    for m in (8, 13, 18, 28, 32):
        c = rng.normal(size=(m, m)) * 1000
        r = O.lap(c)
        i, j = linear_sum_assignment(c)
        assert abs(r.value - c[i, j].sum()) <= 1e-9 * abs(c[i, j].sum())


def test_lap_special_cases():
    m = 9
    c = np.full((m, m), 5.0) - 4.0 * np.eye(m)  # diagonal dominant
    r = O.lap(c)
    assert r.row_to_col.tolist() == list(range(m)) and r.value == m * 1.0
    c = np.full((m, m), 3.25)
    assert O.lap(c).value == m * 3.25


def test_lap_warm_start_same_optimum():
    rng = np.random.default_rng(3)
    for _ in range(40):
        m = int(rng.integers(2, 12))
        c = rng.normal(size=(m, m))
        u0 = rng.normal(size=m)
        a, b = O.lap(c), O.lap(c, u0=u0)
        assert abs(a.value - b.value) <= 1e-12 * m
        assert _reduced(c, b.u, b.v).min() >= -1e-12


def _canonical_by_lp(c, opt):
    """max sum(u) s.t. u_r + v_c <= c_rc, sum u + sum v = opt, u_0 = 0 (HiGHS)."""
    m = c.shape[0]
    nv = 2 * m
    A_ub = np.zeros((m * m, nv))
    b_ub = np.zeros(m * m)
    for r in range(m):
        for col in range(m):
            A_ub[r * m + col, r] = 1
            A_ub[r * m + col, m + col] = 1
            b_ub[r * m + col] = c[r, col]
    A_eq = np.zeros((2, nv))
    A_eq[0, :] = 1
    A_eq[1, 0] = 1
    res = linprog(-np.r_[np.ones(m), np.zeros(m)], A_ub=A_ub, b_ub=b_ub, A_eq=A_eq, b_eq=[opt, 0.0],
                  bounds=[(None, None)] * nv, method="highs")
    assert res.success
    return res.x[:m], res.x[m:]


def test_canonical_dual_is_lp_pointwise_max():
    """The canonical dual maximises sum(u) over the optimal duals with u_0 = 0 (LP),
    and it is the pointwise maximum, so it equals the LP's u exactly up to tolerance."""
    rng = np.random.default_rng(11)
    for trial in range(25):
        m = int(rng.integers(2, 7))
        c = rng.integers(0, 6, (m, m)).astype(float) if trial % 2 else rng.normal(size=(m, m))
        r = O.lap(c)
        u, v = O.lap_canonical(c, r.row_to_col)
        ul, vl = _canonical_by_lp(c, r.value)
        assert np.allclose(u, ul, atol=1e-7), (c, u, ul)
        assert np.allclose(v, vl, atol=1e-7)


def test_canonical_dual_independent_of_optimal_assignment():
    """With ties, every optimal permutation yields the same canonical dual."""
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(200):
        m = int(rng.integers(3, 6))
        c = rng.integers(0, 3, (m, m)).astype(float)
        best, _ = O.lap_brute(c)
        opts = [p for p in itertools.permutations(range(m)) if abs(sum(c[i, p[i]] for i in range(m)) - best) < 1e-12]
        if len(opts) < 2:
            continue
        ref = O.lap_canonical(c, np.array(opts[0], dtype=np.int32))
        for p in opts[1:]:
            u, v = O.lap_canonical(c, np.array(p, dtype=np.int32))
            assert np.array_equal(u, ref[0]) and np.array_equal(v, ref[1])
        checked += 1
    assert checked > 20


def test_canonical_same_for_warm_and_cold():
    rng = np.random.default_rng(9)
    for _ in range(30):
        m = int(rng.integers(2, 10))
        c = rng.normal(size=(m, m))
        a = O.lap(c, canonical=True)
        b = O.lap(c, u0=rng.normal(size=m), canonical=True)
        assert np.allclose(a.u, b.u, atol=1e-12) and np.allclose(a.v, b.v, atol=1e-12)


# ---------------------------------------------------------------- QAP ----
def _qap_brute_py(F, D, B):
    n = F.shape[0]
    best = np.inf
    for p in itertools.permutations(range(n)):
        s = sum(B[i, p[i]] for i in range(n)) + sum(F[i, j] * D[p[i], p[j]] for i in range(n) for j in range(n))
        best = min(best, s)
    return best


def test_qap_brute_vs_python():
    for seed in range(4):
        inst = I.random_instance(6, seed, with_b=True, asymmetric=True)
        val, perm = O.qap_brute(inst.F, inst.D, inst.B)
        assert val == _qap_brute_py(inst.F, inst.D, inst.B)
        assert O.qap_cost(inst.F, inst.D, inst.B, perm) == val


def _residual_cost(st, perm):
    """Residual QAP objective from the oracle's reduced data: sum b' + sum C over i != j."""
    n = st.n
    s = sum(st.bprime[i * n + perm[i]] for i in range(n))
    for i in range(n):
        for j in range(n):
            if i != j:
                s += st.Chat[O.tile_index(n, i, perm[i], j, perm[j])]
    return s


def test_setup_partial_assignment_reduction():
    """const + residual objective == full QAP objective for every completion."""
    rng = np.random.default_rng(2)
    for seed in range(3):
        inst = I.random_instance(6, seed, with_b=True, asymmetric=True)
        part = -np.ones(6, dtype=np.int32)
        fac = rng.permutation(6)[:2]
        loc = rng.permutation(6)[:2]
        part[fac] = loc
        st = O.setup(inst.F, inst.D, inst.B, part)
        free_f = [i for i in range(6) if part[i] < 0]
        free_l = [p for p in range(6) if p not in part]
        for sig in itertools.permutations(range(st.n)):
            full = part.copy()
            for a, b in enumerate(sig):
                full[free_f[a]] = free_l[b]
            assert abs(st.const + _residual_cost(st, sig) - O.qap_cost(inst.F, inst.D, inst.B, full)) < 1e-9


def _gilmore_lawler(F, D, B):
    """Iteration-0 bound in closed form: with D^ = 0 every Z-LAP is 0, so each
    Y-LAP(i,p) is a min scalar product (rearrangement inequality)."""
    n = F.shape[0]
    L = np.zeros((n, n))
    for i in range(n):
        for p in range(n):
            f = np.sort(np.delete(F[i], i))
            d = np.sort(np.delete(D[p], p))[::-1]
            L[i, p] = B[i, p] + F[i, i] * D[p, p] + float(np.dot(f, d))
    r, c = linear_sum_assignment(L)
    return L[r, c].sum()


@pytest.mark.parametrize("which", ["cfg1", "cfg2", "randB", "asym"])
@pytest.mark.parametrize("dual_mode", [0, 1])
def test_iteration0_is_gilmore_lawler(which, dual_mode):
    inst = {"cfg1": lambda: I.config(1), "cfg2": lambda: I.config(2),
            "randB": lambda: I.random_instance(7, 3, with_b=True),
            "asym": lambda: I.random_instance(7, 4, with_b=True, asymmetric=True)}[which]()
    st = O.setup(inst.F, inst.D, inst.B)
    out = O.iterate(st, P1, dual_mode)
    gl = _gilmore_lawler(inst.F, inst.D, inst.B)
    assert abs(out.lb - gl) <= 1e-9 * max(1.0, abs(gl))


@pytest.mark.parametrize("prm", [P1, P0, PX], ids=["P1", "P0", "PX"])
@pytest.mark.parametrize("dual_mode", [0, 1])
def test_bound_valid_and_monotone_small(prm, dual_mode):
    """LB <= OPT (weak duality, Eq. 2.18) and non-decreasing (Theorem 1)."""
    for seed, n in [(0, 5), (1, 6), (2, 7)]:
        inst = I.random_instance(n, seed, with_b=True, asymmetric=(seed == 1))
        opt, _ = O.qap_brute(inst.F, inst.D, inst.B)
        _, lbs, _ = O.run(inst.F, inst.D, inst.B, iters=25, prm=prm, dual_mode=dual_mode)
        for a, b in zip(lbs, lbs[1:]):
            assert b >= a - 1e-9 * max(1.0, abs(a))
        assert max(lbs) <= opt * (1 + 1e-12) + 1e-9


def test_config1_bound_vs_brute_force():
    """n=8, 2x4 grid, 50 iterations: bound below the 8! brute-force optimum, monotone."""
    inst = I.config(1)
    opt, _ = O.qap_brute(inst.F, inst.D, inst.B)
    _, lbs, _ = O.run(inst.F, inst.D, inst.B, iters=50)
    assert all(b >= a - 1e-9 * abs(a) for a, b in zip(lbs, lbs[1:]))
    assert max(lbs) <= opt * (1 + 1e-12) + 1e-9
    assert lbs[-1] > lbs[0]  # the ascent makes progress


def test_partial_node_bound_below_node_optimum():
    inst = I.random_instance(8, 5, with_b=True)
    part = -np.ones(8, dtype=np.int32)
    part[[1, 4]] = [6, 0]
    best = np.inf
    free_f = [i for i in range(8) if part[i] < 0]
    free_l = [p for p in range(8) if p not in part]
    for sig in itertools.permutations(free_l):
        full = part.copy()
        full[free_f] = sig
        best = min(best, O.qap_cost(inst.F, inst.D, inst.B, full))
    _, lbs, _ = O.run(inst.F, inst.D, inst.B, iters=20, partial=part)
    assert max(lbs) <= best + 1e-9
    assert all(b >= a - 1e-9 * abs(a) for a, b in zip(lbs, lbs[1:]))


def test_zero_sum_invariants():
    """The moves only transfer cost inside each symmetry set (Eq. 2.20-2.23):
    every z class sums to its start value 0 and C^_ijpq + C^_jiqp is preserved."""
    inst = I.random_instance(6, 1, with_b=True)
    n = 6
    st = O.setup(inst.F, inst.D, inst.B)
    C0 = st.Chat.copy()
    for _ in range(8):
        O.iterate(st, PX, 1)
    scale = np.abs(st.Dhat).max() + 1
    for i, j, k in itertools.combinations(range(n), 3):
        for p, q, r in itertools.permutations(range(n), 3):
            mem = [((i, j, k), (p, q, r)), ((i, k, j), (p, r, q)), ((j, i, k), (q, p, r)),
                   ((j, k, i), (q, r, p)), ((k, i, j), (r, p, q)), ((k, j, i), (r, q, p))]
            tot = sum(st.Dhat[O.z_index(n, *f, *l)] for f, l in mem)
            assert abs(tot) <= 1e-12 * scale * 6
    for i in range(n):
        for j in range(n):
            for p in range(n):
                for q in range(n):
                    if i == j or p == q:
                        continue
                    a, b = O.tile_index(n, i, p, j, q), O.tile_index(n, j, q, i, p)
                    assert abs((st.Chat[a] + st.Chat[b]) - (C0[a] + C0[b])) <= 1e-9 * (abs(C0[a]) + abs(C0[b]) + 1)


def test_redistribution_hand_example():
    """Hand-computed: one z entry with slack 10, kz=1, distinct phi.  Eq. 2.20: the
    entry drops by 10 and its partners 1..5 gain phi_1..phi_5 * 10."""
    n = 4
    m = n - 2
    T = O.num_tiles(n)
    prm = O.params_array(kz=1.0, ky=0.0, kx=0.0, phi_y=0.0, phi_z=(0.1, 0.2, 0.3, 0.15, 0.25))
    D = np.zeros(O.num_z(n))
    a = O.z_index(n, 0, 1, 2, 0, 1, 2)
    D[a] = 10.0
    z = np.zeros(T * m)
    out = O.redistribute_z(n, prm, D, z, z, np.zeros(T), np.zeros(n * n))
    expect = np.zeros_like(D)
    expect[O.z_index(n, 0, 2, 1, 0, 2, 1)] = 1.0   # phi_1
    expect[O.z_index(n, 1, 0, 2, 1, 0, 2)] = 2.0   # phi_2
    expect[O.z_index(n, 1, 2, 0, 1, 2, 0)] = 3.0   # phi_3
    expect[O.z_index(n, 2, 0, 1, 2, 0, 1)] = 1.5   # phi_4
    expect[O.z_index(n, 2, 1, 0, 2, 1, 0)] = 2.5   # phi_5
    assert np.allclose(out, expect, atol=1e-15)


def test_redistribution_type2_and_type3_hand_example():
    """Type 2 (Eq. 2.22): pi_y = 6 on tile (0,1,0,1) with ky=1 lowers each of its
    (n-2)^2 = 4 entries by 6/(n-2) = 3 and the five partners of each gain
    phi_l*3.  Type 3 (Eq. 2.23): pi_x = 12 on (3,2) with kx=1 lowers every entry
    z_3jk2qr by 12/((n-1)(n-2)) = 2."""
    n = 4
    m = n - 2
    T = O.num_tiles(n)
    prm = O.params_array(kz=0.0, ky=1.0, kx=0.0, phi_y=0.0, phi_z=(0.2,) * 5)
    piy = np.zeros(T)
    piy[O.tile_index(n, 0, 0, 1, 1)] = 6.0
    z = np.zeros(T * m)
    out = O.redistribute_z(n, prm, np.zeros(O.num_z(n)), z, z, piy, np.zeros(n * n))
    for k, r in [(2, 2), (2, 3), (3, 2), (3, 3)]:
        assert out[O.z_index(n, 0, 1, k, 0, 1, r)] == -3.0
        assert abs(out[O.z_index(n, 1, 0, k, 1, 0, r)] - 0.6) < 1e-15   # partner 2 of the entry
        assert abs(out[O.z_index(n, k, 1, 0, r, 1, 0)] - 0.6) < 1e-15   # partner 5
    assert abs(out.sum()) < 1e-12
    prm = O.params_array(kz=0.0, ky=0.0, kx=1.0, phi_y=0.0, phi_z=(0.2,) * 5)
    pix = np.zeros(n * n)
    pix[3 * n + 2] = 12.0
    out = O.redistribute_z(n, prm, np.zeros(O.num_z(n)), z, z, np.zeros(T), pix)
    # every class containing the pair (3,2) has two members led by (3,2): each gives
    # away s = 2 and gets phi*2 = 0.4 from the other; the four other members get 0.8.
    seen = 0
    for j in range(n):
        for q in range(n):
            if j == 3 or q == 2:
                continue
            for k in range(n):
                for r in range(n):
                    if k in (3, j) or r in (2, q):
                        continue
                    assert abs(out[O.z_index(n, 3, j, k, 2, q, r)] - (-1.6)) < 1e-15
                    assert abs(out[O.z_index(n, j, 3, k, q, 2, r)] - 0.8) < 1e-15
                    assert abs(out[O.z_index(n, j, k, 3, q, r, 2)] - 0.8) < 1e-15
                    seen += 1
    assert seen == 3 * 3 * 2 * 2
    assert abs(out.sum()) < 1e-12


def test_y_move_hand_example():
    """Eq. 2.21: u_ijpq += phi*pi(y_ijpq), u_jiqp -= phi*pi(y_ijpq), i.e. C^ moves."""
    n = 3
    T = O.num_tiles(n)
    C = np.arange(T, dtype=float)
    piy = np.zeros(T)
    a, b = O.tile_index(n, 0, 1, 2, 0), O.tile_index(n, 2, 0, 0, 1)
    piy[a] = 4.0
    out = O.redistribute_y(n, 0.25, C, piy)
    exp = C.copy()
    exp[a] -= 1.0
    exp[b] += 1.0
    assert np.array_equal(out, exp)


def test_feasibility_check_gives_optimum():
    """F = 0: every y/z slack is zero, the check (after Algorithm 1) fires, LB = OPT = LAP(b)."""
    inst = I.random_instance(6, 2, with_b=True)
    F = np.zeros_like(inst.F)
    st = O.setup(F, inst.D, inst.B)
    out = O.iterate(st, P1, 1)
    st2 = O.setup(F, inst.D, inst.B)
    Th, xi, psi, _, _ = O.stage_z(6, st2.Dhat)
    assert O.feasibility(6, out.xperm, out.piy, st2.Dhat, xi, psi)
    opt, _ = O.qap_brute(F, inst.D, inst.B)
    assert abs(out.lb - opt) < 1e-9


def test_constant_distance_is_exact_at_iteration0():
    n = 7
    inst = I.random_instance(n, 6, with_b=True)
    D = np.full((n, n), 3.0)
    np.fill_diagonal(D, 0.0)
    opt, _ = O.qap_brute(inst.F, D, inst.B)
    st = O.setup(inst.F, D, inst.B)
    assert abs(O.iterate(st, P1, 1).lb - opt) < 1e-9


def test_rejects_bad_partial():
    inst = I.random_instance(5, 0)
    with pytest.raises(ValueError):
        O.setup(inst.F, inst.D, None, np.array([1, 1, -1, -1, -1], dtype=np.int32))
