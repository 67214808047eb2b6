"""Pins of the oracle's variants (Section 3.4): F (incremental costs), the
two-phase Z solve and the Type 4 rule with annealing (Section 2.3, rule 4;
Section 5).  Every check rests on something other than the oracle's own
formulas: identities of the Lagrangian (F and S reach the same bound because
the previous problem's reduced costs are all tight), conservation of the class
sums by symmetric moves, the complementary-slackness effect of the second
phase, brute-force optima, monotonicity (Theorem 1) and closed forms.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1710_03732_gb300 import instances as I

PRM = O.params_array()


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


def _inst(which):
    if which == "cfg1":
        return I.config(1), None
    if which == "asymB":
        return I.random_instance(7, 21, with_b=True, asymmetric=True), None
    part = -np.ones(9, dtype=np.int32)
    part[[1, 4]] = [6, 2]
    return I.random_instance(9, 22, with_b=True), part


@pytest.mark.parametrize("which", ["cfg1", "asymB", "partial"])
@pytest.mark.parametrize("two_phase", [False, True])
def test_fast_equals_slow(which, two_phase):
    """Eq. 3.6 splits the costs into the previous problem (every reduced cost
    zero, optimum = previous bound) and the increments; with LAPs the split is
    exact and canonical duals shift with the costs, so F and S give the same
    bounds in exact arithmetic (here: up to rounding)."""
    inst, part = _inst(which)
    iters = 20
    _, s_lbs, _ = O.run(inst.F, inst.D, inst.B, iters=iters, partial=part, variant=0, two_phase=two_phase)
    _, f_lbs, _ = O.run(inst.F, inst.D, inst.B, iters=iters, partial=part, variant=1, two_phase=two_phase)
    assert _rel(f_lbs, s_lbs) <= 1e-9


def test_variant_path_equals_plain_path():
    """The variant iteration with no variant switched on (and every Type 4 draw
    rejected: -ln u = 0) reproduces the plain S1 iteration bit for bit, raw and
    canonical, cold and warm."""
    inst = I.random_instance(7, 23, with_b=True)
    n = inst.n
    kf, kl, _ = I.sa_draws(n, 12, 5)
    ng = np.zeros(12)
    for mode in (0, 1):
        for warm in (False, True):
            _, ref, r_out = O.run(inst.F, inst.D, inst.B, iters=12, dual_mode=mode, warm=warm)
            _, got, g_out = O.run(inst.F, inst.D, inst.B, iters=12, dual_mode=mode, warm=warm, sa=(kf, kl, ng),
                                  ub=1000.0)
            assert got == ref
            assert np.array_equal(g_out.xi, r_out.xi) and np.array_equal(g_out.piy, r_out.piy)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("two_phase", [False, True])
def test_monotone_without_annealing(variant, two_phase):
    """Theorem 1: without the Type 4 rule the bound never decreases."""
    inst = I.config(2)
    _, lbs, _ = O.run(inst.F, inst.D, inst.B, iters=15, variant=variant, two_phase=two_phase, threads=4)
    for a, b in zip(lbs, lbs[1:]):
        assert b >= a - 1e-9 * abs(a)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("two_phase", [False, True])
@pytest.mark.parametrize("sa", [False, True])
def test_bounds_below_brute_force_optimum(variant, two_phase, sa):
    """Every variant gives valid lower bounds (Lagrangian duality), the Type 4
    rule included: n = 8 instances against the 8! brute force."""
    for inst in (I.config(1), I.random_instance(8, 24, with_b=True, asymmetric=True)):
        opt, _ = O.qap_brute(inst.F, inst.D, inst.B)
        kw = {}
        if sa:
            kf, kl, ng = I.sa_draws(inst.n, 25, 9)
            kw = dict(sa=(kf, kl, ng * 1e6), ub=opt)  # accept every draw
        tr = []
        _, lbs, _ = O.run(inst.F, inst.D, inst.B, iters=25, variant=variant, two_phase=two_phase, trace=tr, **kw)
        assert max(lbs) <= opt + 1e-9 * abs(opt)
        if sa:
            assert all(t["sa_on"] for t in tr)


@pytest.mark.parametrize("variant", [0, 1])
def test_type4_only_bounded_drop(variant):
    """With kz = ky = kx = phi_y = 0 nothing moves except the Type 4 amounts.
    A rejected draw leaves the bound where it was; an accepted one lowers every
    b'_ip by at most (kf_i + kl_p) nu / n, so the bound drops by at most
    kappa^lb nu / n (one entry per row and per column in the X-LAP)."""
    inst = I.config(1)
    n = inst.n
    prm = O.params_array(kz=0.0, ky=0.0, kx=0.0, phi_y=0.0)
    kf, kl, ng = I.sa_draws(n, 20, 11)
    ng = ng.copy()
    ng[::3] = 0.0  # every third draw rejected
    tr = []
    _, lbs, _ = O.run(inst.F, inst.D, inst.B, iters=20, prm=prm, variant=variant, sa=(kf, kl, ng), ub=118.0,
                      sa_t0=5.0, trace=tr)
    K = kf.sum(axis=1) + kl.sum(axis=1)
    n_acc = 0
    for d in range(19):
        nu = lbs[d]
        if tr[d]["sa_on"]:
            n_acc += 1
            assert lbs[d + 1] >= nu - K[d] * abs(nu) / n - 1e-9 * abs(nu)
        else:
            assert abs(lbs[d + 1] - nu) <= 1e-9 * abs(nu)
    assert 0 < n_acc < 19


def test_schedule_closed_form():
    """T_d = t0 ub cool^floor(d / period); thr_d = -ln(u_d) T_d; K_d = sum of the fractions."""
    n, cnt = 6, 350
    kf, kl, ng = I.sa_draws(n, cnt, 3)
    K, thr = O.sa_schedule(n, kf, kl, ng, ub=250.0, t0=0.04, cool=0.99, period=100)
    for d in range(cnt):
        T = 0.04 * 250.0 * 0.99 ** (d // 100)
        assert abs(thr[d] - ng[d] * T) <= 1e-12 * max(1.0, abs(ng[d] * T))
        assert abs(K[d] - math.fsum(list(kf[d]) + list(kl[d]))) <= 1e-15
        assert K[d] <= 0.25 + 1e-15


def test_type4_amounts_closed_form():
    n = 7
    kf, kl, _ = I.sa_draws(n, 1, 4)
    nu = 321.5
    K = kf[0].sum() + kl[0].sum()
    out = O.sa_term(n, nu, K, K * nu, kf[0], kl[0])
    assert out is not None
    want = (kf[0][:, None] + kl[0][None, :]) * nu / (n * (n - 1) * (n - 2))
    assert np.allclose(out.reshape(n, n), want, rtol=1e-14, atol=0)
    assert O.sa_term(n, nu, K, K * nu * (1 - 1e-12), kf[0], kl[0]) is None


def _state_after(inst, iters, mode=1):
    st = O.setup(inst.F, inst.D, inst.B)
    out = None
    for _ in range(iters):
        out = O.iterate(st, PRM, mode)
    # solve once more on the current costs (no move) for a consistent snapshot
    snap = O.State(st.n, st.const, st.bprime, st.Chat.copy(), st.Dhat.copy())
    out = O.iterate(snap, PRM, mode)
    return st, out


def _classes(n):
    for i in range(n):
        for j in range(i + 1, n):
            for k in range(j + 1, n):
                for p in range(n):
                    for q in range(n):
                        for r in range(n):
                            if len({p, q, r}) < 3:
                                continue
                            f, l3 = (i, j, k), (p, q, r)
                            orders = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
                            yield [O.z_index(n, *[f[o] for o in od], *[l3[o] for o in od]) for od in orders]


def test_phase2_invariants():
    """Second phase of the two-phase Z solve: (a) each class keeps its sum;
    (b) members with slack end with zero slack under the old duals; (c) the
    members without slack share the moved slack equally; (d) no Z-LAP optimum
    decreases (the old duals stay feasible)."""
    inst = I.random_instance(6, 26, with_b=True)
    st, out = _state_after(inst, 6)
    n, m = st.n, st.n - 2
    T = O.num_tiles(n)
    D0 = st.Dhat
    piz = (D0.reshape(T, m, m) - out.xi.reshape(T, m, 1)) - out.psi.reshape(T, 1, m)
    piz = piz.ravel()
    D1 = O.phase2_z(n, D0, out.xi, out.psi)
    tol = 1e-9
    lim = tol * (1 + np.abs(np.repeat(out.xi.reshape(T, m, 1), m, axis=2)).ravel()
                 + np.abs(np.repeat(out.psi.reshape(T, 1, m), m, axis=1)).ravel())
    moved = 0
    for idx in _classes(n):
        idx = np.array(idx)
        assert abs(D1[idx].sum() - D0[idx].sum()) <= 1e-11 * max(1.0, np.abs(D0[idx]).sum())
        basic = piz[idx] <= lim[idx]
        if basic.all() or not basic.any():
            assert np.array_equal(D1[idx], D0[idx])
            continue
        moved += 1
        new_pi = piz[idx] + (D1[idx] - D0[idx])
        assert np.all(np.abs(new_pi[~basic]) <= 1e-9 * max(1.0, np.abs(D0[idx]).max()))
        gains = (D1[idx] - D0[idx])[basic]
        assert np.allclose(gains, piz[idx][~basic].sum() / basic.sum(), rtol=1e-12, atol=1e-12)
    assert moved > 0
    th0, _, _, _, _ = O.stage_z(n, D0)
    th1, _, _, _, _ = O.stage_z(n, D1)
    assert np.all(th1 >= th0 - 1e-9 * np.maximum(1.0, np.abs(th0)))
    assert np.any(th1 > th0 + 1e-9)


@pytest.mark.parametrize("with_sa", [False, True])
def test_move_sums(with_sa):
    """Sums over all entries: the S z move conserves sum D^ (every pool is handed
    on with weights summing to 1); the F z move leaves sum pi_z + sum of the
    tile terms (the Type 4 amounts cancel); the F y and x moves leave
    (1 - ky) sum pi_y and (1 - kx) sum pi_x."""
    inst = I.random_instance(6, 27, with_b=True, asymmetric=True)
    st, out = _state_after(inst, 5)
    n, m = st.n, st.n - 2
    T = O.num_tiles(n)
    prm = O.params_array(kz=0.7, ky=0.4, kx=0.9, phi_y=0.3, phi_z=(0.1, 0.3, 0.15, 0.25, 0.2))
    kz, ky, kx, phi_y = prm[:4]
    sa = None
    if with_sa:
        sa = np.linspace(0.1, 0.9, n * n)
    piz = ((st.Dhat.reshape(T, m, m) - out.xi.reshape(T, m, 1)) - out.psi.reshape(T, 1, m)).ravel()
    Ds = O.redistribute_z_v(n, prm, st.Dhat, out.xi, out.psi, out.piy, out.pix, variant=0, sa=sa)
    assert abs(Ds.sum() - st.Dhat.sum()) <= 1e-10 * max(1.0, np.abs(st.Dhat).sum())
    Df = O.redistribute_z_v(n, prm, st.Dhat, out.xi, out.psi, out.piy, out.pix, variant=1, sa=sa)
    # tile term per z: cy pi_y(tile) + cx pi_x(i p), each tile has m*m entries
    ip = np.repeat(np.arange(n * n), (n - 1) * (n - 1))
    ty = ky / (n - 2) * out.piy + kx / ((n - 1) * (n - 2)) * out.pix[ip]
    want = piz.sum() + m * m * ty.sum()
    assert abs(Df.sum() - want) <= 1e-10 * max(1.0, np.abs(piz).sum() + m * m * np.abs(ty).sum())
    C = st.Chat.copy()
    O.lib().or_redistribute_y_fast(n, float(ky), float(phi_y), O._d(C), O._d(out.piy))
    assert abs(C.sum() - (1 - ky) * out.piy.sum()) <= 1e-11 * max(1.0, np.abs(out.piy).sum())
    bx = np.zeros(n * n)
    O.lib().or_move_x_fast(n, float(kx), O._d(bx), O._d(out.pix))
    assert np.allclose(bx, (1 - kx) * out.pix, rtol=1e-15, atol=0)


# ----------------------------------------------------------- half-Z scheme ----
def _lower_mask(n):
    """Tiles (i,p,j,q) with i > j (lower order) and the matching z entries."""
    m = n - 2
    T = O.num_tiles(n)
    low = np.zeros(T, dtype=bool)
    for i in range(n):
        for p in range(n):
            for j in range(n):
                for q in range(n):
                    if i != j and p != q and i > j:
                        low[O.tile_index(n, i, p, j, q)] = True
    return low, np.repeat(low, m * m)


def test_half_lower_members_stay_zero():
    """The lower-order z keep cost 0 and their (skipped) Z-LAPs optimum 0 and zero
    duals -- so skipping them is exact: solving them anyway changes nothing."""
    inst = I.random_instance(7, 41, with_b=True, asymmetric=True)
    st = O.setup(inst.F, inst.D, inst.B)
    n, m = st.n, st.n - 2
    low_t, low_z = _lower_mask(n)
    for _ in range(6):
        out = O.iterate_half(st, dual_mode=1)
        assert np.all(st.Dhat[low_z] == 0.0)
        assert np.all(out.Theta[low_t] == 0.0)
    th_all, xi_all, psi_all, _, _ = O.stage_z(n, st.Dhat, dual_mode=1)
    snap = O.State(st.n, st.const, st.bprime, st.Chat.copy(), st.Dhat.copy())
    out = O.iterate_half(snap, dual_mode=1)
    assert np.array_equal(th_all[low_t], np.zeros(low_t.sum()))
    assert np.allclose(th_all, out.Theta, rtol=1e-12, atol=1e-12)
    lowm = np.repeat(low_t, m)
    assert np.all(xi_all[lowm] == 0.0) and np.all(psi_all[lowm] == 0.0)


@pytest.mark.parametrize("which", ["cfg1", "asymB", "partial"])
def test_half_monotone_and_valid(which):
    """Theorem 1 for the half scheme (every reduced cost stays >= 0 under the old
    duals), bounds below the brute-force optimum of every completion."""
    inst, part = _inst(which)
    _, lbs, _ = O.run_half(inst.F, inst.D, inst.B, iters=30, partial=part)
    for a, b in zip(lbs, lbs[1:]):
        assert b >= a - 1e-9 * abs(a)
    if part is None:
        opt, _ = O.qap_brute(inst.F, inst.D, inst.B)
    else:
        free_f = [i for i in range(inst.n) if part[i] < 0]
        free_l = [q for q in range(inst.n) if q not in set(part[part >= 0])]
        import itertools
        opt = np.inf
        for perm in itertools.permutations(free_l):
            full = part.copy()
            full[free_f] = perm
            opt = min(opt, O.qap_cost(inst.F, inst.D, inst.B, full))
    assert max(lbs) <= opt + 1e-9 * abs(opt)


def test_half_reaches_optimum_on_n8_grid():
    """Like the full scheme, the half scheme closes the gap on the n = 8 grid
    (optimum 118 by brute force) -- a broken move or a lost slack stalls below."""
    inst = I.config(1)
    _, lbs, _ = O.run_half(inst.F, inst.D, inst.B, iters=40)
    assert max(lbs) >= 118.0 - 1e-6


def test_half_moves_conserve_pair_and_class_sums():
    """The half-scheme step is a symmetric redistribution: every class's z sum and
    every mirror pair C^_ijpq + C^_jiqp (y move and the y-level x move) keep their
    totals."""
    inst = I.random_instance(6, 42, with_b=True)
    st = O.setup(inst.F, inst.D, inst.B)
    for _ in range(3):
        O.iterate_half(st, dual_mode=0)
    n = st.n
    D0, C0 = st.Dhat.copy(), st.Chat.copy()
    O.iterate_half(st, dual_mode=0)
    for idx in _classes(n):
        idx = np.array(idx)
        assert abs(st.Dhat[idx].sum() - D0[idx].sum()) <= 1e-10 * max(1.0, np.abs(D0[idx]).sum())
    for i in range(n):
        for j in range(i + 1, n):
            for p in range(n):
                for q in range(n):
                    if p == q:
                        continue
                    t, tp = O.tile_index(n, i, p, j, q), O.tile_index(n, j, q, i, p)
                    assert abs((st.Chat[t] + st.Chat[tp]) - (C0[t] + C0[tp])) <= 1e-10 * max(1.0, abs(C0[t]) +
                                                                                             abs(C0[tp]))
