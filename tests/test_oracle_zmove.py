"""Pins for the oracle's z move (Eq. 2.20, 2.22, 2.23 combined as in the proof
of Theorem 1) in each of its branches.

The general branch adds the five partner terms of Eq. 2.20 one at a time; it is
the written definition and is itself pinned by the hand examples in
test_oracle_pins.py and, here, by a per-entry restatement that finds every
partner by permuting the index tuple.  The regrouped branches (all phi equal;
all phi equal with kz = 1, the default preset; the half-Z scheme's member
update) must agree with it element by element to a few units in the last place
of the class's magnitude, and every branch must keep each class sum and each
mirror pair of C^ unchanged."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_1710_03732_gb300 import instances as I

EPS = np.finfo(float).eps
P1 = O.params_array(kz=1.0, ky=0.5, kx=1.0, phi_y=0.5, phi_z=(0.2,) * 5)       # folded (default)
P0 = O.params_array(kz=1.0, ky=1.0, kx=1.0, phi_y=0.0, phi_z=(0.2,) * 5)       # folded
PU = O.params_array(kz=0.7, ky=0.4, kx=0.9, phi_y=0.3, phi_z=(0.2,) * 5)       # uniform, kz != 1
PX = O.params_array(kz=0.8, ky=0.6, kx=0.9, phi_y=0.3, phi_z=(0.1, 0.3, 0.15, 0.25, 0.2))  # general
PRESETS = {"P1": P1, "P0": P0, "PU": PU, "PX": PX}

ORDERS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _entries(n):
    """Every z entry (i,j,k,p,q,r) with its flat index, tile, row k', column r'
    and the id of its symmetry class."""
    m = n - 2
    rows, cls = [], {}
    for f in itertools.permutations(range(n), 3):
        for l3 in itertools.permutations(range(n), 3):
            i, j, k = f
            p, q, r = l3
            key = tuple(sorted(zip(f, l3)))
            cid = cls.setdefault(key, len(cls))
            t = O.tile_index(n, i, p, j, q)
            kk = k - (k > i) - (k > j)
            rr = r - (r > p) - (r > q)
            rows.append((O.z_index(n, i, j, k, p, q, r), t, kk, rr, i * n + p, cid))
    a = np.array(rows, dtype=np.int64)
    assert a.shape[0] == O.num_z(n) and len(np.unique(a[:, 0])) == O.num_z(n)
    assert m >= 1
    return a


def _class_scale(n, prm, D, xi, psi, piy, pix, ent):
    """Per entry: the largest |D^| + |xi| + |psi| + |tile term| over its class
    (the magnitude every rounding in the class is relative to)."""
    m = n - 2
    cy, cx = prm[1] / (n - 2), prm[2] / ((n - 1) * (n - 2))
    idx, t, kk, rr, ip, cid = ent.T
    mag = (np.abs(D[idx]) + np.abs(xi[t * m + kk]) + np.abs(psi[t * m + rr]) + np.abs(cy * piy[t]) +
           np.abs(cx * pix[ip]))
    per_class = np.zeros(cid.max() + 1)
    np.maximum.at(per_class, cid, mag)
    out = np.zeros(O.num_z(n))
    out[idx] = per_class[cid]
    return out


def _mid_ascent(n, seed, prm, iters, dual_mode, with_b=True, asymmetric=False):
    """(state before the move, the iteration's duals) after `iters` iterations."""
    inst = I.random_instance(n, seed, with_b=with_b, asymmetric=asymmetric)
    st = O.setup(inst.F, inst.D, inst.B)
    for _ in range(iters):
        O.iterate(st, prm, dual_mode)
    D0 = st.Dhat.copy()
    out = O.iterate(st, prm, dual_mode)
    return D0, out, st.Dhat.copy()


@pytest.mark.parametrize("name", ["P1", "P0", "PU"])
@pytest.mark.parametrize("n,seed,iters,dual_mode", [(5, 3, 0, 1), (6, 1, 4, 1), (6, 2, 9, 0), (7, 5, 6, 1)])
def test_regrouped_branch_equals_general(name, n, seed, iters, dual_mode):
    """With equal phi the oracle regroups the move (folded when kz = 1); on
    mid-ascent states every entry equals the general branch's to 8 ulps of its
    class's magnitude, and the iteration itself used the regrouped branch."""
    prm = PRESETS[name]
    D0, out, moved = _mid_ascent(n, seed, prm, iters, dual_mode, asymmetric=(seed % 2 == 0))
    auto = O.redistribute_z_form(n, prm, D0, out.xi, out.psi, out.piy, out.pix, form=0)
    gen = O.redistribute_z_form(n, prm, D0, out.xi, out.psi, out.piy, out.pix, form=1)
    assert np.array_equal(auto, moved)  # the branch the iteration takes
    scale = _class_scale(n, prm, D0, out.xi, out.psi, out.piy, out.pix, _entries(n))
    err = np.abs(auto - gen)
    assert np.all(err <= 8 * EPS * scale), f"max error {np.max(err / scale) / EPS:.1f} ulps of the class scale"
    # the move is not trivial here (so the comparison means something)
    assert np.max(np.abs(gen - D0)) > 1e-3 * np.max(scale)


@pytest.mark.parametrize("variant", [0, 1])
def test_regrouped_branch_equals_general_with_type4_amounts(variant):
    """The Type 4 amounts (rule 4) enter every pool; with equal phi, kz = 1 (S:
    folded) and with the F variant (uniform), the regrouped and general
    branches still agree entry by entry."""
    n = 6
    D0, out, _ = _mid_ascent(n, 8, P1, 5, 1)
    rng = np.random.default_rng(variant)
    sa = rng.uniform(0.0, 2.0, n * n)
    auto = O.redistribute_z_form(n, P1, D0, out.xi, out.psi, out.piy, out.pix, form=0, variant=variant, sa=sa)
    gen = O.redistribute_z_form(n, P1, D0, out.xi, out.psi, out.piy, out.pix, form=1, variant=variant, sa=sa)
    scale = _class_scale(n, P1, D0, out.xi, out.psi, out.piy, out.pix, _entries(n)) + 2.0
    assert np.all(np.abs(auto - gen) <= 8 * EPS * scale)


def _partner(f, l3, order):
    return tuple(f[o] for o in order), tuple(l3[o] for o in order)


def test_general_branch_equals_per_entry_definition():
    """Eq. 2.20 read entry by entry: a's five partners are its index tuple with
    the positions permuted as listed; partner b gives a the phi of the slot of
    b's own list in which a appears.  Summed in that order (no regrouping) on
    random slacks, duals and reduced costs with unequal phi, the general branch
    agrees to 8 ulps of the class magnitude."""
    n = 5
    m = n - 2
    rng = np.random.default_rng(11)
    prm = PX
    kz, cy, cx = prm[0], prm[1] / (n - 2), prm[2] / ((n - 1) * (n - 2))
    phi = prm[4:9]
    T = O.num_tiles(n)
    D = rng.uniform(-5, 20, O.num_z(n))
    xi, psi = rng.uniform(-3, 3, T * m), rng.uniform(-3, 3, T * m)
    piy, pix = rng.uniform(0, 4, T), rng.uniform(0, 4, n * n)

    def s_of(f, l3):
        i, j, k = f
        p, q, r = l3
        t = O.tile_index(n, i, p, j, q)
        kk, rr = k - (k > i) - (k > j), r - (r > p) - (r > q)
        piz = D[O.z_index(n, *f, *l3)] - xi[t * m + kk] - psi[t * m + rr]
        return kz * piz + cy * piy[t] + cx * pix[i * n + p]

    expect = np.zeros_like(D)
    for f in itertools.permutations(range(n), 3):
        for l3 in itertools.permutations(range(n), 3):
            a = (f, l3)
            val = D[O.z_index(n, *f, *l3)] - s_of(f, l3)
            for order in ORDERS[1:]:
                b = _partner(f, l3, order)
                slot = [_partner(*b, o2) for o2 in ORDERS[1:]].index(a)
                val += phi[slot] * s_of(*b)
            expect[O.z_index(n, *f, *l3)] = val
    gen = O.redistribute_z_form(n, prm, D, xi, psi, piy, pix, form=1)
    scale = _class_scale(n, prm, D, xi, psi, piy, pix, _entries(n))
    assert np.all(np.abs(gen - expect) <= 8 * EPS * scale)


@pytest.mark.parametrize("name", ["P1", "P0", "PU", "PX"])
def test_zero_sum_invariants_every_branch(name):
    """Each preset's moves only shift cost inside a symmetry set: every z class
    sums to its start value 0 and every C^_ijpq + C^_jiqp is preserved."""
    prm = PRESETS[name]
    n = 6
    inst = I.random_instance(n, 1, with_b=True, asymmetric=True)
    st = O.setup(inst.F, inst.D, inst.B)
    C0 = st.Chat.copy()
    for _ in range(8):
        O.iterate(st, prm, 1)
    ent = _entries(n)
    sums = np.zeros(ent[:, 5].max() + 1)
    np.add.at(sums, ent[:, 5], st.Dhat[ent[:, 0]])
    scale = np.abs(st.Dhat).max() + 1
    assert np.all(np.abs(sums) <= 1e-12 * scale * 6)
    for i, j in itertools.permutations(range(n), 2):
        for p, q in itertools.permutations(range(n), 2):
            a, b = O.tile_index(n, i, p, j, q), O.tile_index(n, j, q, i, p)
            assert abs((st.Chat[a] + st.Chat[b]) - (C0[a] + C0[b])) <= 1e-9 * (abs(C0[a]) + abs(C0[b]) + 1)


def test_folded_hand_example():
    """Default preset (kz = 1, ky = 1/2, phi = 1/5, the folded branch), n = 4:
    one z entry with cost 10 and pi_y = 4 on its tile (so cy pi_y = 1 on each of
    the tile's four entries).  Worked by hand: the entry's pool is 11, it ends at
    10 - 11 = -1 and each of its five partners gains 11/5; the tile's three other
    entries have pool 1, end at -1, and their partners gain 1/5."""
    n = 4
    m = n - 2
    T = O.num_tiles(n)
    D = np.zeros(O.num_z(n))
    D[O.z_index(n, 0, 1, 2, 0, 1, 2)] = 10.0
    piy = np.zeros(T)
    piy[O.tile_index(n, 0, 0, 1, 1)] = 4.0
    z = np.zeros(T * m)
    out = O.redistribute_z(n, P1, D, z, z, piy, np.zeros(n * n))
    expect = np.zeros_like(D)
    for k, r in itertools.product((2, 3), (2, 3)):
        f, l3 = (0, 1, k), (0, 1, r)
        expect[O.z_index(n, *f, *l3)] = -1.0
        gain = 11.0 / 5 if (k, r) == (2, 2) else 1.0 / 5
        for order in ORDERS[1:]:
            expect[O.z_index(n, *_partner(f, l3, order)[0], *_partner(f, l3, order)[1])] += gain
    assert np.max(np.abs(out - expect)) <= 4 * EPS * 11


@pytest.mark.parametrize("n,seed,iters", [(5, 4, 2), (6, 7, 5), (7, 9, 3)])
def test_half_regrouped_equals_plain(n, seed, iters):
    """Half-Z scheme (Section 5): the member update regrouped as
    (D + S/2) - (3/2) s equals the plain (D - s) + s_b/2 + s_c/2 to 8 ulps of
    the class magnitude; the y part is the same code in both forms."""
    inst = I.random_instance(n, seed, with_b=True)
    st = O.setup(inst.F, inst.D, inst.B)
    for _ in range(iters):
        O.iterate_half(st, dual_mode=1)
    D0, C0 = st.Dhat.copy(), st.Chat.copy()
    out = O.iterate_half(st, dual_mode=1)
    prm = np.array(O.HALF_PRM)
    Dr, Cr = O.redistribute_half_form(n, prm, D0, C0, out.xi, out.psi, out.piy, out.pix, form=0)
    Dp, Cp = O.redistribute_half_form(n, prm, D0, C0, out.xi, out.psi, out.piy, out.pix, form=1)
    assert np.array_equal(Dr, st.Dhat) and np.array_equal(Cr, st.Chat)
    assert np.array_equal(Cr, Cp)
    hp = O.params_array(kz=prm[0], ky=prm[1], kx=prm[2], phi_y=prm[3])
    scale = _class_scale(n, hp, D0, out.xi, out.psi, 2 * out.piy, out.pix, _entries(n))
    assert np.all(np.abs(Dr - Dp) <= 8 * EPS * scale)
    assert np.max(np.abs(Dp - D0)) > 1e-3 * np.max(scale)
