"""Pins of the branch-and-bound pieces of the oracle (Section 4).

The child state (parent -> child multiplier warm start) is checked against
what the mathematics fixes: with zero multipliers it is the ordinary QAP
reduction of a partial assignment (or_setup), and for any multipliers the
Lagrangian objective of a full assignment equals its QAP cost (the ascent
steps only move cost between symmetric variables), so the child's objective
of a completion must equal the parent's and the QAP cost of the full
permutation.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_1710_03732_gb300 import instances as I


def _full_perm(partial, free_f, free_l, child_perm):
    full = np.array(partial, dtype=np.int32).copy()
    for a, c in zip(free_f, child_perm):
        full[a] = free_l[c]
    return full


@pytest.mark.parametrize("seed,asym", [(51, False), (52, True)])
def test_child_of_fresh_parent_is_the_qap_reduction(seed, asym):
    inst = I.random_instance(7, seed, with_b=True, asymmetric=asym)
    root = O.setup(inst.F, inst.D, inst.B)
    for f, l in [(0, 0), (3, 5), (6, 2)]:
        ch = O.child_state(root, f, l)
        part = -np.ones(7, dtype=np.int32)
        part[f] = l
        ref = O.setup(inst.F, inst.D, inst.B, part)
        assert ch.const == ref.const
        assert np.array_equal(ch.bprime, ref.bprime)
        assert np.array_equal(ch.Chat, ref.Chat)
        assert np.all(ch.Dhat == 0.0)
    # two levels: (f, l) then the child's (f2, l2) in its own residual indices
    ch = O.child_state(O.child_state(root, 2, 4), 4, 0)  # residual facility 4 = original 5, location 0 = 0
    part = -np.ones(7, dtype=np.int32)
    part[2], part[5] = 4, 0
    ref = O.setup(inst.F, inst.D, inst.B, part)
    assert ch.const == ref.const and np.array_equal(ch.bprime, ref.bprime) and np.array_equal(ch.Chat, ref.Chat)


def test_lagrangian_objective_equals_qap_cost_after_ascent():
    """The ascent steps only move cost between symmetric variables, so every
    permutation keeps its QAP cost under the multiplier-adjusted costs; a
    dropped term or a wrong partner in a move breaks this."""
    inst = I.random_instance(7, 53, with_b=True, asymmetric=True)
    st = O.setup(inst.F, inst.D, inst.B)
    prm = O.params_array(kz=0.8, ky=0.6, kx=0.9, phi_y=0.3, phi_z=(0.1, 0.3, 0.15, 0.25, 0.2))
    for _ in range(6):
        O.iterate(st, prm, 0)
    rng = np.random.default_rng(0)
    for _ in range(20):
        perm = rng.permutation(7).astype(np.int32)
        want = O.qap_cost(inst.F, inst.D, inst.B, perm)
        assert abs(O.lagrangian_objective(st, perm) - want) <= 1e-9 * max(1.0, abs(want))


def test_child_objective_equals_parent_objective():
    """For a parent with nonzero multipliers, every completion of the child has
    the same Lagrangian objective in the child as its full permutation has in
    the parent (= its QAP cost)."""
    inst = I.random_instance(7, 54, with_b=True)
    st = O.setup(inst.F, inst.D, inst.B)
    for _ in range(5):
        O.iterate(st, O.params_array(), 1)
    f, l = 2, 3
    ch = O.child_state(st, f, l)
    part = -np.ones(7, dtype=np.int32)
    part[f] = l
    free_f = [a for a in range(7) if a != f]
    free_l = [q for q in range(7) if q != l]
    rng = np.random.default_rng(1)
    for _ in range(25):
        cp = rng.permutation(6).astype(np.int32)
        full = _full_perm(part, free_f, free_l, cp)
        want = O.qap_cost(inst.F, inst.D, inst.B, full)
        assert abs(O.lagrangian_objective(ch, cp) - want) <= 1e-9 * max(1.0, abs(want))
        assert abs(O.lagrangian_objective(st, full) - want) <= 1e-9 * max(1.0, abs(want))


def test_warm_child_bound_is_valid_and_at_least_the_cold_one():
    """A child started from the parent's multipliers has a valid first bound (below
    the best completion, brute force) that is at least the cold child's first
    bound here (Gilmore-Lawler of the residual problem)."""
    inst = I.random_instance(8, 55, with_b=True, asymmetric=True)
    st = O.setup(inst.F, inst.D, inst.B)
    for _ in range(10):
        O.iterate(st, O.params_array(), 1)
    f, l = 1, 6
    part = -np.ones(8, dtype=np.int32)
    part[f] = l
    free_f = [a for a in range(8) if a != f]
    free_l = [q for q in range(8) if q != l]
    best = min(O.qap_cost(inst.F, inst.D, inst.B, _full_perm(part, free_f, free_l, cp))
               for cp in itertools.permutations(range(7)))
    ch = O.child_state(st, f, l)
    warm = ch.const + O.iterate(ch, O.params_array(), 1).lb
    cold_st = O.setup(inst.F, inst.D, inst.B, part)
    cold = cold_st.const + O.iterate(cold_st, O.params_array(), 1).lb
    assert warm <= best + 1e-9 * abs(best)
    assert warm >= cold - 1e-9 * abs(cold)
