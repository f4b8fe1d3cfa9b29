"""Pins of the oracle's surpluses, index-set coefficients and Dantzig choice
(the paper's Sec. 4.2 knapsack view of the sparse-grid set)."""
import itertools

import numpy as np

from oracle import adaptive, combination, driver


def test_standard_set_gives_the_combination_coefficients():
    for d, w in ((2, 5), (3, 6)):
        top = w + d - 1
        I = [b for b in itertools.product(range(1, top + 1), repeat=d) if sum(b) <= top]
        got = adaptive.coefficients(I)
        want = {tuple(i): c for i, c in combination.index_set(d, w)}
        assert got == want


def test_full_tensor_set_telescopes_to_its_corner():
    I = list(itertools.product(range(1, 5), repeat=2))
    assert adaptive.coefficients(I) == {(4, 4): 1}


def test_surpluses_sum_to_the_combination():
    rng = np.random.default_rng(5)
    I = [(1, 1), (2, 1), (1, 2), (3, 1), (2, 2), (1, 3), (4, 1)]
    vals = {b: rng.standard_normal(7) for b in I}
    s = sum(adaptive.surplus(vals, b) for b in I)
    c = adaptive.coefficients(I)
    comb = sum(c[g] * vals[g] for g in c)
    assert np.abs(s - comb).max() < 1e-14


def test_dantzig_takes_admissible_items_by_profit_within_budget():
    prof = {(1, 1): (1.0, 10.0), (2, 1): (0.5, 5.0), (1, 2): (0.6, 6.0), (2, 2): (0.1, 9.0), (3, 1): (0.2, 4.0)}
    cost = {b: 1 for b in prof}
    # (2,2) has the second highest profit but needs (2,1) and (1,2) first
    assert adaptive.dantzig(prof, cost, 4) == [(1, 1), (1, 2), (2, 1), (2, 2)]
    assert adaptive.dantzig(prof, cost, 2) == [(1, 1), (1, 2)]


def test_profits_of_a_symmetric_problem_are_symmetric_and_decay():
    # every component of the full set max(beta) <= 4, evaluated on a Gauss rule
    from oracle import geometry, problems
    from oracle.galerkin import Component
    pts, wts = driver._fine_rule(2, 16, 4)
    vals, cost = {}, {}
    for b in itertools.product(range(1, 5), repeat=2):
        comp = Component(geometry.make("unit", 2), b, 2).assemble(f=problems.get("sine2").f)
        vals[b] = comp.evaluate(comp.solve(), pts)
        cost[b] = comp.ndof
    prof = adaptive.profits(vals, wts, cost)
    for (a, b), (rev, pr) in prof.items():
        rev2, pr2 = prof[(b, a)]
        assert abs(rev - rev2) <= 1e-9 * max(rev, 1e-300)      # transposed solves: rounding only
    assert prof[(1, 1)][0] > prof[(2, 2)][0] > prof[(3, 3)][0] > prof[(4, 4)][0]
