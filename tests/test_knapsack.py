"""The library's index-set logic (paper_1707_09598_gb300.knapsack) agrees
with the oracle's independent implementation (oracle/adaptive.py)."""
import itertools

import numpy as np

from oracle import adaptive
from paper_1707_09598_gb300 import knapsack


def test_coefficients_agree():
    rng = np.random.default_rng(9)
    for _ in range(20):
        # random admissible 2D / 3D sets
        d = rng.integers(2, 4)
        S = {(1,) * d}
        for _ in range(12):
            b = list(rng.choice(sorted(S)))
            k = rng.integers(d)
            b[k] += 1
            b = tuple(int(v) for v in b)
            if all(b[j] == 1 or tuple(v - (i == j) for i, v in enumerate(b)) in S for j in range(d)):
                S.add(b)
        assert knapsack.set_coefficients(S) == adaptive.coefficients(S)


def test_surpluses_and_choice_agree():
    rng = np.random.default_rng(10)
    levels = list(itertools.product(range(1, 5), repeat=2))
    vals = {b: rng.standard_normal(5) for b in levels}
    s1 = knapsack.surpluses(vals)
    for b in levels:
        assert np.abs(s1[b] - adaptive.surplus(vals, b)).max() < 1e-15
    prof = {b: float(rng.random()) for b in levels}
    cost = {b: int(rng.integers(1, 9)) for b in levels}
    for budget in (5, 20, 60):
        mine = knapsack.choose(prof, cost, budget)
        theirs = adaptive.dantzig({b: (0.0, prof[b]) for b in levels}, cost, budget)
        assert mine == theirs
