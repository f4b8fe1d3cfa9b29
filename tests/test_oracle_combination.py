"""Pins of the oracle's combination technique (Sec. 3, eqs. TD-approx, TD-combi-tec)."""
import itertools
import math

import numpy as np
import pytest

from oracle import combination, driver, geometry, problems
from oracle.galerkin import Component


@pytest.mark.parametrize("d,w,m", [(2, 6, 1), (3, 10, 1), (2, 12, 1), (3, 12, 1), (2, 5, 2),
                                   (3, 7, 2), (2, 0, 0), (3, 4, 0)])
def test_coefficients_expansion_equals_binomial_and_sum_to_one(d, w, m):
    cs = combination.coefficients_by_expansion(d, w, m)
    for i, c in cs.items():
        assert c == combination.coefficient_closed_form(d, w, i)
        assert w <= sum(i) <= w + d - 1 and min(i) >= m
    assert sum(cs.values()) == 1
    # brute-force count of the top d layers of the simplex
    hi = w + d - 1
    brute = [i for i in itertools.product(range(m, hi + 1), repeat=d) if w <= sum(i) <= hi]
    assert len(brute) == len(cs)


def test_component_counts_of_workloads():
    # 2D w=6: 11 grids; 3D w=10: 136 grids, sum |c| = 181; 3D w=12: 199 grids, sum|c| = 265
    for d, w, n, s in [(2, 6, 11, 11), (3, 10, 136, 181), (3, 12, 199, 265), (2, 12, 23, 23)]:
        idx = combination.index_set(d, w)
        assert len(idx) == n
        assert sum(abs(c) for _, c in idx) == s
    # closed-form number of components d=2: (J+1) + J with beta >= 0
    for J in range(1, 8):
        assert len(combination.index_set(2, J - 1, 0)) == 2 * J + 1
        assert len(combination.index_set(3, J - 2, 0)) == math.comb(J + 2, 2) + math.comb(J + 1, 2) + math.comb(J, 2)


def test_example_1():
    """Example 1 (Sec. 3): J = 1, d = 2 gives f_[1,0] + f_[0,1] - f_[0,0]."""
    cs = combination.coefficients_by_expansion(2, 0, 0)      # J = w + d - 1 - d m = 1
    assert cs == {(1, 0): 1, (0, 1): 1, (0, 0): -1}


def _expand(index_set):
    """Coefficients of sum_{beta in set} Delta_beta in terms of f's (eq. Delta-combi-tec)."""
    acc = {}
    for beta in index_set:
        for k in itertools.product((0, 1), repeat=len(beta)):
            idx = tuple(b - kk for b, kk in zip(beta, k))
            if min(idx) >= 0:
                acc[idx] = acc.get(idx, 0) + (-1) ** sum(k)
    return {i: c for i, c in acc.items() if c}


@pytest.mark.parametrize("d,J", [(2, 1), (2, 4), (3, 2), (3, 3)])
def test_telescoping_full_tensor(d, J):
    """sum_{beta <= [J..J]} Delta_beta = f_[J..J] (eq. TP-telescopic)."""
    box = list(itertools.product(range(J + 1), repeat=d))
    assert _expand(box) == {tuple([J] * d): 1}


def test_example_1_plus_delta11_gives_full_tensor():
    sg = combination.coefficients_by_expansion(2, 0, 0)
    d11 = _expand([(1, 1)])
    d11_only = {i: c for i, c in d11.items()}
    total = dict(sg)
    for i, c in d11_only.items():
        total[i] = total.get(i, 0) + c
    assert {i: c for i, c in total.items() if c} == {(1, 1): 1}


def test_neumaier_sum():
    t = np.array([[1e16], [1.0], [-1e16], [1e-3]])
    assert combination.neumaier_sum(t)[0] == 1.001
    rng = np.random.default_rng(0)
    x = rng.standard_normal((200, 5)) * 10.0 ** rng.integers(-8, 8, (200, 5))
    exact = np.array([float(sum(__import__("fractions").Fraction(v) for v in col)) for col in x.T])
    np.testing.assert_allclose(combination.neumaier_sum(x), exact, rtol=1e-15, atol=0)


def test_combination_reproduces_polynomial_exactly():
    """u in the coarsest space: every component equals u, so does the combination."""
    res = driver.solve_components("unit", 2, 2, 4, "poly2")
    pts = np.random.default_rng(1).random((64, 2))
    uc, _ = driver.combined_at(res, pts)
    np.testing.assert_allclose(uc, problems.get("poly2").u(pts), atol=1e-14)
    res3 = driver.solve_components("unit", 3, 2, 4, "poly3")
    uc3, _ = driver.combined_at(res3, pts[:, [0, 1, 0]])
    np.testing.assert_allclose(uc3, problems.get("poly3").u(pts[:, [0, 1, 0]]), atol=1e-14)


def test_tiny_levels_agree_with_full_tensor_solve():
    """w small: the combined solution and the full tensor solve u_[w,w] differ by
    no more than their discretisation errors."""
    prob = problems.get("sine2")
    pts = np.random.default_rng(2).random((200, 2))
    for w in (2, 3):
        res = driver.solve_components("unit", 2, 2, w, "sine2")
        uc, _ = driver.combined_at(res, pts)
        full = Component(geometry.UnitCube(2), (w, w), 2).assemble(f=prob.f)
        uf = full.evaluate(full.solve(), pts)
        ex = prob.u(pts)
        gap = np.max(np.abs(uc - uf))
        assert gap <= np.max(np.abs(uc - ex)) + np.max(np.abs(uf - ex))
        assert gap < 0.05


def test_compensated_combination_matches_an_exactly_rounded_sum():
    """combine (Neumaier) against math.fsum, which is correctly rounded, on
    +-1e16 components that cancel down to O(1) values (the regime of the
    +- combination sum)."""
    import math
    from oracle import combination
    rng = np.random.default_rng(31)
    ng, npts = 40, 25
    big = 1e16 * rng.standard_normal((ng // 2, npts))
    vals = np.vstack([big, big + rng.standard_normal((ng // 2, npts))])
    coef = np.concatenate([-np.ones(ng // 2), np.ones(ng // 2)])
    got = combination.combine(vals, coef)
    ref = np.array([math.fsum(coef * vals[:, j]) for j in range(npts)])
    naive = (coef[:, None] * vals).sum(axis=0)
    # Neumaier: error <= 2 eps |sum| + O(n eps^2) sum |x| (~1e-13 here); the
    # plain sum is off by O(eps sum |x|), of the order of the result itself
    assert np.abs(got - ref).max() < 1e-12
    assert np.abs(naive - ref).max() > 1.0
