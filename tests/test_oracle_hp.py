"""Pins of the oracle's h-p sparse combination (oracle/hp.py) against facts
that do not come from its own code: the h-sparse closed form of eq.
TD-combi-tec, the same closed form in d + 1 indices, the sparse sum of
hierarchical increments by brute force, the nesting of spline spaces under
degree elevation at fixed continuity, exact reproduction of a polynomial
that lies in every component space, and the exact split of one degree step
into h-sparse combinations."""
import itertools
import math

import numpy as np
import pytest

from oracle import combination, geometry, hp, problems
from oracle.galerkin import Component, Space1D


@pytest.mark.parametrize("d,w", [(2, 2), (2, 5), (3, 3), (3, 5)])
def test_without_degree_steps_it_is_the_h_sparse_set(d, w):
    c = hp.hp_coefficients_by_expansion(d, w, 0)
    assert all(k[d] == 0 for k in c)
    want = {i: combination.coefficient_closed_form(d, w, i)
            for i in itertools.product(range(1, w + d), repeat=d)}
    want = {i: v for i, v in want.items() if v != 0}
    assert {k[:d]: v for k, v in c.items()} == want


@pytest.mark.parametrize("d,w", [(2, 3), (2, 4), (3, 3)])
def test_full_simplex_has_the_closed_form_in_d_plus_1_indices(d, w):
    """With Q >= J the set is the simplex |beta| + q <= J in d + 1 indices,
    whose coefficients are (-1)^t binom(d, t), t = J - |beta| - q, for
    0 <= t <= d (eq. TD-combi-tec with d + 1 directions), and 0 below."""
    J = w + d - 1 - d
    c = hp.hp_coefficients_by_expansion(d, w, J)
    for beta in itertools.product(range(J + 1), repeat=d):
        for q in range(J + 1):
            t = J - sum(beta) - q
            want = (-1) ** t * math.comb(d, t) if 0 <= t <= d else 0
            assert c.get(tuple(b + 1 for b in beta) + (q,), 0) == want


@pytest.mark.parametrize("d,w,Q", [(2, 4, 1), (2, 5, 2), (3, 4, 1), (3, 3, 3)])
def test_combination_is_the_sparse_sum_of_increments(d, w, Q):
    """For component values u_a = sum_{b <= a} g_b (g random), the
    combination equals the sum of g over the set (brute force)."""
    rng = np.random.default_rng(7)
    J = w + d - 1 - d
    box = list(itertools.product(*([range(J + 1)] * d + [range(Q + 1)])))
    g = {a: rng.standard_normal() for a in box}

    def u(a):
        return sum(g[b] for b in box if all(x <= y for x, y in zip(b, a)))

    c = hp.hp_coefficients_by_expansion(d, w, Q)
    comb = sum(v * u(tuple(x - 1 for x in k[:d]) + (k[d],)) for k, v in c.items())
    inside = sum(g[a] for a in box if sum(a[:d]) + a[d] <= J)
    assert abs(comb - inside) < 1e-12 * max(1.0, abs(inside))
    assert sum(c.values()) == 1


@pytest.mark.parametrize("p,r", [(2, 1), (2, 0), (3, 1), (3, 2)])
def test_degree_elevation_at_fixed_continuity_nests_the_spaces(p, r):
    """Every function of S_{p,r} on a mesh is a least-squares-exact
    combination of S_{p+1,r} on the same mesh; S_{p,p-1} is not inside
    S_{p+1,p} (a kink of the degree-p space's derivative of order p cannot be
    matched with one more continuous derivative)."""
    geom = geometry.make("unit", 2)
    t = np.linspace(0.0, 1.0, 1201)
    A = Space1D(3, p, r, geom, 0).values_at(t)
    B = Space1D(3, p + 1, r, geom, 0).values_at(t)
    X = np.linalg.lstsq(B, A, rcond=None)[0]
    assert np.abs(B @ X - A).max() < 1e-12
    if r == p - 1:
        C = Space1D(3, p + 1, p, geom, 0).values_at(t)
        Y = np.linalg.lstsq(C, A, rcond=None)[0]
        assert np.abs(C @ Y - A).max() > 1e-3


def test_polynomial_in_every_space_is_reproduced():
    """u = x(1-x)y(1-y) lies in every Dirichlet spline space of degree >= 2,
    so each Galerkin component returns it and the combination (coefficients
    summing to 1) does too."""
    geom = geometry.make("unit", 2)
    prob = problems.get("poly2")
    pts = np.random.default_rng(3).random((150, 2))
    u, vals, coef = hp.hp_solution(geom, prob.f, 2, 2, 1, 4, 2, pts)
    assert len({k[2] for k in coef}) == 3
    assert np.abs(u - prob.u(geom.map(pts))).max() < 1e-12


def test_continuity_above_the_lowest_degree_is_refused():
    geom = geometry.make("unit", 2)
    with pytest.raises(ValueError):
        hp.hp_solution(geom, problems.get("poly2").f, 2, 2, 2, 3, 1, np.zeros((1, 2)))


def test_one_degree_step_is_two_h_sparse_combinations_of_the_level_below():
    """With Q = 1 the set's sum splits exactly: the h-sparse combination of
    degree p0 at level w, plus those of degrees p0 + 1 and p0 at level
    w - 1 with signs + and - (the q = 1 increments summed over the h-sparse
    set of level w - 1). Built from eq. TD-combi-tec's closed form and
    direct solves, not from the expansion."""
    geom = geometry.make("unit", 2)
    f = problems.get("sine2").f
    pts = np.random.default_rng(4).random((60, 2))
    d, p0, r, w = 2, 2, 1, 4

    def h_sparse(p, lev):
        acc = np.zeros(len(pts))
        for i in itertools.product(range(1, lev + d), repeat=d):
            c = combination.coefficient_closed_form(d, lev, i)
            if c:
                comp = Component(geom, i, p, r).assemble(f=f)
                acc += c * comp.evaluate(comp.solve(), pts)
        return acc

    u, _, _ = hp.hp_solution(geom, f, d, p0, r, w, 1, pts)
    split = h_sparse(p0, w) + h_sparse(p0 + 1, w - 1) - h_sparse(p0, w - 1)
    assert np.abs(u - split).max() < 1e-12
