"""Pins of the two-level combination preconditioner's oracle (oracle/ct.py):
the prolongations are exact knot insertion (P^T A P = A_i where both are
integrated exactly), FD is the exact inverse on the unit square, and B_CT A
is a near-projection (eigenvalues in [0, 1.2], most of them zero)."""
import numpy as np
import pytest

from oracle import ct, galerkin, geometry


@pytest.mark.parametrize("d,levels,J", [(2, [(1, 4), (2, 3), (3, 1)], 4), (3, [(1, 2, 1), (2, 1, 2)], 3)])
def test_prolongation_is_exact_knot_insertion(d, levels, J):
    g = geometry.make("unit", d)
    full = galerkin.Component(g, (J,) * d, 2, 1).assemble()
    for lv in levels:
        C = galerkin.Component(g, lv, 2, 1).assemble()
        P = ct.prolongation(g, 2, 1, lv, J)
        assert abs(P.T @ full.K @ P - C.K).max() < 1e-13 * abs(C.K).max()


def test_prolongation_of_level_to_itself_is_the_identity():
    g = geometry.make("unit", 2)
    np.testing.assert_allclose(ct.prolongation_1d(g, 3, 2, 3, 3), np.eye(2 ** 3 + 1), atol=1e-14)


def test_fd_is_exact_and_the_combination_operator_a_near_projection():
    g = geometry.make("unit", 2)
    T = ct.TwoLevel(g, 2, 2, 1, 4)
    n = T.A.shape[0]
    r = np.random.default_rng(3).standard_normal(n)
    assert np.abs(T.b_fd(T.A @ r) - r).max() < 1e-12
    BA = np.column_stack([T.b_ct(T.A @ e) for e in np.eye(n)])
    ev = np.linalg.eigvals(BA)
    assert np.abs(ev.imag).max() < 1e-8 and ev.real.min() > -1e-8 and ev.real.max() < 1.2
    assert np.mean(ev.real < 1e-6) > 0.5
