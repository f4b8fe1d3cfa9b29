"""Pins of the oracle's 1D spline machinery (Sec. 2.2, eq. Bsp; Sec. 4.4)."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import spline


@pytest.mark.parametrize("p,r,kind,gamma", [(1, 0, "uniform", 1), (2, 1, "uniform", 1),
                                            (3, 2, "uniform", 1), (3, 0, "uniform", 1),
                                            (4, 3, "radical", 3.0), (2, 1, "onesided", 2.0),
                                            (3, 1, "radical", 2.5)])
def test_partition_of_unity_nonnegativity_support(p, r, kind, gamma):
    E = 8
    kn = spline.open_knot_vector(E, p, r, kind, gamma)
    n = spline.n_basis(E, p, r)
    assert len(kn) == n + p + 1
    x = np.concatenate([np.linspace(0, 1, 401), np.random.default_rng(0).random(200)])
    B = spline.bspline_basis(kn, p, x)
    dB = spline.bspline_deriv(kn, p, x)
    assert B.shape == (len(x), n)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(dB.sum(axis=1), 0.0, atol=1e-10)
    assert B.min() >= -1e-15
    # support of B_i is [xi_i, xi_{i+p+1}]
    for i in range(n):
        outside = (x < kn[i]) | (x > kn[i + p + 1])
        assert np.all(B[outside, i] == 0.0)


@pytest.mark.parametrize("p,r", [(1, 0), (2, 1), (3, 2), (2, 0), (4, 3), (4, 1)])
def test_end_interpolation(p, r):
    kn = spline.open_knot_vector(4, p, r)
    B = spline.bspline_basis(kn, p, np.array([0.0, 1.0]))
    e0 = np.zeros(B.shape[1]); e0[0] = 1
    e1 = np.zeros(B.shape[1]); e1[-1] = 1
    np.testing.assert_array_equal(B[0], e0)
    np.testing.assert_array_equal(B[1], e1)


def test_p1_hat_functions_closed_form():
    E = 5
    kn = spline.open_knot_vector(E, 1, 0)
    x = np.linspace(0, 1, 1001)
    B = spline.bspline_basis(kn, 1, x)
    nodes = np.arange(E + 1) / E
    for i in range(E + 1):
        hat = np.maximum(0.0, 1.0 - np.abs(x - nodes[i]) * E)
        np.testing.assert_allclose(B[:, i], hat, atol=1e-13)


@pytest.mark.parametrize("p,r,kind,gamma", [(2, 1, "uniform", 1), (3, 2, "radical", 3.0),
                                            (3, 0, "uniform", 1), (4, 2, "onesided", 2.0)])
def test_against_independent_library_bspline(p, r, kind, gamma):
    """Cross-check with scipy's B-spline evaluator (an independent implementation)."""
    kn = spline.open_knot_vector(8, p, r, kind, gamma)
    n = spline.n_basis(8, p, r)
    x = np.random.default_rng(1).random(300)
    B = spline.bspline_basis(kn, p, x)
    dB = spline.bspline_deriv(kn, p, x)
    for i in range(n):
        c = np.zeros(n); c[i] = 1
        s = BSpline(kn, c, p, extrapolate=False)
        np.testing.assert_allclose(B[:, i], s(x), atol=1e-13)
        np.testing.assert_allclose(dB[:, i], s.derivative()(x), atol=1e-9)


@pytest.mark.parametrize("p,r", [(2, 1), (3, 2), (3, 1), (4, 3)])
def test_continuity_at_interior_knots(p, r):
    """C^r at breakpoints (Sec. 2.2): derivatives of order <= r match across a knot."""
    E = 4
    kn = spline.open_knot_vector(E, p, r)
    n = spline.n_basis(E, p, r)
    eps = 1e-7
    for zj in np.arange(1, E) / E:
        for i in range(n):
            c = np.zeros(n); c[i] = 1
            s = BSpline(kn, c, p)
            for k in range(r + 1):
                dk = s.derivative(k) if k else s
                left, right = dk(zj - eps), dk(zj + eps)
                assert abs(left - right) < 1e-4 * (1 + abs(left)) * max(1, E ** k)
    # the oracle's own derivative is continuous for r >= 1
    if r >= 1:
        x = np.array([z + s for z in np.arange(1, E) / E for s in (-1e-9, 1e-9)])
        dB = spline.bspline_deriv(kn, p, x)
        np.testing.assert_allclose(dB[0::2], dB[1::2], atol=1e-6)


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 5, 6])
def test_gauss_exactness(Q):
    z = np.array([0.0, 0.3, 1.0])
    xi, w = spline.element_quadrature(z, Q)
    np.testing.assert_allclose(w.sum(axis=1), np.diff(z), rtol=1e-14)
    for deg in range(2 * Q):
        exact = (z[1:] ** (deg + 1) - z[:-1] ** (deg + 1)) / (deg + 1)
        np.testing.assert_allclose((w * xi ** deg).sum(axis=1), exact, rtol=1e-13, atol=1e-15)
    # degree 2Q is not integrated exactly by a Q-point rule
    deg = 2 * Q
    exact = (z[1:] ** (deg + 1) - z[:-1] ** (deg + 1)) / (deg + 1)
    assert np.max(np.abs((w * xi ** deg).sum(axis=1) - exact)) > 1e-12


@pytest.mark.parametrize("gamma", [1.0, 2.0, 3.0, 4.5])
def test_radical_map(gamma):
    t = np.linspace(0, 1, 101)
    g = spline.grading_map(t, "radical", gamma)
    assert g[0] == 0.0 and abs(g[-1] - 1.0) < 1e-15
    assert abs(spline.grading_map(np.array([0.5]), "radical", gamma)[0] - 0.5) < 1e-15
    assert np.all(np.diff(g) > 0)
    # symmetric about t = 1/2
    np.testing.assert_allclose(g + g[::-1], 1.0, atol=1e-14)
    if gamma == 1.0:
        np.testing.assert_allclose(g, t, atol=1e-15)
    # continuity at t = 1/2 (both branches meet) and nested dyadic breakpoints
    for E in (4, 8, 16):
        z1 = spline.breakpoints(E, "radical", gamma)
        z2 = spline.breakpoints(2 * E, "radical", gamma)
        np.testing.assert_array_equal(z1, z2[::2])


def test_onesided_map():
    g = spline.grading_map(np.array([0.0, 0.5, 1.0]), "onesided", 3.0)
    np.testing.assert_allclose(g, [0.0, 0.125, 1.0])


def test_knot_multiplicity_and_first_function():
    p, r, E = 3, 1, 4
    kn = spline.open_knot_vector(E, p, r)
    assert list(kn[:4]) == [0, 0, 0, 0] and list(kn[-4:]) == [1, 1, 1, 1]
    assert np.sum(kn == 0.25) == p - r
    z = spline.breakpoints(E)
    first = spline.element_first_function(kn, p, z)
    np.testing.assert_array_equal(first, np.arange(E) * (p - r))
