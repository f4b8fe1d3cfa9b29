"""Pins of the oracle's learned-scaling definitions (features, scaled
fast-diagonalisation preconditioner, training loss and its gradient)."""
import numpy as np
import pytest

from oracle import fd, geometry, learned, spline
from oracle.galerkin import Component


def test_features_equal_a_constant_coefficient_on_the_unit_cube():
    """Identity map and a = alpha: tr(G_q) = d w_q alpha, so c_i = alpha exactly."""
    comp = Component(geometry.make("unit", 3), (2, 3, 1), 3)
    c = learned.features(comp, diffusion=lambda x: np.full(len(x), 2.5))
    np.testing.assert_allclose(c, 2.5, rtol=1e-13)


@pytest.mark.parametrize("p", [2, 3])
def test_features_of_a_linear_coefficient_are_knot_centroids(p):
    """Identity map, a = 1 + 2 x + y/2: c_i is the B-spline-weighted mean of a,
    i.e. a at the centroid of R_i, whose coordinates are the means of the p+2
    knots of each 1D factor (int t B_i / int B_i = (t_i + .. + t_{i+p+1})/(p+2));
    (p+1)-point Gauss integrates these degree p+1 integrands exactly."""
    lv = (3, 2)
    comp = Component(geometry.make("unit", 2), lv, p)
    c = learned.features(comp, diffusion=lambda x: 1.0 + 2.0 * x[:, 0] + 0.5 * x[:, 1])
    cen = []
    for k, l in enumerate(lv):
        kn = spline.open_knot_vector(2 ** l, p, p - 1)
        nf = spline.n_basis(2 ** l, p, p - 1)
        cen.append(np.array([kn[i:i + p + 2].mean() for i in range(1, nf - 1)]))
    ref = 1.0 + 2.0 * cen[0][None, :] + 0.5 * cen[1][:, None]     # direction 1 fastest
    np.testing.assert_allclose(c, ref.ravel(), rtol=1e-13)


def test_scaled_preconditioner_reduces_to_fd_and_is_symmetric():
    lv, p = (3, 2, 2), 3
    n = int(np.prod([2 ** l + 1 for l in lv]))
    rng = np.random.default_rng(4)
    r, y = rng.standard_normal(n), rng.standard_normal(n)
    np.testing.assert_allclose(learned.scaled_fd(lv, p, p - 1, np.ones(n), r), fd.fd_apply(lv, p, p - 1, r),
                               rtol=1e-14)
    S = np.exp(0.3 * rng.standard_normal(n))
    a = y @ learned.scaled_fd(lv, p, p - 1, S, r)
    b = r @ learned.scaled_fd(lv, p, p - 1, S, y)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_loss_vanishes_at_the_exact_scaling_of_a_constant_coefficient():
    """Unit cube, a = alpha: K = alpha K_ref with FD = K_ref^{-1}, so
    S = alpha^{-1/2} gives M = K^{-1}: zero loss and zero gradient on r = K e."""
    lv, p, alpha = (2, 3, 2), 3, 3.7
    comp = Component(geometry.make("unit", 3), lv, p).assemble(diffusion=lambda x: np.full(len(x), alpha))
    e = np.random.default_rng(5).standard_normal(comp.ndof)
    r = comp.K @ e
    L, g = learned.pair_loss_grad(lv, p, p - 1, np.full(comp.ndof, alpha ** -0.5), r, e)
    assert L < 1e-24 and np.linalg.norm(g) < 1e-10
    L1, _ = learned.pair_loss_grad(lv, p, p - 1, np.ones(comp.ndof), r, e)
    assert abs(L1 - (alpha - 1.0) ** 2) < 1e-9          # S = 1: M r = FD K e = alpha e


def test_loss_gradient_matches_finite_differences():
    lv, p = (2, 2, 3), 3
    n = int(np.prod([2 ** l + 1 for l in lv]))
    rng = np.random.default_rng(6)
    r, e = rng.standard_normal(n), rng.standard_normal(n)
    ls = 0.2 * rng.standard_normal(n)
    L, g = learned.pair_loss_grad(lv, p, p - 1, np.exp(ls), r, e)
    h = 1e-6
    for i in rng.choice(n, 25, replace=False):
        dv = np.zeros(n)
        dv[i] = h
        fp, _ = learned.pair_loss_grad(lv, p, p - 1, np.exp(ls + dv), r, e)
        fm, _ = learned.pair_loss_grad(lv, p, p - 1, np.exp(ls - dv), r, e)
        assert abs((fp - fm) / (2 * h) - g[i]) <= 1e-6 * (1.0 + abs(g[i])), i


def test_packed_loss_is_the_mean_over_components():
    grids = [((2, 2), 0, 16), ((1, 3), 16, 16)]     # p = 2 C^1: 2^l interior functions per direction
    rng = np.random.default_rng(7)
    S, r, e = np.exp(0.1 * rng.standard_normal(32)), rng.standard_normal(32), rng.standard_normal(32)
    L, g = learned.packed_loss_grad(grids, 2, 1, S, r, e)
    L0, g0 = learned.pair_loss_grad((2, 2), 2, 1, S[:16], r[:16], e[:16])
    L1, g1 = learned.pair_loss_grad((1, 3), 2, 1, S[16:], r[16:], e[16:])
    assert abs(L - 0.5 * (L0 + L1)) < 1e-14 * L
    np.testing.assert_allclose(g, 0.5 * np.concatenate([g0, g1]), rtol=1e-14)


def test_scaling_bound():
    """S = exp(4 tanh(y/4)): exp(y) to first order near 0, monotone, within e^{+-4}."""
    y = np.linspace(-50, 50, 2001)
    S = learned.scaling_from_output(y)
    assert np.all(np.diff(S) > 0) and S.min() >= np.exp(-4.0) and S.max() <= np.exp(4.0)
    np.testing.assert_allclose(learned.scaling_from_output([1e-3, -2e-3]), np.exp([1e-3, -2e-3]), rtol=1e-9)


def test_untrained_scaling_is_the_inverse_square_root_of_the_coefficient():
    """With the network output 0, S = c^(-1/2); on the unit cube with a
    constant coefficient a (c = a, by the features' pin) M = S FD S = FD / a,
    the inverse of a K. The correction factor exp(4 tanh(y / 4)) is exp(y) to
    first order and within e^(+-4)."""
    c = np.array([0.25, 0.8, 1.0, 1.3, 4.0])
    np.testing.assert_allclose(learned.scaling_from_output(np.zeros_like(c), np.log(c)), c ** -0.5, rtol=1e-15)
    y = np.array([-50.0, -1e-3, 0.0, 2e-3, 50.0])
    f = learned.scaling_from_output(y, np.log(c)) * np.sqrt(c)
    np.testing.assert_allclose(f[1:4], np.exp(y[1:4]), rtol=1e-8)
    assert np.all(np.abs(np.log(f)) <= 4.0 + 1e-12)


def test_energy_norm_loss_gradient_and_exact_scaling():
    """Energy-norm loss: its gradient matches central differences, and it
    vanishes at the exact scaling of a constant coefficient on the unit cube
    (M = FD / alpha = (alpha K)^{-1})."""
    from oracle import geometry
    from oracle.galerkin import Component
    lv, p = (2, 2, 3), 3
    K = Component(geometry.make("unit", 3), lv, p, p - 1).assemble().K.toarray()
    n = K.shape[0]
    rng = np.random.default_rng(6)
    r, e = rng.standard_normal(n), rng.standard_normal(n)
    ls = 0.2 * rng.standard_normal(n)
    L, g = learned.pair_loss_grad(lv, p, p - 1, np.exp(ls), r, e, K=K)
    h = 1e-6
    for i in rng.choice(n, 25, replace=False):
        dv = np.zeros(n)
        dv[i] = h
        fp, _ = learned.pair_loss_grad(lv, p, p - 1, np.exp(ls + dv), r, e, K=K)
        fm, _ = learned.pair_loss_grad(lv, p, p - 1, np.exp(ls - dv), r, e, K=K)
        assert abs((fp - fm) / (2 * h) - g[i]) <= 1e-6 * (1.0 + abs(g[i])), i
    alpha = 2.5
    e = rng.standard_normal(n)
    r = alpha * (K @ e)
    L, g = learned.pair_loss_grad(lv, p, p - 1, np.full(n, alpha ** -0.5), r, e, K=K)
    assert L < 1e-24 and np.linalg.norm(g) < 1e-10
