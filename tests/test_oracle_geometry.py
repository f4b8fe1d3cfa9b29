"""Pins of the oracle's geometry maps and coefficient field that the
learned-preconditioner and L-shape workloads use (eq. F-B-splines; the
perturbed cube and log-normal coefficient are the workloads' own inputs,
not the paper's)."""
import numpy as np
import pytest

from oracle import geometry
from paper_1707_09598_gb300.inputs import lognormal_features, perturbed_cube_patch


def _fd_jacobian(g, xi, h=1e-6):
    cols = []
    for k in range(xi.shape[1]):
        e = np.zeros(xi.shape[1])
        e[k] = h
        cols.append((g.map(xi + e) - g.map(xi - e)) / (2 * h))
    return np.stack(cols, axis=2)


def test_greville_control_points_give_the_identity():
    """Control points at the Greville abscissae reproduce linear functions, so
    the unperturbed patch is exactly x = xi."""
    kn, cp = perturbed_cube_patch(1, amp=0.0)
    g = geometry.BSplinePatch([3, 3, 3], kn, cp)
    xi = np.random.default_rng(3).uniform(0, 1, (50, 3))
    assert np.abs(g.map(xi) - xi).max() < 1e-14
    assert np.abs(g.jacobian(xi) - np.eye(3)[None]).max() < 1e-13


def test_perturbed_patch_jacobian_faces_and_orientation():
    kn, cp = perturbed_cube_patch(1)
    g = geometry.BSplinePatch([3, 3, 3], kn, cp)
    rng = np.random.default_rng(4)
    xi = rng.uniform(0.02, 0.98, (40, 3))
    J = g.jacobian(xi)
    assert np.abs(J - _fd_jacobian(g, xi)).max() < 1e-7
    # only interior control points move: each face of the cube stays in place
    for k in range(3):
        for side in (0.0, 1.0):
            f = rng.uniform(0, 1, (30, 3))
            f[:, k] = side
            assert np.abs(g.map(f)[:, k] - side).max() < 1e-14
    # a valid map of amplitude 0.1: orientation kept everywhere sampled
    xs = rng.uniform(0, 1, (2000, 3))
    assert np.linalg.det(g.jacobian(xs)).min() > 0.0


@pytest.mark.parametrize("signs", [(1, 1), (-1, 1), (-1, -1)])
def test_axis_map(signs):
    g = geometry.AxisMap(signs)
    xi = np.random.default_rng(5).uniform(0, 1, (20, 2))
    assert np.abs(g.jacobian(xi) - _fd_jacobian(g, xi)).max() < 1e-9
    assert np.allclose(np.linalg.det(g.jacobian(xi)), np.prod(signs))


def test_lognormal_field_has_the_squared_exponential_covariance():
    """log a over independent feature draws: mean 0, variance sigma^2 = 0.25
    and correlation exp(-r^2 / (2 ell^2)) with ell = 0.2 (random Fourier
    features of that kernel)."""
    x0 = np.array([[0.3, 0.4, 0.5]])
    pts = np.vstack([x0, x0 + [0.2, 0, 0], x0 + [0, 0.6, 0]])
    samples = []
    for seed in range(400):
        om, ph, amp = lognormal_features(1000 + seed, nfeat=128)
        samples.append(np.log(geometry.lognormal_coefficient(om, ph, amp)(pts)))
    s = np.array(samples)
    assert abs(s[:, 0].mean()) < 0.1
    assert abs(s[:, 0].var() / 0.25 - 1.0) < 0.2
    c = np.corrcoef(s.T)
    assert abs(c[0, 1] - np.exp(-0.5)) < 0.1
    assert abs(c[0, 2] - np.exp(-0.36 / 0.08)) < 0.12
