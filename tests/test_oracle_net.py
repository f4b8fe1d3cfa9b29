"""Pins of the oracle's learned-correction network (forward/backward definitions)."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import net


def _params(d, seed=0, scale=0.3):
    T = 3 ** d
    n = sum(co * ci * T + co for ci, co in zip(net.CIN, net.COUT))
    return np.random.default_rng(seed).standard_normal(n) * scale


@pytest.mark.parametrize("d,shape", [(3, (4, 3, 5)), (2, (6, 4))])
def test_conv_matches_scipy_correlate(d, shape):
    """conv = multi-channel cross-correlation with zero padding (scipy.ndimage)."""
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3,) + tuple(reversed(shape)))
    W = rng.standard_normal((2, 3, 3 ** d))
    Y = net.conv(X, W)
    for co in range(2):
        ref = np.zeros(X.shape[1:])
        for ci in range(3):
            k = np.zeros((3,) * d)
            for t, off in enumerate(net.offsets(d)):
                k[tuple(o + 1 for o in reversed(off))] = W[co, ci, t]
            ref += ndimage.correlate(X[ci], k, mode="constant", cval=0.0)
        np.testing.assert_allclose(Y[co], ref, atol=1e-12)


@pytest.mark.parametrize("d,shape", [(3, (3, 4, 2)), (2, (5, 3))])
def test_backward_matches_finite_differences(d, shape):
    rng = np.random.default_rng(2)
    p = _params(d)
    x = rng.standard_normal((net.CIN[0],) + tuple(reversed(shape)))
    dy = rng.standard_normal(tuple(reversed(shape)))
    g = net.backward(p, x, dy)
    f = lambda q: float(np.sum(dy * net.forward(q, x)[0]))
    idx = rng.choice(p.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p); e[i] = h
        fd = (f(p + e) - f(p - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(g[i])), (i, fd, g[i])


def test_input_gradient_is_adjoint():
    rng = np.random.default_rng(3)
    W = rng.standard_normal((4, 3, 27))
    X = rng.standard_normal((3, 3, 4, 5))
    dY = rng.standard_normal((4, 3, 4, 5))
    lhs = np.sum(dY * net.conv(X, W))
    rhs = np.sum(net.conv_input_grad(dY, W) * X)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_offsets_order():
    off = net.offsets(3)
    assert off[0] == (-1, -1, -1) and off[1] == (0, -1, -1) and off[3] == (-1, 0, -1) and off[9] == (-1, -1, 0)
    assert off[13] == (0, 0, 0)
