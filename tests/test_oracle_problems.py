"""The oracle's manufactured problems: f = -Laplace(u) and grad u, derived
symbolically, against central differences of u (Problem 1)."""
import numpy as np
import pytest

from oracle import problems


@pytest.mark.parametrize("name", ["sine2", "sine3", "poly2", "poly3", "annulus_sinx", "annulus_paper2",
                                  "annulus_paper3"])
def test_source_and_gradient_against_central_differences(name):
    prob = problems.get(name)
    d = prob.d
    rng = np.random.default_rng(11)
    x = rng.uniform(0.2, 0.8, (25, d)) + (np.array([0.6, 0.6, 0.0])[:d] if "annulus" in name else 0.0)
    h = 1e-3
    lap = np.zeros(len(x))
    grad = np.zeros((len(x), d))
    for k in range(d):
        e = np.zeros(d)
        e[k] = h
        up, um, u0 = prob.u(x + e), prob.u(x - e), prob.u(x)
        lap += (up - 2 * u0 + um) / h ** 2
        grad[:, k] = (up - um) / (2 * h)
    scale = max(1.0, np.abs(prob.f(x)).max())
    assert np.abs(prob.f(x) + lap).max() < 1e-4 * scale
    assert np.abs(prob.grad_u(x) - grad).max() < 1e-5 * max(1.0, np.abs(grad).max())


def test_sine_source_closed_form():
    x = np.random.default_rng(12).uniform(0, 1, (10, 2))
    ref = 2 * np.pi ** 2 * np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])
    assert np.abs(problems.get("sine2").f(x) - ref).max() < 1e-12
