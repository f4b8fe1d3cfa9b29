"""Pins of the oracle's linear functional of the combined solution,
l(u) = sum_i c_i int g u_i, computed from the components' load vectors (no
evaluation points; the paper's remark on functionals of the solution, Sec. 1
and Sec. 4.1)."""
import numpy as np

from oracle import driver


def test_exactly_reproduced_solution_gives_the_closed_form():
    # u = x(1-x)y(1-y) lies in every p = 2 component space: every l(u_i) and the
    # combination equal the exact integrals (the Gauss rule is exact here)
    res = driver.solve_components("unit", 2, 2, 4, "poly2")
    vals, comb = driver.functional(res, lambda x: np.ones(len(x)))
    assert np.abs(vals - 1.0 / 36.0).max() < 1e-15
    assert abs(comb - 1.0 / 36.0) < 1e-15
    _, comb = driver.functional(res, lambda x: x[:, 0])
    assert abs(comb - 1.0 / 72.0) < 1e-15


def test_linearity_and_coefficients():
    res = driver.solve_components("unit", 2, 2, 5, "sine2")
    g1 = lambda x: np.ones(len(x))
    g2 = lambda x: np.sin(3 * x[:, 0]) * x[:, 1]
    v1, c1 = driver.functional(res, g1)
    v2, c2 = driver.functional(res, g2)
    v3, c3 = driver.functional(res, lambda x: 2 * g1(x) - 3 * g2(x))
    assert np.abs(v3 - (2 * v1 - 3 * v2)).max() < 1e-14
    assert abs(c3 - (2 * c1 - 3 * c2)) < 1e-14
    coef = np.array([c for _, c, _, _ in res])
    assert abs(c1 - coef @ v1) < 1e-15


def test_converges_to_the_exact_integral():
    # u = sin(pi x) sin(pi y): int u = 4 / pi^2; the error falls with the level
    errs = []
    for w in (3, 4, 5, 6):
        res = driver.solve_components("unit", 2, 2, w, "sine2")
        _, comb = driver.functional(res, lambda x: np.ones(len(x)))
        errs.append(abs(comb - 4.0 / np.pi ** 2))
    assert driver.rate([3, 4, 5, 6], errs) > 2.5
