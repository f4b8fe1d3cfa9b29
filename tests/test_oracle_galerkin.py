"""Pins of the oracle's geometry, assembly and direct solve (Problem 1, Sec. 2.2)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fd, geometry, problems, spline
from oracle.galerkin import Component, stiffness_1d


# -- geometry -------------------------------------------------------------------

def test_annulus_radius_and_jacobian():
    g = geometry.QuarterAnnulus(2)
    xi = np.random.default_rng(0).random((500, 2))
    x = g.map(xi)
    np.testing.assert_allclose(np.hypot(x[:, 0], x[:, 1]), 1.0 + xi[:, 0], rtol=1e-14)
    assert np.all(x >= -1e-15)
    # Jacobian against central differences
    h = 1e-6
    J = g.jacobian(xi)
    for k in range(2):
        e = np.zeros(2); e[k] = h
        fdJ = (g.map(xi + e) - g.map(xi - e)) / (2 * h)
        np.testing.assert_allclose(J[:, :, k], fdJ, atol=1e-8)
    # separable metric: columns orthogonal, |dF/dxi1| = 1
    np.testing.assert_allclose(np.einsum("ni,ni->n", J[:, :, 0], J[:, :, 1]), 0.0, atol=1e-13)
    np.testing.assert_allclose(np.linalg.norm(J[:, :, 0], axis=1), 1.0, rtol=1e-14)
    # corners of the parametric square
    c = g.map(np.array([[0, 0], [1, 0], [0, 1], [1, 1.0]]))
    np.testing.assert_allclose(c, [[1, 0], [2, 0], [0, 1], [0, 2]], atol=1e-15)


def test_annulus_area_by_quadrature():
    g = geometry.QuarterAnnulus(2)
    xi, w = spline.element_quadrature(np.linspace(0, 1, 9), 5)
    X, Y = np.meshgrid(xi.reshape(-1), xi.reshape(-1), indexing="ij")
    WX, WY = np.meshgrid(w.reshape(-1), w.reshape(-1), indexing="ij")
    pts = np.stack([X.reshape(-1), Y.reshape(-1)], 1)
    det = np.linalg.det(g.jacobian(pts))
    assert np.all(det > 0)
    np.testing.assert_allclose(np.sum(WX.reshape(-1) * WY.reshape(-1) * det), 0.75 * np.pi, rtol=1e-12)


# -- assembly -------------------------------------------------------------------

@pytest.mark.parametrize("levels,p,r", [((2, 3), 2, 1), ((3, 1), 3, 2), ((2, 2), 2, 0),
                                        ((1, 2, 2), 2, 1), ((2, 1, 1), 3, 2)])
def test_kronecker_structure_on_unit_cube(levels, p, r):
    """On the unit square/cube K = sum_k M x .. K_k .. x M (1D matrices) exactly."""
    d = len(levels)
    c = Component(geometry.UnitCube(d), levels, p, r).assemble()
    ones = [stiffness_1d(l, p, r) for l in levels]
    K = None
    for k in range(d):
        term = None
        for j in range(d - 1, -1, -1):      # direction d is the slowest factor
            f = sp.csr_matrix(ones[j][0] if j == k else ones[j][1])
            term = f if term is None else sp.kron(term, f)
        K = term if K is None else K + term
    diff = abs(c.K - K.tocsc()).max()
    assert diff < 1e-12 * abs(K).max()


@pytest.mark.parametrize("levels,p,r", [((2, 3), 2, 1), ((1, 2, 2), 3, 2), ((2, 2), 3, 0)])
def test_constant_in_kernel_and_mass_total(levels, p, r):
    d = len(levels)
    c = Component(geometry.UnitCube(d), levels, p, r).assemble(with_mass=True)
    one = np.ones(c.nfull)
    np.testing.assert_allclose(c.K_full @ one, 0.0, atol=1e-11)
    np.testing.assert_allclose(one @ (c.M_full @ one), 1.0, rtol=1e-13)


def _space_coeffs(comp, fun_param):
    """Coefficients (full numbering) of a function of xi that lies in the space.

    Found by collocation at the Greville-like points of each direction, which is
    exact when the function is in the space."""
    d = comp.d
    pts1 = [np.linspace(0, 1, s.nf) for s in comp.spaces]
    V = [comp.spaces[k].values_at(pts1[k]) for k in range(d)]
    grids = np.meshgrid(*pts1[::-1], indexing="ij")
    P = np.stack([g.reshape(-1) for g in grids[::-1]], 1)
    A = V[0]
    for k in range(1, d):
        A = np.kron(V[k], A)
    return np.linalg.solve(A, fun_param(P))


@pytest.mark.parametrize("p", [2, 3])
def test_annulus_harmonic_functions_are_galerkin_exact(p):
    """x and y are harmonic and lie in the NURBS space, so interior rows of K
    annihilate their coefficients up to the Gauss rule's error on the rational
    integrand; that error falls by at least 2^(2p) per uniform refinement."""
    g = geometry.QuarterAnnulus(2)
    for col in range(2):
        prev = None
        for lv in (1, 2, 3, 4):
            comp = Component(g, (lv, lv), p).assemble()
            c = _space_coeffs(comp, lambda P: g.map(P)[:, col])
            res = np.max(np.abs((comp.K_full @ c)[comp.interior]))
            res /= np.max(np.abs(comp.K_full @ np.abs(c)))
            if prev is not None:
                assert res < prev / 2 ** (2 * p)
            prev = res
        assert prev < 1e-8


def test_annulus_basis_scaling_reading():
    """The refined-NURBS basis w_i B_i / W and B_i / W span the same space: same solution."""
    g = geometry.QuarterAnnulus(2)
    prob = problems.get("annulus_paper2")
    comp = Component(g, (2, 3), 2).assemble(f=prob.f)
    u = comp.solve()
    # refined weights of W in the angular space of this component, by collocation
    s = comp.spaces[1]
    t = np.linspace(0, 1, s.nf)
    Bm = spline.bspline_basis(s.knots, 2, t)
    W, _ = g.weight_1d(1, t)
    wref = np.linalg.solve(Bm, W)
    assert np.all(wref > 0)
    # weighted basis: R'_i = w_i R_i; coefficients scale by 1/w_i, values unchanged
    n1 = comp.nf[0]
    wfull = np.repeat(wref, n1)                  # direction 1 fastest
    Dw = sp.diags(wfull[comp.interior])
    K2 = (Dw @ comp.K @ Dw).tocsc()
    b2 = Dw @ comp.b
    import scipy.sparse.linalg as spla
    u2 = spla.spsolve(K2, b2)
    pts = np.random.default_rng(3).random((50, 2))
    v1 = comp.evaluate(u, pts)
    v2 = comp.evaluate(u2 * wfull[comp.interior], pts)
    np.testing.assert_allclose(v1, v2, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("d,levels,p", [(2, (1, 1), 2), (2, (2, 1), 2), (2, (1, 3), 3),
                                        (3, (1, 1, 1), 2), (3, (1, 2, 1), 3)])
def test_exact_reproduction_polynomial(d, levels, p):
    """u = prod x(1-x) lies in every space with p >= 2: the Galerkin solution is u."""
    prob = problems.get("poly%d" % d)
    comp = Component(geometry.UnitCube(d), levels, p).assemble(f=prob.f)
    u = comp.solve()
    pts = np.random.default_rng(4).random((100, d))
    np.testing.assert_allclose(comp.evaluate(u, pts), prob.u(pts), atol=1e-14)


def test_direct_solve_residual():
    prob = problems.get("sine3")
    comp = Component(geometry.UnitCube(3), (2, 1, 2), 3).assemble(f=prob.f)
    u = comp.solve()
    assert np.linalg.norm(comp.b - comp.K @ u) <= 1e-14 * np.linalg.norm(comp.b) * 10


# -- fast diagonalisation --------------------------------------------------------

@pytest.mark.parametrize("levels,p,r", [((2, 3), 2, 1), ((3, 1), 3, 2), ((1, 2, 2), 3, 2),
                                        ((2, 1, 1), 2, 0)])
def test_fd_is_exact_inverse_on_unit_cube(levels, p, r):
    d = len(levels)
    comp = Component(geometry.UnitCube(d), levels, p, r).assemble()
    rv = np.random.default_rng(5).standard_normal(comp.ndof)
    z = fd.fd_apply(levels, p, r, rv)
    np.testing.assert_allclose(comp.K @ z, rv, rtol=1e-9, atol=1e-9 * np.abs(rv).max())


def test_fd_eig_properties():
    lam, U = fd.eig_1d(5, 3, 2)
    K, M = stiffness_1d(5, 3, 2)
    np.testing.assert_allclose(U.T @ M @ U, np.eye(len(lam)), atol=1e-10)
    np.testing.assert_allclose(K @ U, M @ U * lam[None, :], atol=1e-8 * lam.max())
    assert np.all(lam > 0)


@pytest.mark.parametrize("domain,levels,p", [("annulus", (2, 3, 1), 2), ("unit", (1, 2, 3), 3)])
def test_parametric_gradient_3d_matches_central_differences(domain, levels, p):
    """evaluate_grad in 3D (rational directions included) against central
    differences of evaluate, for random coefficients at interior points."""
    from oracle import geometry
    from oracle.galerkin import Component
    comp = Component(geometry.make(domain, 3), levels, p)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(comp.ndof)
    pts = rng.uniform(0.05, 0.95, size=(20, 3))
    g = comp.evaluate_grad(u, pts)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (comp.evaluate(u, pts + e) - comp.evaluate(u, pts - e)) / (2 * h)
        assert np.abs(g[:, k] - fd).max() < 1e-6 * max(1.0, np.abs(g[:, k]).max()), k


def test_sturm_eigenvalues_closed_form_and_dense_solver():
    """Bisection on the inertia of K - s M: the linear-element pencil has the
    closed form lam_k = 6/h^2 (1 - cos(k pi h)) / (2 + cos(k pi h)); on a
    uniform cubic pencil it agrees with the dense generalised eigensolver."""
    import scipy.linalg as sla
    from oracle import fd
    from oracle.galerkin import stiffness_1d
    K, M = stiffness_1d(5, 1, 0)
    h, n = 1.0 / 32, K.shape[0]
    k = np.arange(1, n + 1)
    closed = 6 / h ** 2 * (1 - np.cos(k * np.pi * h)) / (2 + np.cos(k * np.pi * h))
    js = [0, 1, n // 2, n - 1]
    np.testing.assert_allclose(fd.sturm_eigenvalues(K, M, js), closed[js], rtol=1e-13)
    K, M = stiffness_1d(4, 3, 2)
    ref = sla.eigh(K, M, eigvals_only=True)
    js = [0, 3, 9, K.shape[0] - 1]
    np.testing.assert_allclose(fd.sturm_eigenvalues(K, M, js), ref[js], rtol=1e-12)
