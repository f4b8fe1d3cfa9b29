"""Whole-method runs of the oracle: every component, then the combination.

TEST INFRASTRUCTURE: see the package header.

solve_components  assemble + direct-solve every component of the index set
                  (Sec. 3, eq. TD-combi-tec; Sec. 4.1: direct solver)
combined_at       evaluate each component at parametric points and combine
errors            L2 / H1 errors of the combined solution against the exact
                  u, by Gauss quadrature on a fine parametric mesh mapped by F
rate              least-squares slope of log2(error) against the level
                  (Sec. 4.2: rates fitted with a polynomial fit)
functional        l(u) = int g u of the combined solution from the
                  components' load vectors (no evaluation points)
"""
import numpy as np

from . import combination, geometry, problems, spline
from .galerkin import Component


def solve_components(domain, d, p, w, problem, r=None, min_level=1,
                     kind="uniform", gamma=1.0, only=None):
    """Solve the components (all, or the listed multi-indices `only`).

    Returns a list of (i, c_i, component, solution coefficients).
    """
    geom = geometry.make(domain, d)
    prob = problems.get(problem)
    out = []
    for i, c in combination.index_set(d, w, min_level):
        if only is not None and tuple(i) not in only:
            continue
        comp = Component(geom, i, p, r, kind, gamma).assemble(f=prob.f)
        out.append((i, c, comp, comp.solve()))
    return out


def combined_at(results, pts):
    vals = np.stack([comp.evaluate(u, pts) for _, _, comp, u in results])
    coeffs = np.array([c for _, c, _, _ in results], dtype=np.float64)
    return combination.combine(vals, coeffs), vals


def _fine_rule(d, nel, Q):
    z = np.linspace(0.0, 1.0, nel + 1)
    xi, w = spline.element_quadrature(z, Q)
    xi, w = xi.reshape(-1), w.reshape(-1)
    grids = np.meshgrid(*([xi] * d), indexing="ij")
    wg = np.meshgrid(*([w] * d), indexing="ij")
    pts = np.stack([g.reshape(-1) for g in grids], axis=1)
    wts = np.prod(np.stack([g.reshape(-1) for g in wg], axis=1), axis=1)
    return pts, wts


def errors(results, problem, nel=64, Q=None, with_h1=True):
    """(L2, H1-seminorm) errors of sum_i c_i u_i against the exact solution.

    The integrals over Omega = F(Omega_hat) use a (p+2)-point Gauss rule on a
    uniform parametric mesh of nel^d elements, with weights times |det J|.
    """
    comp0 = results[0][2]
    geom, d, p = comp0.geom, comp0.d, comp0.p
    prob = problems.get(problem)
    Q = p + 2 if Q is None else Q
    pts, wts = _fine_rule(d, nel, Q)
    J = geom.jacobian(pts)
    det = np.abs(np.linalg.det(J))
    x = geom.map(pts)
    coeffs = np.array([c for _, c, _, _ in results], dtype=np.float64)
    uh = combination.combine(np.stack([cp.evaluate(u, pts) for _, _, cp, u in results]), coeffs)
    e2 = np.sum(wts * det * (prob.u(x) - uh) ** 2)
    out = [np.sqrt(e2)]
    if with_h1:
        gh = [cp.evaluate_grad(u, pts) for _, _, cp, u in results]
        gref = np.tensordot(coeffs, np.stack(gh), axes=1)          # [P, d] parametric
        gx = np.linalg.solve(np.transpose(J, (0, 2, 1)), gref[..., None])[..., 0]
        h2 = np.sum(wts * det * np.sum((prob.grad_u(x) - gx) ** 2, axis=1))
        out.append(np.sqrt(h2))
    return tuple(out)


def rate(levels, errs):
    """Least-squares slope s in log2(err) ~ -s * level."""
    A = np.vstack([np.asarray(levels, dtype=np.float64), np.ones(len(levels))]).T
    slope, _ = np.linalg.lstsq(A, np.log2(np.asarray(errs)), rcond=None)[0]
    return -slope


def functional(results, g):
    """Linear functional l(u) = int_Omega g u dx of the combined solution,
    without evaluating it anywhere: sum_i c_i l(u_i), with l(u_i) = b_g . u_i,
    b_g the Galerkin load vector of g in component i's space (the same rule as
    the right-hand side, Sec. 2.2). Returns (per-component values, combined
    value with Neumaier compensation, eq. TD-combi-tec)."""
    vals, coef = [], []
    for _, c, comp, u in results:
        vals.append(float(comp.load_vector(g) @ u))
        coef.append(c)
    vals = np.array(vals)
    return vals, float(combination.combine(vals[:, None], np.array(coef, dtype=np.float64))[0])
