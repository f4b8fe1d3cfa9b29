"""Geometry maps F of the oracle (paper Sec. 2.2, eq. F-B-splines and NURBS).

TEST INFRASTRUCTURE: see the package header.

A geometry exposes
  d                    dimension
  map(xi)              x = F(xi), xi [N, d] -> [N, d]
  jacobian(xi)         J[n, i, k] = dx_i / dxi_k
  weight_1d(k, t)      (W_k(t), W_k'(t)): the rational weight function of
                       parametric direction k (1 and 0 for polynomial directions)

Reading of "verbatim for NURBS" (Sec. 2.2): the discrete space of a
component is the NURBS space obtained by refining the geometry's NURBS. The
geometry's weight function W is a tensor product of 1D weight functions W_k
for the domains used here, and refinement does not change W, so that space
equals span{ prod_k B_{i_k}(xi_k) / W_k(xi_k) }. A Galerkin solution is a
function of the space alone, so this basis (which differs from the refined
NURBS basis only by the positive scalings w_i) gives the same solution.
"""
import numpy as np

from . import spline


class UnitCube:
    """Identity map on [0,1]^d (the unit square or cube)."""

    def __init__(self, d):
        self.d = d

    def map(self, xi):
        return np.array(xi, dtype=np.float64, copy=True)

    def jacobian(self, xi):
        n = np.asarray(xi).shape[0]
        return np.broadcast_to(np.eye(self.d), (n, self.d, self.d)).copy()

    def weight_1d(self, k, t):
        t = np.asarray(t, dtype=np.float64)
        return np.ones_like(t), np.zeros_like(t)

    def measure(self):
        return 1.0


class QuarterAnnulus:
    """Quarter annulus with radii 1 and 2 in the first quadrant (Sec. 4.2).

    Parametrised as a NURBS patch: direction 1 radial, degree 1, control radii
    1 and 2; direction 2 angular, degree 2, control points (1,0), (1,1), (0,1)
    times the radius with weights 1, sqrt(2)/2, 1. In 3D the patch is extruded
    along z in [0, 1] (direction 3, degree 1). Both evaluated through the
    oracle's Cox-de Boor routine.
    """

    R_IN, R_OUT = 1.0, 2.0

    def __init__(self, d=2):
        self.d = d
        self.k1 = np.array([0.0, 0.0, 1.0, 1.0])
        self.k2 = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
        self.rad = np.array([self.R_IN, self.R_OUT])
        self.ang = np.array([[1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
        self.wang = np.array([1.0, np.sqrt(2.0) / 2.0, 1.0])

    def _angular(self, t):
        """Rational quarter circle c(t), its derivative, W and W'."""
        N = spline.bspline_basis(self.k2, 2, t)
        dN = spline.bspline_deriv(self.k2, 2, t)
        W = N @ self.wang
        dW = dN @ self.wang
        A = (N * self.wang[None, :]) @ self.ang
        dA = (dN * self.wang[None, :]) @ self.ang
        c = A / W[:, None]
        dc = (dA * W[:, None] - A * dW[:, None]) / (W ** 2)[:, None]
        return c, dc, W, dW

    def _radial(self, t):
        N = spline.bspline_basis(self.k1, 1, t)
        dN = spline.bspline_deriv(self.k1, 1, t)
        return N @ self.rad, dN @ self.rad

    def map(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        rho, _ = self._radial(xi[:, 0])
        c, _, _, _ = self._angular(xi[:, 1])
        x = rho[:, None] * c
        if self.d == 3:
            x = np.concatenate([x, xi[:, 2:3]], axis=1)
        return x

    def jacobian(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        n = xi.shape[0]
        rho, drho = self._radial(xi[:, 0])
        c, dc, _, _ = self._angular(xi[:, 1])
        J = np.zeros((n, self.d, self.d))
        J[:, 0:2, 0] = drho[:, None] * c
        J[:, 0:2, 1] = rho[:, None] * dc
        if self.d == 3:
            J[:, 2, 2] = 1.0
        return J

    def weight_1d(self, k, t):
        t = np.asarray(t, dtype=np.float64)
        if k == 1:
            _, _, W, dW = self._angular(t)
            return W, dW
        return np.ones_like(t), np.zeros_like(t)

    def measure(self):
        return 0.75 * np.pi * (1.0 if self.d == 2 else 1.0)


class BSplinePatch:
    """Tensor-product B-spline patch F(xi) = sum_i P_i prod_k N_{i_k}(xi_k)
    (eq. F-B-splines) with polynomial (weight 1) directions, evaluated with the
    oracle's Cox-de Boor routine."""

    def __init__(self, degrees, knots, cps):
        self.d = len(degrees)
        self.deg = list(degrees)
        self.knots = [np.asarray(k, dtype=np.float64) for k in knots]
        self.ncp = [len(k) - p - 1 for k, p in zip(self.knots, self.deg)]
        self.cp = np.asarray(cps, dtype=np.float64).reshape(self.ncp[::-1] + [self.d])

    def _basis(self, xi):
        N = [spline.bspline_basis(self.knots[k], self.deg[k], xi[:, k]) for k in range(self.d)]
        dN = [spline.bspline_deriv(self.knots[k], self.deg[k], xi[:, k]) for k in range(self.d)]
        return N, dN

    def map(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        N, _ = self._basis(xi)
        if self.d == 3:
            return np.einsum("pc,pb,pa,cbai->pi", N[2], N[1], N[0], self.cp, optimize=True)
        return np.einsum("pb,pa,bai->pi", N[1], N[0], self.cp)

    def jacobian(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        N, dN = self._basis(xi)
        cols = []
        for k in range(self.d):
            f = [dN[j] if j == k else N[j] for j in range(self.d)]
            if self.d == 3:
                cols.append(np.einsum("pc,pb,pa,cbai->pi", f[2], f[1], f[0], self.cp, optimize=True))
            else:
                cols.append(np.einsum("pb,pa,bai->pi", f[1], f[0], self.cp))
        return np.stack(cols, axis=2)

    def weight_1d(self, k, t):
        t = np.asarray(t, dtype=np.float64)
        return np.ones_like(t), np.zeros_like(t)


class AxisMap:
    """x = s * xi with s in {-1, 1}^d: the unit square or cube reflected along
    the directions with s_k = -1 (a bilinear patch of the L-shaped domain;
    its Jacobian diag(s) may reverse orientation)."""

    def __init__(self, signs):
        self.s = np.asarray(signs, dtype=np.float64)
        self.d = len(self.s)

    def map(self, xi):
        return np.asarray(xi, dtype=np.float64) * self.s[None, :]

    def jacobian(self, xi):
        n = np.asarray(xi).shape[0]
        return np.broadcast_to(np.diag(self.s), (n, self.d, self.d)).copy()

    def weight_1d(self, k, t):
        t = np.asarray(t, dtype=np.float64)
        return np.ones_like(t), np.zeros_like(t)


def lognormal_coefficient(omega, phase, amp):
    """a(x) = exp(amp * sum_f cos(omega_f . x + phase_f)) (random Fourier features)."""
    omega = np.asarray(omega, dtype=np.float64)
    phase = np.asarray(phase, dtype=np.float64)

    def a(x):
        x = np.asarray(x, dtype=np.float64)
        return np.exp(amp * np.cos(x @ omega.T + phase[None, :]).sum(axis=1))
    return a


def make(name, d):
    if name in ("unit", "square", "cube"):
        return UnitCube(d)
    if name == "annulus":
        return QuarterAnnulus(d)
    raise ValueError(name)
