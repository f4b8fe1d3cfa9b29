"""1D spline machinery of the oracle (paper Sec. 2.2, eq. Bsp; Sec. 3; Sec. 4.4).

TEST INFRASTRUCTURE: see the package header. Plain, slow, FP64.
"""
import numpy as np


# ----------------------------------------------------------------------------
# Breakpoints and knot vectors
# ----------------------------------------------------------------------------

def grading_map(t, kind="uniform", gamma=1.0):
    """Breakpoint map g: [0,1] -> [0,1] applied to equispaced t.

    kind "uniform":  g(t) = t.
    kind "radical":  the symmetric radical map of Sec. 4.4 ("Radical meshes in
                     the parametric domain"): t^gamma / 2^(1-gamma) for t <= 1/2
                     and 1 - (1-t)^gamma / 2^(1-gamma) otherwise. The printed
                     denominator "1/2^(gamma-1)" is read as 2^(1-gamma), i.e.
                     g(t) = 2^(gamma-1) t^gamma, which makes g(1/2) = 1/2.
    kind "onesided": g(t) = t^gamma, graded toward t = 0 (not in the paper; the
                     one-sided grading of the L-shape workload).
    gamma = 1 recovers the uniform mesh for both graded kinds.
    """
    t = np.asarray(t, dtype=np.float64)
    if kind == "uniform":
        return t.copy()
    if kind == "radical":
        c = 2.0 ** (gamma - 1.0)
        return np.where(t <= 0.5, c * t ** gamma, 1.0 - c * (1.0 - t) ** gamma)
    if kind == "onesided":
        return t ** gamma
    raise ValueError(kind)


def breakpoints(E, kind="uniform", gamma=1.0):
    """Z = [zeta_0 .. zeta_E]: E elements, images of j/E under the grading map."""
    z = grading_map(np.arange(E + 1, dtype=np.float64) / E, kind, gamma)
    z[0], z[-1] = 0.0, 1.0
    return z


def open_knot_vector(E, p, r, kind="uniform", gamma=1.0):
    """Open knot vector of degree p with E elements and continuity C^r.

    Sec. 2.2: the end knots have multiplicity p+1 (open vector); an interior
    breakpoint of multiplicity m gives continuity C^(p-m), so C^r uses
    m = p - r. Returns the knots as a float64 array of length n + p + 1 with
    n = E (p - r) + r + 1 basis functions.
    """
    if not (0 <= r <= p - 1):
        raise ValueError("continuity r must satisfy 0 <= r <= p-1")
    z = breakpoints(E, kind, gamma)
    m = p - r
    knots = [z[0]] * (p + 1)
    for j in range(1, E):
        knots += [z[j]] * m
    knots += [z[-1]] * (p + 1)
    return np.array(knots, dtype=np.float64)


def n_basis(E, p, r):
    """Number of B-splines of degree p, C^r, on E elements (open knots)."""
    return E * (p - r) + r + 1


# ----------------------------------------------------------------------------
# Gauss-Legendre rule
# ----------------------------------------------------------------------------

def gauss_legendre(Q):
    """Q-point Gauss-Legendre nodes and weights on [-1, 1] (numpy's leggauss)."""
    x, w = np.polynomial.legendre.leggauss(Q)
    return x.astype(np.float64), w.astype(np.float64)


def element_quadrature(z, Q):
    """Gauss points/weights on each element [z_e, z_{e+1}].

    Returns xi [E, Q] and w [E, Q]; w includes the Jacobian h_e / 2.
    """
    t, wt = gauss_legendre(Q)
    a, b = z[:-1], z[1:]
    h = b - a
    xi = a[:, None] + 0.5 * (1.0 + t[None, :]) * h[:, None]
    w = 0.5 * h[:, None] * wt[None, :]
    return xi, w


# ----------------------------------------------------------------------------
# Cox-de Boor recursion (eq. Bsp)
# ----------------------------------------------------------------------------

def _ratio(num, den):
    """num / den with the convention 0/0 = 0 (and x/0 = 0 where den == 0)."""
    out = np.zeros(np.broadcast(num, den).shape)
    nz = den != 0.0
    np.divide(num, den, out=out, where=nz)
    return out


def _degree0(knots, xi):
    """B_{i,0}(xi) for every i: indicator of [xi_i, xi_{i+1}).

    At the right end of the parameter interval the half-open intervals give
    zero everywhere; we close the last non-degenerate interval there so that
    B_{n,p}(1) = 1 (interpolation at the end knots, Sec. 2.2).
    """
    xi = np.asarray(xi, dtype=np.float64)
    lo, hi = knots[:-1], knots[1:]
    N0 = ((lo[None, :] <= xi[:, None]) & (xi[:, None] < hi[None, :])).astype(np.float64)
    last = np.nonzero(hi > lo)[0][-1]
    at_end = xi >= knots[-1]
    N0[at_end, :] = 0.0
    N0[at_end, last] = 1.0
    return N0


def cox_de_boor_all(knots, p, xi):
    """All B-splines of degree 0..p at the points xi, by eq. Bsp.

    Returns a list N with N[k] of shape [len(xi), len(knots) - 1 - k] holding
    B_{i,k}(xi). The recursion is the literal one of eq. Bsp:
    B_{i,k} = (xi - xi_i)/(xi_{i+k} - xi_i) B_{i,k-1}
            + (xi_{i+k+1} - xi)/(xi_{i+k+1} - xi_{i+1}) B_{i+1,k-1}, 0/0 = 0.
    """
    xi = np.asarray(xi, dtype=np.float64)
    N = [_degree0(knots, xi)]
    m = len(knots) - 1
    for k in range(1, p + 1):
        prev = N[-1]
        cnt = m - k
        i = np.arange(cnt)
        left = _ratio(xi[:, None] - knots[i][None, :], (knots[i + k] - knots[i])[None, :])
        right = _ratio(knots[i + k + 1][None, :] - xi[:, None],
                       (knots[i + k + 1] - knots[i + 1])[None, :])
        N.append(left * prev[:, :cnt] + right * prev[:, 1:cnt + 1])
    return N


def bspline_basis(knots, p, xi):
    """B_{i,p}(xi), i = 0..n-1: array [len(xi), n]."""
    return cox_de_boor_all(knots, p, xi)[p]


def bspline_deriv(knots, p, xi):
    """d/dxi B_{i,p}(xi): array [len(xi), n].

    Standard derivative formula (de Boor): B'_{i,p} = p/(xi_{i+p}-xi_i) B_{i,p-1}
    - p/(xi_{i+p+1}-xi_{i+1}) B_{i+1,p-1}, with 0/0 = 0.
    """
    if p == 0:
        return np.zeros_like(bspline_basis(knots, 0, xi))
    Nm = cox_de_boor_all(knots, p - 1, xi)[p - 1]
    n = len(knots) - p - 1
    i = np.arange(n)
    a = _ratio(np.full(n, float(p)), knots[i + p] - knots[i])
    b = _ratio(np.full(n, float(p)), knots[i + p + 1] - knots[i + 1])
    return a[None, :] * Nm[:, :n] - b[None, :] * Nm[:, 1:n + 1]


def element_first_function(knots, p, z):
    """Index of the first nonzero B-spline on each element [z_e, z_{e+1}].

    Found by locating each element midpoint in the knot vector: the span s with
    xi_s <= mid < xi_{s+1}; the nonzero functions are s-p .. s.
    """
    mid = 0.5 * (z[:-1] + z[1:])
    s = np.searchsorted(knots, mid, side="right") - 1
    return s - p
