"""Multi-patch components: the L-shaped domain with Dirichlet data.

TEST INFRASTRUCTURE: see the package header. Not in the paper's experiments
(its multi-patch example, the horseshoe, is out of scope); the L-shape is a
standard singular test of graded meshes, which is the paper's topic in
Sec. 4.4.

Domain (-1,1)^2 minus [0,1] x [-1,0], split into three unit squares. Each
one is the image of [0,1]^2 under x = s * xi, with the parametric origin at
the re-entrant corner (0,0):

    patch 0: (0,1) x (0,1),    s = ( 1,  1)
    patch 1: (-1,0) x (0,1),   s = (-1,  1)
    patch 2: (-1,0) x (-1,0),  s = (-1, -1)

Interfaces: side xi_1 = 0 of patches 0 and 1 (the segment x = 0, 0 < y < 1,
with the same parameter xi_2 on both); side xi_2 = 0 of patches 1 and 2
(y = 0, -1 < x < 0, same xi_1). Every other side is a Dirichlet side. A
component (i_1, i_2) uses the same knot vector of level i_k in direction k on
every patch, graded toward xi_k = 0 (the corner). The two traces on an
interface are then the same 1D spline space. Conforming C^0 gluing merges
the trace functions of the two sides into one global function.

Boundary data g (readings; the paper is silent on nonhomogeneous data):
corner coefficients interpolate g at the patch corners. The remaining
coefficients of each Dirichlet side are the L2 projection of g onto the
side's 1D spline space, with the corner coefficients fixed. The projection
uses the parametric measure, which is arc length for these unit sides, and
p+1 Gauss points per element, the rule of the assembly. Then
b_I <- b_I - K_IB g_B.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import spline
from .galerkin import Component
from .geometry import AxisMap

SIGNS = ((1.0, 1.0), (-1.0, 1.0), (-1.0, -1.0))
# Dirichlet sides per patch: (direction, end) with end 0 at xi_k = 0, 1 at xi_k = 1
DIRICHLET = (((1, 0), (0, 1), (1, 1)),           # patch 0: y = 0 (x > 0), x = 1, y = 1
             ((0, 1), (1, 1)),                   # patch 1: x = -1, y = 1
             ((0, 0), (0, 1), (1, 1)))           # patch 2: x = 0 (y < 0), x = -1, y = -1
# interface sides: (patch a, patch b, direction whose index is 0 on the side)
INTERFACES = ((0, 1, 0), (1, 2, 1))


def physical(patch, xi):
    return np.asarray(xi, dtype=np.float64) * np.asarray(SIGNS[patch])[None, :]


class LShapeComponent:
    """Glued, Dirichlet-lifted system of one component grid on the L-shape."""

    def __init__(self, levels, p, r=None, kind="onesided", gamma=1.0):
        self.levels = tuple(int(v) for v in levels)
        self.p = p
        self.r = p - 1 if r is None else r
        self.kind, self.gamma = kind, gamma
        self.patches = [Component(AxisMap(s), self.levels, p, self.r, kind, gamma) for s in SIGNS]
        self.nf = self.patches[0].nf                     # functions per direction (same on every patch)
        nf0, nf1 = self.nf
        # global ids of each patch's functions, local full index a + nf0 * b
        ids = []
        nxt = 0
        for q in range(3):
            gid = -np.ones(nf0 * nf1, dtype=np.int64)
            for (pa, pb, k) in INTERFACES:
                if pb != q:
                    continue
                # the side with index 0 in direction k: copy the ids of patch pa
                for t in range(self.nf[1 - k]):
                    loc = (0 + nf0 * t) if k == 0 else (t + nf0 * 0)
                    gid[loc] = ids[pa][loc]
            new = gid < 0
            gid[new] = nxt + np.arange(new.sum())
            nxt += int(new.sum())
            ids.append(gid)
        self.ids = ids
        self.nglob = nxt
        dirich = np.zeros(nxt, dtype=bool)
        for q in range(3):
            for (k, end) in DIRICHLET[q]:
                dirich[ids[q][self._side(k, end)]] = True
        self.dirichlet = dirich
        self.interior = np.nonzero(~dirich)[0]
        self.boundary = np.nonzero(dirich)[0]
        self.ndof = len(self.interior)

    def _side(self, k, end):
        """Local full indices of the functions on side (k, end), ordered along the side."""
        nf0, nf1 = self.nf
        i = 0 if end == 0 else self.nf[k] - 1
        t = np.arange(self.nf[1 - k])
        return (i + nf0 * t) if k == 0 else (t + nf0 * i)

    # -- assembly ---------------------------------------------------------------
    def assemble(self, f=None, g=None):
        """Glued stiffness over all functions, load vector, boundary lifting.

        f(x) is the source (None: 0); g(x) the Dirichlet data (None: 0)."""
        rows, cols, vals = [], [], []
        b = np.zeros(self.nglob)
        for q in range(3):
            comp = self.patches[q].assemble(f=f if f is not None else (lambda x: np.zeros(len(x))))
            Kf = comp.K_full.tocoo()
            rows.append(self.ids[q][Kf.row])
            cols.append(self.ids[q][Kf.col])
            vals.append(Kf.data)
            np.add.at(b, self.ids[q], comp.b_full)
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.nglob, self.nglob))
        self.K_glob = K
        self.gB = self.boundary_coefficients(g)
        I, B = self.interior, self.boundary
        self.K = K[I][:, I].tocsc()
        self.b = b[I] - K[I][:, B] @ self.gB[B]
        return self

    def boundary_coefficients(self, g):
        """Global coefficient vector holding g's lifting on the Dirichlet functions."""
        c = np.zeros(self.nglob)
        if g is None:
            return c
        for q in range(3):
            for (k, end) in DIRICHLET[q]:
                sp1 = self.patches[q].spaces[1 - k]           # the side's parameter direction
                side = self._side(k, end)
                xi_fixed = 0.0 if end == 0 else 1.0
                coef = self._project(sp1, lambda t: g(physical(q, self._side_points(k, xi_fixed, t))))
                c[self.ids[q][side]] = coef
        return c

    @staticmethod
    def _side_points(k, fixed, t):
        pts = np.zeros((len(t), 2))
        pts[:, k] = fixed
        pts[:, 1 - k] = t
        return pts

    def _project(self, s, gfun):
        """Coefficients c_0..c_{nf-1} on one side: ends interpolate g, the
        interior ones are the L2 projection (p+1 Gauss points per element)."""
        p, nf = self.p, s.nf
        M = np.zeros((nf, nf))
        rhs = np.zeros(nf)
        for e in range(s.E):
            idx = s.first[e] + np.arange(p + 1)
            gv = gfun(s.xi[e])
            for qq in range(s.Q):
                M[np.ix_(idx, idx)] += s.w[e, qq] * np.outer(s.R[e, qq], s.R[e, qq])
                rhs[idx] += s.w[e, qq] * gv[qq] * s.R[e, qq]
        c = np.zeros(nf)
        c[0] = gfun(np.array([0.0]))[0]
        c[-1] = gfun(np.array([1.0]))[0]
        inner = slice(1, nf - 1)
        r = rhs[inner] - M[inner, 0] * c[0] - M[inner, -1] * c[-1]
        c[inner] = np.linalg.solve(M[inner, inner], r)
        return c

    def solve(self, b=None):
        """Sparse direct solve of the interior system (the paper's solver,
        Sec. 4.1), with iterative refinement: x += LU^{-1}(b - K x) while the
        correction shrinks (at most 6 steps). Strong one-sided grading makes
        these systems very ill-conditioned (gamma = 3, w = 11: cond ~ 1e12,
        elements of relative size 1e-9 at the corner; symmetric diagonal
        equilibration still leaves 4e9). There, threshold-pivoted sparse LU
        leaves a solution error of ~5e-8. Refinement removes part of it, down
        to the floor of the FP64 residual: relative ~1e-8 for the most
        anisotropic components. That floor bounds how closely any FP64 solver
        can agree with this reference for such systems."""
        rhs = self.b if b is None else b
        lu = spla.splu(self.K)
        x = lu.solve(rhs)
        prev = np.inf
        for _ in range(6):
            dx = lu.solve(rhs - self.K @ x)
            nd = np.linalg.norm(dx)
            x = x + dx
            if nd >= 0.5 * prev or nd <= 1e-17 * np.linalg.norm(x):
                break
            prev = nd
        return x

    def solve_extended(self, b=None, steps=20):
        """The same system solved to beyond FP64's reach: iterative refinement
        whose residual b - K x and iterate x are kept in extended precision
        (numpy longdouble: 64-bit significand on x86, 113-bit on AArch64),
        corrections from the FP64 sparse LU. K is the FP64 assembled matrix,
        taken as exact; the iteration converges to its solution (relative
        residual ~1e-13 where the FP64 refinement stalls at ~1e-10 on the most
        graded systems) and is the reference the FP64 solvers are measured
        against (its own floor, extended unit roundoff times the condition,
        is ~1e-13 relative on those systems with the x86 format). Returns
        float64 coefficients."""
        rhs = self.b if b is None else b          # float64, or longdouble for an exactly known b
        K = self.K.tocsr()
        data = K.data.astype(np.longdouble)
        nz = np.diff(K.indptr) > 0
        starts = K.indptr[:-1][nz]

        def residual(x):
            prod = data * x[K.indices]
            kx = np.zeros(K.shape[0], dtype=np.longdouble)
            kx[nz] = np.add.reduceat(prod, starts)
            return np.asarray(rhs, dtype=np.longdouble) - kx

        lu = spla.splu(self.K)
        x = lu.solve(np.asarray(rhs, dtype=np.float64)).astype(np.longdouble)
        prev = np.inf
        for _ in range(steps):       # until the corrections stop shrinking
            dx = lu.solve(np.asarray(residual(x), dtype=np.float64))
            nd = np.linalg.norm(dx)
            x = x + dx
            if nd >= 0.5 * prev or nd <= 1e-18 * float(np.linalg.norm(np.asarray(x, dtype=np.float64))):
                break
            prev = nd
        return np.asarray(x, dtype=np.float64)

    def full(self, u):
        """Global coefficients: interior from u, boundary from the lifting."""
        c = self.gB.copy()
        c[self.interior] = u
        return c

    # -- evaluation -------------------------------------------------------------
    def evaluate(self, u, patch, xi):
        """Values and physical gradients of the glued solution at parametric
        points xi [P, 2] of the given patches [P]."""
        c = self.full(u)
        patch = np.asarray(patch)
        xi = np.asarray(xi, dtype=np.float64)
        val = np.zeros(len(xi))
        grad = np.zeros((len(xi), 2))
        for q in range(3):
            sel = np.nonzero(patch == q)[0]
            if len(sel) == 0:
                continue
            C = c[self.ids[q]].reshape(self.nf[1], self.nf[0])
            comp = self.patches[q]
            v0 = comp.spaces[0].values_at(xi[sel, 0])
            v1 = comp.spaces[1].values_at(xi[sel, 1])
            d0 = comp.spaces[0].derivs_at(xi[sel, 0])
            d1 = comp.spaces[1].derivs_at(xi[sel, 1])
            val[sel] = np.einsum("pj,ji,pi->p", v1, C, v0)
            g0 = np.einsum("pj,ji,pi->p", v1, C, d0)
            g1 = np.einsum("pj,ji,pi->p", d1, C, v0)
            s = SIGNS[q]                                     # J = diag(s), grad_x = J^{-T} grad_xi
            grad[sel, 0] = g0 * s[0]
            grad[sel, 1] = g1 * s[1]
        return val, grad


def error_points(nel=64, nq=4):
    """Gauss points and weights of a uniform nel x nel mesh on every patch:
    (patch ids, parametric points, weights); |det J| = 1 on every patch."""
    z = np.linspace(0.0, 1.0, nel + 1)
    x, w = spline.element_quadrature(z, nq)
    x, w = x.reshape(-1), w.reshape(-1)
    X0, X1 = np.meshgrid(x, x, indexing="xy")
    W = np.outer(w, w)
    pts = np.stack([X0.reshape(-1), X1.reshape(-1)], 1)
    ww = W.reshape(-1)
    P = np.concatenate([np.full(len(pts), q) for q in range(3)])
    return P, np.concatenate([pts] * 3), np.concatenate([ww] * 3)


def errors(val, grad, u, du, patch, xi, w):
    """L2 norm and H1 seminorm of (u_h - u) by quadrature on the error points."""
    x = np.concatenate([physical(q, xi[patch == q]) for q in range(3)])
    order = np.concatenate([np.nonzero(patch == q)[0] for q in range(3)])
    ex = np.empty(len(xi))
    ex[order] = u(x)
    dex = np.empty((len(xi), 2))
    dex[order] = du(x)
    l2 = np.sqrt(np.sum(w * (val - ex) ** 2))
    h1 = np.sqrt(np.sum(w * np.sum((grad - dex) ** 2, axis=1)))
    return l2, h1


# -- the data of the L-shape workload ------------------------------------------------

def theta(x):
    """Polar angle in [0, 2pi) measured from the positive x axis."""
    t = np.arctan2(x[:, 1], x[:, 0])
    return np.where(t < 0, t + 2 * np.pi, t)


def corner_u(x):
    """u = r^(2/3) sin(2 theta / 3): harmonic, zero on the two sides at the corner."""
    r = np.hypot(x[:, 0], x[:, 1])
    return r ** (2.0 / 3.0) * np.sin(2.0 * theta(x) / 3.0)


def corner_grad(x):
    r = np.hypot(x[:, 0], x[:, 1])
    th = theta(x)
    ur = (2.0 / 3.0) * r ** (-1.0 / 3.0) * np.sin(2.0 * th / 3.0)
    ut = (2.0 / 3.0) * r ** (-1.0 / 3.0) * np.cos(2.0 * th / 3.0)   # (1/r) du/dtheta
    c, s = np.cos(th), np.sin(th)
    return np.stack([ur * c - ut * s, ur * s + ut * c], 1)


def harmonic_quadratic(x):
    """u = 1 + 2x - 3y + (x^2 - y^2)/2 + xy: harmonic, in every p >= 2 space of
    the affine patches."""
    X, Y = x[:, 0], x[:, 1]
    return 1.0 + 2.0 * X - 3.0 * Y + 0.5 * (X * X - Y * Y) + X * Y


def solve_combination(w, p=2, kind="onesided", gamma=1.0, g=corner_u, min_level=1):
    """Solve every component of level w (2D) on the L-shape; returns
    [(levels, coefficient, component, interior solution)]."""
    from .combination import index_set
    out = []
    for i, c in index_set(2, w, min_level):
        comp = LShapeComponent(i, p, kind=kind, gamma=gamma).assemble(g=g)
        out.append((i, c, comp, comp.solve()))
    return out


def combined(results, patch, xi):
    """Combined values and physical gradients sum_i c_i u_i (Neumaier-compensated)."""
    from .combination import combine
    vals, g0, g1, coef = [], [], [], []
    for (_, c, comp, u) in results:
        v, gr = comp.evaluate(u, patch, xi)
        vals.append(v)
        g0.append(gr[:, 0])
        g1.append(gr[:, 1])
        coef.append(c)
    return combine(vals, coef), np.stack([combine(g0, coef), combine(g1, coef)], 1)


# lowest kept function per direction on each patch: 0 where the low side is a
# patch interface (natural condition in the local problem), 1 where it is a
# Dirichlet side
KEPT_LO = ((0, 1), (0, 0), (1, 0))


def schwarz_apply(comp, r):
    """Weighted additive Schwarz over the patches (the definition the CUDA
    preconditioner of multi-patch plans implements; not in the paper):

        z = sum_q E_q^T D_q A_q^{-1} D_q E_q r,

    A_q = the patch's stiffness on the tensor set of its functions
    [lo_0, nf_0 - 2] x [lo_1, nf_1 - 2] (natural condition at interface sides),
    E_q = restriction of the glued interior vector to that set, zero at a
    function of the set that is not an unknown (patch 1's corner function);
    E_q^T adds back and drops that function. D_q = 1 / (number of patches
    sharing the function): 1/2 on interface functions, the Neumann-Neumann
    weighting (without it the interface is corrected twice and the condition
    number grows like h^-2). r is in the component's interior ordering; comp
    must be assembled."""
    nf0, nf1 = comp.nf
    pos = -np.ones(comp.nglob, dtype=np.int64)
    pos[comp.interior] = np.arange(comp.ndof)
    z = np.zeros(comp.ndof)
    for q in range(3):
        lo0, lo1 = KEPT_LO[q]
        a, b = np.meshgrid(np.arange(lo0, nf0 - 1), np.arange(lo1, nf1 - 1), indexing="xy")
        a, b = a.reshape(-1), b.reshape(-1)
        loc = a + nf0 * b
        p = pos[comp.ids[q][loc]]                      # -1: not an unknown
        shared = 1 + ((a == 0) & (lo0 == 0)).astype(int) + ((b == 0) & (lo1 == 0)).astype(int)
        w = np.where(p >= 0, 1.0 / shared, 0.0)
        A = comp.patches[q].K_full[loc][:, loc].toarray()
        zl = np.linalg.solve(A, w * np.where(p >= 0, r[np.maximum(p, 0)], 0.0)) * w
        ok = p >= 0
        np.add.at(z, p[ok], zl[ok])
    return z
