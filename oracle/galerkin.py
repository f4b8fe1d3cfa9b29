"""Galerkin discretisation of one component grid (paper Problem 1, Sec. 2.2).

TEST INFRASTRUCTURE: see the package header.

A component is the tensor-product spline space with 2^{i_k} elements in
direction k, degree p and continuity C^r, pulled back through the geometry F
(eqs. spline_space_phys, u-IGA-approx). The oracle assembles the stiffness
matrix and load vector element by element with (p+1)^d Gauss points,

    K_ij = sum_q w_q |det J_q| a(x_q) grad R_i(xi_q)^T (J_q^T J_q)^{-1} grad R_j(xi_q)
    b_i  = sum_q w_q |det J_q| f(x_q) R_i(xi_q),

removes the Dirichlet boundary functions (the first and last function of each
direction, which are the only ones that do not vanish on the boundary of an
open knot vector) and solves with a sparse direct LU (the paper's choice of a
direct solver, Sec. 4.1).

Numbering: the full 1D index runs 0..nf_k-1; interior DoFs are 1..nf_k-2.
Vectors are stored with direction 1 fastest.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import spline


class Space1D:
    """One direction of one component: knots, Gauss points and basis tables."""

    def __init__(self, level, p, r, geom, k, kind="uniform", gamma=1.0):
        self.level, self.p, self.r = level, p, r
        self.E = 2 ** level
        self.Q = p + 1
        self.z = spline.breakpoints(self.E, kind, gamma)
        self.knots = spline.open_knot_vector(self.E, p, r, kind, gamma)
        self.nf = spline.n_basis(self.E, p, r)
        self.n = self.nf - 2
        self.xi, self.w = spline.element_quadrature(self.z, self.Q)
        self.first = spline.element_first_function(self.knots, p, self.z)
        flat = self.xi.reshape(-1)
        B = spline.bspline_basis(self.knots, p, flat)
        dB = spline.bspline_deriv(self.knots, p, flat)
        W, dW = geom.weight_1d(k, flat)
        R = B / W[:, None]
        dR = (dB * W[:, None] - B * dW[:, None]) / (W ** 2)[:, None]
        # local tables [E, Q, p+1]: the p+1 functions first[e] .. first[e]+p
        e = np.repeat(np.arange(self.E), self.Q)
        cols = self.first[e][:, None] + np.arange(p + 1)[None, :]
        rows = np.arange(len(flat))[:, None]
        self.R = R[rows, cols].reshape(self.E, self.Q, p + 1)
        self.dR = dR[rows, cols].reshape(self.E, self.Q, p + 1)
        self.geom, self.k = geom, k

    def values_at(self, t):
        """All nf functions R_i(t) = B_i(t)/W_k(t) at arbitrary points: [len(t), nf]."""
        B = spline.bspline_basis(self.knots, self.p, t)
        W, _ = self.geom.weight_1d(self.k, t)
        return B / W[:, None]

    def derivs_at(self, t):
        B = spline.bspline_basis(self.knots, self.p, t)
        dB = spline.bspline_deriv(self.knots, self.p, t)
        W, dW = self.geom.weight_1d(self.k, t)
        return (dB * W[:, None] - B * dW[:, None]) / (W ** 2)[:, None]


class Component:
    """Assembled Dirichlet-eliminated system of one component grid."""

    def __init__(self, geom, levels, p, r=None, kind="uniform", gamma=1.0):
        self.geom = geom
        self.d = geom.d
        self.levels = tuple(int(v) for v in levels)
        self.p = p
        self.r = p - 1 if r is None else r
        self.spaces = [Space1D(l, p, self.r, geom, k, kind, gamma)
                       for k, l in enumerate(self.levels)]
        self.nf = [s.nf for s in self.spaces]
        self.n = [s.n for s in self.spaces]
        self.ndof = int(np.prod(self.n))
        self.nfull = int(np.prod(self.nf))
        full = np.arange(self.nfull)
        inner = np.ones(self.nfull, dtype=bool)
        rem = full.copy()
        for k in range(self.d):
            g = rem % self.nf[k]
            rem //= self.nf[k]
            inner &= (g >= 1) & (g <= self.nf[k] - 2)
        self.interior = np.nonzero(inner)[0]   # increasing = packed order

    # -- element loop ---------------------------------------------------------
    def _element_batches(self, batch):
        E = [s.E for s in self.spaces]
        tot = int(np.prod(E))
        for s0 in range(0, tot, batch):
            ids = np.arange(s0, min(tot, s0 + batch))
            em = []
            rem = ids.copy()
            for k in range(self.d):
                em.append(rem % E[k])
                rem //= E[k]
            yield em

    def _element_data(self, em):
        """Values, reference gradients, qp coordinates and weights of a batch."""
        d, P1 = self.d, self.p + 1
        Rs = [self.spaces[k].R[em[k]] for k in range(d)]     # [nb, Q, P1]
        dRs = [self.spaces[k].dR[em[k]] for k in range(d)]
        xis = [self.spaces[k].xi[em[k]] for k in range(d)]   # [nb, Q]
        ws = [self.spaces[k].w[em[k]] for k in range(d)]
        nb = len(em[0])
        if d == 2:
            val = np.einsum("eqa,erb->erqba", Rs[0], Rs[1])
            g1 = np.einsum("eqa,erb->erqba", dRs[0], Rs[1])
            g2 = np.einsum("eqa,erb->erqba", Rs[0], dRs[1])
            grads = [g1, g2]
            X = np.stack(np.broadcast_arrays(xis[0][:, None, :], xis[1][:, :, None]), -1)
            W = ws[1][:, :, None] * ws[0][:, None, :]
        else:
            val = np.einsum("eqa,erb,esc->esrqcba", Rs[0], Rs[1], Rs[2])
            g1 = np.einsum("eqa,erb,esc->esrqcba", dRs[0], Rs[1], Rs[2])
            g2 = np.einsum("eqa,erb,esc->esrqcba", Rs[0], dRs[1], Rs[2])
            g3 = np.einsum("eqa,erb,esc->esrqcba", Rs[0], Rs[1], dRs[2])
            grads = [g1, g2, g3]
            X = np.stack(np.broadcast_arrays(xis[0][:, None, None, :],
                                             xis[1][:, None, :, None],
                                             xis[2][:, :, None, None]), -1)
            W = ws[2][:, :, None, None] * ws[1][:, None, :, None] * ws[0][:, None, None, :]
        nq = P1 ** d
        val = val.reshape(nb, nq, nq)
        grad = np.stack([g.reshape(nb, nq, nq) for g in grads], axis=-1)  # [nb,q,A,d]
        X = X.reshape(nb * nq, d)
        W = W.reshape(nb, nq)
        # global full indices of the local functions A (direction 1 fastest)
        gidx = np.zeros((nb, 1), dtype=np.int64)
        stride = 1
        loc = np.zeros((nb, nq), dtype=np.int64)
        a = np.arange(nq)
        for k in range(d):
            ak = (a // (P1 ** k)) % P1
            loc += (self.spaces[k].first[em[k]][:, None] + ak[None, :]) * stride
            stride *= self.nf[k]
        del gidx
        return val, grad, X, W, loc

    def assemble(self, f=None, diffusion=None, batch=512, with_mass=False):
        """Assemble K (and b if f is given) over all elements; Dirichlet-eliminate."""
        rows, cols, vals, mvals = [], [], [], []
        bfull = np.zeros(self.nfull)
        d = self.d
        for em in self._element_batches(batch):
            val, grad, Xi, W, loc = self._element_data(em)
            nb, nq = W.shape
            J = self.geom.jacobian(Xi).reshape(nb, nq, d, d)
            det = np.linalg.det(J)
            if not (np.all(det > 0) or np.all(det < 0)):
                raise ValueError("Jacobian determinant vanishes or changes sign")
            JtJinv = np.linalg.inv(np.einsum("eqik,eqil->eqkl", J, J))
            coef = (W * np.abs(det))
            x = self.geom.map(Xi)
            if diffusion is not None:
                coef = coef * diffusion(x).reshape(nb, nq)
            G = JtJinv * coef[:, :, None, None]                      # [nb,q,d,d]
            T = np.einsum("eqAk,eqkl->eqAl", grad, G)                # [nb,q,A,d]
            Ke = np.matmul(T.transpose(0, 2, 1, 3).reshape(nb, nq, nq * d),
                           grad.transpose(0, 1, 3, 2).reshape(nb, nq * d, nq))
            rows.append(np.repeat(loc, nq, axis=1).reshape(-1))
            cols.append(np.tile(loc, (1, nq)).reshape(-1))
            vals.append(Ke.reshape(-1))
            if with_mass:
                Me = np.einsum("eqA,eq,eqB->eAB", val, W * np.abs(det), val)
                mvals.append(Me.reshape(-1))
            if f is not None:
                fx = f(x).reshape(nb, nq)
                be = np.einsum("eqA,eq->eA", val, W * np.abs(det) * fx)
                np.add.at(bfull, loc.reshape(-1), be.reshape(-1))
        r = np.concatenate(rows)
        c = np.concatenate(cols)
        K = sp.csr_matrix((np.concatenate(vals), (r, c)), shape=(self.nfull, self.nfull))
        self.K_full = K
        if with_mass:
            self.M_full = sp.csr_matrix((np.concatenate(mvals), (r, c)),
                                        shape=(self.nfull, self.nfull))
        I = self.interior
        self.K = K[I][:, I].tocsc()
        self.b_full = bfull
        self.b = bfull[I] if f is not None else None
        return self

    def load_vector(self, g):
        """b_i = sum_q w_q |det J_q| g(x_q) R_i(xi_q) over the interior
        functions: the load vector of g (the assembly's rule), without
        touching the assembled system."""
        bfull = np.zeros(self.nfull)
        for em in self._element_batches(512):
            val, _, Xi, W, loc = self._element_data(em)
            nb, nq = W.shape
            det = np.abs(np.linalg.det(self.geom.jacobian(Xi).reshape(nb, nq, self.d, self.d)))
            gx = g(self.geom.map(Xi)).reshape(nb, nq)
            np.add.at(bfull, loc.reshape(-1), np.einsum("eqA,eq->eA", val, W * det * gx).reshape(-1))
        return bfull[self.interior]

    def solve(self, b=None):
        """Sparse direct solve of the Dirichlet-eliminated system (Sec. 4.1)."""
        rhs = self.b if b is None else b
        lu = spla.splu(self.K)
        return lu.solve(rhs)

    # -- evaluation -----------------------------------------------------------
    def full_coeffs(self, u):
        c = np.zeros(self.nfull)
        c[self.interior] = u
        return c.reshape(self.nf[::-1])   # axes (.., dir2, dir1)

    def evaluate(self, u, pts):
        """u_n(F(xi)) = sum_i c_i R_i(xi) at parametric points pts [P, d]."""
        C = self.full_coeffs(u)
        vals = [self.spaces[k].values_at(pts[:, k]) for k in range(self.d)]
        if self.d == 2:
            return np.einsum("pj,ji,pi->p", vals[1], C, vals[0])
        return np.einsum("pk,kji,pj,pi->p", vals[2], C, vals[1], vals[0], optimize=True)

    def evaluate_grad(self, u, pts):
        """Parametric gradient of u_n at pts: [P, d]."""
        C = self.full_coeffs(u)
        vals = [self.spaces[k].values_at(pts[:, k]) for k in range(self.d)]
        ders = [self.spaces[k].derivs_at(pts[:, k]) for k in range(self.d)]
        out = []
        for l in range(self.d):
            f = [ders[k] if k == l else vals[k] for k in range(self.d)]
            if self.d == 2:
                out.append(np.einsum("pj,ji,pi->p", f[1], C, f[0]))
            else:
                out.append(np.einsum("pk,kji,pj,pi->p", f[2], C, f[1], f[0], optimize=True))
        return np.stack(out, axis=1)


def stiffness_1d(level, p, r, kind="uniform", gamma=1.0, geom=None, k=0):
    """1D parametric stiffness and mass matrices of the interior basis functions.

    K_ij = int_0^1 R_i' R_j', M_ij = int_0^1 R_i R_j by (p+1)-point Gauss
    quadrature per element; dense, interior functions 1..nf-2 only. R are the
    B-splines of direction k divided by that direction's rational weight
    function of `geom` (plain B-splines when geom is None).
    """
    from .geometry import UnitCube
    s = Space1D(level, p, r, UnitCube(1) if geom is None else geom, 0 if geom is None else k, kind, gamma)
    K = np.zeros((s.nf, s.nf))
    M = np.zeros((s.nf, s.nf))
    for e in range(s.E):
        idx = s.first[e] + np.arange(p + 1)
        for q in range(s.Q):
            K[np.ix_(idx, idx)] += s.w[e, q] * np.outer(s.dR[e, q], s.dR[e, q])
            M[np.ix_(idx, idx)] += s.w[e, q] * np.outer(s.R[e, q], s.R[e, q])
    return K[1:-1, 1:-1], M[1:-1, 1:-1]
