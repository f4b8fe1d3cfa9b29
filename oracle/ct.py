"""The combination technique as a preconditioner of the full tensor-product
solve (the paper's closing remark, Sec. 5): the definitions the CUDA library's
two-level preconditioner is checked against.

TEST INFRASTRUCTURE: see the package header.

Full system A u = b on the tensor grid with every level J. Combination
operator over the components i of level w = J (eq. TD-combi-tec):

    B_CT = sum_i c_i P_i A_i^{-1} P_i^T,

P_i the prolongation of component i's space into the full space. The spaces
are nested (uniform knots, the same degree and continuity), so every coarse
B-spline is a combination of fine ones; here the coefficients are found by
least squares at 8 n_f + 3 points, exact up to rounding because the
representation exists. The two-level preconditioner is FD + B_CT, FD the fast
diagonalisation of the full grid's parametric 1D matrices.
"""
import numpy as np
import scipy.linalg as sl
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import combination, galerkin, spline


def prolongation_1d(geom, p, r, lc, lf, k=0):
    """Fine-space coefficients of every interior coarse B-spline of direction
    k: [n_f - 2, n_c - 2], column j = coarse function j + 1."""
    sc = galerkin.Space1D(lc, p, r, geom, k)
    sf = galerkin.Space1D(lf, p, r, geom, k)
    t = np.linspace(0.0, 1.0, 8 * sf.nf + 3)
    Bc = spline.bspline_basis(sc.knots, p, t)[:, 1:-1]
    Bf = spline.bspline_basis(sf.knots, p, t)[:, 1:-1]
    T = np.linalg.lstsq(Bf, Bc, rcond=None)[0]
    if np.abs(Bf @ T - Bc).max() > 1e-12:
        raise ValueError("the coarse space is not contained in the fine one")
    return np.where(np.abs(T) < 1e-14, 0.0, T)


def prolongation(geom, p, r, levels, J):
    """P_i = P_{d-1} x .. x P_0 (direction 0 fastest), sparse."""
    P = None
    for k, lc in enumerate(levels):
        Pk = sp.csr_matrix(prolongation_1d(geom, p, r, lc, J, k))
        P = Pk if P is None else sp.kron(Pk, P).tocsr()
    return P


class TwoLevel:
    """The full system of level J and its combination operator over the
    components of level w = J (min level 1), with the diffusion coefficient
    `diffusion` (a function of the physical points) and load f."""

    def __init__(self, geom, d, p, r, J, diffusion=None, f=None):
        self.full = galerkin.Component(geom, (J,) * d, p, r).assemble(
            f=f if f is not None else (lambda x: np.ones(len(x))), diffusion=diffusion)
        self.A, self.b = self.full.K, self.full.b
        self.comps = []
        for lv, c in combination.index_set(d, J, 1):
            C = galerkin.Component(geom, lv, p, r).assemble(diffusion=diffusion)
            self.comps.append((lv, c, prolongation(geom, p, r, lv, J), spla.splu(C.K.tocsc())))
        K0, M0 = galerkin.stiffness_1d(J, p, r)
        K0 = K0.toarray() if hasattr(K0, "toarray") else np.asarray(K0)
        M0 = M0.toarray() if hasattr(M0, "toarray") else np.asarray(M0)
        self.lam, self.U = sl.eigh(K0, M0)
        self.d = d

    def b_ct(self, v):
        out = np.zeros(self.A.shape[0])
        for _, c, P, lu in self.comps:
            out += c * (P @ lu.solve(P.T @ v))
        return out

    def b_fd(self, v):
        n, U, lam = len(self.lam), self.U, self.lam
        if self.d == 2:
            W = U.T @ v.reshape(n, n) @ U
            return (U @ (W / (lam[:, None] + lam[None, :])) @ U.T).reshape(-1)
        W = np.einsum("ia,jb,kc,ijk->abc", U, U, U, v.reshape(n, n, n))
        W /= lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
        return np.einsum("ia,jb,kc,abc->ijk", U, U, U, W).reshape(-1)

    def cg_iterations(self, B, tol=1e-10):
        it = [0]

        def cb(_):
            it[0] += 1
        M = spla.LinearOperator(self.A.shape, matvec=B)
        x, info = spla.cg(self.A, self.b, rtol=tol, maxiter=3000, M=M, callback=cb)
        if info != 0:
            raise RuntimeError("CG did not converge")
        return it[0], x
