"""The combination technique as a preconditioner for the full tensor-product
solve (the paper's closing remark, Sec. 5), studied on the CPU with the
oracle's matrices (the GPU version is `sgiga_ct_attach`, checked against
oracle/ct.py in tests/test_gpu_ct.py).

Full system: A u = b on the tensor grid with every level J (2D quarter annulus,
p = 2, C^1, diffusion coefficient a(x)). Combination operator:

  B_CT = sum_i c_i P_i A_i^{-1} P_i^T,

over the components of level w = J (eq. TD-combi-tec). P_i is the prolongation
of component i's space into the full space by knot insertion (the spaces are
nested). FD: the fast-diagonalisation preconditioner of the full grid's
parametric constant-coefficient 1D matrices.

Findings pinned here:
- B_CT A is a near-projection: real eigenvalues in [0, ~1.1], most of them
  zero (the sparse-grid spaces span a small part of the full space). So B_CT
  alone is no preconditioner, and the stationary iteration u += B_CT (b - A u)
  stalls at the combination technique's own error.
- With a coefficient jump (10x across x = 1) that iteration keeps a residual
  of order one (0.86 at J = 5; at J = 6 it grows from 2.6 to 4.2).
- Added to FD (additive two-level, SPD), it saves under a quarter of the CG
  iterations. Each application costs a solve of every component, about as
  much as the sparse-grid solve itself.
"""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import combination, galerkin, geometry, spline

P_DEG, R_CONT = 2, 1
COEF = {"exp": lambda x: np.exp(np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1])),
        "jump": lambda x: np.where(x[:, 0] > 1.0, 10.0, 1.0)}


def prolongation_1d(geom, lc, lf):
    """Fine-space coefficients of every interior coarse B-spline (knot
    insertion), by least squares at 8 n_f + 3 points; exact up to rounding
    because the spaces are nested."""
    sc = galerkin.Space1D(lc, P_DEG, R_CONT, geom, 0)
    sf = galerkin.Space1D(lf, P_DEG, R_CONT, geom, 0)
    t = np.linspace(0.0, 1.0, 8 * sf.nf + 3)
    Bc = spline.bspline_basis(sc.knots, P_DEG, t)[:, 1:-1]
    Bf = spline.bspline_basis(sf.knots, P_DEG, t)[:, 1:-1]
    T = np.linalg.lstsq(Bf, Bc, rcond=None)[0]
    assert np.abs(Bf @ T - Bc).max() < 1e-12          # nested: exact representation
    return sp.csr_matrix(np.where(np.abs(T) < 1e-14, 0.0, T))


def setup(J, coef):
    geom = geometry.make("annulus", 2)
    full = galerkin.Component(geom, (J, J), P_DEG, R_CONT).assemble(f=lambda x: np.ones(len(x)),
                                                                   diffusion=COEF[coef])
    A, b = full.K, full.b
    comps = []
    for lv, c in combination.index_set(2, J, 1):
        C = galerkin.Component(geom, lv, P_DEG, R_CONT).assemble(diffusion=COEF[coef])
        P = sp.kron(prolongation_1d(geom, lv[1], J), prolongation_1d(geom, lv[0], J)).tocsr()
        comps.append((c, P, spla.splu(C.K.tocsc())))

    def B_ct(v):
        out = np.zeros(A.shape[0])
        for c, P, lu in comps:
            out += c * (P @ lu.solve(P.T @ v))
        return out

    K0, M0 = galerkin.stiffness_1d(J, P_DEG, R_CONT)
    K0 = K0.toarray() if hasattr(K0, "toarray") else np.asarray(K0)
    M0 = M0.toarray() if hasattr(M0, "toarray") else np.asarray(M0)
    lam, U = sl.eigh(K0, M0)
    D = 1.0 / (lam[:, None] + lam[None, :])

    def B_fd(v):
        W = U.T @ v.reshape(len(lam), len(lam)) @ U
        return (U @ (W * D) @ U.T).reshape(-1)

    return A, b, B_ct, B_fd


def cg_iterations(A, b, B):
    it = [0]

    def cb(_):
        it[0] += 1
    M = spla.LinearOperator(A.shape, matvec=B)
    x, info = spla.cg(A, b, rtol=1e-10, maxiter=3000, M=M, callback=cb)
    assert info == 0 and np.linalg.norm(b - A @ x) <= 1.01e-10 * np.linalg.norm(b)
    return it[0]


def test_prolongation_is_exact_knot_insertion():
    """P^T A P = A_i for nested spaces where both are integrated exactly (unit
    square, constant coefficient: polynomial integrands). On the annulus the
    component matrices differ from P^T A P by their own quadrature error
    (1e-4 .. 2e-2 relative at these levels), as in the combination technique
    itself."""
    geom = geometry.make("unit", 2)
    full = galerkin.Component(geom, (4, 4), P_DEG, R_CONT).assemble()
    for lv in [(1, 4), (2, 3), (3, 1)]:
        C = galerkin.Component(geom, lv, P_DEG, R_CONT).assemble()
        P = sp.kron(prolongation_1d(geom, lv[1], 4), prolongation_1d(geom, lv[0], 4))
        assert abs(P.T @ full.K @ P - C.K).max() < 1e-13 * abs(C.K).max()


def test_combination_operator_is_a_rank_deficient_near_projection():
    A, b, B_ct, _ = setup(4, "exp")
    n = A.shape[0]
    BA = np.column_stack([B_ct(A @ e) for e in np.eye(n)])
    ev = np.linalg.eigvals(BA)
    assert np.abs(ev.imag).max() < 1e-8
    assert ev.real.min() > -1e-8 and ev.real.max() < 1.2
    assert np.mean(ev.real < 1e-6) > 0.5                # most of the full space untouched
    # the stationary iteration stalls at the combination technique's error
    x = np.zeros(n)
    res = []
    for _ in range(10):
        x = x + B_ct(b - A @ x)
        res.append(np.linalg.norm(b - A @ x) / np.linalg.norm(b))
    assert res[-1] > 0.5 * res[0] > 1e-4


def test_combination_iteration_stalls_at_order_one_with_a_coefficient_jump():
    A, b, B_ct, _ = setup(5, "jump")
    x = np.zeros(A.shape[0])
    for _ in range(30):
        x = x + B_ct(b - A @ x)
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) > 0.5


@pytest.mark.parametrize("coef", ["exp", "jump"])
def test_additive_two_level_saves_little(coef):
    A, b, B_ct, B_fd = setup(5, coef)
    n_fd = cg_iterations(A, b, B_fd)
    n_2l = cg_iterations(A, b, lambda v: B_fd(v) + B_ct(v))
    assert n_2l <= n_fd and n_2l > 0.75 * n_fd, (n_fd, n_2l)
