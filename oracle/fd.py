"""Fast-diagonalisation (FD) preconditioner of the oracle, from its definition.

TEST INFRASTRUCTURE: see the package header.

Not in the paper (it cites fast-diagonalisation solvers as related fast-IGA
work and lists combining them with sparse grids as future work, Sec. 5). For a
component with interior 1D parametric matrices K_k, M_k (galerkin.stiffness_1d,
in the basis of the component's own direction k: B-splines divided by the
geometry's rational weight function of that direction)
and the generalised eigenpairs K_k U_k = M_k U_k Lambda_k, U_k^T M_k U_k = I,

    P^{-1} r = (U_d x ... x U_1) diag(sum_k s_k lambda_{k,i_k})^{-1} (U_d x ... x U_1)^T r

with per-direction scales s_k (1 unless given). On the unit square/cube with
s = 1 the Galerkin matrix is exactly sum_k M_d x .. K_k .. x M_1, so P^{-1} is
its exact inverse (pinned against the sparse direct solve).
"""
import numpy as np
import scipy.linalg as sla

from .galerkin import stiffness_1d


def eig_1d(level, p, r, kind="uniform", gamma=1.0, geom=None, k=0):
    """Generalised eigenpairs of (K, M) in 1D, eigenvalues ascending."""
    K, M = stiffness_1d(level, p, r, kind, gamma, geom, k)
    lam, U = sla.eigh(K, M)
    return lam, U


def fd_apply(levels, p, r, rvec, scales=None, kind="uniform", gamma=1.0, geom=None):
    d = len(levels)
    s = np.ones(d) if scales is None else np.asarray(scales, dtype=np.float64)
    eig = [eig_1d(l, p, r, kind, gamma, geom, k) for k, l in enumerate(levels)]
    n = [len(e[0]) for e in eig]
    T = np.asarray(rvec, dtype=np.float64).reshape(n[::-1])   # axes (.., dir2, dir1)
    # forward transform along every direction: T <- U_k^T T
    for k in range(d):
        ax = d - 1 - k
        T = np.moveaxis(np.tensordot(eig[k][1].T, T, axes=([1], [ax])), 0, ax)
    D = np.zeros(n[::-1])
    for k in range(d):
        ax = d - 1 - k
        shape = [1] * d
        shape[ax] = n[k]
        D = D + s[k] * eig[k][0].reshape(shape)
    T = T / D
    for k in range(d):
        ax = d - 1 - k
        T = np.moveaxis(np.tensordot(eig[k][1], T, axes=([1], [ax])), 0, ax)
    return T.reshape(-1)
