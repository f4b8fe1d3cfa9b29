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


def sturm_eigenvalues(K, M, js, dtype=np.longdouble, bw=None):
    """Eigenvalues number js (ascending, 0-based) of the symmetric-definite
    pencil (K, M) by bisection on the inertia of K - s M: by Sylvester's law of
    inertia the number of eigenvalues below s is the number of negative pivots
    of its LDL^T factorisation (M positive definite). Written out entry by
    entry in `dtype` (extended precision by default) for banded K, M of
    bandwidth bw; it forms neither M^{-1} nor a Cholesky factor of M, so graded
    meshes (ill-conditioned M) keep their accuracy. Returns float64 values."""
    K = np.asarray(K, dtype=dtype)
    M = np.asarray(M, dtype=dtype)
    n = K.shape[0]
    if bw is None:
        bw = max(abs(i - j) for i, j in zip(*np.nonzero(np.asarray(K, dtype=np.float64))))

    eps = np.finfo(dtype).eps

    def count(s):
        A = K - s * M
        floor = eps * eps * np.abs(A).max()
        L = np.zeros((n, n), dtype=dtype)
        D = np.zeros(n, dtype=dtype)
        neg = 0
        for i in range(n):
            lo = max(0, i - bw)
            for j in range(lo, i):
                v = A[i, j] - sum(L[i, k] * D[k] * L[j, k] for k in range(max(lo, j - bw), j))
                L[i, j] = v / D[j]
            d = A[i, i] - sum(L[i, k] * L[i, k] * D[k] for k in range(lo, i))
            if abs(d) < floor:
                d = -floor
            D[i] = d
            neg += d < 0
        return neg

    # first bound and descent factor are no powers of 2 (a bisection point equal
    # to some K_ii / M_ii would make a pivot vanish exactly)
    hi = dtype(2.17) * max(K[i, i] / M[i, i] for i in range(n))
    while count(hi) < n:
        hi = hi * 4
    out = []
    for j in js:
        lo, h = dtype(0), hi
        while h - lo > 4 * eps * h:
            mid = (lo + h) / 2 if lo > 0 and h < 2 * lo else (np.sqrt(lo * h) if lo > 0 else h / 7)
            if not (lo < mid < h):
                break
            if count(mid) > j:
                h = mid
            else:
                lo = mid
        out.append(float((lo + h) / 2 if lo > 0 else h / 2))
    return np.array(out)
