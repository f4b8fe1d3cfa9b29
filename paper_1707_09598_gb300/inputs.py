"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method: only point lattices and seeded
random numbers. Both sides draw their inputs from here so that a parity test
feeds the same numbers to each.
"""
import numpy as np


def eval_points(d, k):
    """Parametric evaluation lattice {j/k : j = 0..k}^d, direction 1 fastest.

    Returns an array [P, d] with P = (k+1)^d, float64. The boundary points are
    included (the 257 x 257 lattice of the 2D unit-square workload is k = 256).
    """
    t = np.arange(k + 1, dtype=np.float64) / k
    grids = np.meshgrid(*([t] * d), indexing="ij")
    # direction 1 fastest: reverse the axis order before flattening
    cols = [g.transpose(tuple(range(d))[::-1]).reshape(-1) for g in grids]
    return np.ascontiguousarray(np.stack(cols, axis=1))


def random_points(n, d, seed):
    """n seeded uniform parametric points in [0,1)^d, float64 [n, d]."""
    rng = np.random.default_rng(seed)
    return rng.random((n, d))


def random_vector(n, seed):
    """n seeded standard-normal float64 values."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n)


def perturbed_cube_patch(seed, amp=0.1, elems=2, degree=3):
    """Seeded perturbation of the unit cube as a tensor-product B-spline patch.

    Degree `degree`, `elems` uniform elements per direction (open knots); the
    control points start at the Greville abscissae (the identity map) and every
    control point off the boundary faces moves by amp * U[-1, 1] in each
    coordinate. Returns (knots [3 arrays], control points [n^3, 3], direction 0
    fastest).
    """
    rng = np.random.default_rng(seed)
    p, E = degree, elems
    kn = np.concatenate([np.zeros(p + 1), np.arange(1, E) / E, np.ones(p + 1)])
    n = E + p
    gr = np.array([kn[i + 1:i + p + 1].mean() for i in range(n)])
    cp = np.zeros((n, n, n, 3))
    for c in range(n):
        for b in range(n):
            for a in range(n):
                cp[c, b, a] = (gr[a], gr[b], gr[c])
    inner = np.zeros((n, n, n), dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    disp = amp * (2.0 * rng.random((n, n, n, 3)) - 1.0)
    cp[inner] += disp[inner]
    return [kn.copy(), kn.copy(), kn.copy()], cp.reshape(-1, 3)


def lognormal_features(seed, nfeat=512, sigma=0.5, ell=0.2, d=3):
    """Seeded random Fourier features of a Gaussian field with squared-exponential
    covariance sigma^2 exp(-|x-y|^2 / (2 ell^2)): returns (omega [nfeat, d] with
    N(0, 1/ell^2) entries, phase [nfeat] uniform on [0, 2 pi), amplitude
    sigma sqrt(2 / nfeat)). The field is amplitude * sum_f cos(omega_f . x + phase_f)
    and the coefficient a = exp(field)."""
    rng = np.random.default_rng(seed)
    omega = rng.standard_normal((nfeat, d)) / ell
    phase = 2.0 * np.pi * rng.random(nfeat)
    return omega, phase, sigma * np.sqrt(2.0 / nfeat)
