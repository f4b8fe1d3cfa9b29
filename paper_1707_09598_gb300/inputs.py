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
