"""Combination technique of the oracle (paper Sec. 3).

TEST INFRASTRUCTURE: see the package header.

Level convention. A component is i in N^d with i_k >= m (m = min_level,
default 1) and 2^{i_k} elements in direction k. The paper's multi-index is
beta = i - m, i.e. its 1D hierarchy starts at the space with 2^m elements.
The truncation level is J = w + d - 1 - d m, so that the sparse-grid sum
f_J = sum_{|beta| <= J} Delta_beta (eq. TD-approx) uses the components with
w <= |i| <= w + d - 1.
"""
import itertools
import math

import numpy as np


def _J(d, w, m):
    return w + d - 1 - d * m


def coefficients_by_expansion(d, w, min_level=1):
    """Combination coefficients from the definition (eqs. Delta-op, TD-approx).

    Expand f_J = sum_{beta >= 0, |beta| <= J} Delta_beta with
    Delta_beta = sum_{k in {0,1}^d} (-1)^{|k|} f_{beta - k} (eq. Delta-combi-tec
    applied direction by direction) and f_{beta} = 0 when some beta_k < 0.
    Returns {i: c_i} over the components with a nonzero coefficient, i = beta + m.
    """
    J = _J(d, w, min_level)
    if J < 0:
        raise ValueError("level too small for min_level")
    acc = {}
    for beta in itertools.product(range(J + 1), repeat=d):
        if sum(beta) > J:
            continue
        for k in itertools.product((0, 1), repeat=d):
            idx = tuple(b - kk for b, kk in zip(beta, k))
            if min(idx) < 0:
                continue
            acc[idx] = acc.get(idx, 0) + (-1) ** sum(k)
    out = {}
    for beta, c in acc.items():
        if c != 0:
            out[tuple(b + min_level for b in beta)] = c
    return out


def coefficient_closed_form(d, w, i):
    """(-1)^{w+d-1-|i|} binom(d-1, w+d-1-|i|) (second line of eq. TD-combi-tec)."""
    t = w + d - 1 - sum(i)
    if t < 0 or t > d - 1:
        return 0
    return (-1) ** t * math.comb(d - 1, t)


def index_set(d, w, min_level=1):
    """Components and coefficients, ordered by (|i| descending, then lexicographic).

    Enumerated by brute force over the box and filtered by w <= |i| <= w+d-1.
    """
    hi = w + d - 1 - (d - 1) * min_level
    out = []
    for i in itertools.product(range(min_level, hi + 1), repeat=d):
        if w <= sum(i) <= w + d - 1:
            out.append(tuple(i))
    out.sort(key=lambda t: (-sum(t), t))
    coef = coefficients_by_expansion(d, w, min_level)
    return [(i, coef[i]) for i in out]


def neumaier_sum(terms):
    """Neumaier-compensated sum along axis 0 of an array [n, ...] (FP64)."""
    terms = np.asarray(terms, dtype=np.float64)
    s = np.zeros(terms.shape[1:])
    c = np.zeros(terms.shape[1:])
    for t in terms:
        u = s + t
        big = np.abs(s) >= np.abs(t)
        c += np.where(big, (s - u) + t, (t - u) + s)
        s = u
    return s + c


def combine(values, coeffs):
    """u_J(x) = sum_i c_i u_i(x) with Neumaier compensation (eq. TD-combi-tec).

    values [ngrids, P], coeffs [ngrids].
    """
    values = np.asarray(values, dtype=np.float64)
    coeffs = np.asarray(coeffs, dtype=np.float64)
    return neumaier_sum(values * coeffs[:, None])
