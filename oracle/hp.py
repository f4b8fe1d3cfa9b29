"""h-p sparse combination of the oracle: the combination technique with the
spline degree as one more index. The paper builds its sparse grids by
h-refinement alone; it names a p-sparsification, or a combined h-p version,
as possible (Sec. 2.2) and as a direction for further work (Sec. 5), without
fixing a construction. This module takes the following reading.

TEST INFRASTRUCTURE: see the package header.

Component (i, q): the spline space of degree p0 + q with continuity C^r at
every interior breakpoint, on the mesh with 2^{i_k} elements in direction k
(eq. u-IGA-approx, Dirichlet functions removed). One r <= p0 - 1 serves every
degree, so that raising the degree keeps each space inside the next one on
the same mesh (a piecewise polynomial of degree p with C^r joints is one of
degree p + 1 with C^r joints), just as refining the mesh does (Sec. 3).

Index set of level w with Q degree steps: (beta, q) with beta = i - m >= 0
(m = min_level), 0 <= q <= Q and |beta| + q <= J, J = w + d - 1 - d m as in
eq. TD-approx. The approximation is the sum of Delta_{beta,q} over that set,
where Delta is the difference operator of eq. Delta-combi-tec taken in all
d + 1 indices (u of an index with a negative entry is 0). Expanded, it is a
sum of component solutions with integer coefficients. Q = 0 is the h-sparse
set of eq. TD-combi-tec.
"""
import itertools

import numpy as np

from . import combination
from .galerkin import Component


def hp_index_set(d, w, Q, min_level=1):
    """The (beta, q) of the set, beta = i - min_level, as tuples of d + 1."""
    J = w + d - 1 - d * min_level
    if J < 0 or Q < 0:
        raise ValueError("level too small for min_level, or Q < 0")
    out = []
    for t in itertools.product(range(J + 1), repeat=d):
        for q in range(Q + 1):
            if sum(t) + q <= J:
                out.append(tuple(t) + (q,))
    return out


def hp_coefficients_by_expansion(d, w, Q, min_level=1):
    """{(i_1, .., i_d, q): c} over the components with a nonzero coefficient:
    every Delta_{beta,q} of the set expanded into (-1)^{|k|} u_{(beta,q) - k},
    k in {0,1}^{d+1}, terms with a negative index dropped."""
    acc = {}
    for a in hp_index_set(d, w, Q, min_level):
        for k in itertools.product((0, 1), repeat=d + 1):
            idx = tuple(x - y for x, y in zip(a, k))
            if min(idx) < 0:
                continue
            acc[idx] = acc.get(idx, 0) + (-1) ** sum(k)
    return {tuple(b + min_level for b in a[:d]) + (a[d],): c for a, c in acc.items() if c != 0}


def hp_solution(geom, f, d, p0, r, w, Q, pts, min_level=1):
    """Combined value at parametric points pts [P, d] and the per-component
    values {(i.., q): values}: each component assembled by Gauss quadrature
    and solved by a sparse direct solve (Sec. 4.1), then the Neumaier sum
    with the coefficients above (eq. TD-combi-tec)."""
    if r > p0 - 1:
        raise ValueError("continuity r must be at most p0 - 1")
    coef = hp_coefficients_by_expansion(d, w, Q, min_level)
    vals = {}
    for key in sorted(coef):
        comp = Component(geom, key[:d], p0 + key[d], r).assemble(f=f)
        vals[key] = comp.evaluate(comp.solve(), pts)
    keys = sorted(coef)
    u = combination.combine(np.array([vals[k] for k in keys]), np.array([coef[k] for k in keys], float))
    return u, vals, coef
