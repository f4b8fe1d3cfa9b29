"""Hierarchical surpluses, their profits and the knapsack (Dantzig) choice of
the sparse-grid index set (the paper's Sec. 4.2 discussion of optimal sets).

TEST INFRASTRUCTURE: see the package header.

  Delta_beta(u) = sum_{k in {0,1}^d} (-1)^{|k|} u_{beta - k}     (eq. Delta-combi-tec)

with u_gamma = 0 when some gamma_k is below the coarsest level. A set I of
multi-indices gives u_I = sum_{beta in I} Delta_beta(u). Collecting the terms
per component gives combination coefficients:

  c_gamma = sum_{k in {0,1}^d} (-1)^{|k|} [gamma + k in I].

For the standard set {|beta| <= J} these are the coefficients of eq.
TD-combi-tec. Revenue of Delta_beta: its L2 norm. Cost: the degrees of
freedom of component beta. Profit: revenue / cost. The Dantzig method sorts
by profit and takes items until the budget is spent. Here, an item is taken
only once its backward neighbours are in the set (admissible sets, so that
the coefficient formula only involves components in I).
"""
import itertools

import numpy as np


def corners(d):
    return list(itertools.product((0, 1), repeat=d))


def coefficients(index_set):
    """Combination coefficients of an index set {beta} (a dict beta -> c)."""
    I = set(tuple(b) for b in index_set)
    d = len(next(iter(I)))
    out = {}
    for g in I:
        c = 0
        for k in corners(d):
            if tuple(gi + ki for gi, ki in zip(g, k)) in I:
                c += (-1) ** sum(k)
        if c != 0:
            out[g] = c
    return out


def surplus(values, beta, min_level=1):
    """Delta_beta from component values (dict level tuple -> array)."""
    acc = None
    for k in corners(len(beta)):
        g = tuple(b - kk for b, kk in zip(beta, k))
        if min(g) < min_level:
            continue
        term = (-1) ** sum(k) * values[g]
        acc = term if acc is None else acc + term
    return acc


def profits(values, weights, costs, min_level=1):
    """(revenue, profit) of every surplus of the full set of the given values:
    revenue = sqrt(sum_q w_q Delta_beta(x_q)^2), profit = revenue / cost."""
    out = {}
    for beta in values:
        delta = surplus(values, beta, min_level)
        rev = float(np.sqrt(np.sum(weights * delta * delta)))
        out[beta] = (rev, rev / costs[beta])
    return out


def admissible(beta, chosen, min_level=1):
    return all(b == min_level or tuple(bb - (j == k) for j, bb in enumerate(beta)) in chosen
               for k, b in enumerate(beta))


def dantzig(prof, costs, budget, min_level=1):
    """Items by decreasing profit, each once admissible, until the next one
    would exceed the budget. Returns the chosen set (a list, in choice order)."""
    order = sorted(prof, key=lambda b: (-prof[b][1], b))
    chosen, spent = [], 0
    done = set()
    progress = True
    while progress:
        progress = False
        for b in order:
            if b in done or not admissible(b, done, min_level):
                continue
            if spent + costs[b] > budget:
                return chosen
            chosen.append(b)
            done.add(b)
            spent += costs[b]
            progress = True
            break
    return chosen
