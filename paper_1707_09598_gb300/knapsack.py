"""Index sets chosen by the profits of their hierarchical surpluses (the
knapsack view of the sparse-grid set, Sec. 4.2; Dantzig method). Host-side
set logic around the solver: the solves and evaluations run in the library.

For a set I of multi-indices, u_I = sum_{beta in I} Delta_beta with
Delta_beta = sum_{k in {0,1}^d} (-1)^{|k|} u_{beta-k} (eq. Delta-combi-tec),
which is the combination sum_gamma c_gamma u_gamma with
c_gamma = sum_k (-1)^{|k|} [gamma + k in I].
"""
import numpy as np


def _shifts(d):
    """(offset, sign) for the 2^d corners of the unit cube."""
    out = []
    for m in range(1 << d):
        off = tuple((m >> k) & 1 for k in range(d))
        out.append((off, -1 if bin(m).count("1") % 2 else 1))
    return out


def set_coefficients(levels):
    """{gamma: c_gamma} for the index set `levels` (zero coefficients dropped)."""
    S = {tuple(int(v) for v in b) for b in levels}
    d = len(next(iter(S)))
    out = {}
    for g in S:
        c = sum(sign for off, sign in _shifts(d) if tuple(a + o for a, o in zip(g, off)) in S)
        if c:
            out[g] = c
    return out


def surpluses(u, min_level=1):
    """{beta: Delta_beta} from component values u (dict beta -> array)."""
    d = len(next(iter(u)))
    out = {}
    for beta in u:
        acc = np.zeros_like(next(iter(u.values())))
        for off, sign in _shifts(d):
            g = tuple(b - o for b, o in zip(beta, off))
            if min(g) >= min_level:
                acc = acc + sign * u[g]
        out[beta] = acc
    return out


def choose(profit, cost, budget, min_level=1):
    """Admissible Dantzig choice: repeatedly take the highest-profit index
    whose backward neighbours are taken, until the next would exceed the
    budget. Returns the chosen indices in order."""
    taken, spent = [], 0
    have = set()
    cand = sorted(profit, key=lambda b: (-profit[b], b))
    while True:
        nxt = None
        for b in cand:
            if b in have:
                continue
            ok = all(b[k] == min_level or tuple(v - (j == k) for j, v in enumerate(b)) in have
                     for k in range(len(b)))
            if ok:
                nxt = b
                break
        if nxt is None or spent + cost[nxt] > budget:
            return taken
        taken.append(nxt)
        have.add(nxt)
        spent += cost[nxt]
