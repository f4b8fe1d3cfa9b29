"""The knapsack choice of the sparse-grid index set (Sec. 4.2, optimal
sets) from profits computed on the GPU: every component of a full square of
levels is solved and evaluated through the C ABI, the host set logic forms
the hierarchical surpluses (eq. Delta-combi-tec), their revenues and profits
(revenue / degrees of freedom) and the admissible Dantzig choice. The same
from the oracle's solves and its own set routines gives the same profits and
the same chosen sets."""
import itertools
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_09598_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_1707_09598_gb300 import sgiga
    return sgiga


def test_dantzig_choice_from_gpu_profits_equals_the_oracle(sg):
    from oracle import adaptive, geometry, problems
    from oracle.galerkin import Component
    from paper_1707_09598_gb300 import knapsack
    from paper_1707_09598_gb300.inputs import random_points
    L, p, npts = 5, 2, 400
    levels = list(itertools.product(range(1, L + 1), repeat=2))
    xi = np.ascontiguousarray(random_points(npts, 2, seed=84))
    wts = np.full(npts, 1.0 / npts)
    # GPU: one plan over the whole square, every component solved and evaluated
    with sg.Plan(2, p, 2, domain="annulus", components=levels, coefficients=[1.0] * len(levels)) as P:
        sg.sgiga_set_rhs_builtin(P.handle, "annulus_paper")
        sg.sgiga_solve(P.handle, 1e-13, 400)
        ng = P.info.ngrids
        uc = np.zeros(ng * npts)
        sg.sgiga_eval(P.handle, xi, npts, uc)
        info = [sg.sgiga_grid_info(P.handle, g) for g in range(ng)]
    vals = {tuple(info[g].levels[:2]): uc[g * npts:(g + 1) * npts] for g in range(ng)}
    cost = {tuple(info[g].levels[:2]): int(info[g].ndof) for g in range(ng)}
    assert sorted(vals) == sorted(levels)
    sur = knapsack.surpluses(vals)
    rev = {b: float(np.sqrt(np.sum(wts * sur[b] ** 2))) for b in levels}
    prof = {b: rev[b] / cost[b] for b in levels}
    # oracle: its own solves, surpluses, profits and choice
    geom = geometry.make("annulus", 2)
    f = problems.get("annulus_paper2").f
    ovals, ocost = {}, {}
    for b in levels:
        comp = Component(geom, b, p).assemble(f=f)
        ovals[b] = comp.evaluate(comp.solve(), xi)
        ocost[b] = comp.K.shape[0]
    assert ocost == cost
    oprof = adaptive.profits(ovals, wts, ocost)
    top = max(r for r, _ in oprof.values())
    for b in levels:
        assert abs(rev[b] - oprof[b][0]) < 1e-8 * oprof[b][0] + 1e-12 * top, (b, rev[b], oprof[b][0])
    # the ordering is decided by relative gaps far above those differences
    ps = sorted(v for _, v in oprof.values())
    assert min((b - a) / b for a, b in zip(ps, ps[1:])) > 1e-5
    total = sum(cost.values())
    for budget in (total // 20, total // 8, total // 3, total):
        mine = knapsack.choose(prof, cost, budget)
        theirs = adaptive.dantzig(oprof, ocost, budget)
        assert mine == theirs, budget
        assert mine and sum(cost[b] for b in mine) <= budget
    # the chosen sets are admissible, so their coefficients combine the surpluses
    chosen = knapsack.choose(prof, cost, total // 3)
    coef = knapsack.set_coefficients(chosen)
    comb = sum(c * vals[g] for g, c in coef.items())
    assert np.abs(comb - sum(sur[b] for b in chosen)).max() < 1e-12 * np.abs(comb).max()
