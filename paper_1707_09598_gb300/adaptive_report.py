"""Profits of the hierarchical surpluses and knapsack-chosen index sets on the
quarter annulus (the paper's Sec. 4.2 discussion of optimal sets), through
the C ABI.

Every component of the full set {beta : 1 <= beta_k <= J} is solved in one
plan (FP64, batched FD-PCG to 1e-12) and evaluated on the error rule of
rates_report (values only). The surpluses
Delta_beta = sum_k (-1)^|k| u_{beta-k} then give revenue = ||Delta_beta||_L2
(the rule's weights times |det J|), cost = the DoFs of component beta, and
profit = revenue / cost. For each budget (the DoFs of the standard
sparse-grid set of level w), the admissible Dantzig choice
(paper_1707_09598_gb300.knapsack) picks a set. A plan over exactly that set,
with the coefficients of its surpluses, is solved, and its L2 error against
the exact u is compared with the standard set's. Prints one JSON line.

  python -m paper_1707_09598_gb300.adaptive_report [--J 8] [--p 2] [--r 1]
"""
import argparse
import itertools
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1707_09598_gb300 import knapsack, rates_report, sgiga  # noqa: E402


def values_at(P, xi_d, npts):
    ng = P.info.ngrids
    uc = torch.zeros(ng * npts, dtype=torch.float64, device="cuda")
    sgiga.sgiga_eval(P.handle, xi_d, npts, uc)
    return uc.view(ng, npts).cpu().numpy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--J", type=int, default=8)
    ap.add_argument("--p", type=int, default=2)
    ap.add_argument("--r", type=int, default=1)
    ap.add_argument("--nel", type=int, default=64)
    ap.add_argument("--source", default="paper", choices=["paper", "one"],
                    help="paper: the regular u of Sec. 4.2 (errors against it); one: f = 1, the "
                         "low-regularity problem of Sec. 4.3 (errors against the full tensor solution beta = (J, J))")
    a = ap.parse_args()
    src = "annulus_paper" if a.source == "paper" else "one"
    stream = torch.cuda.Stream()
    # torch's fills and reads of the buffers handed to the plan run on the
    # plan's stream, in order with its calls
    torch.cuda.set_stream(stream)
    xi, wt = rates_report.rule(a.nel, a.p + 2)
    npts = len(xi)
    xi_d = torch.as_tensor(xi, device="cuda")
    full = [b for b in itertools.product(range(1, a.J + 1), repeat=2)]
    P = sgiga.Plan(2, a.p, 2, domain="annulus", continuity=a.r, stream=stream, components=full,
                   coefficients=[1.0] * len(full))
    sgiga.sgiga_set_rhs_builtin(P.handle, src)
    sgiga.sgiga_solve(P.handle, 1e-12, 1000)
    x = torch.zeros(npts * 2, dtype=torch.float64, device="cuda")
    det = torch.zeros(npts, dtype=torch.float64, device="cuda")
    sgiga.sgiga_map_points(P.handle, xi_d, None, npts, x, det)
    w = wt * np.abs(det.cpu().numpy())
    ue, _ = rates_report.exact(x.cpu().numpy().reshape(-1, 2))
    vals = values_at(P, xi_d, npts)
    u = {tuple(g.levels[:2]): vals[k] for k, g in enumerate(P.grids)}
    cost = {tuple(g.levels[:2]): int(g.ndof) for g in P.grids}
    P.close()
    if a.source == "one":
        ue = u[(a.J, a.J)]          # reference: the full tensor solution of the top level
    delta = knapsack.surpluses(u)
    revenue = {b: float(np.sqrt(np.sum(w * delta[b] ** 2))) for b in delta}
    profit = {b: revenue[b] / cost[b] for b in delta}

    def l2_error(coef):
        uI = sum(c * u[g] for g, c in coef.items())
        return float(np.sqrt(np.sum(w * (uI - ue) ** 2)))

    rows = []
    for wl in range(3, (a.J if a.source == "paper" else a.J - 2) + 1):
        std = [b for b in full if sum(b) <= wl + 1]           # |beta| <= w + d - 1
        budget = sum(cost[b] for b in std)
        chosen = knapsack.choose(profit, cost, budget)
        c_std, c_ks = knapsack.set_coefficients(std), knapsack.set_coefficients(chosen)
        # the chosen set solved on its own plan (coefficients of its surpluses)
        comps = sorted(c_ks)
        Q = sgiga.Plan(2, a.p, 2, domain="annulus", continuity=a.r, stream=stream, components=comps,
                       coefficients=[c_ks[g] for g in comps])
        sgiga.sgiga_set_rhs_builtin(Q.handle, src)
        sgiga.sgiga_solve(Q.handle, 1e-12, 1000)
        uc = torch.zeros(len(comps) * npts, dtype=torch.float64, device="cuda")
        sgiga.sgiga_eval(Q.handle, xi_d, npts, uc)
        ucomb = torch.zeros(npts, dtype=torch.float64, device="cuda")
        sgiga.sgiga_combine(Q.handle, uc, npts, ucomb)
        Q.close()
        err_plan = float(np.sqrt(np.sum(w * (ucomb.cpu().numpy() - ue) ** 2)))
        rows.append({"w": wl, "budget_dofs": budget, "standard_l2": l2_error(c_std),
                     "knapsack_l2": err_plan, "knapsack_l2_from_full_plan": l2_error(c_ks),
                     "knapsack_set": sorted(chosen), "knapsack_dofs": sum(cost[b] for b in chosen),
                     "same_as_standard": sorted(chosen) == sorted(std)})
    out = {"workload": "quarter annulus, %s, p = %d C^%d, full set max beta <= %d"
                       % ("u = -(x^2+y^2-1)(x^2+y^2-4) x y^2" if a.source == "paper" else
                          "f = 1 (errors against the full tensor solution beta = (J, J))", a.p, a.r, a.J),
           "profits": {"%d,%d" % b: profit[b] for b in sorted(profit)},
           "revenues": {"%d,%d" % b: revenue[b] for b in sorted(revenue)},
           "costs": {"%d,%d" % b: cost[b] for b in sorted(cost)}, "budgets": rows}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
