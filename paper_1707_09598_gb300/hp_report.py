"""Error, DoFs and solve time of the h-p sparse combination against the
h-sparse one (Q = 0), on the quarter annulus with the regular u of the
paper's Table 2 (Sec. 4.2), through the C ABI.

For each Q and level w: one FP64 plan per degree p0 .. p0 + Q at
continuity r (paper_1707_09598_gb300.hp_sparse), batched FD-PCG to 1e-12,
values of every component at the points of a (p0 + Q + 2)-point Gauss rule
on nel^d elements (sgiga_eval), their combination over all plans
(sgiga_combine_plans), and the L2 error against the exact u with weights
times |det J| (sgiga_map_points). The solve time is CUDA-event time on the
plans' stream around the solves of all plans (plans built beforehand).
Prints one JSON line.

  python -m paper_1707_09598_gb300.hp_report [--d 2] [--p0 2] [--r 1] [--wmin 3] [--wmax 9] [--Qs 0,1,2]
"""
import argparse
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1707_09598_gb300 import hp_sparse, rates_report, sgiga  # noqa: E402


def run(d, p0, r, w, Q, nel, stream):
    xi, wt = rates_report.rule(nel, p0 + Q + 2, d)
    npts = len(xi)
    with torch.cuda.stream(stream):
        xi_d = torch.as_tensor(xi, device="cuda")
        with hp_sparse.HPCombination(d, p0, r, w, Q, domain="annulus", stream=stream) as H:
            H.set_rhs_builtin("annulus_paper")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            stats = H.solve(1e-12, 2000)
            e1.record(stream)
            torch.cuda.synchronize()
            uc = torch.zeros(H.ngrids * npts, dtype=torch.float64, device="cuda")
            u = torch.zeros(npts, dtype=torch.float64, device="cuda")
            H.eval_combine(xi_d, npts, uc, u)
            x = torch.zeros(npts * d, dtype=torch.float64, device="cuda")
            det = torch.zeros(npts, dtype=torch.float64, device="cuda")
            sgiga.sgiga_map_points(H.plans[0][1].handle, xi_d, None, npts, x, det)
            ue, _ = rates_report.exact(x.cpu().numpy().reshape(-1, d))
            du = u.cpu().numpy() - ue
            l2 = float(np.sqrt(np.sum(wt * np.abs(det.cpu().numpy()) * du * du)))
            return {"w": w, "Q": Q, "degrees": [p for p, _ in H.plans], "ngrids": H.ngrids, "ndof": H.ndof,
                    "ngrids_per_degree": [P.info.ngrids for _, P in H.plans],
                    "ndof_per_degree": [P.info.ndof for _, P in H.plans],
                    "iterations": [s.iterations for s in stats], "solve_ms": e0.elapsed_time(e1), "l2": l2}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--p0", type=int, default=2)
    ap.add_argument("--r", type=int, default=1)
    ap.add_argument("--wmin", type=int, default=3)
    ap.add_argument("--wmax", type=int, default=9)
    ap.add_argument("--Qs", default="0,1,2")
    ap.add_argument("--nel", type=int, default=64)
    a = ap.parse_args()
    stream = torch.cuda.Stream()
    rows = []
    for Q in [int(v) for v in a.Qs.split(",")]:
        for w in range(a.wmin, a.wmax + 1):
            rows.append(run(a.d, a.p0, a.r, w, Q, a.nel, stream))
    print(json.dumps({"workload": "quarter annulus, u of Table 2, d=%d, p0=%d, C^%d" % (a.d, a.p0, a.r),
                      "rows": rows}))


if __name__ == "__main__":
    main()
