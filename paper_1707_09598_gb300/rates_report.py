"""Convergence rates of the combined solution on the quarter annulus (the
measurements of the paper's Table 2, Sec. 4.2), computed through the C ABI.

-Laplace u = f on the quarter annulus (radii 1 and 2; d = 3: extruded over
z in [0, 1]), u = -(x^2+y^2-1)(x^2+y^2-4) x y^2 [sin(pi z)] (the paper's
regular solution), homogeneous Dirichlet data, p = 2 (C^0, C^1) and p = 3
(C^0, C^1, C^2), levels w = wmin..wmax.
Every level is solved in FP64 (batched FD-PCG to 1e-12). The combined values
and gradients come from sgiga_eval_grad + sgiga_combine, and the physical
points and |det J| from sgiga_map_points. L2 and H1-seminorm errors use a
(p+2)-point Gauss rule on a uniform nel^d parametric mesh with weights
times |det J|, the rule of the oracle's error routine. Rates are
least-squares slopes of log2(error) against w, over all levels and over the
last four. Prints one JSON line.

  python -m paper_1707_09598_gb300.rates_report [--d 2] [--wmin 3] [--wmax 10] [--nel 64]
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

from paper_1707_09598_gb300 import sgiga  # noqa: E402

# Table 2, SG-IGA rows: d -> (r, p) -> (H1 rate, L2 rate)
TABLE2_D = {
    2: {(0, 2): (2.29, 3.03), (1, 2): (2.16, 3.04), (0, 3): (3.21, 3.94), (1, 3): (3.05, 3.93),
        (2, 3): (3.06, 4.15)},
    3: {(0, 2): (2.38, 3.12), (1, 2): (2.23, 3.08), (0, 3): (3.30, 4.00), (1, 3): (3.13, 3.93),
        (2, 3): (3.15, 4.26)},
}
TABLE2 = TABLE2_D[2]


def exact(x):
    """u = -phi x y^2 [sin(pi z)] with phi = (r^2 - 1)(r^2 - 4);
    d phi/dx = (2 r^2 - 5) 2x. x is [npts][d]."""
    X, Y = x[:, 0], x[:, 1]
    r2 = X * X + Y * Y
    phi = (r2 - 1.0) * (r2 - 4.0)
    g = 2.0 * r2 - 5.0
    u = -phi * X * Y * Y
    ux = -(g * 2.0 * X) * X * Y * Y - phi * Y * Y
    uy = -(g * 2.0 * Y) * X * Y * Y - phi * 2.0 * X * Y
    if x.shape[1] == 2:
        return u, np.stack([ux, uy], 1)
    s, c = np.sin(np.pi * x[:, 2]), np.cos(np.pi * x[:, 2])
    return u * s, np.stack([ux * s, uy * s, u * np.pi * c], 1)


def rule(nel, Q, d=2):
    t, w = np.polynomial.legendre.leggauss(Q)
    z = np.linspace(0.0, 1.0, nel + 1)
    h = np.diff(z)
    x = (z[:-1, None] + 0.5 * h[:, None] * (t[None, :] + 1.0)).reshape(-1)
    wx = (0.5 * h[:, None] * w[None, :]).reshape(-1)
    X = np.meshgrid(*([x] * d), indexing="ij")
    W = np.meshgrid(*([wx] * d), indexing="ij")
    return (np.ascontiguousarray(np.stack([a.reshape(-1) for a in X], 1)),
            np.prod(np.stack([a.reshape(-1) for a in W], 1), 1))


def errors_at(P, xi, wt, npts, stream):
    """(L2, H1) errors of the plan's combined solution at the rule's points."""
    d = P.info.d
    xi_d = torch.as_tensor(xi, device="cuda")
    x = torch.zeros(npts * d, dtype=torch.float64, device="cuda")
    det = torch.zeros(npts, dtype=torch.float64, device="cuda")
    sgiga.sgiga_map_points(P.handle, xi_d, None, npts, x, det)
    ng = P.info.ngrids
    uc = torch.zeros(ng * npts, dtype=torch.float64, device="cuda")
    gc = torch.zeros(d * ng * npts, dtype=torch.float64, device="cuda")
    sgiga.sgiga_eval_grad(P.handle, xi_d, None, npts, uc, gc)
    u = torch.zeros(npts, dtype=torch.float64, device="cuda")
    sgiga.sgiga_combine(P.handle, uc, npts, u)
    gs = []
    for k in range(d):
        gk = torch.zeros_like(u)
        sgiga.sgiga_combine(P.handle, gc[k * ng * npts:(k + 1) * ng * npts], npts, gk)
        gs.append(gk.cpu().numpy())
    xh = x.cpu().numpy().reshape(-1, d)
    w = wt * np.abs(det.cpu().numpy())
    ue, ge = exact(xh)
    du = u.cpu().numpy() - ue
    dg = np.stack(gs, 1) - ge
    return float(np.sqrt(np.sum(w * du * du))), float(np.sqrt(np.sum(w * np.sum(dg * dg, 1))))


def rate(levels, errs):
    A = np.vstack([np.asarray(levels, float), np.ones(len(levels))]).T
    return float(-np.linalg.lstsq(A, np.log2(np.asarray(errs)), rcond=None)[0][0])


def run_case(p, r, ws, nel, stream, d=2):
    xi, wt = rule(nel, p + 2, d)
    npts = len(xi)
    rows = []
    # torch's fills and reads of the buffers handed to the plan run on the
    # plan's stream, in order with its calls
    with torch.cuda.stream(stream):
        for w in ws:
            P = sgiga.Plan(d, p, w, domain="annulus", continuity=r, stream=stream)
            sgiga.sgiga_set_rhs_builtin(P.handle, "annulus_paper")
            st, _ = sgiga.sgiga_solve(P.handle, 1e-12, 500)
            l2, h1 = errors_at(P, xi, wt, npts, stream)
            rows.append({"w": w, "ngrids": P.info.ngrids, "ndof": P.info.ndof, "l2": l2, "h1": h1,
                         "iterations": st.iterations})
            P.close()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--wmin", type=int, default=3)
    ap.add_argument("--wmax", type=int, default=10)
    ap.add_argument("--nel", type=int, default=64)
    a = ap.parse_args()
    stream = torch.cuda.Stream()
    sol = "-(x^2+y^2-1)(x^2+y^2-4) x y^2" + (" sin(pi z)" if a.d == 3 else "")
    out = {"workload": "quarter annulus, u = %s, d = %d, FP64 batched FD-PCG to 1e-12" % (sol, a.d),
           "error_rule": "(p+2)-point Gauss on a uniform %d^%d parametric mesh, weights x |det J|" % (a.nel, a.d),
           "cases": {}}
    ws = list(range(a.wmin, a.wmax + 1))
    for (r, p), (h1_ref, l2_ref) in TABLE2_D[a.d].items():
        rows = run_case(p, r, ws, a.nel, stream, a.d)
        L, H = [x["l2"] for x in rows], [x["h1"] for x in rows]
        out["cases"]["p=%d C^%d" % (p, r)] = {
            "levels": rows, "rate_l2": rate(ws, L), "rate_h1": rate(ws, H),
            "rate_l2_last4": rate(ws[-4:], L[-4:]), "rate_h1_last4": rate(ws[-4:], H[-4:]),
            "rate_l2_w3_7": rate(ws[:5], L[:5]), "rate_h1_w3_7": rate(ws[:5], H[:5]),
            "table2": {"l2": l2_ref, "h1": h1_ref}}
        print("p=%d C^%d: L2 %.2f / w<=7 %.2f (Table 2 %.2f), H1 %.2f / w<=7 %.2f (Table 2 %.2f)" %
              (p, r, rate(ws, L), rate(ws[:5], L[:5]), l2_ref, rate(ws, H), rate(ws[:5], H[:5]), h1_ref),
              file=sys.stderr, flush=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
