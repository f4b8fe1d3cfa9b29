"""Convergence rates of the combined solution on the quarter annulus (the
measurements of the paper's Tables 2 and 3, Sec. 4.2-4.3, and of the rates
against the grading exponent, Sec. 4.4), computed through the C ABI.

-Laplace u = f on the quarter annulus (radii 1 and 2; d = 3: extruded over
z in [0, 1]) with homogeneous Dirichlet data, levels w = wmin..wmax, every
level solved in FP64 (batched FD-PCG to 1e-12).
  --source paper  u = -(x^2+y^2-1)(x^2+y^2-4) x y^2 [sin(pi z)] (Table 2);
                  errors against it.
  --source one    f = 1 (Table 3): u has corner (and edge) singularities and
                  no closed form. Errors are measured against the full
                  tensor-product solution with every level = ref-level, on
                  the same knots.
  --grading radical --gammas g1,g2,..  the symmetric radical meshes of
                  Sec. 4.4, one rate pair per exponent.
The combined values and gradients come from sgiga_eval_grad + sgiga_combine,
and the physical points and |det J| from sgiga_map_points. L2 and
H1-seminorm errors use a (p+2)-point Gauss rule on nel^d elements, with
weights times |det J|. On uniform meshes this is the rule of the oracle's
error routine. On graded meshes the elements are the images of the uniform
ones under the grading map. Rates are least-squares slopes of log2(error)
against w. Prints one JSON line.

  python -m paper_1707_09598_gb300.rates_report [--d 2] [--wmin 3] [--wmax 10] [--nel 64]
      [--source one --ref-level 12] [--grading radical --gammas 1,2,3] [--cases 2:0,3:2]
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

# Table 3 (f = 1, low-regular u; SG-IGA rows): d -> (r, p) -> (H1 rate, L2 rate)
TABLE3_D = {
    2: {(0, 2): (1.35, 1.72), (1, 2): (1.20, 1.72), (0, 3): (1.26, 1.74), (1, 3): (1.25, 1.78),
        (2, 3): (1.19, 1.58)},
    3: {(0, 2): (1.30, 1.62), (1, 2): (1.22, 1.63), (0, 3): (1.30, 1.71), (1, 3): (1.28, 1.75),
        (2, 3): (1.20, 1.55)},
}


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


def grading_map(t, grading="uniform", gamma=1.0):
    """Breakpoint map of the plan's knots and its derivative: t for uniform
    meshes; the symmetric radical map 2^(gamma-1) t^gamma (t <= 1/2), mirrored
    above 1/2 (Sec. 4.4)."""
    if grading == "uniform" or gamma == 1.0:
        return t, np.ones_like(t)
    c = 2.0 ** (gamma - 1.0)
    lo = t <= 0.5
    s = np.where(lo, t, 1.0 - t)
    g = c * s ** gamma
    return np.where(lo, g, 1.0 - g), c * gamma * s ** (gamma - 1.0)


def rule(nel, Q, d=2, grading="uniform", gamma=1.0):
    """Q-point Gauss rule on nel^d elements; on a graded plan the elements are
    the images of a uniform mesh under the plan's grading map, so the rule
    clusters where the mesh does (weights times the map's derivative)."""
    t, w = np.polynomial.legendre.leggauss(Q)
    z = np.linspace(0.0, 1.0, nel + 1)
    h = np.diff(z)
    x = (z[:-1, None] + 0.5 * h[:, None] * (t[None, :] + 1.0)).reshape(-1)
    wx = (0.5 * h[:, None] * w[None, :]).reshape(-1)
    x, dg = grading_map(x, grading, gamma)
    wx = wx * dg
    X = np.meshgrid(*([x] * d), indexing="ij")
    W = np.meshgrid(*([wx] * d), indexing="ij")
    return (np.ascontiguousarray(np.stack([a.reshape(-1) for a in X], 1)),
            np.prod(np.stack([a.reshape(-1) for a in W], 1), 1))


def fields_at(P, xi_d, npts):
    """Combined value [npts] and physical gradient [npts][d] of the plan's
    solution at parametric points (sgiga_eval_grad + sgiga_combine)."""
    d, ng = P.info.d, P.info.ngrids
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
    return u.cpu().numpy(), np.stack(gs, 1)


def errors_at(P, xi, wt, npts, stream, ref=None):
    """(L2, H1) errors of the plan's combined solution at the rule's points,
    against the exact u, or against ref = (values, gradients) at the points."""
    d = P.info.d
    xi_d = torch.as_tensor(xi, device="cuda")
    x = torch.zeros(npts * d, dtype=torch.float64, device="cuda")
    det = torch.zeros(npts, dtype=torch.float64, device="cuda")
    sgiga.sgiga_map_points(P.handle, xi_d, None, npts, x, det)
    u, g = fields_at(P, xi_d, npts)
    w = wt * np.abs(det.cpu().numpy())
    ue, ge = exact(x.cpu().numpy().reshape(-1, d)) if ref is None else ref
    du = u - ue
    dg = g - ge
    return float(np.sqrt(np.sum(w * du * du))), float(np.sqrt(np.sum(w * np.sum(dg * dg, 1))))


def rate(levels, errs):
    A = np.vstack([np.asarray(levels, float), np.ones(len(levels))]).T
    return float(-np.linalg.lstsq(A, np.log2(np.asarray(errs)), rcond=None)[0][0])


def solve(P, src, tol=1e-12):
    """Solve to tol; a run that stops at max_iter above tol (the residual
    floor of strongly graded meshes) is kept, with its residual recorded."""
    sgiga.sgiga_set_rhs_builtin(P.handle, src)
    st, rc = sgiga.sgiga_solve(P.handle, tol, 2000, check=False)
    if rc not in (sgiga.SGIGA_OK, sgiga.SGIGA_ERR_NOT_CONVERGED):
        sgiga._check(rc)
    return {"iterations": st.iterations, "converged": rc == sgiga.SGIGA_OK,
            "max_rel_residual": st.max_rel_residual}


def run_case(p, r, ws, nel, stream, d=2, source="paper", grading="uniform", gamma=1.0, ref_level=None):
    """Solve levels ws and return their errors. source "paper": the regular u
    (Table 2), errors against it. source "one": f = 1 (Table 3), errors
    against the full tensor-product solution with every level ref_level on
    the same mesh family (one component, coefficient 1)."""
    xi, wt = rule(nel, p + 2, d, grading, gamma)
    npts = len(xi)
    src = "annulus_paper" if source == "paper" else "one"
    kw = dict(domain="annulus", continuity=r, grading=grading, gamma=gamma, stream=stream)
    rows = []
    # torch's fills and reads of the buffers handed to the plan run on the
    # plan's stream, in order with its calls
    with torch.cuda.stream(stream):
        ref = None
        if source == "one":
            R = sgiga.Plan(d, p, 2, components=[(ref_level,) * d], coefficients=[1.0], **kw)
            info = solve(R, src)
            ref = fields_at(R, torch.as_tensor(xi, device="cuda"), npts)
            ref_info = dict(level=ref_level, ndof=R.info.ndof, **info)
            R.close()
        for w in ws:
            P = sgiga.Plan(d, p, w, **kw)
            info = solve(P, src)
            l2, h1 = errors_at(P, xi, wt, npts, stream, ref)
            rows.append(dict(w=w, ngrids=P.info.ngrids, ndof=P.info.ndof, l2=l2, h1=h1, **info))
            if ref is not None:
                rows[-1]["reference"] = ref_info
            P.close()
    return rows


def parse_cases(text, table):
    if not text:
        return [(p, r) for (r, p) in table]
    return [tuple(int(v) for v in c.split(":")) for c in text.split(",")]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--wmin", type=int, default=3)
    ap.add_argument("--wmax", type=int, default=10)
    ap.add_argument("--nel", type=int, default=64)
    ap.add_argument("--source", default="paper", choices=["paper", "one"],
                    help="paper: the regular u (Table 2); one: f = 1 (Table 3), errors against a full tensor solution")
    ap.add_argument("--ref-level", type=int, default=None, help="level of the reference (default wmax + 2)")
    ap.add_argument("--grading", default="uniform", choices=["uniform", "radical"])
    ap.add_argument("--gammas", default="1", help="comma-separated grading exponents (a sweep with radical)")
    ap.add_argument("--cases", default="", help="p:r list, e.g. 2:0,2:1,4:3 (default: the table's rows)")
    a = ap.parse_args()
    stream = torch.cuda.Stream()
    table = (TABLE2_D if a.source == "paper" else TABLE3_D)[a.d]
    ref_level = a.ref_level if a.ref_level is not None else a.wmax + 2
    if a.source == "paper":
        sol = "u = -(x^2+y^2-1)(x^2+y^2-4) x y^2" + (" sin(pi z)" if a.d == 3 else "")
    else:
        sol = "f = 1, errors against the full tensor solution of level %d" % ref_level
    out = {"workload": "quarter annulus, %s, d = %d, %s mesh, FP64 batched FD-PCG to 1e-12" % (sol, a.d, a.grading),
           "error_rule": "(p+2)-point Gauss on %d^%d elements (images of a uniform mesh under the grading map), "
                         "weights x |det J|" % (a.nel, a.d),
           "cases": {}}
    ws = list(range(a.wmin, a.wmax + 1))
    for gamma in [float(g) for g in a.gammas.split(",")]:
        for p, r in parse_cases(a.cases, table):
            rows = run_case(p, r, ws, a.nel, stream, a.d, a.source, a.grading, gamma, ref_level)
            L, H = [x["l2"] for x in rows], [x["h1"] for x in rows]
            h1_ref, l2_ref = table.get((r, p), (None, None)) if gamma == 1.0 else (None, None)
            key = "p=%d C^%d" % (p, r) + ("" if a.grading == "uniform" else " gamma=%g" % gamma)
            out["cases"][key] = {
                "levels": rows, "rate_l2": rate(ws, L), "rate_h1": rate(ws, H),
                "rate_l2_last4": rate(ws[-4:], L[-4:]), "rate_h1_last4": rate(ws[-4:], H[-4:]),
                "rate_l2_first5": rate(ws[:5], L[:5]), "rate_h1_first5": rate(ws[:5], H[:5]),
                "printed": {"l2": l2_ref, "h1": h1_ref}}
            print("%s: L2 %.2f / first 5 %.2f / last 4 %.2f (printed %s), H1 %.2f / first 5 %.2f / last 4 %.2f "
                  "(printed %s); max residual %.1e" %
                  (key, rate(ws, L), rate(ws[:5], L[:5]), rate(ws[-4:], L[-4:]), l2_ref, rate(ws, H),
                   rate(ws[:5], H[:5]), rate(ws[-4:], H[-4:]), h1_ref, max(max(x["max_rel_residual"], x.get("reference", x)["max_rel_residual"]) for x in rows)),
                  file=sys.stderr, flush=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
