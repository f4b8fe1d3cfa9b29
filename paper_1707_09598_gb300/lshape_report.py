"""Combined L2 / H1 error against level on the L-shaped domain.

-Laplace u = 0 on (-1,1)^2 minus [0,1] x [-1,0] (three glued bilinear patches),
u = r^(2/3) sin(2 theta/3) on the boundary, p = 2 C^1, one-sided grading
t^gamma toward the re-entrant corner, levels w = 5..11, batched
mixed-precision PCG (FP32 inner solve, FP64 refinement) to relative residual
1e-10. The errors of the combined solution sum_i c_i u_i against the exact u
are integrated with 4 x 4 Gauss points on a uniform 64 x 64 mesh of every
patch (|det J| = 1); the values and gradients come from sgiga_eval_grad and
sgiga_combine. Prints one JSON line with, per gamma, the errors per level, the
least-squares rates in w, and the solve times (CUDA events on the plan's
stream).

  python -m paper_1707_09598_gb300.lshape_report [--wmin 5] [--wmax 11] [--precision mixed]
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

SIGNS = np.array([[1.0, 1.0], [-1.0, 1.0], [-1.0, -1.0]])


def error_rule(nel=64, nq=4):
    t, w = np.polynomial.legendre.leggauss(nq)
    z = np.linspace(0.0, 1.0, nel + 1)
    h = np.diff(z)
    x = (z[:-1, None] + 0.5 * h[:, None] * (t[None, :] + 1.0)).reshape(-1)
    wx = (0.5 * h[:, None] * w[None, :]).reshape(-1)
    X0, X1 = np.meshgrid(x, x, indexing="xy")
    xi = np.stack([X0.reshape(-1), X1.reshape(-1)], 1)
    wt = np.outer(wx, wx).reshape(-1)
    patch = np.repeat(np.arange(3), len(xi)).astype(np.int32)
    return np.concatenate([xi] * 3), patch, np.concatenate([wt] * 3)


def exact(x):
    r = np.hypot(x[:, 0], x[:, 1])
    th = np.arctan2(x[:, 1], x[:, 0])
    th = np.where(th < 0, th + 2 * np.pi, th)
    u = r ** (2 / 3) * np.sin(2 * th / 3)
    ur = (2 / 3) * r ** (-1 / 3) * np.sin(2 * th / 3)
    ut = (2 / 3) * r ** (-1 / 3) * np.cos(2 * th / 3)
    c, s = np.cos(th), np.sin(th)
    return u, np.stack([ur * c - ut * s, ur * s + ut * c], 1)


def rate(levels, errs):
    A = np.vstack([np.asarray(levels, float), np.ones(len(levels))]).T
    return float(-np.linalg.lstsq(A, np.log2(np.asarray(errs)), rcond=None)[0][0])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--wmin", type=int, default=5)
    ap.add_argument("--wmax", type=int, default=11)
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--tol-gamma3", type=float, default=1e-9,
                    help="gamma = 3 at w = 11: the FP64 true residual floors near 3e-10 (cond ~1e12)")
    a = ap.parse_args()
    xi, patch, wt = error_rule()
    x = xi * SIGNS[patch]
    ue, ge = exact(x)
    npts = len(xi)
    stream = torch.cuda.Stream()
    # torch's fills and reads of the buffers handed to the plan run on the
    # plan's stream, in order with its calls
    torch.cuda.set_stream(stream)
    xi_d = torch.as_tensor(xi, device="cuda")
    patch_d = torch.as_tensor(patch, device="cuda")
    out = {"workload": "L-shape, 3 glued bilinear patches, u = r^(2/3) sin(2 theta/3) Dirichlet data, f = 0, p = 2 C^1, "
                       "one-sided grading toward the corner, %s PCG to %g (gamma = 3: %g)" % (a.precision, a.tol, a.tol_gamma3),
           "error_rule": "4x4 Gauss points on a uniform 64x64 mesh per patch", "results": {}}
    for gamma in (1.0, 2.0, 3.0):
        rows = []
        for w in range(a.wmin, a.wmax + 1):
            P = sgiga.Plan(2, 2, w, domain="lshape", grading="onesided", gamma=gamma, precision=a.precision,
                           stream=stream)
            sgiga.sgiga_autotune(P.handle, reps=2)
            sgiga.sgiga_set_rhs_builtin(P.handle, "lshape_corner")
            tol = a.tol_gamma3 if gamma == 3.0 else a.tol
            sgiga.sgiga_solve(P.handle, tol, 3000, check=False)      # warm-up (graph capture)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            st, rc = sgiga.sgiga_solve(P.handle, tol, 3000, check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            print("gamma=%g w=%d rc=%d outer=%d inner=%d fallback=%d maxres=%.2e" %
                  (gamma, w, rc, st.iterations, st.inner_iterations, st.fallback, st.max_rel_residual),
                  file=sys.stderr, flush=True)
            ng = P.info.ngrids
            uc = torch.zeros(ng * npts, dtype=torch.float64, device="cuda")
            gc = torch.zeros(2 * ng * npts, dtype=torch.float64, device="cuda")
            sgiga.sgiga_eval_grad(P.handle, xi_d, patch_d, npts, uc, gc)
            u = torch.zeros(npts, dtype=torch.float64, device="cuda")
            g0 = torch.zeros_like(u)
            g1 = torch.zeros_like(u)
            sgiga.sgiga_combine(P.handle, uc, npts, u)
            sgiga.sgiga_combine(P.handle, gc[:ng * npts], npts, g0)
            sgiga.sgiga_combine(P.handle, gc[ng * npts:], npts, g1)
            du = u.cpu().numpy() - ue
            dg = np.stack([g0.cpu().numpy(), g1.cpu().numpy()], 1) - ge
            l2 = float(np.sqrt(np.sum(wt * du * du)))
            h1 = float(np.sqrt(np.sum(wt * np.sum(dg * dg, 1))))
            rows.append({"w": w, "tol": tol, "ngrids": ng, "ndof": P.info.ndof, "l2": l2, "h1": h1,
                         "solve_ms": e0.elapsed_time(e1), "outer": st.iterations, "inner": st.inner_iterations,
                         "max_rel_residual": st.max_rel_residual, "fp64_fallback": bool(st.fallback & 2),
                         "rc": rc})
            P.close()
        ws = [r["w"] for r in rows]
        out["results"]["gamma=%g" % gamma] = {
            "levels": rows, "rate_l2": rate(ws, [r["l2"] for r in rows]),
            "rate_h1": rate(ws, [r["h1"] for r in rows])}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
