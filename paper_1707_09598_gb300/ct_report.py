"""The combination technique as a preconditioner of the full tensor-product
solve (the paper's closing remark, Sec. 5), measured: the full system of
level J (unit square or cube, or the quarter annulus; p = 2 C^1,
a(x) = exp(sin 3x cos 2y), f = 1)
solved by FP64 FD-PCG alone and by flexible CG with FD + B_CT, B_CT over the
components of level w = J solved by the combination plan's batched PCG.

  python -m paper_1707_09598_gb300.ct_report [--d 2] [--domain unit] [--levels 6,7,8] [--inner-tol 1e-6]

Prints one markdown row per level: outer iterations, total inner iterations
and CUDA-event milliseconds of both solves to a relative residual of 1e-10.
"""
import argparse
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1707_09598_gb300 import sgiga  # noqa: E402


def coefficient(x):
    return np.exp(np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1]))


def set_coefficient(P, d):
    xq = np.zeros(d * P.info.nqp)
    sgiga.sgiga_qp_coords(P.handle, xq)
    sgiga.sgiga_set_coefficient_qp(P.handle, coefficient(xq.reshape(d, -1).T))


def timed(P, tol):
    st = None
    best = 1e30
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        st, _ = sgiga.sgiga_solve(P.handle, tol, 1000)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return st, best


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--domain", default="unit", choices=["unit", "annulus"])
    ap.add_argument("--levels", default="6,7,8")
    ap.add_argument("--inner-tol", type=float, default=1e-6)
    a = ap.parse_args()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    print("| domain | d | J | full DoFs | components | FD: iterations / ms | FD + CT: outer / inner iterations / ms |")
    print("|---|---|---|---|---|---|---|")
    for J in (int(v) for v in a.levels.split(",")):
        full = sgiga.Plan(a.d, 2, 2 * J, domain=a.domain, continuity=1, components=[(J,) * a.d], coefficients=[1.0],
                          stream=stream)
        comb = sgiga.Plan(a.d, 2, J, domain=a.domain, continuity=1, stream=stream)
        with full, comb:
            for P in (full, comb):
                set_coefficient(P, a.d)
            sgiga.sgiga_autotune(comb.handle, reps=2)
            sgiga.sgiga_set_rhs_builtin(full.handle, "one")
            s1, t1 = timed(full, 1e-10)
            sgiga.sgiga_ct_attach(full.handle, comb.handle, a.inner_tol, 500)
            s2, t2 = timed(full, 1e-10)
            sgiga.sgiga_ct_attach(full.handle, None)
            print("| %s | %d | %d | %d | %d | %d / %.2f | %d / %d / %.2f |" % (
                a.domain, a.d, J, full.info.ndof, comb.info.ngrids, s1.iterations, t1, s2.iterations,
                s2.inner_iterations, t2))


if __name__ == "__main__":
    main()
