"""Learned-preconditioner comparison on the perturbed-cube workload.

3D Poisson -div(a grad u) = 1 on the unit cube mapped by a seeded cubic
B-spline perturbation (amplitude 0.1) with a log-normal coefficient a
(std 0.5, correlation length 0.2, random Fourier features), p = 3, level w
(12 by default: 199 components). Solves the same problem four ways and prints
one JSON line:

  fp64_fd      plain FP64 FD-preconditioned CG, tolerance 1e-12 (reference)
  fp64_fd_per_grid  plain FP64 FD-CG one component grid at a time (a plan
               per grid, stream-ordered host loop, no batching, no graph)
  mixed_fd     FP32 inner FD-CG inside FP64 refinement
  mixed_learned  FP32 inner flexible CG with M(r) = S * FD(S * r), S = exp(N(phi))
               from the trained network (training: target_pairs
               residual/error pairs from the plan's own CG)
  mixed_scaled   the same with the network-free scaling S = c^(-1/2)

with wall time (CUDA events on the plan's stream), iterations, and the
relative L2 of each solution's combined values (17^3 lattice) against the
fp64_fd reference.

The mixed plans run each FP32 inner solve to --inner-tol (1e-3, the fastest
of 1e-2 .. 1e-6 measured on this workload; 3 refinement steps either way).

  python -m paper_1707_09598_gb300.learned_report [--w 12] [--pairs 10000] [--epochs 6] [--inner-tol 1e-3]
      [--inner-tol-sweep 1e-2,3e-3,1e-3,1e-4,1e-5,1e-6]
"""
import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1707_09598_gb300 import sgiga  # noqa: E402
from paper_1707_09598_gb300.inputs import eval_points, lognormal_features, perturbed_cube_patch  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--w", type=int, default=12)
    ap.add_argument("--pairs", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=2)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--nfeat", type=int, default=128)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--inner-tol-sweep", default="",
                    help="comma-separated inner tolerances: also time the mixed FD solve at each (best of 3)")
    ap.add_argument("--inner-tol", type=float, default=1e-3,
                    help="relative tolerance of each FP32 inner solve of the mixed plans (measured best of "
                         "1e-2 .. 1e-6 on this workload; the library default is 1e-5)")
    a = ap.parse_args()
    kn, cp = perturbed_cube_patch(1)
    om, ph, amp = lognormal_features(2, nfeat=a.nfeat)
    stream = torch.cuda.Stream()
    # torch's fills and reads of the buffers handed to the plan run on the
    # plan's stream, in order with its calls
    torch.cuda.set_stream(stream)
    pts = torch.as_tensor(eval_points(3, 16), device="cuda")
    out = {"workload": "perturbed cube (amp 0.1, seed 1), log-normal a (std 0.5, ell 0.2, %d features, seed 2), "
                       "f = 1, p = 3, w = %d" % (a.nfeat, a.w)}

    def plan(precision, precond):
        t0 = time.perf_counter()
        P = sgiga.Plan(3, 3, a.w, domain="patch", patch=([3, 3, 3], kn, cp), precision=precision,
                       precond=precond, stream=stream)
        sgiga.sgiga_set_coefficient(P.handle, om, ph, amp)
        sgiga.sgiga_autotune(P.handle, reps=2)     # tiles and preconditioner layout, measured
        sgiga.sgiga_set_rhs_builtin(P.handle, "one")
        return P, time.perf_counter() - t0

    def timed_solve(P, tol, maxit):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        st, rc = sgiga.sgiga_solve(P.handle, tol, maxit, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        return st, rc, e0.elapsed_time(e1)

    def combined(P):
        uc = torch.zeros(P.info.ngrids * len(pts), dtype=torch.float64, device="cuda")
        sgiga.sgiga_eval(P.handle, pts, len(pts), uc)
        u = torch.zeros(len(pts), dtype=torch.float64, device="cuda")
        sgiga.sgiga_combine(P.handle, uc, len(pts), u)
        return u.cpu().numpy()

    P, ps = plan("fp64", "fd")
    out["ngrids"], out["ndof"] = P.info.ngrids, P.info.ndof
    timed_solve(P, 1e-12, 2000)               # warm-up
    st, rc, ms = timed_solve(P, 1e-12, 2000)
    ref = combined(P)
    out["fp64_fd"] = {"ms": ms, "iterations": st.iterations, "rc": rc, "plan_s": ps}
    st, rc, ms = timed_solve(P, a.tol, 2000)
    out["fp64_fd_at_tol"] = {"ms": ms, "iterations": st.iterations, "rc": rc,
                             "rel_l2_vs_ref": float(np.linalg.norm(combined(P) - ref) / np.linalg.norm(ref))}
    # plain per-grid FP64 PCG: one plan per component, solved one after the other
    comps = [tuple(g.levels[:3]) for g in P.grids]
    coefs = [g.coeff for g in P.grids]
    P.close()
    t0 = time.perf_counter()
    singles = []
    for cl in comps:
        Q = sgiga.Plan(3, 3, a.w, domain="patch", patch=([3, 3, 3], kn, cp), stream=stream, components=[cl])
        sgiga.sgiga_set_coefficient(Q.handle, om, ph, amp)
        sgiga.sgiga_set_rhs_builtin(Q.handle, "one")
        sgiga.sgiga_set_solver_options(Q.handle, use_graph=False)
        singles.append(Q)
    setup_s = time.perf_counter() - t0
    for Q in singles[:4]:                      # warm-up of the kernels
        sgiga.sgiga_solve(Q.handle, a.tol, 2000, check=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    its = 0
    for Q in singles:
        st, _ = sgiga.sgiga_solve(Q.handle, a.tol, 2000, check=False)
        its = max(its, st.iterations)
    e1.record(stream)
    torch.cuda.synchronize()
    acc = np.zeros(len(pts))
    for Q, c in zip(singles, coefs):
        uq = torch.zeros(len(pts), dtype=torch.float64, device="cuda")
        sgiga.sgiga_eval(Q.handle, pts, len(pts), uq)
        acc += c * uq.cpu().numpy()
        Q.close()
    out["fp64_fd_per_grid"] = {"ms": e0.elapsed_time(e1), "iterations": its, "plans": len(singles),
                               "setup_s": setup_s,
                               "rel_l2_vs_ref": float(np.linalg.norm(acc - ref) / np.linalg.norm(ref))}
    P, ps = plan("mixed", "learned")
    sgiga.sgiga_set_solver_options(P.handle, use_graph=True, inner_tol=a.inner_tol, inner_max=100)
    out["inner_tol"] = a.inner_tol
    st, rc, ms = timed_solve(P, a.tol, 50)    # warm-up, also the learned path before training (= FD)
    st, rc, ms = timed_solve(P, a.tol, 50)
    out["mixed_fd"] = {"ms": ms, "outer": st.iterations, "inner": st.inner_iterations, "rc": rc,
                       "rel_l2_vs_ref": float(np.linalg.norm(combined(P) - ref) / np.linalg.norm(ref))}
    if a.inner_tol_sweep:
        sweep = []
        for t in [float(v) for v in a.inner_tol_sweep.split(",")]:
            sgiga.sgiga_set_solver_options(P.handle, use_graph=True, inner_tol=t, inner_max=100)
            timed_solve(P, a.tol, 50)
            runs = [timed_solve(P, a.tol, 50) for _ in range(3)]
            st_t, rc_t, _ = runs[-1]
            sweep.append({"inner_tol": t, "ms": min(r[2] for r in runs), "outer": st_t.iterations,
                          "inner": st_t.inner_iterations, "rc": rc_t,
                          "rel_l2_vs_ref": float(np.linalg.norm(combined(P) - ref) / np.linalg.norm(ref))})
        out["mixed_fd_inner_tol_sweep"] = sweep
        sgiga.sgiga_set_solver_options(P.handle, use_graph=True, inner_tol=a.inner_tol, inner_max=100)
    sgiga.sgiga_net_init(P.handle, 11)
    tr = sgiga.sgiga_train_net(P.handle, target_pairs=a.pairs, max_iter_record=30, epochs=a.epochs, lr=a.lr,
                               seed=100, batch=a.batch)
    out["training"] = {"pairs": tr.pairs, "samples": tr.samples, "rhs": tr.rhs, "steps": tr.steps,
                       "loss_first_epoch": tr.loss_first_epoch, "loss_last_epoch": tr.loss_last_epoch,
                       "seconds": tr.seconds}
    sgiga.sgiga_set_rhs_builtin(P.handle, "one")
    timed_solve(P, a.tol, 50)
    st, rc, ms = timed_solve(P, a.tol, 50)
    out["mixed_learned"] = {"ms": ms, "outer": st.iterations, "inner": st.inner_iterations, "rc": rc,
                            "fallback": st.fallback,
                            "rel_l2_vs_ref": float(np.linalg.norm(combined(P) - ref) / np.linalg.norm(ref))}
    phi = torch.zeros(P.info.ndof, dtype=torch.float32, device="cuda")
    sgiga.sgiga_net_features(P.handle, phi)
    sgiga.sgiga_net_set_scaling(P.handle, torch.exp(-0.5 * phi).contiguous())
    timed_solve(P, a.tol, 50)
    st, rc, ms = timed_solve(P, a.tol, 50)
    out["mixed_scaled"] = {"ms": ms, "outer": st.iterations, "inner": st.inner_iterations, "rc": rc,
                           "fallback": st.fallback,
                           "rel_l2_vs_ref": float(np.linalg.norm(combined(P) - ref) / np.linalg.norm(ref))}
    P.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
