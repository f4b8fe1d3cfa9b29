"""Run one operation of the library repeatedly on a fixed workload (for timing
and profiler captures of a single kernel family).

  python -m paper_1707_09598_gb300.kernel_driver --op apply --reps 3 [--d 3 --p 3 --w 10]

Ops: apply (stiffness apply), apply_f32 / precond_f32 (the FP32 kernels of
the mixed-precision plan), precond (fast diagonalisation), rhs (load
vector), solve (batched PCG), eval (evaluation + combination on the 17^d
lattice), solve_scaled (the perturbed-cube mixed solve with the scaled
preconditioner S * FD(S * r), S = c^(-1/2), to 1e-8 with inner solves to
1e-3: the kernels of the learned + mixed solve without its training),
solve_mixed (the same mixed solve with the plain FD preconditioner).
--coef sets the log-normal coefficient (128 Fourier features, seed 2);
--host-loop runs the CG loops from the host (profilers then list every
kernel). Prints the mean CUDA-event time per repetition.
"""
import argparse
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1707_09598_gb300 import sgiga  # noqa: E402
from paper_1707_09598_gb300.inputs import eval_points, random_vector  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="apply", choices=["apply", "apply_f32", "precond", "precond_f32", "rhs", "solve",
                                                      "eval", "solve_scaled", "solve_mixed"])
    ap.add_argument("--coef", action="store_true")
    ap.add_argument("--inner-tol", type=float, default=1e-3, help="inner FP32 tolerance of the mixed solves")
    ap.add_argument("--host-loop", action="store_true")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--d", type=int, default=3)
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--w", type=int, default=10)
    ap.add_argument("--domain", default="unit", help="unit, annulus or perturbed (cube with a seeded cubic perturbation)")
    ap.add_argument("--tune", action="store_true", help="run the autotuner first")
    ap.add_argument("--fd-split", default=None, help="ks,grouped: the preconditioner's item depth and layout")
    ap.add_argument("--tiling", default=None,
                    help="budget,qpcap,nthreads,prefetch: set the operator's decomposition (after --tune, if given)")
    a = ap.parse_args()
    stream = torch.cuda.Stream()
    # torch's fills and reads of the buffers handed to the plan run on the
    # plan's stream, in order with its calls
    torch.cuda.set_stream(stream)
    f32 = a.op.endswith("_f32") or a.op in ("solve_scaled", "solve_mixed")
    kw = {}
    if a.domain == "perturbed":   # the learned-preconditioner geometry: seeded cubic perturbation, general metric
        from paper_1707_09598_gb300.inputs import perturbed_cube_patch
        kn, cp = perturbed_cube_patch(1)
        kw = dict(domain="patch", patch=([3, 3, 3], kn, cp))
    else:
        kw = dict(domain=a.domain)
    P = sgiga.Plan(a.d, a.p, a.w, stream=stream, precision="mixed" if f32 else "fp64",
                   precond="learned" if a.op == "solve_scaled" else "fd", **kw)
    if a.coef or a.op == "solve_scaled":
        from paper_1707_09598_gb300.inputs import lognormal_features
        om, ph, amp = lognormal_features(2, nfeat=128)
        sgiga.sgiga_set_coefficient(P.handle, om, ph, amp)
    if a.tune:
        t = sgiga.sgiga_autotune(P.handle, reps=3)
        print("autotune: best %d/%d/%d threads prefetch %d, %.4f ms; fd ks %d %s; candidates %s" % (
            t.budget[t.best], t.qpcap[t.best], t.nthreads[t.best], t.best_prefetch, t.best_ms, t.fd_ks[t.fd_best],
            "grouped" if t.fd_grouped[t.fd_best] else "per piece",
            " ".join("%d/%d/%d/%d:%.4f" % (t.budget[i], t.qpcap[i], t.nthreads[i], t.prefetch[i], t.ms[i])
                     for i in range(t.ncand))))
    if a.tiling:
        b, q, nt, pf = (int(v) for v in a.tiling.split(","))
        sgiga.sgiga_set_tiling(P.handle, b, q, nt, pf)
    if a.fd_split:
        ks, grp = (int(v) for v in a.fd_split.split(","))
        sgiga.sgiga_set_precond_split(P.handle, ks, bool(grp))
    if a.op in ("solve_scaled", "solve_mixed"):
        sgiga.sgiga_set_solver_options(P.handle, use_graph=not a.host_loop, inner_tol=a.inner_tol, inner_max=100)
    if a.op == "solve_scaled":
        phi = torch.zeros(P.info.ndof, dtype=torch.float32, device="cuda")
        sgiga.sgiga_net_features(P.handle, phi)
        sgiga.sgiga_net_set_scaling(P.handle, torch.exp(-0.5 * phi).contiguous())
    elif a.host_loop and a.op != "solve_mixed":
        sgiga.sgiga_set_solver_options(P.handle, use_graph=False)
    n = P.info.ndof
    x = torch.as_tensor(random_vector(n, 1), device="cuda")
    if f32:
        x = x.float()
    y = torch.zeros_like(x)
    src = {"unit": "sine", "annulus": "annulus_paper"}.get(a.domain, "one")
    sgiga.sgiga_set_rhs_builtin(P.handle, src)
    pts = torch.as_tensor(eval_points(a.d, 16), device="cuda")
    uc = torch.zeros(P.info.ngrids * len(pts), dtype=torch.float64, device="cuda")
    u = torch.zeros(len(pts), dtype=torch.float64, device="cuda")

    def op():
        if a.op == "apply":
            sgiga.sgiga_apply(P.handle, x, y)
        elif a.op == "apply_f32":
            sgiga.sgiga_apply_f32(P.handle, x, y)
        elif a.op == "precond_f32":
            sgiga.sgiga_precond_f32(P.handle, x, y)
        elif a.op == "precond":
            sgiga.sgiga_precond(P.handle, x, y)
        elif a.op == "rhs":
            sgiga.sgiga_set_rhs_builtin(P.handle, src)
        elif a.op == "solve":
            sgiga.sgiga_solve(P.handle, 1e-12, 50)
        elif a.op in ("solve_scaled", "solve_mixed"):
            sgiga.sgiga_solve(P.handle, 1e-8, 50)
        else:
            sgiga.sgiga_eval(P.handle, pts, len(pts), uc)
            sgiga.sgiga_combine(P.handle, uc, len(pts), u)

    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.reps):
        op()
    e1.record(stream)
    torch.cuda.synchronize()
    extra = ""
    if a.op in ("solve_scaled", "solve_mixed", "solve"):
        st, _ = sgiga.sgiga_solve(P.handle, 1e-8 if a.op != "solve" else 1e-12, 50, check=False)
        extra = " outer=%d inner=%d max_rel_residual=%.3g" % (st.iterations, st.inner_iterations, st.max_rel_residual)
    print("op=%s reps=%d mean_ms=%.4f ndof=%d nqp=%d ntiles=%d%s" %
          (a.op, a.reps, e0.elapsed_time(e1) / a.reps, n, P.info.nqp, P.info.ntiles, extra))
    P.close()


if __name__ == "__main__":
    main()
