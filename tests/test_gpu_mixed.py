"""Mixed-precision path (FP32 inner solve, FP64 iterative refinement) against the oracle.

The FP32 operator is checked against the oracle's assembled matrix at FP32
accuracy; the refined solutions against the oracle's direct solves at the
mixed-path target (relative L2 1e-8 of the combined solution), including the
full-size quarter-annulus workload (p = 2, 3, 4, w = 12) against stored
oracle values.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import combination, fd, geometry, problems  # noqa: E402
from oracle.galerkin import Component  # noqa: E402
from paper_1707_09598_gb300.inputs import eval_points, random_points, random_vector  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_09598_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_1707_09598_gb300 import sgiga
    return sgiga


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    # (domain, d, p, w, grading, gamma, source, oracle problem)
    ("unit", 3, 3, 6, "uniform", 1.0, "sine", "sine3"),
    ("annulus", 2, 3, 8, "uniform", 1.0, "annulus", "annulus_sinx"),
    ("annulus", 2, 2, 7, "radical", 2.0, "annulus_paper", "annulus_paper2"),
    ("unit", 2, 4, 8, "onesided", 2.0, "sine", "sine2"),
]


@pytest.mark.parametrize("case", CASES)
def test_fp32_apply(sg, case):
    domain, d, p, w, grading, gamma, src, pname = case
    with sg.Plan(d, p, w, domain=domain, grading=grading, gamma=gamma, precision="mixed") as P:
        n = P.info.ndof
        x = random_vector(n, seed=41)
        y = torch.zeros(n, dtype=torch.float32, device="cuda")
        sg.sgiga_apply_f32(P.handle, torch.as_tensor(x, dtype=torch.float32, device="cuda"), y)
        y = y.double().cpu().numpy()
        geom = geometry.make(domain, d)
        for g in P.grids[:: max(1, len(P.grids) // 5)]:
            comp = Component(geom, tuple(g.levels[:d]), p, None, grading, gamma).assemble()
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            ref = comp.K @ x[sl].astype(np.float32).astype(np.float64)
            # FP32 data and accumulation: error a few ulp of the operator's scale
            assert _rel(y[sl], ref) < 2e-5, (g.levels[:d], _rel(y[sl], ref))


@pytest.mark.parametrize("case", CASES[:2])
def test_fp32_preconditioner(sg, case):
    """FP32 fast diagonalisation against the oracle's FP64 one: the error is the
    FP32 rounding of the eigenvectors and of the mode products."""
    domain, d, p, w, grading, gamma, src, pname = case
    with sg.Plan(d, p, w, domain=domain, grading=grading, gamma=gamma, precision="mixed") as P:
        n = P.info.ndof
        rv = random_vector(n, seed=43)
        z = torch.zeros(n, dtype=torch.float32, device="cuda")
        sg.sgiga_precond_f32(P.handle, torch.as_tensor(rv, dtype=torch.float32, device="cuda"), z)
        z = z.double().cpu().numpy()
        geom = geometry.make(domain, d)
        for g in P.grids[:: max(1, len(P.grids) // 5)]:
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            ref = fd.fd_apply(tuple(g.levels[:d]), p, p - 1, rv[sl].astype(np.float32).astype(np.float64),
                              kind=grading, gamma=gamma, geom=geom)
            assert _rel(z[sl], ref) < 1e-4, (g.levels[:d], _rel(z[sl], ref))
        with pytest.raises(TypeError):
            sg.sgiga_precond_f32(P.handle, torch.zeros(n, dtype=torch.float64, device="cuda"), z)


@pytest.mark.parametrize("case", CASES)
def test_mixed_solve_against_oracle(sg, case):
    domain, d, p, w, grading, gamma, src, pname = case
    prob = problems.get(pname)
    geom = geometry.make(domain, d)
    pts = random_points(400, d, seed=42)
    with sg.Plan(d, p, w, domain=domain, grading=grading, gamma=gamma, precision="mixed") as P:
        sg.sgiga_set_rhs_builtin(P.handle, src)
        st, _ = sg.sgiga_solve(P.handle, 1e-11, 20)
        assert st.converged == P.info.ngrids
        assert st.max_rel_residual <= 1e-11
        u = np.zeros(P.info.ndof)
        sg.sgiga_get_solution(P.handle, u)
        uc = np.zeros(P.info.ngrids * len(pts))
        sg.sgiga_eval(P.handle, np.ascontiguousarray(pts), len(pts), uc)
        uu = np.zeros(len(pts))
        sg.sgiga_combine(P.handle, uc, len(pts), uu)
        vals, coeffs = [], []
        for g in P.grids:
            comp = Component(geom, tuple(g.levels[:d]), p, None, grading, gamma).assemble(f=prob.f)
            uo = comp.solve()
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            assert _rel(u[sl], uo) < 1e-8, (g.levels[:d], _rel(u[sl], uo))
            vals.append(comp.evaluate(uo, pts))
            coeffs.append(g.coeff)
        ref = combination.combine(np.stack(vals), np.array(coeffs, dtype=np.float64))
        assert _rel(uu, ref) < 1e-8


@pytest.mark.parametrize("p", [2, 3, 4])
def test_annulus_w12_full_size_mixed(sg, p):
    """Quarter annulus, u = x y (r^2-1)(r^2-4) sin x, p = 2, 3, 4, w = 12 (23
    components): mixed-precision solve refined to 1e-10, combined values on the
    65 x 65 lattice against stored oracle values (target 1e-8)."""
    gold = np.loadtxt(os.path.join(GOLD, "annulus_p%d_w12.txt" % p))
    pts = eval_points(2, 64)
    with sg.Plan(2, p, 12, domain="annulus", precision="mixed") as P:
        assert P.info.ngrids == 23
        sg.sgiga_set_rhs_builtin(P.handle, "annulus")
        st, _ = sg.sgiga_solve(P.handle, 1e-10, 30)
        assert st.converged == 23
        uc = np.zeros(P.info.ngrids * len(pts))
        sg.sgiga_eval(P.handle, np.ascontiguousarray(pts), len(pts), uc)
        uu = np.zeros(len(pts))
        sg.sgiga_combine(P.handle, uc, len(pts), uu)
        assert _rel(uu, gold[:, 0]) < 1e-8, _rel(uu, gold[:, 0])
        ucn = uc.reshape(P.info.ngrids, len(pts))
        levels = [tuple(g.levels[:2]) for g in P.grids]
        for col, sel in enumerate([(12, 1), (6, 6), (1, 12)]):
            assert _rel(ucn[levels.index(sel)], gold[:, 1 + col]) < 1e-8


@pytest.mark.gpu
def test_fp32_apply_under_every_tiling_and_prefetch(sg):
    """The FP32 3D operator at every decomposition the autotuner may choose
    (tile policy, 256 or 128 threads, L2 prefetch of the metric planes whole,
    capped or off) against the oracle's assembled K on sampled components of
    an annulus (general metric) plan with several tiles per component; the
    tilings only reorder FP32 sums (atomics), so the results agree to a few
    ulp. Out-of-range settings are argument errors."""
    d, p, w = 3, 3, 7
    with sg.Plan(d, p, w, domain="annulus", precision="mixed") as P:
        n = P.info.ndof
        x = random_vector(n, seed=47)
        xd = torch.as_tensor(x, dtype=torch.float32, device="cuda")
        geom = geometry.make("annulus", d)
        refs = {}
        for g in P.grids[:: max(1, len(P.grids) // 4)]:
            comp = Component(geom, tuple(g.levels[:d]), p, None, "uniform", 1.0).assemble()
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            refs[sl] = comp.K @ x[sl].astype(np.float32).astype(np.float64)
        first = None
        for budget, qpcap in ((48 * 1024, 4096), (110 * 1024, 16384), (200 * 1024, 32768)):
            for nth in (256, 128):
                for pf in (0, 1024, 16, -1):
                    sg.sgiga_set_tiling(P.handle, budget, qpcap, nth, pf)
                    y = torch.zeros(n, dtype=torch.float32, device="cuda")
                    sg.sgiga_apply_f32(P.handle, xd, y)
                    yh = y.double().cpu().numpy()
                    for sl, ref in refs.items():
                        assert _rel(yh[sl], ref) < 2e-5, (budget, qpcap, nth, pf, _rel(yh[sl], ref))
                    if first is None:
                        first = yh
                    assert _rel(yh, first) < 2e-6
        for bad in ((8 * 1024, 4096, 256, 0), (110 * 1024, 16, 256, 0), (110 * 1024, 4096, 64, 0),
                    (110 * 1024, 4096, 256, 24)):
            with pytest.raises(sg.SgigaError) as ei:
                sg.sgiga_set_tiling(P.handle, *bad)
            assert ei.value.code == sg.SGIGA_ERR_ARG


@pytest.mark.gpu
def test_autotune_chooses_the_solve_precision(sg):
    """On the unit cube the FD preconditioner is the exact inverse (K is a
    sum of Kronecker products of the same 1D pencils), so FP64 PCG converges
    in one or two iterations and beats the mixed solve's refinement steps: the
    autotuner switches the MIXED plan's solve to FP64, whose result then meets
    the FP64 bound against the oracle's sparse direct solves, with the FP64
    or the FP32 preconditioner, whichever the probe found faster."""
    with sg.Plan(3, 3, 6, domain="unit", precision="mixed") as P:
        sg.sgiga_set_rhs_builtin(P.handle, "sine")
        b0 = np.zeros(P.info.ndof)
        sg.sgiga_get_rhs(P.handle, b0)
        res = sg.sgiga_autotune(P.handle, reps=2)
        assert res.solve_precision == sg.PREC["fp64"], (res.solve_ms_fp64, res.solve_ms_fp64_fd32, res.solve_ms_mixed)
        chosen = res.solve_ms_fp64_fd32 if res.solve_fp32_precond else res.solve_ms_fp64
        assert 0 < chosen < res.solve_ms_mixed
        print("probe ms: fp64 %.3f, fp64 with fp32 FD %.3f, mixed %.3f; fp32 preconditioner %d"
              % (res.solve_ms_fp64, res.solve_ms_fp64_fd32, res.solve_ms_mixed, res.solve_fp32_precond))
        b1 = np.zeros(P.info.ndof)
        sg.sgiga_get_rhs(P.handle, b1)
        assert np.array_equal(b0, b1)          # the probe solves leave the load vector
        st, rc = sg.sgiga_solve(P.handle, 1e-12, 50)
        assert rc == sg.SGIGA_OK and st.inner_iterations == 0
        u = np.zeros(P.info.ndof)
        sg.sgiga_get_solution(P.handle, u)
        geom = geometry.make("unit", 3)
        f = problems.get("sine3").f
        for g in P.grids[:: max(1, len(P.grids) // 4)]:
            comp = Component(geom, tuple(g.levels[:3]), 3).assemble(f=f)
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            assert _rel(u[sl], comp.solve()) < 1e-10
