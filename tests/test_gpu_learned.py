"""Perturbed-cube geometry with a log-normal coefficient, and the learned
correction network (kernels against the oracle network, training, flexible CG
with the learned preconditioner against FD alone, checkpoints)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import geometry, net, problems  # noqa: E402
from oracle.galerkin import Component  # noqa: E402
from paper_1707_09598_gb300.inputs import (lognormal_features, perturbed_cube_patch,  # noqa: E402
                                           random_points, random_vector)


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
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _patch_plan(sg, w, p=3, precision="fp64", precond="fd", nfeat=64):
    kn, cp = perturbed_cube_patch(1)
    P = sg.Plan(3, p, w, domain="patch", patch=([3, 3, 3], kn, cp), precision=precision, precond=precond)
    om, ph, amp = lognormal_features(2, nfeat=nfeat)
    sg.sgiga_set_coefficient(P.handle, om, ph, amp)
    geom = geometry.BSplinePatch([3, 3, 3], kn, cp)
    return P, geom, geometry.lognormal_coefficient(om, ph, amp)


def test_perturbed_cube_with_coefficient(sg):
    """Operator, load vector (f = 1) and FP64 solve on the seeded perturbed cube
    with the log-normal coefficient, against the oracle's assembly and LU."""
    P, geom, a = _patch_plan(sg, 5)
    with P:
        n = P.info.ndof
        x = random_vector(n, 51)
        y = torch.zeros(n, dtype=torch.float64, device="cuda")
        sg.sgiga_apply(P.handle, torch.as_tensor(x, device="cuda"), y)
        y = y.cpu().numpy()
        sg.sgiga_set_rhs_builtin(P.handle, "one")
        st, _ = sg.sgiga_solve(P.handle, 1e-12, 400)
        u = np.zeros(n)
        sg.sgiga_get_solution(P.handle, u)
        prob = problems.get("one3")
        for g in P.grids[:: max(1, len(P.grids) // 6)]:
            comp = Component(geom, tuple(g.levels), 3).assemble(f=prob.f, diffusion=a)
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            assert _rel(y[sl], comp.K @ x[sl]) < 1e-12, tuple(g.levels)
            assert _rel(u[sl], comp.solve()) < 1e-9, tuple(g.levels)


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-12, 1e-9), ("mixed", 1e-10, 1e-7)])
def test_perturbed_cube_full_size_sampled_components(sg, precision, tol, bound):
    """The learned-preconditioner workload at its full size (p = 3, w = 12, 199
    components, 3.03 M DoFs, 128 Fourier features), solved by the plan as the
    report solves it. Sampled components (the longest in directions 0 and 2 at
    |i| = 12, and the cube-shaped one) are compared, by their values on the
    17^3 lattice, with the oracle's assembly and direct solve of the same
    component."""
    from paper_1707_09598_gb300.inputs import eval_points
    kn, cp = perturbed_cube_patch(1)
    om, ph, amp = lognormal_features(2, nfeat=128)
    geom = geometry.BSplinePatch([3, 3, 3], kn, cp)
    a = geometry.lognormal_coefficient(om, ph, amp)
    pts = eval_points(3, 16)
    npts = len(pts)
    sample = [(10, 1, 1), (1, 1, 10), (4, 4, 4)]
    with sg.Plan(3, 3, 12, domain="patch", patch=([3, 3, 3], kn, cp), precision=precision) as P:
        assert P.info.ngrids == 199 and P.info.ndof == 3026945
        sg.sgiga_set_coefficient(P.handle, om, ph, amp)
        sg.sgiga_set_rhs_builtin(P.handle, "one")
        st, _ = sg.sgiga_solve(P.handle, tol, 3000)
        uc = torch.zeros(P.info.ngrids * npts, dtype=torch.float64, device="cuda")
        sg.sgiga_eval(P.handle, torch.as_tensor(pts, device="cuda"), npts, uc)
        uc = uc.cpu().numpy().reshape(P.info.ngrids, npts)
        levels = [tuple(g.levels[:3]) for g in P.grids]
    prob = problems.get("one3")
    for lv in sample:
        comp = Component(geom, lv, 3).assemble(f=prob.f, diffusion=a)
        ref = comp.evaluate(comp.solve(), pts)
        assert _rel(uc[levels.index(lv)], ref) < bound, (lv, _rel(uc[levels.index(lv)], ref))


def _bf16(x):
    return torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def test_network_kernels_against_oracle(sg):
    """Forward and backward of the CUDA network (BF16 weights, FP32 accumulation)
    against the oracle's FP64 network with the same BF16-rounded weights."""
    with sg.Plan(3, 2, 4, precision="mixed", precond="learned") as P:
        sg.sgiga_net_init(P.handle, 7)
        params = sg.sgiga_net_get_params(P.handle).astype(np.float64)
        npar = params.size
        # round weights (not biases) as the kernels do
        T = 27
        q, o = params.copy(), 0
        for ci, co in zip(net.CIN, net.COUT):
            q[o:o + co * ci * T] = _bf16(q[o:o + co * ci * T])
            o += co * ci * T + co
        assert o == npar
        n = P.info.ndof
        rng = np.random.default_rng(5)
        inp = rng.standard_normal((2, n)).astype(np.float32)
        dy = rng.standard_normal(n).astype(np.float32)
        out = torch.zeros(n, dtype=torch.float32, device="cuda")
        sg.sgiga_net_forward(P.handle, torch.as_tensor(inp, device="cuda"), out)
        grad = sg.sgiga_net_backward(P.handle, torch.as_tensor(inp, device="cuda"),
                                     torch.as_tensor(dy, device="cuda"))
        out = out.cpu().numpy()
        shapes = [tuple(g.n[:3]) for g in P.grids]
        xs = net.split_packed(inp.astype(np.float64), shapes)
        dys = net.split_packed(dy.astype(np.float64), shapes)
        ref = np.concatenate([net.forward(q, x)[0].ravel() for x in xs])
        assert _rel(out, ref) < 2e-5
        gref = sum(net.backward(q, x, d_) for x, d_ in zip(xs, dys))
        o = 0
        for ci, co in zip(net.CIN, net.COUT):
            for sl in (slice(o, o + co * ci * T), slice(o + co * ci * T, o + co * ci * T + co)):
                assert _rel(grad[sl], gref[sl]) < 1e-4
            o += co * ci * T + co


def test_training_and_learned_flexible_cg(sg, tmp_path):
    """Train on the plan's own CG pairs; the learned flexible CG (inner FP32 solve
    of the mixed path) converges to the same solution as FD alone; report the
    inner iterations of both; a checkpoint restores the same network."""
    P, geom, a = _patch_plan(sg, 6, precision="mixed", precond="learned")
    with P:
        sg.sgiga_net_init(P.handle, 11)
        st = sg.sgiga_train_net(P.handle, target_pairs=4000, max_iter_record=25, epochs=4, lr=2e-3, seed=100)
        assert st.pairs >= 4000 and st.loss_last_epoch < st.loss_first_epoch
        sg.sgiga_set_rhs_builtin(P.handle, "one")
        s_l, _ = sg.sgiga_solve(P.handle, 1e-10, 30)
        u_l = np.zeros(P.info.ndof)
        sg.sgiga_get_solution(P.handle, u_l)
        path = str(tmp_path / "net.bin")
        sg.sgiga_net_save(P.handle, path)
        params = sg.sgiga_net_get_params(P.handle)
    P2, _, _ = _patch_plan(sg, 6, precision="mixed", precond="fd")
    with P2:
        sg.sgiga_set_rhs_builtin(P2.handle, "one")
        s_f, _ = sg.sgiga_solve(P2.handle, 1e-10, 30)
        u_f = np.zeros(P2.info.ndof)
        sg.sgiga_get_solution(P2.handle, u_f)
    assert _rel(u_l, u_f) < 1e-8
    print("inner iterations: learned %d, FD %d; loss %.3f -> %.3f"
          % (s_l.inner_iterations, s_f.inner_iterations, st.loss_first_epoch, st.loss_last_epoch))
    P3, _, _ = _patch_plan(sg, 6, precision="mixed", precond="learned")
    with P3:
        sg.sgiga_net_load(P3.handle, path)
        np.testing.assert_array_equal(sg.sgiga_net_get_params(P3.handle), params)
