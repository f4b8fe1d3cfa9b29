"""Perturbed-cube geometry with a log-normal coefficient, and the learned
scaling of the preconditioner (features, network kernels and the training
loss against the oracle, training, the gain of the learned flexible CG over
FD alone, checkpoints)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import geometry, learned, net, problems  # noqa: E402
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


def test_coefficient_given_at_quadrature_points(sg):
    """A coefficient passed as values at the quadrature points (the oracle's
    a(x) at the plan's own quadrature coordinates) gives the operator of the
    oracle's assembly with that a, and the same operator as the plan's own
    Fourier-feature evaluation of it."""
    P, geom, a = _patch_plan(sg, 5)
    kn, cp = perturbed_cube_patch(1)
    with P, sg.Plan(3, 3, 5, domain="patch", patch=([3, 3, 3], kn, cp)) as Q:
        xq = np.zeros(3 * Q.info.nqp)
        sg.sgiga_qp_coords(Q.handle, xq)
        aq = a(xq.reshape(3, -1).T)
        sg.sgiga_set_coefficient_qp(Q.handle, aq)
        n = P.info.ndof
        x = torch.as_tensor(random_vector(n, 52), device="cuda")
        y1 = torch.zeros(n, dtype=torch.float64, device="cuda")
        y2 = torch.zeros_like(y1)
        sg.sgiga_apply(P.handle, x, y1)
        sg.sgiga_apply(Q.handle, x, y2)
        y1, y2, xh = y1.cpu().numpy(), y2.cpu().numpy(), x.cpu().numpy()
        assert _rel(y2, y1) < 1e-13
        for g in Q.grids[:: max(1, len(Q.grids) // 4)]:
            comp = Component(geom, tuple(g.levels), 3).assemble(diffusion=a)
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            assert _rel(y2[sl], comp.K @ xh[sl]) < 1e-12, tuple(g.levels)
        sg.sgiga_set_coefficient_qp(Q.handle, None)      # back to a = 1
        y3 = torch.zeros(n, dtype=torch.float64, device="cuda")
        sg.sgiga_apply(Q.handle, x, y3)
        g = Q.grids[0]
        comp = Component(geom, tuple(g.levels), 3).assemble()
        sl = slice(g.dof_off, g.dof_off + g.ndof)
        assert _rel(y3.cpu().numpy()[sl], comp.K @ xh[sl]) < 1e-12


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-12, 1e-10), ("mixed", 1e-9, 1e-8)])
def test_perturbed_cube_full_size_against_stored_oracle(sg, precision, tol, bound):
    """The learned-preconditioner workload at its full size (p = 3, w = 12, 199
    components, 3.03 M DoFs, 128 Fourier features), solved by the plan as the
    benchmark solves it: the combined values on the 17^3 lattice, and three
    components' values, against the oracle's assembly, direct solve and
    combination of all 199 components (tests/golden/perturbed_p3_w12.txt,
    written by tests/golden/make_golden.py from the oracle alone)."""
    from paper_1707_09598_gb300.inputs import eval_points
    gold = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "perturbed_p3_w12.txt"))
    kn, cp = perturbed_cube_patch(1)
    om, ph, amp = lognormal_features(2, nfeat=128)
    pts = eval_points(3, 16)
    npts = len(pts)
    sample = [(12, 1, 1), (1, 1, 12), (4, 5, 5)]
    with sg.Plan(3, 3, 12, domain="patch", patch=([3, 3, 3], kn, cp), precision=precision) as P:
        assert P.info.ngrids == 199 and P.info.ndof == 3026945
        sg.sgiga_set_coefficient(P.handle, om, ph, amp)
        sg.sgiga_set_rhs_builtin(P.handle, "one")
        st, _ = sg.sgiga_solve(P.handle, tol, 3000)
        uc = torch.zeros(P.info.ngrids * npts, dtype=torch.float64, device="cuda")
        sg.sgiga_eval(P.handle, torch.as_tensor(pts, device="cuda"), npts, uc)
        u = torch.zeros(npts, dtype=torch.float64, device="cuda")
        sg.sgiga_combine(P.handle, uc, npts, u)
        uc = uc.cpu().numpy().reshape(P.info.ngrids, npts)
        levels = [tuple(g.levels[:3]) for g in P.grids]
    err = _rel(u.cpu().numpy(), gold[:, 0])
    print("%s combined rel. L2 vs oracle %.2e" % (precision, err))
    assert err < bound, err
    for c, lv in enumerate(sample):
        assert _rel(uc[levels.index(lv)], gold[:, 1 + c]) < bound, lv


def _bf16(x):
    return torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def _bf16_t(x):
    return _bf16(np.asarray(x)).reshape(np.shape(x))


def _emulated_net(params, x, dy, d):
    """The network with the kernels' storage precision emulated around the
    oracle's FP64 convolutions: the 32-channel activations and their data
    gradients are stored as BF16 (rounded to nearest), everything else FP64."""
    T = 3 ** d
    (W1, b1), (W2, b2), (W3, b3) = net.unpack(params, d)
    A1 = _bf16_t(np.maximum(net.conv(x, W1, b1), 0.0))
    A2 = _bf16_t(np.maximum(net.conv(A1, W2, b2), 0.0))
    Y = net.conv(A2, W3, b3)[0]
    dY = dy[None]
    gW3 = net.conv_weight_grad(dY, A2, T)
    gb3 = dY.reshape(1, -1).sum(axis=1)
    dA2 = _bf16_t(net.conv_input_grad(dY, W3) * (A2 > 0))
    gW2 = net.conv_weight_grad(dA2, A1, T)
    gb2 = dA2.reshape(32, -1).sum(axis=1)
    dA1 = _bf16_t(net.conv_input_grad(dA2, W2) * (A1 > 0))
    gW1 = net.conv_weight_grad(dA1, x, T)
    gb1 = dA1.reshape(32, -1).sum(axis=1)
    return Y, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


@pytest.mark.parametrize("d,p,w", [(3, 2, 4), (2, 3, 6)])
def test_network_kernels_against_oracle(sg, d, p, w):
    """Forward and backward of the CUDA network (BF16 weights and 32-channel
    activations, FP32 accumulation; the 32 x 32 layer on the tensor cores)
    against the oracle's FP64 network with the same BF16 weights and the
    activations rounded to BF16 where the kernels store them. The bounds allow
    an activation that rounds the other way in one of the two (one BF16 unit,
    2^-8 relative, in a few entries) and FP32 accumulation order."""
    with sg.Plan(d, p, w, precision="mixed", precond="learned") as P:
        sg.sgiga_net_init(P.handle, 7)
        # the initial last layer is zero: give it random weights so that every
        # layer's forward and backward paths are exercised
        params = sg.sgiga_net_get_params(P.handle)
        T = 3 ** d
        nlast = 32 * T + 1
        params[-nlast:] = np.random.default_rng(8).uniform(-0.1, 0.1, nlast).astype(np.float32)
        sg.sgiga_net_set_params(P.handle, params)
        params = sg.sgiga_net_get_params(P.handle).astype(np.float64)
        npar = params.size
        # round weights (not biases) as the kernels do
        T = 3 ** d
        q, o = params.copy(), 0
        for ci, co in zip(net.CIN, net.COUT):
            q[o:o + co * ci * T] = _bf16(q[o:o + co * ci * T])
            o += co * ci * T + co
        assert o == npar
        n = P.info.ndof
        rng = np.random.default_rng(5)
        inp = rng.standard_normal((1, n)).astype(np.float32)
        dy = rng.standard_normal(n).astype(np.float32)
        out = torch.zeros(n, dtype=torch.float32, device="cuda")
        sg.sgiga_net_forward(P.handle, torch.as_tensor(inp, device="cuda"), out)
        grad = sg.sgiga_net_backward(P.handle, torch.as_tensor(inp, device="cuda"),
                                     torch.as_tensor(dy, device="cuda"))
        out = out.cpu().numpy()
        shapes = [tuple(g.n[:d]) for g in P.grids]
        xs = net.split_packed(inp.astype(np.float64), shapes)
        dys = net.split_packed(dy.astype(np.float64), shapes)
        res = [_emulated_net(q, x, d_, d) for x, d_ in zip(xs, dys)]
        ref = np.concatenate([r[0].ravel() for r in res])
        assert _rel(out, ref) < 2e-4, _rel(out, ref)
        gref = sum(r[1] for r in res)
        o = 0
        for ci, co in zip(net.CIN, net.COUT):
            for sl in (slice(o, o + co * ci * T), slice(o + co * ci * T, o + co * ci * T + co)):
                assert _rel(grad[sl], gref[sl]) < 1e-3, (ci, co, _rel(grad[sl], gref[sl]))
            o += co * ci * T + co


def test_features_against_oracle(sg):
    """phi = log c of every DoF (load vectors of tr(G) and d w on the device)
    against the oracle's definition on sampled components."""
    P, geom, a = _patch_plan(sg, 5, precision="mixed", precond="learned")
    with P:
        phi = np.zeros(P.info.ndof, dtype=np.float32)
        sg.sgiga_net_features(P.handle, phi)
        for g in P.grids[:: max(1, len(P.grids) // 5)]:
            comp = Component(geom, tuple(g.levels), 3)
            ref = np.log(learned.features(comp, diffusion=a))
            got = phi[g.dof_off:g.dof_off + g.ndof].astype(np.float64)
            assert np.max(np.abs(got - ref)) < 2e-6, tuple(g.levels)


def test_scaling_from_the_network_against_oracle(sg):
    """S on the device from the network output y = N(phi) and the feature
    phi: the oracle's S = exp(-phi / 2 + 4 tanh(y / 4)) of the same y and
    phi, to FP32 rounding; the untrained network (last layer zero) gives the
    network-free scaling c^(-1/2); after one set of random parameters the
    device S still follows the oracle's formula."""
    P, geom, a = _patch_plan(sg, 4, precision="mixed", precond="learned")
    with P:
        n = P.info.ndof
        sg.sgiga_net_init(P.handle, 3)
        phi = torch.zeros(n, dtype=torch.float32, device="cuda")
        sg.sgiga_net_features(P.handle, phi)
        y = torch.zeros(n, dtype=torch.float32, device="cuda")
        sg.sgiga_net_forward(P.handle, phi, y)
        S = torch.zeros(n, dtype=torch.float32, device="cuda")
        sg.sgiga_net_scaling(P.handle, S)
        ph, yh, Sh = (t.cpu().numpy().astype(np.float64) for t in (phi, y, S))
        ref = learned.scaling_from_output(yh, ph)
        assert np.max(np.abs(Sh / ref - 1.0)) < 2e-6
        assert np.max(np.abs(yh)) == 0.0 and np.max(np.abs(np.log(Sh) + 0.5 * ph)) < 1e-6
        params = sg.sgiga_net_get_params(P.handle)
        rng = np.random.default_rng(4)
        sg.sgiga_net_set_params(P.handle, (params + 0.05 * rng.standard_normal(params.size)).astype(np.float32))
        sg.sgiga_net_forward(P.handle, phi, y)
        sg.sgiga_net_scaling(P.handle, S)
        yh, Sh = (t.cpu().numpy().astype(np.float64) for t in (y, S))
    assert np.max(np.abs(yh)) > 1e-3
    assert np.max(np.abs(Sh / learned.scaling_from_output(yh, ph) - 1.0)) < 2e-6


@pytest.mark.parametrize("norm", ["euclidean", "energy"])
def test_loss_and_gradient_against_oracle(sg, norm):
    """Training loss of one sample and its gradient with respect to log S (FP32
    preconditioner and, for the energy norm, FP32 operator on the device)
    against the oracle's FP64 definition, at a random positive scaling."""
    P, geom, a = _patch_plan(sg, 4, precision="mixed", precond="learned")
    with P:
        n = P.info.ndof
        rng = np.random.default_rng(9)
        S = np.exp(0.3 * rng.standard_normal(n)).astype(np.float32)
        r = rng.standard_normal(n).astype(np.float32)
        e = rng.standard_normal(n).astype(np.float32)
        sg.sgiga_net_init(P.handle, 1)
        sg.sgiga_net_set_loss_norm(P.handle, norm)
        sg.sgiga_net_set_scaling(P.handle, S)
        grad = torch.zeros(n, dtype=torch.float32, device="cuda")
        loss = sg.sgiga_net_loss_grad(P.handle, torch.as_tensor(r, device="cuda"), torch.as_tensor(e, device="cuda"),
                                      grad)
        grids = [(tuple(g.levels[:3]), g.dof_off, g.ndof) for g in P.grids]
        Ks = None
        if norm == "energy":
            Ks = [Component(geom, lv, 3).assemble(diffusion=a).K for lv, _, _ in grids]
        Lref, gref = learned.packed_loss_grad(grids, 3, 2, S.astype(np.float64), r.astype(np.float64),
                                              e.astype(np.float64), Ks=Ks)
    assert abs(loss - Lref) < 1e-5 * Lref, (loss, Lref)
    assert _rel(grad.cpu().numpy(), gref) < 1e-4


def _timed_solve(sg, P, tol, reps=3):
    best, st = 1e30, None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        st, _ = sg.sgiga_solve(P.handle, tol, 30)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return st, best


def test_learned_scaling_gains_over_fd(sg, tmp_path):
    """What the trained network gains over the method without it: on a
    right-hand side held out of training (f = 1; the network is trained on
    pairs from seeded random right-hand sides), the mixed solve with the
    learned scaling needs fewer inner FP32 iterations and less time than the
    mixed solve with plain FD, both to relative residual 1e-8, and the two
    solutions agree. The network-free scaling S = c^(-1/2) is reported beside
    them. A checkpoint restores the same network."""
    P, geom, a = _patch_plan(sg, 7, precision="mixed", precond="learned")
    with P:
        sg.sgiga_set_solver_options(P.handle, use_graph=True, inner_tol=1e-3, inner_max=100)
        sg.sgiga_net_init(P.handle, 11)
        st = sg.sgiga_train_net(P.handle, target_pairs=3000, max_iter_record=25, epochs=8, lr=1e-3, seed=100,
                                batch=2)
        # training lowers the loss below that of its starting point (the
        # network-free scaling, which the untrained network reproduces) and far
        # below plain FD's
        assert st.pairs >= 3000 and st.loss_last_epoch < st.loss_initial and st.loss_last_epoch < 0.2 * st.loss_fd
        sg.sgiga_set_rhs_builtin(P.handle, "one")
        s_l, ms_l = _timed_solve(sg, P, 1e-8)
        assert s_l.fallback == 0
        u_l = np.zeros(P.info.ndof)
        sg.sgiga_get_solution(P.handle, u_l)
        path = str(tmp_path / "net.bin")
        sg.sgiga_net_save(P.handle, path)
        params = sg.sgiga_net_get_params(P.handle)
        # the same plan with a scaling that needs no network: S = c^(-1/2)
        phi = np.zeros(P.info.ndof, dtype=np.float32)
        sg.sgiga_net_features(P.handle, phi)
        sg.sgiga_net_set_scaling(P.handle, np.exp(-0.5 * phi).astype(np.float32))
        s_h, ms_h = _timed_solve(sg, P, 1e-8)
    P2, _, _ = _patch_plan(sg, 7, precision="mixed", precond="fd")
    with P2:
        sg.sgiga_set_solver_options(P2.handle, use_graph=True, inner_tol=1e-3, inner_max=100)
        sg.sgiga_set_rhs_builtin(P2.handle, "one")
        s_f, ms_f = _timed_solve(sg, P2, 1e-8)
        u_f = np.zeros(P2.info.ndof)
        sg.sgiga_get_solution(P2.handle, u_f)
    print("inner iterations / ms: learned %d / %.2f, c^-1/2 scaling %d / %.2f, FD %d / %.2f; loss FD %.4f, "
          "initial %.4f, epochs %.4f -> %.4f" % (s_l.inner_iterations, ms_l, s_h.inner_iterations, ms_h,
                                                s_f.inner_iterations, ms_f, st.loss_fd, st.loss_initial,
                                                st.loss_first_epoch, st.loss_last_epoch))
    assert _rel(u_l, u_f) < 1e-7
    assert s_l.inner_iterations < s_f.inner_iterations
    assert ms_l < ms_f
    P3, _, _ = _patch_plan(sg, 7, precision="mixed", precond="learned")
    with P3:
        sg.sgiga_net_load(P3.handle, path)
        np.testing.assert_array_equal(sg.sgiga_net_get_params(P3.handle), params)
