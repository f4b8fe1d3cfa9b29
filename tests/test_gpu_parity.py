"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Kernel by kernel (basis tables, geometry coefficients, operator apply, load
vector, preconditioner, solve, evaluation, combination) on seeded inputs, at
sizes the oracle finishes in seconds and that span several tiles, plus the
full-size 3D cube workload against stored oracle values.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import combination, driver, fd, geometry, problems  # noqa: E402
from oracle.galerkin import Component, Space1D  # noqa: E402
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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _geom(domain, d):
    return geometry.make(domain, d)


CASES = [
    # (domain, d, p, r, w, grading, gamma, min_level)
    ("unit", 2, 2, 1, 6, "uniform", 1.0, 1),
    ("unit", 2, 3, 0, 5, "uniform", 1.0, 1),
    ("unit", 2, 4, 3, 9, "radical", 3.0, 1),
    ("annulus", 2, 3, 2, 7, "uniform", 1.0, 1),
    ("annulus", 2, 2, 1, 6, "radical", 2.0, 1),
    ("unit", 3, 3, 2, 5, "uniform", 1.0, 1),
    ("unit", 3, 2, 1, 4, "onesided", 2.0, 1),
    ("unit", 3, 2, 0, 3, "uniform", 1.0, 1),
    ("annulus", 3, 2, 1, 4, "uniform", 1.0, 1),
    ("unit", 2, 2, 1, 2, "uniform", 1.0, 0),
]


def _plan(sg, case, precond="fd"):
    domain, d, p, r, w, grading, gamma, mn = case
    return sg.Plan(d, p, w, domain=domain, continuity=r, min_level=mn, grading=grading, gamma=gamma,
                   precond=precond)


def _component(case, g):
    domain, d, p, r, w, grading, gamma, mn = case
    lv = tuple(g.levels[:d])
    return Component(_geom(domain, d), lv, p, r, grading, gamma)


@pytest.mark.parametrize("case", CASES[:5] + CASES[5:7])
def test_basis_tables(sg, case):
    domain, d, p, r, w, grading, gamma, mn = case
    with _plan(sg, case) as P:
        geom = _geom(domain, d)
        seen = set()
        for g in P.grids:
            for k in range(d):
                key = (k, g.levels[k])
                if key in seen:
                    continue
                seen.add(key)
                xi, wq, R, dR, first = sg.sgiga_basis_table(P.handle, k, g.levels[k])
                s = Space1D(g.levels[k], p, r, geom, k, grading, gamma)
                np.testing.assert_allclose(xi, s.xi.reshape(-1), rtol=0, atol=4e-16)
                np.testing.assert_allclose(wq, s.w.reshape(-1), rtol=1e-14, atol=0)
                np.testing.assert_array_equal(first, s.first)
                np.testing.assert_allclose(R, s.R, rtol=0, atol=1e-14)
                scale = max(1.0, np.abs(s.dR).max())
                np.testing.assert_allclose(dR, s.dR, rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("case", [CASES[3], CASES[4], CASES[8], CASES[0]])
def test_geometry_coefficients(sg, case):
    domain, d, p, r, w, grading, gamma, mn = case
    with _plan(sg, case) as P:
        geom = _geom(domain, d)
        for gi in range(0, P.info.ngrids, max(1, P.info.ngrids // 4)):
            g = P.grids[gi]
            G, mw = sg.sgiga_geometry_coeffs(P.handle, gi)
            comp = _component(case, g)
            # oracle qp lattice in natural order (direction 1 fastest)
            xs = [comp.spaces[k].xi.reshape(-1) for k in range(d)]
            ws = [comp.spaces[k].w.reshape(-1) for k in range(d)]
            mesh = np.meshgrid(*xs[::-1], indexing="ij")
            wmesh = np.meshgrid(*ws[::-1], indexing="ij")
            pts = np.stack([m.reshape(-1) for m in mesh[::-1]], 1)
            wt = np.prod(np.stack([m.reshape(-1) for m in wmesh], 1), axis=1)
            J = geom.jacobian(pts)
            det = np.linalg.det(J)
            Gm = np.linalg.inv(np.einsum("nik,nil->nkl", J, J)) * (wt * np.abs(det))[:, None, None]
            c = 0
            for k in range(d):
                for l in range(k, d):
                    np.testing.assert_allclose(G[c], Gm[:, k, l], rtol=1e-12, atol=1e-15 * np.abs(Gm).max())
                    c += 1
            np.testing.assert_allclose(mw, wt * np.abs(det), rtol=1e-13)


@pytest.mark.parametrize("case", CASES)
def test_apply_and_rhs(sg, case):
    """y = K x for every component against the oracle's assembled K (seeded x),
    and the load vector of a built-in source against the oracle's."""
    domain, d, p, r, w, grading, gamma, mn = case
    src = {"unit": "sine", "annulus": "annulus_paper"}[domain]
    prob = problems.get({("unit", 2): "sine2", ("unit", 3): "sine3", ("annulus", 2): "annulus_paper2",
                         ("annulus", 3): "annulus_paper3"}[(domain, d)])
    with _plan(sg, case) as P:
        n = P.info.ndof
        x = random_vector(n, seed=11)
        y = torch.zeros(n, dtype=torch.float64, device="cuda")
        sg.sgiga_apply(P.handle, _dev(x), y)
        sg.sgiga_set_rhs_builtin(P.handle, src)
        b = torch.zeros(n, dtype=torch.float64, device="cuda")
        sg.sgiga_get_rhs(P.handle, b)
        y, b = y.cpu().numpy(), b.cpu().numpy()
        for g in P.grids:
            if g.ndof == 0:
                continue
            comp = _component(case, g).assemble(f=prob.f)
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            ref = comp.K @ x[sl]
            assert _rel(y[sl], ref) < 1e-13, (g.levels[:d], _rel(y[sl], ref))
            assert _rel(b[sl], comp.b) < 1e-13, (g.levels[:d], _rel(b[sl], comp.b))


MULTI_TILE = [("unit", 2, 3, 2, 10, "uniform", 1.0, 1), ("annulus", 2, 2, 1, 10, "radical", 3.0, 1),
              ("unit", 2, 2, 0, 9, "uniform", 1.0, 1), ("unit", 3, 3, 2, 8, "uniform", 1.0, 1),
              ("annulus", 3, 2, 1, 7, "uniform", 1.0, 1)]


@pytest.mark.parametrize("case", MULTI_TILE)
def test_apply_multi_tile(sg, case):
    """Operator apply and load vector on components that span many tiles
    (sampled components for the 3D cases)."""
    domain, d, p, r, w, grading, gamma, mn = case
    src = {"unit": "sine", "annulus": "annulus_paper"}[domain]
    prob = problems.get({("unit", 2): "sine2", ("unit", 3): "sine3", ("annulus", 2): "annulus_paper2",
                         ("annulus", 3): "annulus_paper3"}[(domain, d)])
    with _plan(sg, case) as P:
        n = P.info.ndof
        x = random_vector(n, seed=21)
        y = torch.zeros(n, dtype=torch.float64, device="cuda")
        sg.sgiga_apply(P.handle, _dev(x), y)
        sg.sgiga_set_rhs_builtin(P.handle, src)
        b = torch.zeros(n, dtype=torch.float64, device="cuda")
        sg.sgiga_get_rhs(P.handle, b)
        y, b = y.cpu().numpy(), b.cpu().numpy()
        grids = list(P.grids)
        if d == 3:
            multi = [g for g in grids if g.ntiles > 1]
            grids = [multi[0], multi[len(multi) // 2], multi[-1], grids[0]]
        assert sum(g.ntiles >= 4 for g in grids) >= 2
        for g in grids:
            comp = _component(case, g).assemble(f=prob.f)
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            assert _rel(y[sl], comp.K @ x[sl]) < 1e-13, (g.levels[:d], g.ntiles)
            assert _rel(b[sl], comp.b) < 1e-13, (g.levels[:d], g.ntiles)


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[3], CASES[5], CASES[7], CASES[8]])
def test_preconditioner(sg, case):
    domain, d, p, r, w, grading, gamma, mn = case
    with _plan(sg, case) as P:
        n = P.info.ndof
        rv = random_vector(n, seed=12)
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        sg.sgiga_precond(P.handle, _dev(rv), z)
        z = z.cpu().numpy()
        geom = _geom(domain, d)
        for g in P.grids:
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            ref = fd.fd_apply(tuple(g.levels[:d]), p, r, rv[sl], kind=grading, gamma=gamma, geom=geom)
            assert _rel(z[sl], ref) < 1e-11, (g.levels[:d], _rel(z[sl], ref))


@pytest.mark.parametrize("grouped", [False, True])
@pytest.mark.parametrize("ks", [16, 32, 64, 128, 256])
def test_preconditioner_split_depths(sg, ks, grouped):
    """Long 1D contractions (per-piece ROWS and TILE items, or level-grouped
    GEMM tiles, split into ks-deep partial sums added atomically) give the
    oracle's FD result at every depth."""
    case = ("unit", 3, 3, 2, 10, "uniform", 1.0, 1)
    with _plan(sg, case) as P:
        sg.sgiga_set_precond_split(P.handle, ks, grouped)
        n = P.info.ndof
        rv = random_vector(n, seed=13)
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        sg.sgiga_precond(P.handle, _dev(rv), z)
        z = z.cpu().numpy()
        # components whose long direction is split: ROWS (few columns) and TILE (>= 64 columns)
        pick = [(8, 1, 1), (1, 9, 1), (6, 4, 2), (2, 3, 7), (7, 2, 2), (4, 4, 4)]
        seen = 0
        for g in P.grids:
            lv = tuple(g.levels[:3])
            if lv not in pick:
                continue
            seen += 1
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            ref = fd.fd_apply(lv, 3, 2, rv[sl], kind="uniform", gamma=1.0, geom=None)
            assert _rel(z[sl], ref) < 1e-11, (lv, ks, _rel(z[sl], ref))
        assert seen == len(pick)
    with _plan(sg, case) as P:
        with pytest.raises(sg.SgigaError):
            sg.sgiga_set_precond_split(P.handle, 24)


# (domain, d, p, w, grading, gamma, direction, levels): the 1D eigenproblems
# the plan solves on the device (bisection on the banded pencil, inverse
# iteration), against the oracle's dense FP64 generalised eigensolver
EIG_CASES = [
    ("unit", 3, 3, 10, "uniform", 1.0, 0, (1, 4, 10)),
    ("unit", 2, 3, 12, "uniform", 1.0, 0, (12,)),
    ("unit", 2, 1, 8, "uniform", 1.0, 1, (3, 8)),
    ("unit", 2, 2, 9, "radical", 3.0, 0, (2, 6, 9)),
    ("unit", 2, 4, 8, "onesided", 3.0, 1, (5, 8)),
    ("annulus", 2, 2, 9, "uniform", 1.0, 1, (2, 9)),
]


@pytest.mark.parametrize("case", EIG_CASES)
def test_eigenpairs(sg, case):
    domain, d, p, w, grading, gamma, k, levels = case
    from oracle.galerkin import stiffness_1d
    import scipy.sparse as spm
    geom = geometry.make(domain, d) if domain != "unit" else None
    with sg.Plan(d, p, w, domain=domain, grading=grading, gamma=gamma) as P:
        for lv in levels:
            K, M = stiffness_1d(lv, p, p - 1, grading, gamma, geom, k)
            n = K.shape[0]
            U, lam = sg.sgiga_fd_eigen(P.handle, k, lv, n)
            assert np.all(np.diff(lam) >= 0) and lam[0] > 0
            Ks, Ms = spm.csr_matrix(K), spm.csr_matrix(M)
            MU = Ms @ U
            # inverse iteration leaves an M-orthogonality error of order eps ||K|| / gap
            assert np.abs(U.T @ MU - np.eye(n)).max() < 1e-9, lv
            assert np.abs(Ks @ U - MU * lam[None, :]).max() < 1e-10 * lam.max(), lv
            if grading == "uniform" and n <= 1100:
                lam_o = fd.eig_1d(lv, p, p - 1, grading, gamma, geom, k)[0]
                np.testing.assert_allclose(lam, lam_o, rtol=1e-9)
            if grading != "uniform":
                # graded meshes: M is ill-conditioned and the dense FP64 solver
                # (Cholesky of M) loses digits; the oracle's extended-precision
                # bisection on the inertia of K - s M does not
                js = sorted({j for j in (0, 4, n // 2, n - 1) if j < n})
                ref = fd.sturm_eigenvalues(K, M, js)
                np.testing.assert_allclose(lam[js], ref, rtol=1e-10)


@pytest.mark.parametrize("case", CASES)
def test_solve_eval_combine(sg, case):
    """Batched PCG solution of every component against the oracle's direct
    solve, then evaluation and the combination at parametric points."""
    domain, d, p, r, w, grading, gamma, mn = case
    src = {"unit": "sine", "annulus": "annulus_paper"}[domain]
    pname = {("unit", 2): "sine2", ("unit", 3): "sine3", ("annulus", 2): "annulus_paper2",
             ("annulus", 3): "annulus_paper3"}[(domain, d)]
    prob = problems.get(pname)
    with _plan(sg, case) as P:
        sg.sgiga_set_rhs_builtin(P.handle, src)
        st, _ = sg.sgiga_solve(P.handle, 1e-13, 200)
        u = torch.zeros(P.info.ndof, dtype=torch.float64, device="cuda")
        sg.sgiga_get_solution(P.handle, u)
        u = u.cpu().numpy()
        pts = random_points(300, d, seed=13)
        pts[:8] = np.array([[0.0] * d, [1.0] * d, [0.5] * d, [1.0] + [0.0] * (d - 1),
                            [0.25] * d, [0.75] * d, [0.0] + [1.0] * (d - 1), [1.0 / 3] * d])
        uc = torch.zeros(P.info.ngrids * len(pts), dtype=torch.float64, device="cuda")
        sg.sgiga_eval(P.handle, _dev(pts), len(pts), uc)
        uu = torch.zeros(len(pts), dtype=torch.float64, device="cuda")
        sg.sgiga_combine(P.handle, uc, len(pts), uu)
        uc = uc.cpu().numpy().reshape(P.info.ngrids, len(pts))
        vals, coeffs = [], []
        for gi, g in enumerate(P.grids):
            comp = _component(case, g).assemble(f=prob.f)
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            uo = comp.solve() if g.ndof else np.zeros(0)
            if g.ndof:
                assert _rel(u[sl], uo) < 1e-10, (g.levels[:d], _rel(u[sl], uo))
            vo = comp.evaluate(uo, pts)
            np.testing.assert_allclose(uc[gi], vo, rtol=0, atol=1e-10 * max(1.0, np.abs(vo).max()))
            vals.append(vo)
            coeffs.append(g.coeff)
        ref = combination.combine(np.stack(vals), np.array(coeffs, dtype=np.float64))
        assert _rel(uu.cpu().numpy(), ref) < 1e-10


def test_combine_kernel_against_oracle_sum(sg):
    """The FP64 compensated combination on seeded values of widely varying size."""
    case = CASES[5]
    with _plan(sg, case) as P:
        ng, npts = P.info.ngrids, 1000
        rng = np.random.default_rng(14)
        v = rng.standard_normal((ng, npts)) * 10.0 ** rng.integers(-6, 6, (ng, npts))
        out = torch.zeros(npts, dtype=torch.float64, device="cuda")
        sg.sgiga_combine(P.handle, _dev(v.reshape(-1)), npts, out)
        ref = combination.combine(v, np.array([g.coeff for g in P.grids], dtype=np.float64))
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-15, atol=1e-15 * np.abs(v).max())
        # host buffers go through the same entry point
        host = np.zeros(npts)
        sg.sgiga_combine(P.handle, np.ascontiguousarray(v.reshape(-1)), npts, host)
        np.testing.assert_array_equal(host, out.cpu().numpy())


def test_square_p2_w6_full_lattice(sg):
    """2D unit square, p = 2, C^1, w = 6, combined on the 257 x 257 lattice."""
    case = ("unit", 2, 2, 1, 6, "uniform", 1.0, 1)
    from oracle import driver
    with _plan(sg, case) as P:
        sg.sgiga_set_rhs_builtin(P.handle, "sine")
        sg.sgiga_solve(P.handle, 1e-14, 100)
        pts = eval_points(2, 256)
        uc = torch.zeros(P.info.ngrids * len(pts), dtype=torch.float64, device="cuda")
        sg.sgiga_eval(P.handle, _dev(pts), len(pts), uc)
        uu = np.zeros(len(pts))
        sg.sgiga_combine(P.handle, uc, len(pts), uu)
    res = driver.solve_components("unit", 2, 2, 6, "sine2")
    ref, _ = driver.combined_at(res, pts)
    assert _rel(uu, ref) < 1e-10


def test_cube_p3_w10_full_size(sg):
    """3D unit cube, p = 3, C^2, w = 10 (136 components): combined values and
    selected components at the 17^3 lattice against stored oracle values, and
    sampled components' coefficients against the oracle's direct solve."""
    gold = np.loadtxt(os.path.join(GOLD, "cube_p3_w10.txt"))
    case = ("unit", 3, 3, 2, 10, "uniform", 1.0, 1)
    pts = eval_points(3, 16)
    with _plan(sg, case) as P:
        assert P.info.ngrids == 136 and P.info.ndof == 557030
        assert P.info.diag_metric == 1      # identity map: the cross terms are skipped
        sg.sgiga_set_rhs_builtin(P.handle, "sine")
        st, _ = sg.sgiga_solve(P.handle, 1e-12, 100)
        assert st.converged == 136
        uc = torch.zeros(P.info.ngrids * len(pts), dtype=torch.float64, device="cuda")
        sg.sgiga_eval(P.handle, _dev(pts), len(pts), uc)
        uu = np.zeros(len(pts))
        sg.sgiga_combine(P.handle, uc, len(pts), uu)
        assert _rel(uu, gold[:, 0]) < 1e-10, _rel(uu, gold[:, 0])
        ucn = uc.cpu().numpy().reshape(P.info.ngrids, len(pts))
        levels = [tuple(g.levels[:3]) for g in P.grids]
        for col, sel in enumerate([(10, 1, 1), (4, 4, 4), (1, 5, 4), (3, 3, 4)]):
            gi = levels.index(sel)
            assert _rel(ucn[gi], gold[:, 1 + col]) < 1e-10
        u = torch.zeros(P.info.ndof, dtype=torch.float64, device="cuda")
        sg.sgiga_get_solution(P.handle, u)
        u = u.cpu().numpy()
        prob = problems.get("sine3")
        # coefficients: forward error <= cond(K) x relative residual; at the solve's
        # 1e-12 residual the longest components (n = 1025 x 3 x 3) sit near 1e-10
        # against the direct solve, which carries a rounding error of the same kind
        for sel in [(1, 1, 10), (2, 6, 3)]:
            g = P.grids[levels.index(sel)]
            comp = Component(geometry.UnitCube(3), sel, 3).assemble(f=prob.f)
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            assert _rel(u[sl], comp.solve()) < 1e-9


def test_host_buffers_and_user_rhs(sg):
    """f given at the quadrature points from host memory equals the built-in source."""
    case = CASES[3]
    with _plan(sg, case) as P:
        d = 2
        xq = torch.zeros(d * P.info.nqp, dtype=torch.float64, device="cuda")
        sg.sgiga_qp_coords(P.handle, xq)
        xq = xq.cpu().numpy().reshape(d, -1).T
        f = problems.get("annulus_paper2").f(xq)
        fq = np.zeros(P.info.nqp)
        sg.sgiga_source_at_qp(P.handle, "annulus_paper", fq)
        np.testing.assert_allclose(fq, f, rtol=1e-12, atol=1e-12 * np.abs(f).max())
        sg.sgiga_set_rhs(P.handle, np.ascontiguousarray(f))
        b1 = np.zeros(P.info.ndof)
        sg.sgiga_get_rhs(P.handle, b1)
        sg.sgiga_set_rhs_builtin(P.handle, "annulus_paper")
        b2 = np.zeros(P.info.ndof)
        sg.sgiga_get_rhs(P.handle, b2)
        assert _rel(b1, b2) < 1e-13


def test_pinned_host_rhs_is_read_in_place(sg):
    """f in page-locked host memory (read by the density kernel over the host
    link), in pageable host memory (staged) and on the device give the same
    load vector, bit for bit; the pinned buffer may be reused on return."""
    case = CASES[3]
    with _plan(sg, case) as P:
        fd = torch.zeros(P.info.nqp, dtype=torch.float64, device="cuda")
        sg.sgiga_source_at_qp(P.handle, "annulus_paper", fd)
        fd = fd * 1.5 + 0.25
        fpin = fd.cpu().pin_memory()
        fpage = fd.cpu().numpy().copy()
        out = []
        for f in (fd, fpin, fpage):
            sg.sgiga_set_rhs(P.handle, f)
            b = np.zeros(P.info.ndof)
            sg.sgiga_get_rhs(P.handle, b)
            out.append(b)
        fpin.zero_()                      # read in full before the call returned
        assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
        assert np.abs(out[0]).max() > 0


def test_errors_are_reported_not_crashes(sg):
    with pytest.raises(sg.SgigaError):
        sg.sgiga_plan(4, 2, 6)
    with pytest.raises(sg.SgigaError):
        sg.sgiga_plan(2, 2, 6, continuity=5)
    with _plan(sg, CASES[0]) as P:
        with pytest.raises(sg.SgigaError):
            sg.sgiga_eval(P.handle, _dev(np.array([[1.5, 0.2]])), 1,
                          torch.zeros(P.info.ngrids, dtype=torch.float64, device="cuda"))
        sg.sgiga_set_rhs_builtin(P.handle, "sine")
        st, rc = sg.sgiga_solve(P.handle, 1e-300, 1, check=False)
        assert rc == sg.SGIGA_ERR_NOT_CONVERGED


@pytest.mark.parametrize("case,precision", [(CASES[5], "fp64"), (CASES[3], "mixed")])
def test_graph_loop_matches_host_loop(sg, case, precision):
    """The CG loop captured as one graph (device-side while node) gives the same
    iterations and solution as the host-driven loop."""
    domain, d, p, r, w, grading, gamma, mn = case
    src = {"unit": "sine", "annulus": "annulus_paper"}[domain]
    out = []
    with sg.Plan(d, p, w, domain=domain, continuity=r, min_level=mn, grading=grading, gamma=gamma,
                 precision=precision) as P:
        for use_graph in (True, False, True):
            sg.sgiga_set_solver_options(P.handle, use_graph=use_graph)
            sg.sgiga_set_rhs_builtin(P.handle, src)
            st, _ = sg.sgiga_solve(P.handle, 1e-12, 50)
            u = np.zeros(P.info.ndof)
            sg.sgiga_get_solution(P.handle, u)
            out.append((st.iterations, st.inner_iterations, u))
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert _rel(out[0][2], out[1][2]) < 1e-12 and _rel(out[2][2], out[1][2]) < 1e-12


def test_autotune_keeps_the_operator(sg):
    """The tile autotuner re-plans tiles and geometry planes; K x is unchanged."""
    case = ("unit", 3, 3, 2, 7, "uniform", 1.0, 1)
    with _plan(sg, case) as P:
        n = P.info.ndof
        x = _dev(random_vector(n, 61))
        y0 = torch.zeros_like(x)
        sg.sgiga_apply(P.handle, x, y0)
        rv = _dev(random_vector(n, 62))
        z0 = torch.zeros_like(x)
        sg.sgiga_precond(P.handle, rv, z0)
        res = sg.sgiga_autotune(P.handle, reps=2)
        assert res.ncand >= 4 and 0 <= res.best < res.ncand and res.best_ms > 0
        assert res.fd_ncand == 8 and 0 <= res.fd_best < 8 and res.fd_ms[res.fd_best] > 0 and res.fd_nitems > 0
        z1 = torch.zeros_like(x)
        sg.sgiga_precond(P.handle, rv, z1)
        assert _rel(z1.cpu().numpy(), z0.cpu().numpy()) < 1e-13
        y1 = torch.zeros_like(x)
        sg.sgiga_apply(P.handle, x, y1)
        assert _rel(y1.cpu().numpy(), y0.cpu().numpy()) < 1e-13
        sg.sgiga_set_rhs_builtin(P.handle, "sine")
        st, _ = sg.sgiga_solve(P.handle, 1e-12, 50)
        u = np.zeros(n)
        sg.sgiga_get_solution(P.handle, u)
        g = P.grids[0]
        comp = _component(case, g).assemble(f=problems.get("sine3").f)
        assert _rel(u[g.dof_off:g.dof_off + g.ndof], comp.solve()) < 1e-10


def test_component_subset_plan(sg):
    """A plan restricted to one component (the per-grid comparator) solves that
    component exactly as the batched plan does."""
    case = ("unit", 3, 3, 2, 7, "uniform", 1.0, 1)
    with _plan(sg, case) as P:
        sg.sgiga_set_rhs_builtin(P.handle, "sine")
        sg.sgiga_solve(P.handle, 1e-12, 50)
        u = np.zeros(P.info.ndof)
        sg.sgiga_get_solution(P.handle, u)
        g = P.grids[3]
        lv = tuple(g.levels[:3])
        with sg.Plan(3, 3, 7, components=[lv]) as Q:
            assert Q.info.ngrids == 1 and Q.info.ndof == g.ndof and Q.grids[0].coeff == g.coeff
            sg.sgiga_set_solver_options(Q.handle, use_graph=False)
            sg.sgiga_set_rhs_builtin(Q.handle, "sine")
            sg.sgiga_solve(Q.handle, 1e-12, 50)
            v = np.zeros(Q.info.ndof)
            sg.sgiga_get_solution(Q.handle, v)
        assert _rel(v, u[g.dof_off:g.dof_off + g.ndof]) < 1e-12
    with pytest.raises(sg.SgigaError):
        sg.Plan(3, 3, 7, components=[(7, 7, 7)])


@pytest.mark.parametrize("case", [CASES[0], CASES[3], CASES[5]])
def test_functional_against_oracle(sg, case):
    """l(u) = sum_g c_g int q u_g from the load vector of q, without evaluation
    points, matches the oracle's (per component and combined)."""
    domain, d, p, r, w, grading, gamma, mn = case
    prob = {"unit": "sine%d" % d, "annulus": "annulus_sinx"}[domain]
    if domain == "annulus" and d == 3:
        pytest.skip("no 3D annulus source")
    src = {"unit": "sine", "annulus": "annulus"}[domain]
    with _plan(sg, case) as P:
        sg.sgiga_set_rhs_builtin(P.handle, src)
        sg.sgiga_solve(P.handle, 1e-13, 100)
        xq = torch.zeros(d * P.info.nqp, dtype=torch.float64, device="cuda")   # device buffer
        sg.sgiga_qp_coords(P.handle, xq)
        xq = xq.cpu().numpy().reshape(d, -1).T
        qfun = lambda x: 1.0 + np.cos(2.0 * x[:, 0]) * x[:, 1]
        vals, comb = sg.sgiga_functional(P.handle, np.ascontiguousarray(qfun(xq)))
        res = []
        for g in P.grids:
            comp = _component(case, g).assemble(f=problems.get(prob).f)
            res.append((tuple(g.levels[:d]), g.coeff, comp, comp.solve()))
        ov, oc = driver.functional(res, qfun)
        assert _rel(vals, ov) < 1e-10
        assert abs(comb - oc) <= 1e-10 * abs(oc)


def test_host_pointers_are_refused_not_dereferenced(sg):
    """Entry points whose kernels read caller buffers refuse host memory with
    an error status (the binding accepts numpy arrays; a kernel would fault)."""
    with _plan(sg, CASES[0]) as P:
        n = P.info.ndof
        xh, yh = np.zeros(n), np.zeros(n)
        for fn in (sg.sgiga_apply, sg.sgiga_precond):
            with pytest.raises(sg.SgigaError):
                fn(P.handle, xh, yh)
        # host buffers are fine where the call stages them
        xq = np.zeros(2 * P.info.nqp)
        sg.sgiga_qp_coords(P.handle, xq)
        xd = torch.zeros(2 * P.info.nqp, dtype=torch.float64, device="cuda")
        sg.sgiga_qp_coords(P.handle, xd)
        assert np.abs(xd.cpu().numpy() - xq).max() == 0.0
