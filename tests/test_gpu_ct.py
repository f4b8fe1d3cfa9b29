"""The combination technique as a preconditioner of the full tensor-product
solve (the paper's closing remark, Sec. 5), on the GPU: the combination
operator B_CT = sum_i c_i P_i K_i^{-1} P_i^T (knot-insertion prolongations,
the combination plan's batched PCG as K_i^{-1}) against the oracle's (exact
LU solves), and the two-level FD + B_CT solve of the full system against the
oracle's direct solve and its CG iteration counts."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ct, geometry  # noqa: E402
from paper_1707_09598_gb300.inputs import random_vector  # noqa: E402


def _coef(x):
    """a(x) = exp(sin(3 x) cos(2 y)): smooth, varying by e^(+-1)."""
    return np.exp(np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1]))


@pytest.fixture
def stream():
    """A side stream that is torch's current stream for the test only (the
    plans run on it, so torch's fills and reads are ordered with their calls)."""
    s = torch.cuda.Stream()
    prev = torch.cuda.current_stream()
    torch.cuda.set_stream(s)
    yield s
    torch.cuda.synchronize()
    torch.cuda.set_stream(prev)


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_09598_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_1707_09598_gb300 import sgiga
    return sgiga


def _set_coef(sg, P, d):
    xq = np.zeros(d * P.info.nqp)
    sg.sgiga_qp_coords(P.handle, xq)
    sg.sgiga_set_coefficient_qp(P.handle, _coef(xq.reshape(d, -1).T))


def _plans(sg, d, p, r, J, stream):
    full = sg.Plan(d, p, 2 * J, continuity=r, components=[(J,) * d], coefficients=[1.0], stream=stream)
    comb = sg.Plan(d, p, J, continuity=r, stream=stream)
    for P in (full, comb):
        _set_coef(sg, P, d)
    return full, comb


@pytest.mark.parametrize("d,J", [(2, 5), (3, 3)])
def test_combination_operator_against_oracle(sg, stream, d, J):
    full, comb = _plans(sg, d, 2, 1, J, stream)
    with full, comb:
        sg.sgiga_ct_attach(full.handle, comb.handle, 1e-13, 2000)
        n = full.info.ndof
        r = random_vector(n, 71)
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        sg.sgiga_ct_apply(full.handle, torch.as_tensor(r, device="cuda"), z)
        z = z.cpu().numpy()
        sg.sgiga_ct_attach(full.handle, None)
    T = ct.TwoLevel(geometry.make("unit", d), d, 2, 1, J, diffusion=_coef)
    assert T.A.shape[0] == n
    ref = T.b_ct(r)
    assert np.linalg.norm(z - ref) / np.linalg.norm(ref) < 1e-9


def test_two_level_solve_against_oracle(sg, stream):
    """FD + B_CT in flexible CG on the GPU: the solution equals the oracle's
    direct solve, and the outer iteration counts with and without B_CT are
    within one of the oracle's standard PCG counts (exact inner solves there)."""
    d, J = 2, 6
    full, comb = _plans(sg, d, 2, 1, J, stream)
    T = ct.TwoLevel(geometry.make("unit", d), d, 2, 1, J, diffusion=_coef)
    n_fd, _ = T.cg_iterations(T.b_fd)
    n_2l, _ = T.cg_iterations(lambda v: T.b_fd(v) + T.b_ct(v))
    u_ref = T.full.solve()
    with full, comb:
        sg.sgiga_set_rhs_builtin(full.handle, "one")
        st_fd, _ = sg.sgiga_solve(full.handle, 1e-10, 500)
        sg.sgiga_ct_attach(full.handle, comb.handle, 1e-12, 2000)
        st_2l, _ = sg.sgiga_solve(full.handle, 1e-10, 500)
        u = np.zeros(full.info.ndof)
        sg.sgiga_get_solution(full.handle, u)
        sg.sgiga_ct_attach(full.handle, None)
    print("outer iterations: FD %d (oracle %d), FD + CT %d (oracle %d), inner %d"
          % (st_fd.iterations, n_fd, st_2l.iterations, n_2l, st_2l.inner_iterations))
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-8
    assert abs(st_fd.iterations - n_fd) <= 1 and abs(st_2l.iterations - n_2l) <= 1
    assert st_2l.inner_iterations > 0


def test_attach_refuses_mismatched_plans(sg):
    with sg.Plan(2, 2, 8, components=[(4, 4)], coefficients=[1.0]) as full, \
            sg.Plan(2, 2, 5) as finer, sg.Plan(2, 3, 4) as other_p, \
            sg.Plan(2, 2, 4, precision="mixed") as mixed, sg.Plan(2, 2, 4) as ok:
        for bad in (finer, other_p, mixed, full):
            with pytest.raises(sg.SgigaError) as ei:
                sg.sgiga_ct_attach(full.handle, bad.handle)
            assert ei.value.code == sg.SGIGA_ERR_ARG
        with pytest.raises(sg.SgigaError):
            sg.sgiga_ct_attach(ok.handle, full.handle)       # the full plan needs one component
        sg.sgiga_ct_attach(full.handle, ok.handle)
        sg.sgiga_ct_attach(full.handle, None)
        r = torch.zeros(full.info.ndof, dtype=torch.float64, device="cuda")
        with pytest.raises(sg.SgigaError):
            sg.sgiga_ct_apply(full.handle, r, r)
