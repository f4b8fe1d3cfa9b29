"""h-p sparse combination on the GPU against the oracle (oracle/hp.py): one
plan per degree (p0 .. p0 + Q at one continuity r), FP64 batched FD-PCG,
evaluation, and sgiga_combine_plans over all plans' components."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import combination, geometry, hp, problems  # noqa: E402
from paper_1707_09598_gb300.inputs import eval_points, random_points  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_09598_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_1707_09598_gb300 import hp_sparse, sgiga
    return sgiga, hp_sparse


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# (domain, d, p0, r, w, Q, plan source, oracle problem)
CASES = [
    ("unit", 2, 2, 1, 5, 1, "sine", "sine2"),
    ("unit", 2, 2, 1, 5, 2, "sine", "sine2"),
    ("annulus", 2, 2, 1, 5, 1, "annulus_paper", "annulus_paper2"),
    ("unit", 3, 2, 1, 4, 1, "sine", "sine3"),
]


@pytest.mark.parametrize("case", CASES)
def test_hp_combination_matches_the_oracle(sg, case):
    """Every component's values and the combined values at a lattice and at
    random points, against the oracle's direct solves and its Neumaier sum
    with the expanded coefficients: relative L2 1e-10 (FP64 path)."""
    sgiga, hps = sg
    domain, d, p0, r, w, Q, src, prob = case
    xi = np.ascontiguousarray(np.vstack([eval_points(d, 8), random_points(40, d, seed=91)]))
    npts = len(xi)
    with hps.HPCombination(d, p0, r, w, Q, domain=domain) as H:
        assert {k for k in H.component_keys()} == set(H.coef)
        H.set_rhs_builtin(src)
        stats = H.solve(1e-13, 400)          # raises unless every plan converged
        assert len(stats) == len(H.plans) == Q + 1
        uc = np.zeros(H.ngrids * npts)
        u = np.zeros(npts)
        H.eval_combine(xi, npts, uc, u)
        keys = H.component_keys()
    ref, vals, coef = hp.hp_solution(geometry.make(domain, d), problems.get(prob).f, d, p0, r, w, Q, xi)
    assert coef == H.coef
    uc = uc.reshape(len(keys), npts)
    for row, k in enumerate(keys):
        assert _rel(uc[row], vals[k]) < 1e-10, k
    assert _rel(u, ref) < 1e-10


def test_combine_plans_is_the_compensated_sum(sg):
    """sgiga_combine_plans over the plans of a combination equals the
    oracle's Neumaier sum of the same rows with each plan's coefficients, for
    host and for device buffers, on values spanning 1e-6 .. 1e6."""
    sgiga, hps = sg
    npts = 257
    with hps.HPCombination(2, 2, 1, 5, 2) as H:
        coef = np.array([g.coeff for _, P in H.plans for g in P.grids], dtype=np.float64)
        rng = np.random.default_rng(5)
        vals = rng.standard_normal((H.ngrids, npts)) * 10.0 ** rng.integers(-6, 7, (H.ngrids, 1))
        ref = combination.combine(vals, coef)
        handles = [P.handle for _, P in H.plans]
        ud = torch.zeros(npts, dtype=torch.float64, device="cuda")
        sgiga.sgiga_combine_plans(handles, torch.as_tensor(vals.reshape(-1), device="cuda"), npts, ud)
        np.testing.assert_allclose(ud.cpu().numpy(), ref, rtol=1e-15, atol=1e-15 * np.abs(vals).max())
        # host buffers go through the same kernel
        u = np.zeros(npts)
        sgiga.sgiga_combine_plans(handles, np.ascontiguousarray(vals.reshape(-1)), npts, u)
        np.testing.assert_array_equal(u, ud.cpu().numpy())


def test_combine_plans_refuses_mismatched_plans(sg):
    sgiga, hps = sg
    u = np.zeros(4)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with sgiga.Plan(2, 2, 3) as A, sgiga.Plan(3, 2, 3) as B:
        vals = np.zeros((A.info.ngrids + B.info.ngrids) * 4)
        with pytest.raises(sgiga.SgigaError) as ei:
            sgiga.sgiga_combine_plans([A.handle, B.handle], vals, 4, u)
        assert ei.value.code == sgiga.SGIGA_ERR_ARG
        with pytest.raises(sgiga.SgigaError) as ei:
            sgiga.sgiga_combine_plans([], vals, 4, u)
        assert ei.value.code == sgiga.SGIGA_ERR_ARG
    with sgiga.Plan(2, 2, 3, stream=s1) as A, sgiga.Plan(2, 3, 3, stream=s2) as B:
        vals = np.zeros((A.info.ngrids + B.info.ngrids) * 4)
        with pytest.raises(sgiga.SgigaError) as ei:
            sgiga.sgiga_combine_plans([A.handle, B.handle], vals, 4, u)
        assert ei.value.code == sgiga.SGIGA_ERR_ARG
