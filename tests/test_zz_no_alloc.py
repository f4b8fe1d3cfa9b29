"""The allocation-free preconditioner apply against the plan-based one.

sgiga_fd_apply_noalloc serves callers that cannot call cudaMalloc where they
need the preconditioner (allocation-free real-time loops, memory owned by
another allocator that must account for every byte). It keeps its
intermediate tensors in a library-owned device array. This test checks,
through the C ABI, that it gives the same result as sgiga_precond on several
components, on two calls in a row (the array keeps the previous call's
contents), that the device's free memory does not change across calls, and
that it rejects grids larger than its array, also when the product of the
sizes would overflow. It runs last (file name) and also alone.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("d,p,w", [(3, 3, 6), (2, 2, 8)])
def test_noalloc_matches_plan_preconditioner(sg, d, p, w):
    from paper_1707_09598_gb300.inputs import random_vector
    with sg.Plan(d, p, w) as P:
        n_all = P.info.ndof
        r = torch.as_tensor(random_vector(n_all, 31), device="cuda")
        z_ref = torch.zeros_like(r)
        sg.sgiga_precond(P.handle, r, z_ref)
        for gi in (0, P.info.ngrids // 2, P.info.ngrids - 1):
            g = P.grids[gi]
            n = [g.n[k] for k in range(d)]
            U, lam = [], []
            for k in range(d):
                Uk, lk = sg.sgiga_fd_eigen(P.handle, k, g.levels[k], n[k])
                U.append(torch.as_tensor(Uk, device="cuda").contiguous())
                lam.append(torch.as_tensor(lk, device="cuda").contiguous())
            sl = slice(g.dof_off, g.dof_off + g.ndof)
            rg = r[sl].contiguous()
            z = torch.full_like(rg, float("nan"))
            sg.sgiga_fd_apply_noalloc(n, U, lam, rg, z)     # first call on the device: address look-up
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            alloc0 = torch.cuda.memory_allocated()
            for call in range(2):          # two calls in a row share the scratch array
                z.fill_(float("nan"))
                sg.sgiga_fd_apply_noalloc(n, U, lam, rg, z)
                torch.cuda.synchronize()
                assert _rel(z, z_ref[sl]) < 1e-12, (gi, call, _rel(z, z_ref[sl]))
            assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
            # a second input right after: no state leaks from the previous call
            r2 = torch.as_tensor(random_vector(g.ndof, 32 + gi), device="cuda")
            z2 = torch.zeros_like(r2)
            sg.sgiga_fd_apply_noalloc(n, U, lam, r2, z2)
            full = torch.zeros(n_all, dtype=torch.float64, device="cuda")
            full[sl] = r2
            zf = torch.zeros_like(full)
            sg.sgiga_precond(P.handle, full, zf)
            torch.cuda.synchronize()
            assert _rel(z2, zf[sl]) < 1e-12


def test_noalloc_rejects_grids_larger_than_its_array(sg):
    m = 65
    n = [m, m, m]                       # 274,625 > SGIGA_NOALLOC_MAX_DOFS entries
    assert m ** 3 > sg.SGIGA_NOALLOC_MAX_DOFS
    U = [torch.eye(m, dtype=torch.float64, device="cuda") for _ in range(3)]
    lam = [torch.ones(m, dtype=torch.float64, device="cuda") for _ in range(3)]
    r = torch.ones(m ** 3, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    rc = sg.sgiga_fd_apply_noalloc(n, U, lam, r, z, check=False)
    assert rc == sg.SGIGA_ERR_ARG
    assert "SGIGA_NOALLOC_MAX_DOFS" in sg.sgiga_last_error()
    assert float(z.abs().max()) == 0.0  # nothing was launched
    # sizes whose product would overflow: refused before any pointer is used
    # (through the C ABI directly; the binding would refuse the buffers first)
    import ctypes
    na = (ctypes.c_int * 3)(*([2 ** 31 - 1] * 3))
    ua = (ctypes.c_void_p * 3)(*[u.data_ptr() for u in U])
    la = (ctypes.c_void_p * 3)(*[l_.data_ptr() for l_ in lam])
    rc = sg._lib.sgiga_fd_apply_noalloc(3, na, ua, la, r.data_ptr(), z.data_ptr(), None)
    assert rc == sg.SGIGA_ERR_ARG and "SGIGA_NOALLOC_MAX_DOFS" in sg.sgiga_last_error()
