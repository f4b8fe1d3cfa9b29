"""Failure handling made on the host: invalid plans, non-finite inputs,
corrupted checkpoints and an iteration limit that is too small each return
an error status (no call aborts, no GPU fault is provoked). The plan checks
run without a GPU; the input checks need one and are marked gpu."""
import ctypes
import os

import numpy as np
import pytest

from paper_1707_09598_gb300 import build


@pytest.fixture(scope="module")
def sg():
    if not os.path.exists(build.LIB):
        build.build()
    from paper_1707_09598_gb300 import sgiga
    return sgiga


def _raw_plan(sg, **over):
    """sgiga_plan through the C ABI with a config whose fields may be invalid."""
    cfg = sg.sgiga_config(3, 3, -1, 6, 1, 0, 0, 1.0, 0, 0, None)
    for k, v in over.items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p()
    rc = sg._lib.sgiga_plan(ctypes.byref(cfg), None, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("field,value", [
    ("d", 4), ("d", 1), ("p", 0), ("p", 9), ("continuity", 3), ("min_level", -1), ("w", -5),
    ("domain", 9), ("grading", 7), ("precision", 5), ("precond", 8),
])
def test_invalid_plan_configuration_is_an_argument_error(sg, field, value):
    rc, h = _raw_plan(sg, **{field: value})
    assert rc == sg.SGIGA_ERR_ARG and not h.value
    assert sg.sgiga_last_error()


def test_invalid_combinations_are_argument_errors(sg):
    # the L-shaped domain is 2D; the learned preconditioner needs the mixed precision
    assert _raw_plan(sg, domain=3)[0] == sg.SGIGA_ERR_ARG
    assert _raw_plan(sg, precond=2)[0] == sg.SGIGA_ERR_ARG
    assert _raw_plan(sg, grading=1, gamma=0.0)[0] == sg.SGIGA_ERR_ARG
    assert _raw_plan(sg, domain=2)[0] == sg.SGIGA_ERR_ARG          # a user patch without a patch


def test_null_arguments(sg):
    h = ctypes.c_void_p()
    assert sg._lib.sgiga_plan(None, None, ctypes.byref(h)) == sg.SGIGA_ERR_ARG
    assert sg._lib.sgiga_solve(None, ctypes.c_double(1e-8), 10, None) == sg.SGIGA_ERR_ARG
    assert sg._lib.sgiga_apply(None, None, None) == sg.SGIGA_ERR_ARG
    sg._lib.sgiga_destroy(None)     # no-op


@pytest.mark.gpu
def test_non_finite_inputs_are_argument_errors(sg, tmp_path):
    """A NaN in f at one quadrature point makes sgiga_solve return
    SGIGA_ERR_ARG before iterating; a non-positive or NaN coefficient is
    refused and the plan keeps a = 1 (it still solves); a corrupted network
    checkpoint is refused; an iteration limit of 1 gives
    SGIGA_ERR_NOT_CONVERGED."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with sg.Plan(2, 2, 5, precision="mixed", precond="learned") as P:
        f = torch.ones(P.info.nqp, dtype=torch.float64, device="cuda")
        f[P.info.nqp // 3] = float("nan")
        sg.sgiga_set_rhs(P.handle, f)
        st, rc = sg.sgiga_solve(P.handle, 1e-8, 20, check=False)
        assert rc == sg.SGIGA_ERR_ARG and "not finite" in sg.sgiga_last_error()
        a = np.ones(P.info.nqp)
        a[7] = -1.0
        with pytest.raises(sg.SgigaError) as ei:
            sg.sgiga_set_coefficient_qp(P.handle, a)
        assert ei.value.code == sg.SGIGA_ERR_ARG
        a[7] = np.nan
        with pytest.raises(sg.SgigaError):
            sg.sgiga_set_coefficient_qp(P.handle, a)
        sg.sgiga_set_rhs_builtin(P.handle, "sine")
        st, rc = sg.sgiga_solve(P.handle, 1e-8, 20, check=False)
        assert rc == sg.SGIGA_OK
        st, rc = sg.sgiga_solve(P.handle, 1e-12, 1, check=False)
        assert rc == sg.SGIGA_ERR_NOT_CONVERGED
        bad = tmp_path / "net.bin"
        bad.write_bytes(b"SGIGANET" + b"\x02\x00\x00\x00" + b"\x00" * 40)
        with pytest.raises(sg.SgigaError) as ei:
            sg.sgiga_net_load(P.handle, str(bad))
        assert ei.value.code == sg.SGIGA_ERR_ARG
