"""The checked build (-DSGIGA_CHECKED): the same library with bounds checks
in the operator and preconditioner kernels. It runs the 3D FP32 and FP64
operators, both preconditioner layouts, a 2D L-shape (aliased pieces) and a
mixed solve in a child process and must record no failed check and give the
default build's results. The default build reports that it has no checks."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, %(root)r)
from paper_1707_09598_gb300 import sgiga
from paper_1707_09598_gb300.inputs import random_vector
out = {"checked": sgiga.sgiga_build_checked(), "sites": [], "vals": {}}
with sgiga.Plan(3, 3, 7, domain="annulus", precision="mixed") as P:
    n = P.info.ndof
    x = torch.as_tensor(random_vector(n, 5), device="cuda")
    y = torch.zeros_like(x)
    sgiga.sgiga_apply(P.handle, x, y)
    yf = torch.zeros(n, dtype=torch.float32, device="cuda")
    sgiga.sgiga_apply_f32(P.handle, x.float(), yf)
    z = torch.zeros_like(x)
    vals = [y.norm().item(), yf.double().norm().item()]
    for grouped in (0, 1):
        sgiga.sgiga_set_precond_split(P.handle, 32, grouped)
        sgiga.sgiga_precond(P.handle, x, z)
        vals.append(z.norm().item())
    sgiga.sgiga_set_rhs_builtin(P.handle, "annulus_paper")
    st, rc = sgiga.sgiga_solve(P.handle, 1e-8, 50)
    u = np.zeros(n)
    sgiga.sgiga_get_solution(P.handle, u)
    vals.append(float(np.linalg.norm(u)))
    out["sites"].append(sgiga.sgiga_check_site(P.handle))
    out["vals"]["annulus3"] = vals
with sgiga.Plan(2, 2, 6, domain="lshape", grading="onesided", gamma=2.0) as P:
    sgiga.sgiga_set_rhs_builtin(P.handle, "lshape_corner")
    st, rc = sgiga.sgiga_solve(P.handle, 1e-11, 2000)
    u = np.zeros(P.info.ndof)
    sgiga.sgiga_get_solution(P.handle, u)
    out["sites"].append(sgiga.sgiga_check_site(P.handle))
    out["vals"]["lshape"] = [float(np.linalg.norm(u))]
print("RESULT " + json.dumps(out))
"""


def _run(lib=None):
    env = dict(os.environ)
    if lib:
        env["SGIGA_LIB"] = lib
    else:
        env.pop("SGIGA_LIB", None)
    r = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}], capture_output=True, text=True, env=env,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_checked_build_records_no_failed_check_and_agrees():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_09598_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    lib = build.build(checked=True)
    base = _run()
    chk = _run(lib)
    assert base["checked"] == 0 and chk["checked"] == 1
    assert chk["sites"] == [0, 0] and base["sites"] == [0, 0]
    for key, vals in base["vals"].items():
        np.testing.assert_allclose(chk["vals"][key], vals, rtol=1e-6)
