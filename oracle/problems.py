"""Manufactured Poisson problems of the oracle (Problem 1; Sec. 4.2).

TEST INFRASTRUCTURE: see the package header.

Each problem gives the exact solution u (when known), its gradient, and the
source f = -Laplace(u), all derived here symbolically with sympy so that f is
never typed in by hand on the oracle side.
"""
import functools

import numpy as np
import sympy as sy

_X = sy.symbols("x y z", real=True)

# name -> (d, expression of u or None, constant f when u is unknown)
_DEFS = {
    # unit square / cube, u = prod sin(pi x_k)
    "sine2": (2, lambda x, y, z: sy.sin(sy.pi * x) * sy.sin(sy.pi * y), None),
    "sine3": (3, lambda x, y, z: sy.sin(sy.pi * x) * sy.sin(sy.pi * y) * sy.sin(sy.pi * z), None),
    # polynomial that lies in every component space with p >= 2 on the unit square/cube
    "poly2": (2, lambda x, y, z: x * (1 - x) * y * (1 - y), None),
    "poly3": (3, lambda x, y, z: x * (1 - x) * y * (1 - y) * z * (1 - z), None),
    # quarter annulus: the workload's solution u = x y (r^2-1)(r^2-4) sin(x)
    "annulus_sinx": (2, lambda x, y, z: x * y * (x**2 + y**2 - 1) * (x**2 + y**2 - 4) * sy.sin(x), None),
    # quarter annulus: the paper's regular solution (Sec. 4.2), d = 2 and 3
    "annulus_paper2": (2, lambda x, y, z: -(x**2 + y**2 - 1) * (x**2 + y**2 - 4) * x * y**2, None),
    "annulus_paper3": (3, lambda x, y, z: -(x**2 + y**2 - 1) * (x**2 + y**2 - 4) * x * y**2
                       * sy.sin(sy.pi * z), None),
    # f = 1 (low-regularity tests of Sec. 4.3); exact u unknown
    "one2": (2, None, 1.0),
    "one3": (3, None, 1.0),
}


class Problem:
    def __init__(self, name):
        d, uf, fconst = _DEFS[name]
        self.name, self.d = name, d
        xs = _X[:d]
        if uf is None:
            self.u = None
            self.grad_u = None
            c = float(fconst)
            self.f = lambda pts: np.full(np.asarray(pts).shape[0], c)
            return
        u = uf(*_X)
        f = -sum(sy.diff(u, v, 2) for v in xs)
        self._u_expr, self._f_expr = u, sy.simplify(f)
        ul = sy.lambdify(xs, u, "numpy")
        fl = sy.lambdify(xs, self._f_expr, "numpy")
        gl = [sy.lambdify(xs, sy.diff(u, v), "numpy") for v in xs]

        def wrap(fun):
            def g(pts):
                pts = np.asarray(pts, dtype=np.float64)
                out = fun(*[pts[:, k] for k in range(d)])
                return np.broadcast_to(np.asarray(out, dtype=np.float64), (pts.shape[0],)).copy()
            return g

        self.u = wrap(ul)
        self.f = wrap(fl)
        gw = [wrap(g) for g in gl]
        self.grad_u = lambda pts: np.stack([g(pts) for g in gw], axis=1)


@functools.lru_cache(maxsize=None)
def get(name):
    return Problem(name)
