"""Python binding of the C ABI in include/sgiga.h (argument marshalling only).

Every function has the name of its C entry point and forwards to it through
ctypes; all arithmetic runs in the CUDA library. Buffers may be torch tensors
(CUDA or CPU) or numpy arrays, float64 and contiguous; a host buffer is staged
by the library. Importing this module fails loudly if the library is missing.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SGIGA_LIB selects another build of the library (the checked build)
LIB_PATH = os.environ.get("SGIGA_LIB") or os.path.join(_HERE, "_lib", "libsgiga.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libsgiga.so is not built (%s); run paper_1707_09598_gb300.build.build()" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

SGIGA_OK = 0
SGIGA_ERR_ARG = -1
SGIGA_ERR_NOMEM = -2
SGIGA_ERR_CUDA = -3
SGIGA_ERR_NOT_CONVERGED = -4
SGIGA_ERR_TIMEOUT = -5
SGIGA_ERR_GEOMETRY = -6

DOMAIN = {"unit": 0, "square": 0, "cube": 0, "annulus": 1, "patch": 2, "lshape": 3}
GRADING = {"uniform": 0, "radical": 1, "onesided": 2}
PREC = {"fp64": 0, "mixed": 1, "mixed_fp32": 1}
PRECOND = {"fd": 0, "none": 1, "learned": 2}
SOURCE = {"sine": 0, "poly": 1, "annulus": 2, "annulus_paper": 3, "one": 4, "lshape_corner": 5,
          "harmonic_quadratic": 6}


class sgiga_patch(ctypes.Structure):
    _fields_ = [("deg", ctypes.c_int * 3), ("nknots", ctypes.c_int * 3), ("knots", ctypes.c_void_p * 3),
                ("ncp", ctypes.c_int * 3), ("weights", ctypes.c_void_p * 3), ("cp", ctypes.c_void_p)]


class sgiga_config(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("p", ctypes.c_int), ("continuity", ctypes.c_int), ("w", ctypes.c_int),
                ("min_level", ctypes.c_int), ("domain", ctypes.c_int), ("grading", ctypes.c_int),
                ("gamma", ctypes.c_double), ("precision", ctypes.c_int), ("precond", ctypes.c_int),
                ("patch", ctypes.POINTER(sgiga_patch)), ("ncomponents", ctypes.c_int),
                ("components", ctypes.POINTER(ctypes.c_int)), ("coefficients", ctypes.POINTER(ctypes.c_double))]


class sgiga_info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("p", ctypes.c_int), ("continuity", ctypes.c_int), ("ngrids", ctypes.c_int),
                ("ndof", ctypes.c_longlong), ("nqp", ctypes.c_longlong), ("max_tile_smem", ctypes.c_int),
                ("ntiles", ctypes.c_int), ("diag_metric", ctypes.c_int), ("npatches", ctypes.c_int),
                ("nbpts", ctypes.c_longlong)]


class sgiga_grid(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int * 3), ("n", ctypes.c_int * 3), ("coeff", ctypes.c_int),
                ("ndof", ctypes.c_longlong), ("dof_off", ctypes.c_longlong), ("nqp", ctypes.c_longlong),
                ("qp_off", ctypes.c_longlong), ("tile", ctypes.c_int * 3), ("pencil_dir", ctypes.c_int),
                ("ntiles", ctypes.c_int)]


class sgiga_train_cfg(ctypes.Structure):
    _fields_ = [("target_pairs", ctypes.c_int), ("max_iter_record", ctypes.c_int), ("epochs", ctypes.c_int),
                ("lr", ctypes.c_float), ("seed", ctypes.c_uint), ("batch", ctypes.c_int), ("loss_norm", ctypes.c_int)]


class sgiga_train_stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int), ("samples", ctypes.c_int), ("rhs", ctypes.c_int), ("steps", ctypes.c_int),
                ("loss_first_epoch", ctypes.c_double), ("loss_last_epoch", ctypes.c_double),
                ("seconds", ctypes.c_double), ("loss_initial", ctypes.c_double), ("loss_fd", ctypes.c_double),
                ("loss_epoch", ctypes.c_double * 32), ("logs_min", ctypes.c_double), ("logs_max", ctypes.c_double),
                ("best_epoch", ctypes.c_int), ("val_iters_initial", ctypes.c_int), ("val_iters_best", ctypes.c_int)]


class sgiga_tune_result(ctypes.Structure):
    _fields_ = [("ncand", ctypes.c_int), ("best", ctypes.c_int), ("ntiles", ctypes.c_int), ("best_ms", ctypes.c_double),
                ("ms", ctypes.c_double * 16), ("budget", ctypes.c_int * 16), ("qpcap", ctypes.c_int * 16),
                ("nthreads", ctypes.c_int * 16),
                ("fd_ncand", ctypes.c_int), ("fd_best", ctypes.c_int), ("fd_nitems", ctypes.c_int),
                ("fd_ks", ctypes.c_int * 8), ("fd_ms", ctypes.c_double * 8), ("fd_grouped", ctypes.c_int * 8),
                ("prefetch", ctypes.c_int * 16), ("best_prefetch", ctypes.c_int),
                ("solve_precision", ctypes.c_int), ("solve_ms_fp64", ctypes.c_double),
                ("solve_ms_mixed", ctypes.c_double), ("solve_ms_fp64_fd32", ctypes.c_double),
                ("solve_fp32_precond", ctypes.c_int)]


class sgiga_plan_times_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("total", "host", "basis", "eigen", "fd", "geometry", "vectors",
                                               "coefficient", "autotune")]


class sgiga_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("max_rel_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("inner_iterations", ctypes.c_int), ("fallback", ctypes.c_int)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_longlong
_SIGS = {
    "sgiga_plan": (_I, [ctypes.POINTER(sgiga_config), _P, ctypes.POINTER(_P)]),
    "sgiga_destroy": (None, [_P]),
    "sgiga_plan_info": (_I, [_P, ctypes.POINTER(sgiga_info)]),
    "sgiga_grid_info": (_I, [_P, _I, ctypes.POINTER(sgiga_grid)]),
    "sgiga_plan_times": (_I, [_P, ctypes.POINTER(sgiga_plan_times_t)]),
    "sgiga_qp_coords": (_I, [_P, _P]),
    "sgiga_set_rhs": (_I, [_P, _P]),
    "sgiga_set_rhs_builtin": (_I, [_P, _I]),
    "sgiga_get_rhs": (_I, [_P, _P]),
    "sgiga_set_coefficient": (_I, [_P, _I, _P, _P, _D]),
    "sgiga_set_coefficient_qp": (_I, [_P, _P]),
    "sgiga_source_at_qp": (_I, [_P, _I, _P]),
    "sgiga_apply": (_I, [_P, _P, _P]),
    "sgiga_apply_f32": (_I, [_P, _P, _P]),
    "sgiga_set_precond_split": (_I, [_P, _I, _I]),
    "sgiga_precond_f32": (_I, [_P, _P, _P]),
    "sgiga_precond": (_I, [_P, _P, _P]),
    "sgiga_solve": (_I, [_P, _D, _I, ctypes.POINTER(sgiga_solve_stats)]),
    "sgiga_set_solver_options": (_I, [_P, _I, _D, _I]),
    "sgiga_autotune": (_I, [_P, _I, ctypes.POINTER(sgiga_tune_result)]),
    "sgiga_set_tiling": (_I, [_P, _I, _I, _I, _I]),
    "sgiga_build_checked": (_I, []),
    "sgiga_check_site": (_I, [_P, ctypes.POINTER(ctypes.c_int)]),
    "sgiga_ct_attach": (_I, [_P, _P, ctypes.c_double, _I]),
    "sgiga_ct_apply": (_I, [_P, _P, _P]),
    "sgiga_get_solution": (_I, [_P, _P]),
    "sgiga_set_solution": (_I, [_P, _P]),
    "sgiga_eval": (_I, [_P, _P, _L, _P]),
    "sgiga_eval_grad": (_I, [_P, _P, _P, _L, _P, _P]),
    "sgiga_boundary_points": (_I, [_P, _P]),
    "sgiga_map_points": (_I, [_P, _P, _P, _L, _P, _P]),
    "sgiga_functional": (_I, [_P, _P, _P, _P]),
    "sgiga_set_dirichlet": (_I, [_P, _P]),
    "sgiga_combine": (_I, [_P, _P, _L, _P]),
    "sgiga_combine_plans": (_I, [_I, ctypes.POINTER(_P), _P, _L, _P]),
    "sgiga_basis_table": (_I, [_P, _I, _I, _P, _P, _P, _P, _P]),
    "sgiga_geometry_coeffs": (_I, [_P, _I, _P, _P]),
    "sgiga_fd_eigen": (_I, [_P, _I, _I, _P, _P]),
    "sgiga_fd_apply_noalloc": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_P), ctypes.POINTER(_P), _P, _P, _P]),
    "sgiga_net_init": (_I, [_P, ctypes.c_uint]),
    "sgiga_net_num_params": (_I, [_P]),
    "sgiga_net_get_params": (_I, [_P, _P]),
    "sgiga_net_set_params": (_I, [_P, _P]),
    "sgiga_net_forward": (_I, [_P, _P, _P]),
    "sgiga_net_backward": (_I, [_P, _P, _P, _P]),
    "sgiga_net_features": (_I, [_P, _P]),
    "sgiga_net_scaling": (_I, [_P, _P]),
    "sgiga_net_set_scaling": (_I, [_P, _P]),
    "sgiga_net_loss_grad": (_I, [_P, _P, _P, ctypes.POINTER(_D), _P]),
    "sgiga_net_set_loss_norm": (_I, [_P, _I]),
    "sgiga_train_net": (_I, [_P, ctypes.POINTER(sgiga_train_cfg), ctypes.POINTER(sgiga_train_stats)]),
    "sgiga_net_save": (_I, [_P, ctypes.c_char_p]),
    "sgiga_net_load": (_I, [_P, ctypes.c_char_p]),
    "sgiga_last_error": (ctypes.c_char_p, []),
    "sgiga_launch_count": (ctypes.c_longlong, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = sorted(_SIGS)


class SgigaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("sgiga error %d: %s" % (code, msg))
        self.code = code


def _check(rc):
    if rc != SGIGA_OK:
        raise SgigaError(rc, _lib.sgiga_last_error().decode())
    return rc


def _ptr(buf, n=None, dtype=np.float64):
    """Address of a contiguous buffer (torch tensor or numpy array), checked."""
    if buf is None:
        return None
    if hasattr(buf, "data_ptr"):          # torch tensor
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32}[dtype]
        if buf.dtype != want or not buf.is_contiguous():
            raise TypeError("expected a contiguous %s tensor" % want)
        if n is not None and buf.numel() < n:
            raise ValueError("buffer has %d elements, needs %d" % (buf.numel(), n))
        return buf.data_ptr()
    arr = buf
    if not isinstance(arr, np.ndarray) or arr.dtype != dtype or not arr.flags.c_contiguous:
        raise TypeError("expected a C-contiguous numpy array of %s" % np.dtype(dtype))
    if n is not None and arr.size < n:
        raise ValueError("buffer has %d elements, needs %d" % (arr.size, n))
    return arr.ctypes.data


# --- entry points (same names as the C ABI) ------------------------------------

def sgiga_plan(d, p, w, domain="unit", continuity=-1, min_level=1, grading="uniform", gamma=1.0,
               precision="fp64", precond="fd", stream=None, patch=None, components=None, coefficients=None):
    """patch: (degrees [d], knots [d arrays], control points [n, d]) for domain "patch";
    components: levels of the components to keep (default: the whole index set);
    coefficients: with components, their combination coefficients (an arbitrary index set)."""
    keep = []
    pp = None
    if patch is not None:
        degs, knots, cps = patch
        ps = sgiga_patch()
        for k in range(d):
            kn = np.ascontiguousarray(knots[k], dtype=np.float64)
            keep.append(kn)
            ps.deg[k] = int(degs[k])
            ps.nknots[k] = len(kn)
            ps.knots[k] = kn.ctypes.data
            ps.ncp[k] = len(kn) - int(degs[k]) - 1
            ps.weights[k] = None
        cpa = np.ascontiguousarray(cps, dtype=np.float64)
        keep.append(cpa)
        ps.cp = cpa.ctypes.data
        pp = ctypes.pointer(ps)
    cfg = sgiga_config(d, p, continuity, w, min_level, DOMAIN[domain], GRADING[grading], float(gamma),
                       PREC[precision], PRECOND[precond], pp)
    if components is not None:
        comp = np.ascontiguousarray(np.asarray(components, dtype=np.int32).reshape(-1, d))
        keep.append(comp)
        cfg.ncomponents = len(comp)
        cfg.components = comp.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        if coefficients is not None:
            cf = np.ascontiguousarray(np.asarray(coefficients, dtype=np.float64).reshape(-1))
            if len(cf) != len(comp):
                raise ValueError("one coefficient per component")
            keep.append(cf)
            cfg.coefficients = cf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = _P()
    s = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(_lib.sgiga_plan(ctypes.byref(cfg), s, ctypes.byref(h)))
    return h


def sgiga_destroy(plan):
    _lib.sgiga_destroy(plan)


def sgiga_plan_info(plan):
    out = sgiga_info()
    _check(_lib.sgiga_plan_info(plan, ctypes.byref(out)))
    return out


def sgiga_grid_info(plan, g):
    out = sgiga_grid()
    _check(_lib.sgiga_grid_info(plan, g, ctypes.byref(out)))
    return out


def sgiga_qp_coords(plan, xq):
    _check(_lib.sgiga_qp_coords(plan, _ptr(xq)))


def sgiga_set_rhs(plan, f_qp):
    n = sgiga_plan_info(plan).nqp
    _check(_lib.sgiga_set_rhs(plan, _ptr(f_qp, n)))


def sgiga_set_rhs_builtin(plan, source):
    _check(_lib.sgiga_set_rhs_builtin(plan, SOURCE[source] if isinstance(source, str) else int(source)))


def sgiga_source_at_qp(plan, source, f):
    n = sgiga_plan_info(plan).nqp
    _check(_lib.sgiga_source_at_qp(plan, SOURCE[source] if isinstance(source, str) else int(source), _ptr(f, n)))


def sgiga_set_coefficient(plan, omega, phase, amp):
    om = np.ascontiguousarray(omega, dtype=np.float64)
    ph = np.ascontiguousarray(phase, dtype=np.float64)
    _check(_lib.sgiga_set_coefficient(plan, len(ph), om.ctypes.data, ph.ctypes.data, float(amp)))


def sgiga_set_coefficient_qp(plan, a_qp):
    """a(x) at every quadrature point ([nqp], natural order; host or device), or None."""
    _check(_lib.sgiga_set_coefficient_qp(plan, None if a_qp is None else _ptr(a_qp, sgiga_plan_info(plan).nqp)))


def sgiga_get_rhs(plan, b):
    _check(_lib.sgiga_get_rhs(plan, _ptr(b, sgiga_plan_info(plan).ndof)))


def sgiga_apply(plan, x, y):
    n = sgiga_plan_info(plan).ndof
    _check(_lib.sgiga_apply(plan, _ptr(x, n), _ptr(y, n)))


def sgiga_apply_f32(plan, x, y):
    import torch
    n = sgiga_plan_info(plan).ndof
    for t in (x, y):
        if not (hasattr(t, "dtype") and t.dtype == torch.float32 and t.is_contiguous() and t.numel() >= n):
            raise TypeError("expected contiguous float32 tensors of %d entries" % n)
    _check(_lib.sgiga_apply_f32(plan, x.data_ptr(), y.data_ptr()))


def sgiga_precond(plan, r, z):
    n = sgiga_plan_info(plan).ndof
    _check(_lib.sgiga_precond(plan, _ptr(r, n), _ptr(z, n)))


def sgiga_precond_f32(plan, r, z):
    import torch
    n = sgiga_plan_info(plan).ndof
    for t in (r, z):
        if not (hasattr(t, "dtype") and t.dtype == torch.float32 and t.is_contiguous() and t.numel() >= n):
            raise TypeError("expected contiguous float32 tensors of %d entries" % n)
    _check(_lib.sgiga_precond_f32(plan, r.data_ptr(), z.data_ptr()))


def sgiga_autotune(plan, reps=3):
    out = sgiga_tune_result()
    _check(_lib.sgiga_autotune(plan, int(reps), ctypes.byref(out)))
    return out


def sgiga_build_checked():
    return int(_lib.sgiga_build_checked())


def sgiga_check_site(plan):
    site = ctypes.c_int(0)
    _check(_lib.sgiga_check_site(plan, ctypes.byref(site)))
    return site.value


def sgiga_ct_attach(plan, ct_plan, inner_tol=1e-6, inner_max=200):
    _check(_lib.sgiga_ct_attach(plan, ct_plan, float(inner_tol), int(inner_max)))


def sgiga_ct_apply(plan, r, z):
    n = sgiga_plan_info(plan).ndof
    _check(_lib.sgiga_ct_apply(plan, _ptr(r, n), _ptr(z, n)))


def sgiga_set_tiling(plan, budget, qpcap, nthreads=256, prefetch=0):
    _check(_lib.sgiga_set_tiling(plan, int(budget), int(qpcap), int(nthreads), int(prefetch)))


def sgiga_set_precond_split(plan, ks, grouped=False):
    _check(_lib.sgiga_set_precond_split(plan, int(ks), int(bool(grouped))))


def sgiga_set_solver_options(plan, use_graph=True, inner_tol=1e-5, inner_max=100):
    _check(_lib.sgiga_set_solver_options(plan, int(bool(use_graph)), float(inner_tol), int(inner_max)))


def sgiga_solve(plan, rel_tol, max_iter, check=True):
    st = sgiga_solve_stats()
    rc = _lib.sgiga_solve(plan, float(rel_tol), int(max_iter), ctypes.byref(st))
    if check:
        _check(rc)
    return st, rc


def sgiga_get_solution(plan, u):
    _check(_lib.sgiga_get_solution(plan, _ptr(u, sgiga_plan_info(plan).ndof)))


def sgiga_set_solution(plan, u):
    _check(_lib.sgiga_set_solution(plan, _ptr(u, sgiga_plan_info(plan).ndof)))


def sgiga_eval(plan, xi, npts, u_comp):
    info = sgiga_plan_info(plan)
    _check(_lib.sgiga_eval(plan, _ptr(xi, npts * info.d), int(npts), _ptr(u_comp, npts * info.ngrids)))


def sgiga_eval_grad(plan, xi, patch, npts, u_comp, grad_comp=None):
    """Values [ngrids][npts] and physical gradients [d][ngrids][npts]."""
    info = sgiga_plan_info(plan)
    _check(_lib.sgiga_eval_grad(plan, _ptr(xi, npts * info.d), _ptr(patch, npts, dtype=np.int32), int(npts),
                                _ptr(u_comp, npts * info.ngrids),
                                _ptr(grad_comp, info.d * npts * info.ngrids) if grad_comp is not None else None))


def sgiga_functional(plan, q_qp):
    """(per-component values, combined value) of l(u) = sum_g c_g int q u_g."""
    info = sgiga_plan_info(plan)
    comp = np.zeros(info.ngrids)
    out = np.zeros(1)
    _check(_lib.sgiga_functional(plan, _ptr(q_qp, info.nqp), _ptr(comp), _ptr(out)))
    return comp, float(out[0])


def sgiga_map_points(plan, xi, patch, npts, x, detj=None):
    d = sgiga_plan_info(plan).d
    _check(_lib.sgiga_map_points(plan, _ptr(xi, npts * d), _ptr(patch, npts, dtype=np.int32), int(npts),
                                 _ptr(x, npts * d), _ptr(detj, npts) if detj is not None else None))


def sgiga_boundary_points(plan, xb):
    _check(_lib.sgiga_boundary_points(plan, _ptr(xb, 2 * sgiga_plan_info(plan).nbpts)))


def sgiga_set_dirichlet(plan, g):
    _check(_lib.sgiga_set_dirichlet(plan, None if g is None else _ptr(g, sgiga_plan_info(plan).nbpts)))


def sgiga_combine(plan, u_comp, npts, u):
    info = sgiga_plan_info(plan)
    _check(_lib.sgiga_combine(plan, _ptr(u_comp, npts * info.ngrids), int(npts), _ptr(u, npts)))


def sgiga_combine_plans(plans, u_comp, npts, u):
    """plans: handles; u_comp: their sgiga_eval outputs, concatenated in that order."""
    ng = sum(sgiga_plan_info(h).ngrids for h in plans)
    arr = (_P * len(plans))(*plans)
    _check(_lib.sgiga_combine_plans(len(plans), arr, _ptr(u_comp, npts * ng), int(npts), _ptr(u, npts)))


def sgiga_basis_table(plan, dir, level):
    info = sgiga_plan_info(plan)
    E, Q = 2 ** level, info.p + 1
    xi, w = np.zeros(E * Q), np.zeros(E * Q)
    R, dR = np.zeros(E * Q * (info.p + 1)), np.zeros(E * Q * (info.p + 1))
    first = np.zeros(E, dtype=np.int32)
    _check(_lib.sgiga_basis_table(plan, dir, level, _ptr(xi), _ptr(w), _ptr(R), _ptr(dR),
                                  _ptr(first, dtype=np.int32)))
    return xi, w, R.reshape(E, Q, info.p + 1), dR.reshape(E, Q, info.p + 1), first


def sgiga_geometry_coeffs(plan, g):
    info = sgiga_plan_info(plan)
    gi = sgiga_grid_info(plan, g)
    nc = info.d * (info.d + 1) // 2
    G = np.zeros(nc * gi.nqp)
    mw = np.zeros(gi.nqp)
    _check(_lib.sgiga_geometry_coeffs(plan, g, _ptr(G), _ptr(mw)))
    return G.reshape(nc, gi.nqp), mw


def sgiga_fd_eigen(plan, dir, level, n):
    U = np.zeros(n * n)
    lam = np.zeros(n)
    _check(_lib.sgiga_fd_eigen(plan, dir, level, _ptr(U), _ptr(lam)))
    return U.reshape(n, n), lam


SGIGA_NOALLOC_MAX_DOFS = 262144


def sgiga_fd_apply_noalloc(n, U, lam, r, z, stream=None, check=True):
    """Allocation-free fast-diagonalisation apply for one grid (see include/sgiga.h).

    n: sizes per direction; U, lam: per-direction device tensors; r, z: device
    tensors of prod(n) float64 entries. Returns the status code."""
    d = len(n)
    N = 1
    for v in n:
        N *= int(v)
    na = (_I * d)(*[int(v) for v in n])
    ua = (_P * d)(*[_ptr(u, int(v) * int(v)) for u, v in zip(U, n)])
    la = (_P * d)(*[_ptr(l_, int(v)) for l_, v in zip(lam, n)])
    s = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = _lib.sgiga_fd_apply_noalloc(d, na, ua, la, _ptr(r, N), _ptr(z, N), s)
    if check:
        _check(rc)
    return rc


def sgiga_net_init(plan, seed):
    _check(_lib.sgiga_net_init(plan, int(seed)))


def sgiga_net_num_params(plan):
    n = _lib.sgiga_net_num_params(plan)
    if n < 0:
        _check(n)
    return n


def sgiga_net_get_params(plan):
    out = np.zeros(sgiga_net_num_params(plan), dtype=np.float32)
    _check(_lib.sgiga_net_get_params(plan, out.ctypes.data))
    return out


def sgiga_net_set_params(plan, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != sgiga_net_num_params(plan):
        raise ValueError("wrong parameter count")
    _check(_lib.sgiga_net_set_params(plan, a.ctypes.data))


def _f32dev(t, n):
    if not (hasattr(t, "dtype") and str(t.dtype) == "torch.float32" and t.is_cuda and t.is_contiguous()
            and t.numel() >= n):
        raise TypeError("expected a contiguous CUDA float32 tensor of %d entries" % n)
    return t.data_ptr()


def sgiga_net_forward(plan, inp, out):
    n = sgiga_plan_info(plan).ndof
    _check(_lib.sgiga_net_forward(plan, _f32dev(inp, n), _f32dev(out, n)))


def sgiga_net_backward(plan, inp, dy):
    n = sgiga_plan_info(plan).ndof
    g = np.zeros(sgiga_net_num_params(plan), dtype=np.float32)
    _check(_lib.sgiga_net_backward(plan, _f32dev(inp, n), _f32dev(dy, n), g.ctypes.data))
    return g


def sgiga_net_features(plan, out):
    """phi = log c into a float32 buffer [ndof] (CUDA tensor or numpy array)."""
    n = sgiga_plan_info(plan).ndof
    _check(_lib.sgiga_net_features(plan, _ptr(out, n, np.float32)))


def sgiga_net_scaling(plan, out):
    n = sgiga_plan_info(plan).ndof
    _check(_lib.sgiga_net_scaling(plan, _ptr(out, n, np.float32)))


def sgiga_net_set_scaling(plan, S):
    n = sgiga_plan_info(plan).ndof
    _check(_lib.sgiga_net_set_scaling(plan, _ptr(S, n, np.float32)))


def sgiga_net_set_loss_norm(plan, norm):
    _check(_lib.sgiga_net_set_loss_norm(plan, {"euclidean": 0, "energy": 1}.get(norm, norm)))


def sgiga_net_loss_grad(plan, r, e, grad):
    """(loss, fills grad): the training loss of one sample and its gradient
    with respect to log S (float32 CUDA tensors [ndof])."""
    n = sgiga_plan_info(plan).ndof
    loss = ctypes.c_double()
    _check(_lib.sgiga_net_loss_grad(plan, _f32dev(r, n), _f32dev(e, n), ctypes.byref(loss), _f32dev(grad, n)))
    return loss.value


def sgiga_train_net(plan, target_pairs=10000, max_iter_record=30, epochs=10, lr=1e-3, seed=100, batch=2,
                    loss="euclidean"):
    cfg = sgiga_train_cfg(int(target_pairs), int(max_iter_record), int(epochs), float(lr), int(seed), int(batch),
                          {"euclidean": 0, "energy": 1}[loss])
    st = sgiga_train_stats()
    _check(_lib.sgiga_train_net(plan, ctypes.byref(cfg), ctypes.byref(st)))
    return st


def sgiga_net_save(plan, path):
    _check(_lib.sgiga_net_save(plan, str(path).encode()))


def sgiga_net_load(plan, path):
    _check(_lib.sgiga_net_load(plan, str(path).encode()))


def sgiga_plan_times(plan):
    """Set-up phase times of the plan (seconds), as a dict."""
    t = sgiga_plan_times_t()
    _check(_lib.sgiga_plan_times(plan, ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in sgiga_plan_times_t._fields_}


def sgiga_launch_count():
    return int(_lib.sgiga_launch_count())


def sgiga_last_error():
    return _lib.sgiga_last_error().decode()


class Plan:
    """Owning handle: a plan plus its metadata (marshalling helper only)."""

    def __init__(self, d, p, w, **kw):
        self.handle = sgiga_plan(d, p, w, **kw)
        self.info = sgiga_plan_info(self.handle)
        self.grids = [sgiga_grid_info(self.handle, g) for g in range(self.info.ngrids)]

    def close(self):
        if self.handle:
            sgiga_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
