"""Learned scaling of the fast-diagonalisation preconditioner: the oracle's
definitions of its features, of the scaled preconditioner and of its training
loss with the loss's gradient.

TEST INFRASTRUCTURE: see the package header. Not in the paper (its
conclusions, Sec. 5, name fast solvers used as preconditioners as future
work); this module is the definition the CUDA library is checked against.

Features. For interior function i of a component, the local effective
coefficient
    c_i = sum_q R_i(xi_q) tr(G_q) / (d sum_q R_i(xi_q) w_q),
    G_q = w_q |det J_q| a(x_q) (J_q^T J_q)^{-1},
the R_i-weighted mean of the trace of the Galerkin integrand's metric over
the support of R_i, relative to the parametric Laplacian (G_q = w_q I), the
operator the fast-diagonalisation preconditioner inverts. The network input
is log c_i.

Scaled preconditioner. With a positive scaling S (one value per DoF, from the
network's output y and the feature phi = log c as
S = exp(-phi / 2 + 4 tanh(y / 4)): the network corrects the network-free
scaling c^(-1/2) by a factor within e^(+-4)),
M(r) = S * FD(S * r), elementwise products: symmetric positive definite
whenever FD is.

Loss of one (residual, error) pair of one component:
    L = ||M(r) - e||^2 / ||e||^2,
or in the component's energy norm (M(r) - e)^T K (M(r) - e) / e^T K e, and
with several components the mean over them. Its gradient with respect to
log S_i (FD symmetric):
    dL/dlog S_i = S_i (delta_i FD(S r)_i + r_i FD(S delta)_i),
    delta = 2 (M(r) - e) / ||e||^2.
"""
import numpy as np

from . import fd


def scaling_from_output(y, phi=0.0):
    """S = exp(-phi / 2 + 4 tanh(y / 4)) of the network output y at the
    feature phi = log c."""
    y = np.asarray(y, dtype=np.float64)
    return np.exp(-0.5 * np.asarray(phi, dtype=np.float64) + 4.0 * np.tanh(y / 4.0))


def features(comp, diffusion=None):
    """c_i of every interior function of an assembled-geometry component
    (galerkin.Component), in packed order."""
    d = comp.d
    num = np.zeros(comp.nfull)
    den = np.zeros(comp.nfull)
    for em in comp._element_batches(512):
        val, _, Xi, W, loc = comp._element_data(em)
        nb, nq = W.shape
        J = comp.geom.jacobian(Xi).reshape(nb, nq, d, d)
        det = np.abs(np.linalg.det(J))
        JtJinv = np.linalg.inv(np.einsum("eqik,eqil->eqkl", J, J))
        tr = np.trace(JtJinv, axis1=2, axis2=3) * det
        if diffusion is not None:
            tr = tr * diffusion(comp.geom.map(Xi)).reshape(nb, nq)
        np.add.at(num, loc.reshape(-1), np.einsum("eqA,eq->eA", val, W * tr).reshape(-1))
        np.add.at(den, loc.reshape(-1), np.einsum("eqA,eq->eA", val, d * W).reshape(-1))
    return (num / den)[comp.interior]


def scaled_fd(levels, p, r, S, rvec, geom=None):
    """M(r) = S * FD(S * r) for one component."""
    S = np.asarray(S, dtype=np.float64)
    return S * fd.fd_apply(levels, p, r, S * np.asarray(rvec, dtype=np.float64), geom=geom)


def pair_loss_grad(levels, p, r, S, rvec, evec, geom=None, K=None):
    """(L, dL/dlog S) of one pair of one component. With the component's
    stiffness K the loss is in its energy norm,
        L = (M(r) - e)^T K (M(r) - e) / e^T K e,
    and delta = 2 K (M(r) - e) / e^T K e (K symmetric)."""
    S = np.asarray(S, dtype=np.float64)
    rvec = np.asarray(rvec, dtype=np.float64)
    evec = np.asarray(evec, dtype=np.float64)
    z1 = fd.fd_apply(levels, p, r, S * rvec, geom=geom)
    m = S * z1
    res = m - evec
    if K is None:
        ee = float(evec @ evec)
        L = float(res @ res) / ee
        delta = 2.0 * res / ee
    else:
        ee = float(evec @ (K @ evec))
        Kres = K @ res
        L = float(res @ Kres) / ee
        delta = 2.0 * Kres / ee
    z2 = fd.fd_apply(levels, p, r, S * delta, geom=geom)
    return L, S * (delta * z1 + rvec * z2)


def packed_loss_grad(grids, p, r, S, rvec, evec, geom=None, Ks=None):
    """Mean loss over the components of packed vectors, and its gradient.

    grids: per component (levels, dof_off, ndof); Ks: per component its
    stiffness matrix (energy-norm loss), or None (Euclidean)."""
    S = np.asarray(S, dtype=np.float64)
    grad = np.zeros_like(S)
    tot = 0.0
    for gi, (levels, off, n) in enumerate(grids):
        sl = slice(off, off + n)
        L, g = pair_loss_grad(levels, p, r, S[sl], rvec[sl], evec[sl], geom=geom,
                              K=None if Ks is None else Ks[gi])
        tot += L
        grad[sl] = g
    return tot / len(grids), grad / len(grids)
