"""Network of the learned preconditioner scaling: plain FP64 forward and backward.

TEST INFRASTRUCTURE: see the package header. Not in the paper (it is the
CUDA library's learned scaling of its preconditioner, see oracle.learned);
this module is the definition its kernels are checked against.

N(x) on each component's DoF tensor (shape (n_d, .., n_1), direction 1
fastest in the packed vector), zero padding, channels 1 -> 32 -> 32 -> 1
(input: the log of the local effective coefficient; output: log S):
    Z1 = conv(x, W1) + b1,  A1 = relu(Z1)
    Z2 = conv(A1, W2) + b2, A2 = relu(Z2)
    Y  = conv(A2, W3) + b3
conv(X, W)[co][v] = sum_{ci, t} W[co][ci][t] X[ci][v + offset(t)], offsets in
{-1, 0, 1}^d with the offset of direction 1 varying fastest over t.
Parameters are one vector: W1 [32][1][T], b1 [32], W2 [32][32][T], b2 [32],
W3 [1][32][T], b3 [1] (T = 3^d).
"""
import itertools

import numpy as np

CIN = (1, 32, 32)
COUT = (32, 32, 1)


def offsets(d):
    """Tap offsets (direction 1 first in each tuple), tap index fastest in direction 1."""
    out = []
    for t in itertools.product((-1, 0, 1), repeat=d):
        out.append(tuple(reversed(t)))          # product varies the last slot fastest
    return out


def unpack(params, d):
    T = 3 ** d
    p = np.asarray(params, dtype=np.float64)
    layers, o = [], 0
    for ci, co in zip(CIN, COUT):
        W = p[o:o + co * ci * T].reshape(co, ci, T)
        o += co * ci * T
        b = p[o:o + co]
        o += co
        layers.append((W, b))
    assert o == p.size
    return layers


def _shift(X, off):
    """Y[v] = X[v + off] with zeros outside; X has shape (C, n_d, .., n_1); off
    is (o_1, .., o_d) with o_1 for the last axis."""
    d = len(off)
    Y = np.zeros_like(X)
    src, dst = [slice(None)], [slice(None)]
    for k in range(d):
        o = off[k]
        ax_len = X.shape[X.ndim - 1 - k]
        if o >= 0:
            s, t = slice(o, ax_len), slice(0, ax_len - o)
        else:
            s, t = slice(0, ax_len + o), slice(-o, ax_len)
        src.insert(1, s)
        dst.insert(1, t)
    Y[tuple(dst)] = X[tuple(src)]
    return Y


def conv(X, W, b=None):
    """X (Cin, *shape) -> (Cout, *shape)."""
    d = X.ndim - 1
    offs = offsets(d)
    Y = np.zeros((W.shape[0],) + X.shape[1:])
    for t, off in enumerate(offs):
        Y += np.tensordot(W[:, :, t], _shift(X, off), axes=([1], [0]))
    if b is not None:
        Y += b.reshape((-1,) + (1,) * d)
    return Y


def conv_input_grad(dY, W):
    """Gradient of sum(dY * conv(X, W)) with respect to X."""
    d = dY.ndim - 1
    dX = np.zeros((W.shape[1],) + dY.shape[1:])
    for t, off in enumerate(offsets(d)):
        neg = tuple(-o for o in off)
        dX += _shift(np.tensordot(W[:, :, t].T, dY, axes=([1], [0])), neg)
    return dX


def conv_weight_grad(dY, X, T):
    """Gradient of sum(dY * conv(X, W)) with respect to W: [Cout][Cin][T]."""
    d = X.ndim - 1
    G = np.zeros((dY.shape[0], X.shape[0], T))
    for t, off in enumerate(offsets(d)):
        G[:, :, t] = np.tensordot(dY, _shift(X, off), axes=(list(range(1, d + 1)), list(range(1, d + 1))))
    return G


def forward(params, x):
    """x: (1, *shape) for one component; returns Y (shape) and the activations."""
    d = x.ndim - 1
    (W1, b1), (W2, b2), (W3, b3) = unpack(params, d)
    A1 = np.maximum(conv(x, W1, b1), 0.0)
    A2 = np.maximum(conv(A1, W2, b2), 0.0)
    Y = conv(A2, W3, b3)
    return Y[0], (x, A1, A2)


def backward(params, x, dy):
    """Gradient of sum(dy * N(x)) with respect to the parameter vector."""
    d = x.ndim - 1
    T = 3 ** d
    (W1, b1), (W2, b2), (W3, b3) = unpack(params, d)
    _, (A0, A1, A2) = forward(params, x)
    dY = dy[None]
    gW3 = conv_weight_grad(dY, A2, T)
    gb3 = dY.reshape(1, -1).sum(axis=1)
    dA2 = conv_input_grad(dY, W3) * (A2 > 0)
    gW2 = conv_weight_grad(dA2, A1, T)
    gb2 = dA2.reshape(32, -1).sum(axis=1)
    dA1 = conv_input_grad(dA2, W2) * (A1 > 0)
    gW1 = conv_weight_grad(dA1, A0, T)
    gb1 = dA1.reshape(32, -1).sum(axis=1)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def split_packed(vec, shapes, nch=None):
    """Packed vector(s) of all components -> list of per-component tensors.

    shapes: per component (n_1, .., n_d); vec: (C, ndof) or (ndof,)."""
    out, o = [], 0
    v = np.asarray(vec)
    for sh in shapes:
        n = int(np.prod(sh))
        if v.ndim == 2:
            out.append(v[:, o:o + n].reshape((v.shape[0],) + tuple(reversed(sh))))
        else:
            out.append(v[o:o + n].reshape(tuple(reversed(sh))))
        o += n
    return out
