"""Learned surrogate of the compressed Bloch model: a small MLP and its Sobolev loss.

The paper names surrogate models as a remedy for the cost of the partial-derivative
computations (Discussion).  The surrogate maps tissue parameters to the coefficients of
the echo time course in a fixed time basis U (see model.project_onto_basis):

    u = ((ln T1 - mu1) / s1, (ln T2 - mu2) / s2, (B1 - mu3) / s3)
    a1 = tanh(W1 u + b1), a2 = tanh(W2 a1 + b2), a3 = tanh(W3 a2 + b3)
    c  = scale * (W4 a3 + b4)                        (R coefficients)

and its derivatives dc/dln T1, dc/dln T2 come from forward-mode tangents through the
same layers (the tangent of u along ln T1 is (1/s1, 0, 0), along ln T2 (0, 1/s2, 0);
a tanh layer maps a tangent t to (1 - a^2) * (W t)).  Training minimises the Sobolev
loss

    L = 1/B sum_b sum_r [ (c - c*)^2 + lam ((dc1 - dc1*)^2 + (dc2 - dc2*)^2) ] / scale_r^2

against projected simulations (c* = U^T m_y, dc*_k = U^T dm_y/dln T_k).  Everything
here is float64 NumPy with a hand-written backward pass, pinned by central
differences in tests/test_oracle_surrogate.py.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(hidden: int, rank: int):
    return [(hidden, 3), (hidden, hidden), (hidden, hidden), (rank, hidden)]


def num_params(hidden: int, rank: int) -> int:
    return sum(o * i + o for o, i in layer_shapes(hidden, rank))


def unpack(theta, hidden, rank):
    """Flat parameter vector -> [(W, b), ...] in the layout W_l (row-major [out][in]) then b_l."""
    out, k = [], 0
    for o, i in layer_shapes(hidden, rank):
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def forward(theta, x, norm, scale, hidden, rank):
    """x: [3, B] (ln T1, ln T2, B1). Returns (c, dc1, dc2) each [R, B] and the cache."""
    layers = unpack(np.asarray(theta, np.float64), hidden, rank)
    mu = np.array([norm[0], norm[2], norm[4]])[:, None]
    sd = np.array([norm[1], norm[3], norm[5]])[:, None]
    u = (np.asarray(x, np.float64) - mu) / sd
    B = u.shape[1]
    t1 = np.zeros_like(u)
    t1[0] = 1.0 / sd[0, 0]
    t2 = np.zeros_like(u)
    t2[1] = 1.0 / sd[1, 0]
    cache = []
    a, s1, s2 = u, t1, t2
    for li, (W, b) in enumerate(layers):
        z = W @ a + b[:, None]
        zt1 = W @ s1
        zt2 = W @ s2
        cache.append((a, s1, s2, z, zt1, zt2))
        if li < len(layers) - 1:
            a = np.tanh(z)
            d = 1.0 - a * a
            s1, s2 = d * zt1, d * zt2
        else:
            a, s1, s2 = z, zt1, zt2
    sc = np.asarray(scale, np.float64)[:, None]
    return sc * a, sc * s1, sc * s2, cache


def loss(theta, x, target, norm, scale, hidden, rank, lam):
    """Sobolev loss; target = (c*, dc1*, dc2*) each [R, B]."""
    c, d1, d2, _ = forward(theta, x, norm, scale, hidden, rank)
    sc = np.asarray(scale, np.float64)[:, None]
    B = c.shape[1]
    r0 = (c - target[0]) / sc
    r1 = (d1 - target[1]) / sc
    r2 = (d2 - target[2]) / sc
    return float((np.sum(r0 * r0) + lam * (np.sum(r1 * r1) + np.sum(r2 * r2))) / B)


def loss_grad(theta, x, target, norm, scale, hidden, rank, lam):
    """(loss, dloss/dtheta) by the chain rule through values and tangents."""
    theta = np.asarray(theta, np.float64)
    layers = unpack(theta, hidden, rank)
    c, d1, d2, cache = forward(theta, x, norm, scale, hidden, rank)
    sc = np.asarray(scale, np.float64)[:, None]
    B = c.shape[1]
    r0 = (c - target[0]) / sc
    r1 = (d1 - target[1]) / sc
    r2 = (d2 - target[2]) / sc
    L = float((np.sum(r0 * r0) + lam * (np.sum(r1 * r1) + np.sum(r2 * r2))) / B)
    # gradients w.r.t. the last layer's pre-scale outputs
    ga = 2.0 * r0 / B          # d/d(c / sc) * 1 / sc * sc
    gs1 = 2.0 * lam * r1 / B
    gs2 = 2.0 * lam * r2 / B
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        a_in, s1_in, s2_in, z, zt1, zt2 = cache[li]
        if li == len(layers) - 1:
            gz, gzt1, gzt2 = ga, gs1, gs2
        else:
            a = np.tanh(z)
            d = 1.0 - a * a
            gzt1 = gs1 * d
            gzt2 = gs2 * d
            # s_k = d * zt_k with d = 1 - tanh(z)^2: dd/dz = -2 a d
            gd = gs1 * zt1 + gs2 * zt2
            gz = (ga + gd * (-2.0 * a)) * d
        gW = gz @ a_in.T + gzt1 @ s1_in.T + gzt2 @ s2_in.T
        gb = gz.sum(axis=1)
        grads.append((gW, gb))
        ga = W.T @ gz
        gs1 = W.T @ gzt1
        gs2 = W.T @ gzt2
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return L, flat
