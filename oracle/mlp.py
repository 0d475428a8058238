"""Oracle: node-wise MLP for the learned CG initial guess (TEST INFRASTRUCTURE ONLY).

The paper has no learned component; this restates, in plain FP64 NumPy, the
network the CUDA library trains and evaluates (a fully connected net with tanh
hidden layers and a linear output, mean-squared-error loss, Adam) so that the
GPU forward pass, gradients and parameter updates can be checked.

Parameter layout (shared convention, not code): for layer l with fan-in a and
fan-out b, W_l is stored row-major [a, b] followed by the bias [b]; layers
are concatenated in order.  Inputs are standardised with (x - shift) * scale
before the first layer and outputs are multiplied by out_scale after the last.

Parity status: pinned (central finite differences of the loss for every
parameter block; Adam's first step equals lr * sign(g) by its definition).
"""
from __future__ import annotations

import numpy as np


def layer_shapes(n_in, width, depth, n_out):
    dims = [n_in] + [width] * depth + [n_out]
    return [(dims[i], dims[i + 1]) for i in range(len(dims) - 1)]


def unpack(theta, shapes):
    out, o = [], 0
    for a, b in shapes:
        W = theta[o:o + a * b].reshape(a, b)
        o += a * b
        bias = theta[o:o + b]
        o += b
        out.append((W, bias))
    return out


def forward(theta, shapes, X, shift, scale, out_scale):
    """Returns (Y, cache) with Y = out_scale * (last linear layer)."""
    h = (X - shift) * scale
    cache = [h]
    layers = unpack(theta, shapes)
    for li, (W, b) in enumerate(layers):
        z = h @ W + b
        h = z if li == len(layers) - 1 else np.tanh(z)
        cache.append(h)
    return h * out_scale, cache


def loss_and_grad(theta, shapes, X, Y, shift, scale, out_scale):
    """Mean over samples and outputs of (pred - Y)^2 and its gradient."""
    pred, cache = forward(theta, shapes, X, shift, scale, out_scale)
    n, m = Y.shape
    diff = pred - Y
    loss = float((diff ** 2).sum() / (n * m))
    layers = unpack(theta, shapes)
    grads = [None] * len(layers)
    d = 2.0 * diff / (n * m) * out_scale          # dL/d(last linear output)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        h_in = cache[li]
        grads[li] = (h_in.T @ d, d.sum(axis=0))
        if li > 0:
            d = (d @ W.T) * (1.0 - cache[li] ** 2)  # tanh' = 1 - tanh^2
    g = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, g


def node_features(coords, cells, T=None, dist=None):
    """Features [n, 8]: x, y, z, T, grad T, dist.

    grad T at a node is the volume-weighted mean over its cells of grad T_h at
    the cell centroid, where T_h is the interpolant in the cell's Lagrange
    space (P1 or P2); evaluated generically from the barycentric basis
    polynomials of oracle.fem.
    """
    from fractions import Fraction

    from . import fem
    n = coords.shape[0]
    F = np.zeros((n, 8))
    F[:, :3] = coords
    if T is None:
        return F
    F[:, 3] = T
    degree = 1 if cells.shape[1] == 4 else 2
    phi = fem.basis_polys(degree)
    lam = (Fraction(1, 4),) * 4
    # d phi_c / d lambda_k at the centroid
    dphi = np.array([[float(sum(c * e[k] * np.prod([lam[q] ** (e[q] - (q == k)) for q in range(4)])
                                for e, c in p.items() if e[k] > 0)) for k in range(4)] for p in phi])
    G, vol = fem.barycentric_gradients(coords[cells[:, :4]])
    grad = np.einsum("ec,ck,ekd->ed", T[cells], dphi, G)       # [cells, 3]
    gsum = np.zeros((n, 3))
    wsum = np.zeros(n)
    for a in range(cells.shape[1]):
        np.add.at(gsum, cells[:, a], vol[:, None] * grad)
        np.add.at(wsum, cells[:, a], vol)
    F[:, 4:7] = gsum / np.where(wsum > 0, wsum, 1.0)[:, None]
    if dist is not None:
        F[:, 7] = dist
    return F


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); t counts from 1."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
