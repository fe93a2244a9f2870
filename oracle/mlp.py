"""FP64 reference of the warm-start network (test infrastructure only).

The learned warm start is not part of the paper: it is a small multilayer
perceptron that maps features of a composite-cell problem to a prediction of
its X dual (the Sinkhorn initialisation alpha_init of Alg. 1 / Alg. 4). This
module is the plain CPU definition of that network, its loss and its gradient,
against which the library's BF16/FP32 GPU kernels are checked.

Network: layer widths dims = (d_0, ..., d_L); layer l maps d_{l-1} -> d_l by
z = W_l h + b_l, with W_l of shape (d_l, d_{l-1}) (row n holds the weights into
output n); hidden layers apply SiLU(z) = z / (1 + exp(-z)), the output layer is
linear.

Loss over a batch of B rows: L = (1 / B) sum_b sum_j w_j (y_bj - t_bj)^2 with
per-output weights w_j.

Parameters are one flat vector: W_1 (row-major), b_1, W_2, b_2, ...
"""

from __future__ import annotations

import numpy as np

DIMS = (336, 256, 256, 256, 320)


def n_params(dims=DIMS) -> int:
    return sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(len(dims) - 1))


def unflatten(p, dims=DIMS):
    out, o = [], 0
    for l in range(len(dims) - 1):
        k, n = dims[l], dims[l + 1]
        W = p[o:o + n * k].reshape(n, k)
        o += n * k
        b = p[o:o + n]
        o += n
        out.append((W, b))
    assert o == len(p)
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    """d/dz [z sigma(z)] = sigma(z) (1 + z (1 - sigma(z)))."""
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, X, dims=DIMS):
    """Outputs (B, d_L) and the per-layer inputs / pre-activations."""
    layers = unflatten(np.asarray(p, dtype=np.float64), dims)
    h = np.asarray(X, dtype=np.float64)
    hs, zs = [], []
    for l, (W, b) in enumerate(layers):
        hs.append(h)
        z = h @ W.T + b
        zs.append(z)
        h = silu(z) if l < len(layers) - 1 else z
    return h, (hs, zs)


def loss(p, X, T, w, dims=DIMS) -> float:
    y, _ = forward(p, X, dims)
    return float(np.sum(w[None, :] * (y - T) ** 2) / X.shape[0])


def loss_and_grad(p, X, T, w, dims=DIMS):
    """Loss and its gradient with respect to the flat parameters (backpropagation)."""
    layers = unflatten(np.asarray(p, dtype=np.float64), dims)
    y, (hs, zs) = forward(p, X, dims)
    B = X.shape[0]
    L = float(np.sum(w[None, :] * (y - T) ** 2) / B)
    g = 2.0 * w[None, :] * (y - T) / B          # dL/dz of the output layer
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = (g.T @ hs[l], g.sum(axis=0))
        if l > 0:
            g = (g @ W) * silu_grad(zs[l - 1])
    flat = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return L, flat
