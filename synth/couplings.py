"""Initial couplings for the iteration, as inputs.

A coupling is returned as three flat arrays (x index, y index, mass) with
x = p * N2 + q for pixel (p, q). `boxes_from_coupling` converts it to the
basic-cell state both sides read: for each basic cell X_i (an s x s pixel
block, index i = (p // s) * (N2 // s) + q // s) the Y-marginal of the coupling
restricted to X_i x Y (Eq. basic-cell-Y-marginal), stored on its bounding box
as (o1, o2, dense float64 array).
"""

from __future__ import annotations

import numpy as np


def _monotone_1d(p: np.ndarray, q: np.ndarray):
    """North-west-corner (monotone) coupling of two 1-D histograms.

    Returns (i, j, mass) with sum_j mass = p[i], sum_i mass = q[j]. q is
    rescaled to the total of p first.
    """
    P = np.concatenate([[0.0], np.cumsum(p)])
    Q = np.concatenate([[0.0], np.cumsum(q)])
    Q *= P[-1] / Q[-1]
    Q[-1] = P[-1]
    br = np.unique(np.concatenate([P, Q]))
    m = np.diff(br)
    mid = 0.5 * (br[:-1] + br[1:])
    i = np.searchsorted(P, mid, side="right") - 1
    j = np.searchsorted(Q, mid, side="right") - 1
    ok = (m > 0) & (i >= 0) & (i < len(p)) & (j >= 0) & (j < len(q))
    return i[ok], j[ok], m[ok]


def knothe_rosenblatt(mu: np.ndarray, nu: np.ndarray):
    """Discrete Knothe-Rosenblatt coupling of two grid measures.

    The axis-1 marginals are coupled monotonically; for every coupled pair of
    rows (p, p') with mass m, the conditional axis-2 distributions
    mu[p, :] / mu_row[p] and nu[p', :] / nu_row[p'] are coupled monotonically
    with total mass m. Exactly feasible up to float64 rounding.
    """
    N1, N2 = mu.shape
    mr = mu.sum(axis=1)
    nr = nu.sum(axis=1)
    pi, pj, pm = _monotone_1d(mr, nr)
    xs, ys, ms = [], [], []
    for a, b, m in zip(pi, pj, pm):
        ca = mu[a] * (m / mr[a])
        cb = nu[b] * (m / nr[b])
        qi, qj, qm = _monotone_1d(ca, cb)
        xs.append(a * N2 + qi)
        ys.append(b * N2 + qj)
        ms.append(qm)
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(ms)


def product_coupling(mu: np.ndarray, nu: np.ndarray):
    """mu (x) nu as a flat (x, y, mass) list (only for small grids)."""
    n = mu.size
    x = np.repeat(np.arange(n), n)
    y = np.tile(np.arange(n), n)
    return x, y, (mu.reshape(-1)[:, None] * nu.reshape(-1)[None, :]).reshape(-1)


def rotation_coupling(mu: np.ndarray):
    """(id, T0)_# mu for the quarter turn T0 of Eq. (T0) on the pixel grid."""
    N = mu.shape[0]
    p, q = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    # (x1, x2) -> (-x2, x1): pixel (p, q) -> (N - 1 - q, p)
    y = (N - 1 - q) * N + p
    return (p * N + q).reshape(-1), y.reshape(-1), mu.reshape(-1).copy()


def boxes_from_coupling(shape, s: int, x, y, mass):
    """Basic-cell Y-marginals of a sparse coupling, on their bounding boxes."""
    N1, N2 = shape
    n2 = N2 // s
    px, qx = np.divmod(x, N2)
    cell = (px // s) * n2 + (qx // s)
    py, qy = np.divmod(y, N2)
    order = np.argsort(cell, kind="stable")
    cell, py, qy, mass = cell[order], py[order], qy[order], mass[order]
    nb = (N1 // s) * n2
    starts = np.searchsorted(cell, np.arange(nb + 1))
    boxes = []
    for i in range(nb):
        a, b = starts[i], starts[i + 1]
        r, c, m = py[a:b], qy[a:b], mass[a:b]
        keep = m > 0
        r, c, m = r[keep], c[keep], m[keep]
        o1, o2 = int(r.min()), int(c.min())
        arr = np.zeros((int(r.max()) - o1 + 1, int(c.max()) - o2 + 1))
        np.add.at(arr, (r - o1, c - o2), m)
        boxes.append((o1, o2, arr))
    return boxes
