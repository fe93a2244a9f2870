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


def rotation_contraction_coupling(mu: np.ndarray, theta_deg: float):
    """(id, T)_# mu for T(x) = c R_theta x on [-1, 1]^2, with the contraction
    c = 1 / (cos theta + sin theta) that makes the rotated square fit into
    [-1, 1]^2 (the initial plan and target of Section 5.3). On the pixel grid
    each pixel's mass goes to the four pixels around T(its centre) with bilinear
    weights (indices clipped to the grid), so nu is by construction the exact
    second marginal of the returned coupling.

    Returns (x index, y index, mass, nu) with nu an (N, N) array summing to 1.
    """
    N = mu.shape[0]
    th = np.deg2rad(theta_deg)
    c = 1.0 / (abs(np.cos(th)) + abs(np.sin(th)))
    t = 2.0 * (np.arange(N) + 0.5) / N - 1.0
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    Y1 = c * (np.cos(th) * X1 - np.sin(th) * X2)
    Y2 = c * (np.sin(th) * X1 + np.cos(th) * X2)
    # continuous pixel coordinates of the image points
    q1 = (Y1 + 1.0) * N / 2.0 - 0.5
    q2 = (Y2 + 1.0) * N / 2.0 - 0.5
    f1, f2 = np.floor(q1), np.floor(q2)
    w1, w2 = q1 - f1, q2 - f2
    xs, ys, ms = [], [], []
    xi = (np.arange(N)[:, None] * N + np.arange(N)[None, :]).reshape(-1)
    m = mu.reshape(-1)
    for d1, a1 in ((0, 1.0 - w1), (1, w1)):
        for d2, a2 in ((0, 1.0 - w2), (1, w2)):
            r = np.clip(f1 + d1, 0, N - 1).astype(np.int64).reshape(-1)
            k = np.clip(f2 + d2, 0, N - 1).astype(np.int64).reshape(-1)
            wt = (a1 * a2).reshape(-1) * m
            ok = wt > 0
            xs.append(xi[ok])
            ys.append((r * N + k)[ok])
            ms.append(wt[ok])
    x, y, mass = np.concatenate(xs), np.concatenate(ys), np.concatenate(ms)
    nu = np.bincount(y, weights=mass, minlength=N * N).reshape(N, N)
    return x, y, mass, nu


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


def coarsen(a: np.ndarray) -> np.ndarray:
    """2 x 2 pixel sums (a measure on an N x N grid -> N/2 x N/2)."""
    n1, n2 = a.shape
    return a.reshape(n1 // 2, 2, n2 // 2, 2).sum(axis=(1, 3))


def prolongate(boxes_c, mu, nu, s: int, noise: float = 0.01, seed: int = 0, tol: float = 1e-13,
               max_sweeps: int = 500, trunc: float = 0.0, rebalance: str = "project"):
    """A fine initial plan from a coarse one (input recipe of the large 1024 x 1024
    configuration). boxes_c: basic-cell Y-marginals [(o1, o2, array)] of a plan
    for the 2 x 2-coarsened measures (coarsen(mu), coarsen(nu)) with the same
    cell size s; mu, nu the fine measures. Parent basic cell i -> its 4 children
    i' and coarse pixel y -> its 4 fine pixels y':
        nu_i'(y') = (m_i' / m_i) nu_i(parent(y')) nu(y') / coarsen(nu)(parent(y')),
    which has both fine marginals exactly; then 1 % seeded multiplicative noise
    (u ~ U[-1, 1]) and a rebalancing to the exact marginals:
      * rebalance="project" (default): within each (parent cell, coarse pixel)
        block of 4 children x 4 fine pixels the base plan is a (x) b
        (a_k = share of child k, b_q = share of fine pixel q); the noise is
        entry-wise base * noise * u~ with u~ = u minus its b-weighted row means
        and a-weighted column means (plus the joint mean), which has zero row and
        column sums in every block: both marginals stay exact in exact
        arithmetic (float64 rounding only) and every entry stays within
        (1 +- 4 noise) of its base value;
      * rebalance="ipf": entries times (1 + noise u), then iterative proportional
        fitting on that support (rows: basic masses m_i', columns: nu) until both
        L1 errors are below tol or max_sweeps sweeps.
    Optionally the entries below `trunc` are dropped and the rows scaled back to
    m_i' (the dropped mass then shows in the Y error). Returns [(o1, o2, array)]
    on minimal boxes."""
    rng = np.random.default_rng(seed)
    N1, N2 = mu.shape
    n2 = N2 // s
    nc2 = (N2 // 2) // s
    m = mu.reshape(N1 // s, s, n2, s).sum(axis=(1, 3)).reshape(-1)
    nuc = coarsen(nu)
    # blocks: one per (parent cell, coarse pixel with mass); children k (4) x fine pixels q (4)
    blk_cell, blk_pix, blk_val = [], [], []
    for ic, (o1, o2, a) in enumerate(boxes_c):
        a = np.asarray(a, dtype=np.float64)
        if a.size == 0:
            continue
        bi, bj = divmod(ic, nc2)
        mi = m.reshape(N1 // s, n2)[2 * bi:2 * bi + 2, 2 * bj:2 * bj + 2].reshape(-1)
        kids = np.array([(2 * bi + di) * n2 + 2 * bj + dj for di in (0, 1) for dj in (0, 1)])
        r, c = np.nonzero(a > 0)
        if r.size == 0:
            continue
        Y1, Y2 = 2 * (o1 + r), 2 * (o2 + c)
        fr = np.stack([Y1, Y1, Y1 + 1, Y1 + 1], axis=1)          # fine pixels q of each coarse pixel
        fc = np.stack([Y2, Y2 + 1, Y2, Y2 + 1], axis=1)
        share = nu[fr, fc] / nuc[o1 + r, o2 + c][:, None]          # b_q
        ak = mi / mi.sum()                                         # a_k
        base = a[r, c][:, None, None] * ak[None, :, None] * share[:, None, :]
        blk_cell.append(np.broadcast_to(kids[None, :, None], base.shape))
        blk_pix.append(np.broadcast_to((fr * N2 + fc)[:, None, :], base.shape))
        blk_val.append(base)
    base = np.concatenate(blk_val)                                 # (nblk, 4, 4)
    cell_b = np.concatenate(blk_cell)
    pix_b = np.concatenate(blk_pix)
    u = rng.uniform(-1.0, 1.0, size=base.shape)
    nuf = nu.reshape(-1)
    if rebalance == "project":
        tot = base.sum(axis=(1, 2), keepdims=True)
        ak = base.sum(axis=2, keepdims=True) / tot                 # (nblk, 4, 1)
        bq = base.sum(axis=1, keepdims=True) / tot                 # (nblk, 1, 4)
        ut = u - (u * bq).sum(axis=2, keepdims=True) - (ak * u).sum(axis=1, keepdims=True) \
            + (ak * u * bq).sum(axis=(1, 2), keepdims=True)
        val3 = base * (1.0 + noise * ut)
        cell, pix, val = cell_b.reshape(-1), pix_b.reshape(-1), val3.reshape(-1)
    elif rebalance == "ipf":
        cell, pix = cell_b.reshape(-1), pix_b.reshape(-1)
        val = (base * (1.0 + noise * u)).reshape(-1)
        for _ in range(max_sweeps):
            rs = np.bincount(cell, weights=val, minlength=len(m))
            val *= (m / rs)[cell]
            cs = np.bincount(pix, weights=val, minlength=nuf.size)
            ex = np.abs(rs - m).sum()
            val *= np.where(cs > 0, nuf / np.where(cs > 0, cs, 1.0), 1.0)[pix]
            rs2 = np.bincount(cell, weights=val, minlength=len(m))
            if np.abs(rs2 - m).sum() < tol and ex < tol:
                break
    else:
        raise ValueError("rebalance must be 'project' or 'ipf'")
    keep = val > 0
    cell, pix, val = cell[keep], pix[keep], val[keep]
    # drop entries below trunc, then the rows back to their masses (the dropped
    # mass, <= trunc per entry, goes to the Y error)
    if trunc > 0.0:
        val[val < trunc] = 0.0
        rs = np.bincount(cell, weights=val, minlength=len(m))
        val *= np.where(rs > 0, m / np.where(rs > 0, rs, 1.0), 0.0)[cell]
    out = []
    order = np.argsort(cell, kind="stable")
    cell, pix, val = cell[order], pix[order], val[order]
    starts = np.searchsorted(cell, np.arange(len(m) + 1))
    for c in range(len(m)):
        sl = slice(starts[c], starts[c + 1])
        p, v = pix[sl], val[sl]
        nz = v > 0
        p, v = p[nz], v[nz]
        if p.size == 0:
            out.append((0, 0, np.zeros((0, 0))))
            continue
        r, q = p // N2, p % N2
        o1, o2 = int(r.min()), int(q.min())
        arr = np.zeros((int(r.max()) - o1 + 1, int(q.max()) - o2 + 1))
        np.add.at(arr, (r - o1, q - o2), v)
        out.append((o1, o2, arr))
    return out
