"""Cell-LSE microbenchmark inputs: independent cells with an m x m box each.

The paper measures its cell solver alone on batches of independent problems of
one box size (Appendix A, Fig. 10). Here the same setting is embedded in a grid
problem the library takes as it is: on an N x N grid with N = 16384 / m and
4 x 4 basic cells, every A-cell (2 x 2 basic cells, an 8 x 8 X block) gets its
own m x m box, placed over the block and clipped to the grid, holding a seeded
random Gaussian (centre within m/8 of the box centre, per-axis sigma in
[m/8, m/4], floor 1e-3 of the peak) normalised to the block's mass; its four
members share it equally. nu is the sum of the boxes, so the plan is feasible
exactly. There are (2048 / m)^2 A-cells and the boxes cover 2048^2 pixels in
all, the cell counts of a 2048 x 2048 batch tiled by m x m boxes.

mu is uniform, eps = 2 h^2 (h = 1 / N). No arithmetic of the method is here:
only the data (measures and the initial basic-cell boxes).
"""

from __future__ import annotations

import numpy as np

SIDES = (8, 16, 32, 64, 128)


def cell_lse_sweep(m: int, seed: int = 0):
    """Return (mu, nu, eps, s, (hdr, data)) for box side m (a power of two, 8..128).

    hdr: (nbasic, 4) int32 rows (o1, o2, h, w) in row-major basic-cell order;
    data: the boxes' values, row-major, concatenated in the same order (float64).
    """
    if m not in SIDES:
        raise ValueError("box side must be one of %s" % (SIDES,))
    s = 4
    N = 16384 // m
    nA = N // (2 * s)
    rng = np.random.default_rng(seed)
    mu = np.full((N, N), 1.0 / (N * N))
    o = np.clip(2 * s * np.arange(nA) + s - m // 2, 0, N - m)
    ctr = (m - 1) / 2.0 + rng.uniform(-m / 8.0, m / 8.0, size=(nA, nA, 2))
    sig = rng.uniform(m / 8.0, m / 4.0, size=(nA, nA, 2))
    y = np.arange(m, dtype=np.float64)
    g1 = np.exp(-0.5 * ((y[None, None, :] - ctr[..., 0:1]) / sig[..., 0:1]) ** 2)  # (nA, nA, m)
    g2 = np.exp(-0.5 * ((y[None, None, :] - ctr[..., 1:2]) / sig[..., 1:2]) ** 2)
    g = g1[..., :, None] * g2[..., None, :] + 1e-3
    g *= (4.0 * s * s / (N * N)) / g.sum(axis=(2, 3), keepdims=True)  # mass of the 8 x 8 block
    nu = np.zeros((N, N))
    for a in range(nA):
        for b in range(nA):
            nu[o[a]:o[a] + m, o[b]:o[b] + m] += g[a, b]
    n = N // s
    q = g / 4.0
    data = np.repeat(np.repeat(q, 2, axis=0), 2, axis=1).reshape(-1)  # basic cell (r, c) -> A-cell (r//2, c//2)
    r = np.arange(n)
    hdr = np.zeros((n, n, 4), dtype=np.int32)
    hdr[..., 0] = o[r // 2][:, None]
    hdr[..., 1] = o[r // 2][None, :]
    hdr[..., 2] = m
    hdr[..., 3] = m
    return mu, nu, 2.0 / (N * N), s, (hdr.reshape(-1, 4), data)
