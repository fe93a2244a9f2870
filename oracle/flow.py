"""The flow update (Section 3.2) on the basic-cell box state.

Edge candidates are product gluing candidates (Def. 3.7 with gamma_ij the
product coupling, Remark 3.8): pi_hat_ij = mu_j/m_j (x) nu_i/m_i for j != i, and
pi_hat_ii = pi_i/m_i (Def. 3.4). The edge cost Eq. (edge-cost) is then

    c_bar_ij = <c, mu_j/m_j (x) nu_i/m_i> - <c, pi_i> / m_i   (j != i),
    c_bar_ii = 0,

evaluated here as the explicit double sum over X_j x box(nu_i). <c, pi_i> = D_i
comes from the latest half-iteration. The min-cost flow Eq. (MinCostFlow) over
the mass-preserving flows of Eq. (div-constraint-single-cell) is solved as a
linear program by scipy's HiGHS (a library LP solver standing in for the
paper's OR-tools), and the new basic-cell Y-marginals follow
Eq. (flow-update-cell-marginals): nu_hat_j = sum_{i in N(j)} w_ij nu_i / m_i,
truncated, re-boxed and rescaled to m_j like the half-iteration output.

Reading: the min-cost flow is solved over the reals (the paper does not say how
it scaled masses for an integer solver).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog

from .cell import sq_cost
from .domdec import Box, box_pixels, embed, truncate_box, union_header


def edge_costs(geom, mu, boxes, D, hgrid) -> np.ndarray:
    """c_bar (nb, 5) in the neighbour order of Geometry.neighbours(); NaN where no edge."""
    nbr = geom.neighbours()
    m = geom.basic_masses(mu)
    cbar = np.full((geom.nb, 5), np.nan)
    for i in range(geom.nb):
        b = boxes[i]
        Y = box_pixels(b.o1, b.o2, b.h, b.w)
        nu_i = b.a.reshape(-1) / m[i]
        for k in range(5):
            j = nbr[i, k]
            if j < 0:
                continue
            if j == i:
                cbar[i, k] = 0.0
                continue
            Xj = geom.cell_pixels(j)
            mu_j = mu[Xj[:, 0], Xj[:, 1]] / m[j]
            cand = float(mu_j @ sq_cost(Xj, Y, hgrid) @ nu_i)
            cbar[i, k] = cand - D[i] / m[i]
    return cbar


def flow_arcs(nbr):
    ii, kk = np.nonzero(nbr >= 0)
    return ii, kk, nbr[ii, kk]


def min_cost_flow(nbr, cbar, m):
    """Solve Eq. (MinCostFlow). Returns (w (nb, 5), optimal value, dual potentials)."""
    nb = len(m)
    ii, kk, jj = flow_arcs(nbr)
    na = len(ii)
    cols = np.arange(na)
    rows = np.concatenate([ii, nb + jj])
    A = sp.csr_matrix((np.ones(2 * na), (rows, np.concatenate([cols, cols]))), shape=(2 * nb, na))
    b = np.concatenate([m, m])
    # tight feasibility tolerances: HiGHS' defaults (1e-7) let flows go slightly
    # negative, which violates w >= 0 of the flow definition (Section 3.1)
    res = linprog(cbar[ii, kk], A_eq=A, b_eq=b, bounds=(0, None), method="highs-ds",
                  options=dict(primal_feasibility_tolerance=1e-10, dual_feasibility_tolerance=1e-10))
    if res.status != 0:
        raise RuntimeError("min-cost flow LP failed: " + res.message)
    w = np.zeros((nb, 5))
    w[ii, kk] = res.x
    duals = res.eqlin.marginals if hasattr(res, "eqlin") else None
    return w, float(res.fun), duals


def exchange(geom, boxes, w, nbr, m, thr=1e-15):
    """nu_hat_j = sum_{i in N(j)} w_ij nu_i / m_i (Eq. flow-update-cell-marginals), re-boxed."""
    incoming = [[] for _ in range(geom.nb)]
    for i in range(geom.nb):
        for k in range(5):
            j = nbr[i, k]
            if j >= 0 and w[i, k] > 0:
                incoming[j].append((i, w[i, k]))
    out = []
    for j in range(geom.nb):
        srcs = [boxes[i] for i, _ in incoming[j]]
        if not srcs:
            out.append(Box(0, 0, np.zeros((0, 0))))
            continue
        o1, o2, h, wd = union_header(srcs)
        acc = np.zeros((h, wd))
        for i, wij in incoming[j]:
            acc += (wij / m[i]) * embed(boxes[i], o1, o2, h, wd)
        out.append(truncate_box(acc, o1, o2, thr, m[j]))
    return out
