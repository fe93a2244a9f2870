"""The flow update (Section 3.2) on the basic-cell box state.

Edge candidates are gluing candidates (Def. 3.7): with gamma_ij the product
coupling (Remark 3.8, eps_gamma = inf), pi_hat_ij = mu_j/m_j (x) nu_i/m_i for
j != i, and pi_hat_ii = pi_i/m_i (Def. 3.4); with an entropic gamma_ij (small
eps_gamma) see gluing_plan / edge_costs_glued below. For the product candidate
the edge cost Eq. (edge-cost) is

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

from .cell import cell_sinkhorn, gibbs_plan, sq_cost
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


def gluing_plan(geom, mu, i, j, hgrid, eps_gamma, tol=1e-13, max_iter=1000000):
    """gamma_ij in Pi(mu_i/m_i, mu_j/m_j) for the gluing edge candidate (Def. 3.7,
    Remark 3.8): the entropic optimal plan between the normalised basic-cell
    measures for the squared distance on X with regularisation eps_gamma (the
    paper's small-eps_gamma choice), solved by the oracle's dense log-domain
    Sinkhorn (cell.cell_sinkhorn: Y-marginal mu_j/m_j exact, X-marginal within
    tol); eps_gamma = inf gives the product coupling. Rows over X_i, columns
    over X_j, in Geometry.cell_pixels order."""
    Xi, Xj = geom.cell_pixels(i), geom.cell_pixels(j)
    a = mu[Xi[:, 0], Xi[:, 1]]
    b = mu[Xj[:, 0], Xj[:, 1]]
    a, b = a / a.sum(), b / b.sum()
    if not np.isfinite(eps_gamma):
        return np.outer(a, b)
    C = sq_cost(Xi, Xj, hgrid)
    res = cell_sinkhorn(a, b, C, eps_gamma, np.zeros(len(a)), tol=tol, max_iter=max_iter)
    return gibbs_plan(res["alpha"], res["beta_t"], a, b, C, eps_gamma)


def gluing_plans(geom, mu, hgrid, eps_gamma):
    """gamma_ij for every edge (i, j) of the neighbourhood set with j != i, keyed
    by (i, k) with j = Geometry.neighbours()[i, k]."""
    nbr = geom.neighbours()
    return {(i, k): gluing_plan(geom, mu, i, int(nbr[i, k]), hgrid, eps_gamma)
            for i in range(geom.nb) for k in range(1, 5) if nbr[i, k] >= 0}


def glued_candidate(G, pi_i, mu_i):
    """pi_hat_ij on X_j x Y from gamma_ij (G, rows X_i, columns X_j) and the
    basic-cell plan pi_i (rows X_i) by Eq. (glued-plan): the disintegration of
    gamma_ij at x' (G[x', .] m_i / mu(x')) times the disintegration of pi_i at
    x' (pi_i(x', .) / mu(x')), integrated against mu_i / m_i, i.e.
        pi_hat_ij(x, y) = sum_{x'} G[x', x] pi_i(x', y) / mu(x'),
    the matrix product of Remark 3.8."""
    return G.T @ (pi_i / mu_i[:, None])


def edge_costs_glued(geom, mu, plans, D, hgrid, gammas) -> np.ndarray:
    """c_bar (nb, 5) of Eq. (edge-cost) with gluing edge candidates:
    c_bar_ij = <c, pi_hat_ij> - D_i / m_i, pi_hat_ij = glued_candidate(gamma_ij, pi_i),
    evaluated as explicit sums over X_j x Y. plans[i] = (Y pixels (ny, 2), pi_i
    (s^2, ny)): the basic cell's part of the Gibbs cell plan of the latest
    half-iteration, the plan D_i = <c, pi_i> comes from (reading: both terms from
    the same plan, before balancing)."""
    nbr = geom.neighbours()
    m = geom.basic_masses(mu)
    cbar = np.full((geom.nb, 5), np.nan)
    for i in range(geom.nb):
        Y, pi_i = plans[i]
        Xi = geom.cell_pixels(i)
        mu_i = mu[Xi[:, 0], Xi[:, 1]]
        for k in range(5):
            j = nbr[i, k]
            if j < 0:
                continue
            if j == i:
                cbar[i, k] = 0.0
                continue
            Xj = geom.cell_pixels(j)
            cand = glued_candidate(gammas[(i, k)], pi_i, mu_i)
            cbar[i, k] = float(np.sum(sq_cost(Xj, Y, hgrid) * cand)) - D[i] / m[i]
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
