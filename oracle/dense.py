"""Full-plan versions for tiny grids (a few hundred pixels), used to pin the box oracle.

The plan pi is an explicit (N1*N2) x (N1*N2) float64 matrix; pixel x = p*N2 + q.

* `global_sinkhorn`: the global problem Eq. (entropic-transport), solved with the
  same log-domain iteration as a cell (a single cell covering X).
* `objective`: <c, pi> + eps KL(pi | mu (x) nu) with KL of Eq. (KL).
* `domdec_iter`: Alg. 1 literally on the explicit plan (no boxes, no balancing).
* `flow_update`: Def. 3.4 literally, with the product gluing candidates of
  Remark 3.8 built as explicit matrices; c_bar_ij = <c, pi_hat_ij - pi_hat_ii>
  (Eq. edge-cost) summed over the matrices.
"""

from __future__ import annotations

import numpy as np

from .cell import cell_sinkhorn, gibbs_plan, sq_cost
from .flow import min_cost_flow


def pixels(N1, N2):
    p, q = np.meshgrid(np.arange(N1), np.arange(N2), indexing="ij")
    return np.stack([p.reshape(-1), q.reshape(-1)], axis=1)


def cost_matrix(N1, N2, hgrid):
    P = pixels(N1, N2)
    return sq_cost(P, P, hgrid)


def kl(pi, ref):
    """KL(pi | ref) = sum phi(pi/ref) ref with phi(s) = s log s - s + 1, Eq. (KL)."""
    pos = pi > 0
    val = np.sum(pi[pos] * np.log(pi[pos] / ref[pos])) - pi.sum() + ref.sum()
    if np.any(pos & (ref <= 0)):
        return np.inf
    return float(val)


def objective(pi, mu, nu, C, eps):
    ref = np.outer(mu.reshape(-1), nu.reshape(-1))
    return float(np.sum(C * pi)) + eps * kl(pi, ref)


def global_sinkhorn(mu, nu, eps, hgrid, tol=1e-13, max_iter=200000):
    N1, N2 = mu.shape
    C = cost_matrix(N1, N2, hgrid)
    mu_x, nu_y = mu.reshape(-1), nu.reshape(-1)
    res = cell_sinkhorn(mu_x, nu_y, C, eps, np.zeros(len(mu_x)), tol, max_iter)
    return gibbs_plan(res["alpha"], res["beta_t"], mu_x, nu_y, C, eps), res


def product_plan(mu, nu):
    return np.outer(mu.reshape(-1), nu.reshape(-1))


def cell_rows(geom, i):
    X = geom.cell_pixels(i)
    return X[:, 0] * geom.N2 + X[:, 1]


def domdec_iter(pi, geom, part, mu, C, eps, tol=1e-12, max_iter=200000, alpha_prev=None):
    """Alg. 1 on the explicit plan. Returns (new plan, alphas)."""
    pi = pi.copy()
    mu_f = mu.reshape(-1)
    alphas = []
    for J, members in enumerate(geom.partition(part)):
        rows = np.concatenate([cell_rows(geom, i) for i in members])
        nuJ = pi[rows].sum(axis=0)
        supp = nuJ > 0
        a0 = np.zeros(len(rows)) if alpha_prev is None else alpha_prev[J]
        res = cell_sinkhorn(mu_f[rows], nuJ[supp], C[np.ix_(rows, np.nonzero(supp)[0])], eps, a0, tol, max_iter)
        block = np.zeros((len(rows), pi.shape[1]))
        block[:, supp] = gibbs_plan(res["alpha"], res["beta_t"], mu_f[rows], nuJ[supp],
                                    C[np.ix_(rows, np.nonzero(supp)[0])], eps)
        pi[rows] = block
        alphas.append(res["alpha"])
    return pi, alphas


def flow_update(pi, geom, mu, C, gammas=None):
    """Def. 3.4 with gluing candidates: product (gammas None) or from the plans
    gamma_ij in `gammas` ((i, k) -> rows X_i, columns X_j), Eq. (glued-plan).
    Returns (new plan, w, c_bar, value)."""
    mu_f = mu.reshape(-1)
    nbr = geom.neighbours()
    m = geom.basic_masses(mu)
    rows = [cell_rows(geom, i) for i in range(geom.nb)]
    nu_i = [pi[r].sum(axis=0) for r in rows]

    def cand(i, j, k):  # pi_hat_ij restricted to X_j x Y
        if i == j:
            return pi[rows[i]] / m[i]
        if gammas is not None:  # sum_{x'} gamma(x', x) pi_i(x', y) / mu(x')
            return gammas[(i, k)].T @ (pi[rows[i]] / mu_f[rows[i]][:, None])
        return np.outer(mu_f[rows[j]] / m[j], nu_i[i] / m[i])

    cbar = np.full((geom.nb, 5), np.nan)
    for i in range(geom.nb):
        for k in range(5):
            j = nbr[i, k]
            if j >= 0:
                cbar[i, k] = float(np.sum(C[rows[j]] * cand(i, j, k)) - np.sum(C[rows[i]] * cand(i, i, 0)))
    w, value, _ = min_cost_flow(nbr, cbar, m)
    new = np.zeros_like(pi)
    for i in range(geom.nb):
        for k in range(5):
            j = nbr[i, k]
            if j >= 0 and w[i, k] > 0:
                new[rows[j]] += w[i, k] * cand(i, j, k)
    return new, w, cbar, value
