"""Pins for the oracle's flow update (oracle.flow, oracle.dense.flow_update).

* product plan: edge costs are potential differences and the flow update is a
  fixed point (Section 3.3, first paragraph);
* singleton cells (s = 1): Eq. (edge-cost) reduces to Eq. (CostCoefficientSimple);
* the min-cost flow LP against brute-force vertex enumeration and against
  networkx's network simplex on an integer instance;
* Lemma 3.5 (marginals), Eq. (total-cost-update) and Lemma 3.9 (KL) on full plans;
* the box version against the full-plan Def. 3.4.
"""

import itertools

import networkx as nx
import numpy as np
import pytest

import synth
from oracle import dense
from oracle.domdec import embed, l1_y_error
from oracle.flow import edge_costs, exchange, min_cost_flow, flow_arcs
from oracle.geometry import Geometry
from oracle.hybrid import OracleDD


def _problem(N=8, seed=20):
    mu = synth.gaussian_mixture(N, 2, (0.1, 0.3), 1e-2, seed=seed)
    nu = synth.gaussian_mixture(N, 2, (0.1, 0.3), 1e-2, seed=seed + 1)
    return mu, nu


def test_product_plan_costs_are_potential_differences():
    N, s = 8, 2
    mu, nu = _problem(N)
    g = Geometry(N, N, s)
    C = dense.cost_matrix(N, N, 1.0 / N)
    pi = dense.product_plan(mu, nu)
    new, w, cbar, value = dense.flow_update(pi, g, mu, C)
    nbr = g.neighbours()
    for i in range(g.nb):
        for k in range(1, 5):
            j = nbr[i, k]
            if j >= 0:
                back = list(nbr[j]).index(i)
                assert cbar[i, k] == pytest.approx(-cbar[j, back], abs=1e-15)
    # around every unit square of the cell grid the costs sum to zero
    for bi in range(g.n1 - 1):
        for bj in range(g.n2 - 1):
            a, b, c, d = bi * g.n2 + bj, bi * g.n2 + bj + 1, (bi + 1) * g.n2 + bj + 1, (bi + 1) * g.n2 + bj
            cyc = cbar[a, 4] + cbar[b, 2] + cbar[c, 3] + cbar[d, 1]
            assert abs(cyc) < 1e-15
    assert abs(value) < 1e-15
    assert np.abs(new - pi).sum() < 1e-14          # fixed point


def test_singleton_cells_reduce_to_simple_costs():
    N, s = 4, 1
    mu, nu = _problem(N)
    o = OracleDD(mu, nu, 2.0 / N ** 2, s, tol=1e-12)
    o.iterate(0)
    o.iterate(1)
    g = o.geom
    cbar = edge_costs(g, mu, o.boxes, o.D, 1.0 / N)
    nbr = g.neighbours()
    h = 1.0 / N
    P = dense.pixels(N, N)
    for i in range(g.nb):
        b = o.boxes[i]
        nu_i = embed(b, 0, 0, N, N).reshape(-1) / mu.reshape(-1)[i]
        for k in range(5):
            j = nbr[i, k]
            if j < 0:
                continue
            # Eq. (CostCoefficientSimple): < c(x_j, .) - c(x_i, .), nu_i / m_i >
            cj = h * h * ((P - P[j]) ** 2).sum(axis=1)
            ci = h * h * ((P - P[i]) ** 2).sum(axis=1)
            assert cbar[i, k] == pytest.approx(float((cj - ci) @ nu_i), abs=1e-12)


def _vertex_enumeration(nbr, cbar, m):
    ii, kk, jj = flow_arcs(nbr)
    na, nb = len(ii), len(m)
    A = np.zeros((2 * nb, na))
    A[ii, np.arange(na)] = 1
    A[nb + jj, np.arange(na)] = 1
    b = np.concatenate([m, m])
    A, b = A[:-1], b[:-1]                       # one redundant constraint
    best = np.inf
    for cols in itertools.combinations(range(na), A.shape[0]):
        B = A[:, cols]
        if abs(np.linalg.det(B)) < 1e-12:
            continue
        x = np.linalg.solve(B, b)
        if (x >= -1e-12).all():
            best = min(best, float(cbar[ii[list(cols)], kk[list(cols)]] @ x))
    return best


@pytest.mark.parametrize("seed", range(4))
def test_min_cost_flow_vs_vertex_enumeration(seed):
    g = Geometry(4, 4, 2)            # a 2 x 2 grid of basic cells, 12 arcs
    rng = np.random.default_rng(seed)
    nbr = g.neighbours()
    cbar = np.where(nbr >= 0, rng.normal(size=nbr.shape), np.nan)
    cbar[:, 0] = 0.0
    m = rng.random(g.nb) + 0.2
    w, val, _ = min_cost_flow(nbr, cbar, m)
    assert val == pytest.approx(_vertex_enumeration(nbr, cbar, m), abs=1e-12)
    assert val <= 1e-15               # the stationary flow is feasible (Lemma 3.6)
    ii, kk, jj = flow_arcs(nbr)
    assert np.allclose(w.sum(axis=1), m, atol=1e-13)
    inflow = np.zeros(g.nb)
    np.add.at(inflow, jj, w[ii, kk])
    assert np.allclose(inflow, m, atol=1e-13)


@pytest.mark.parametrize("seed", range(3))
def test_min_cost_flow_vs_network_simplex(seed):
    g = Geometry(12, 12, 2)
    rng = np.random.default_rng(seed)
    nbr = g.neighbours()
    cost = np.where(nbr >= 0, rng.integers(-50, 50, size=nbr.shape), 0)
    cost[:, 0] = 0
    mass = rng.integers(5, 40, size=g.nb)
    G = nx.DiGraph()
    for i in range(g.nb):
        G.add_node(("s", i), demand=-int(mass[i]))
        G.add_node(("t", i), demand=int(mass[i]))
    ii, kk, jj = flow_arcs(nbr)
    for i, k, j in zip(ii, kk, jj):
        G.add_edge(("s", i), ("t", j), weight=int(cost[i, k]))
    ref = nx.network_simplex(G)[0]
    _, val, _ = min_cost_flow(nbr, cost.astype(float), mass.astype(float))
    assert val == pytest.approx(ref, abs=1e-7)


def test_flow_update_lemmas_on_full_plan():
    """Lemma 3.5, Eq. (total-cost-update), Lemma 3.9 and the box version, on a rotated plan."""
    N, s = 8, 2
    mu = synth.four_bumps(N)
    eps = 1.0 / N ** 2
    g = Geometry(N, N, s)
    C = dense.cost_matrix(N, N, 1.0 / N)
    pi = np.zeros((N * N, N * N))
    x, y, mm = synth.rotation_coupling(mu)
    pi[x, y] = mm
    pi, _ = dense.domdec_iter(pi, g, 0, mu, C, eps, tol=1e-12)
    new, w, cbar, value = dense.flow_update(pi, g, mu, C)
    assert value < -1e-6                                        # there is curl to remove
    assert np.abs(new.sum(axis=0) - pi.sum(axis=0)).sum() < 1e-14   # Y marginal kept
    assert np.abs(new.sum(axis=1) - pi.sum(axis=1)).sum() < 1e-12   # X marginal kept
    ref = np.outer(mu.reshape(-1), mu.reshape(-1))
    assert float((C * new).sum() - (C * pi).sum()) == pytest.approx(value, rel=1e-12, abs=1e-16)
    assert dense.kl(new, ref) <= dense.kl(pi, ref) + 1e-14       # Lemma 3.9
    # box version of the same step
    boxes = synth.boxes_from_coupling(mu.shape, s, x, y, mm)
    o = OracleDD(mu, mu, eps, s, boxes=boxes, tol=1e-12)
    o.iterate(0)
    f = o.flow_update()
    assert f["value"] == pytest.approx(value, rel=1e-9)
    assert np.allclose(f["cbar"][~np.isnan(cbar)], cbar[~np.isnan(cbar)], rtol=1e-8, atol=1e-14)
    for i in range(g.nb):
        ref_i = new[dense.cell_rows(g, i)].sum(axis=0).reshape(N, N)
        assert np.abs(embed(o.boxes[i], 0, 0, N, N) - ref_i).sum() < 1e-10
    assert l1_y_error(o.boxes, mu) < 1e-13
    m = g.basic_masses(mu)
    assert np.allclose([b.a.sum() for b in o.boxes], m, rtol=1e-10, atol=0)


def _small_gluing(N=8, s=2, seed=3):
    mu = synth.gaussian_mixture(N, 2, (0.1, 0.3), 1e-2, seed=seed)
    g = Geometry(N, N, s)
    return mu, g


def test_gluing_plan_is_a_coupling_and_limits():
    """gamma_ij (Def. 3.7): a coupling of mu_i/m_i and mu_j/m_j (both marginals to
    1e-12); eps_gamma = inf is the product coupling; for a small eps_gamma it
    concentrates on the optimal assignment between the two blocks (adjacent
    blocks of a constant measure: the translation by one cell, mass on the
    shifted pixel >= 0.99)."""
    from oracle.flow import gluing_plan

    mu, g = _small_gluing()
    nbr = g.neighbours()
    for i in (0, 5, 9):
        for k in range(1, 5):
            j = nbr[i, k]
            if j < 0:
                continue
            G = gluing_plan(g, mu, i, j, 1.0 / 8, (0.5 / 8) ** 2)
            Xi, Xj = g.cell_pixels(i), g.cell_pixels(j)
            a = mu[Xi[:, 0], Xi[:, 1]]
            b = mu[Xj[:, 0], Xj[:, 1]]
            assert np.abs(G.sum(axis=1) - a / a.sum()).sum() < 1e-12
            assert np.abs(G.sum(axis=0) - b / b.sum()).sum() < 1e-12
            P = gluing_plan(g, mu, i, j, 1.0 / 8, np.inf)
            assert np.allclose(P, np.outer(a / a.sum(), b / b.sum()), rtol=1e-15)
    # constant measure: the small-eps plan is (nearly) the translation
    N, s = 8, 4
    mu = np.full((N, N), 1.0 / N ** 2)
    g = Geometry(N, N, s)
    G = gluing_plan(g, mu, 0, 1, 1.0 / N, (0.1 / N) ** 2)
    Xi, Xj = g.cell_pixels(0), g.cell_pixels(1)
    shifted = [int(np.flatnonzero((Xj == Xi[q] + np.array([0, s])).all(axis=1))[0]) for q in range(len(Xi))]
    assert min(G[q, shifted[q]] * len(Xi) for q in range(len(Xi))) >= 0.99


def test_glued_candidate_lemma_3_9_items_1_and_2():
    """Lemma 3.9 (1): pi_hat_ij in Pi(mu_j/m_j, nu_i/m_i); (2): its density w.r.t.
    mu_j (x) nu is (1/m_j) int dpi_i/d(mu_i (x) nu)(x', y) d(gamma_ij)_x(x') with
    (gamma_ij)_x the disintegration against the mu_j/m_j marginal -- computed
    here by that formula, independently of the matrix product."""
    from oracle.flow import glued_candidate, gluing_plan

    N, s = 8, 2
    mu, g = _small_gluing(N, s)
    nu = synth.gaussian_mixture(N, 2, (0.1, 0.3), 1e-2, seed=4)
    C = dense.cost_matrix(N, N, 1.0 / N)
    pi, _ = dense.global_sinkhorn(mu, nu, 4.0 / N ** 2, 1.0 / N, tol=1e-14)
    m = g.basic_masses(mu)
    nbr = g.neighbours()
    nuf = nu.reshape(-1)
    for i in (0, 6, 10):
        rows_i = dense.cell_rows(g, i)
        mu_i = mu.reshape(-1)[rows_i]
        pi_i = pi[rows_i]
        for k in range(1, 5):
            j = nbr[i, k]
            if j < 0:
                continue
            G = gluing_plan(g, mu, i, j, 1.0 / N, (0.5 / N) ** 2)
            cand = glued_candidate(G, pi_i, mu_i)
            mu_j = mu.reshape(-1)[dense.cell_rows(g, j)]
            assert np.abs(cand.sum(axis=1) - mu_j / m[j]).sum() < 1e-12
            assert np.abs(cand.sum(axis=0) - pi_i.sum(axis=0) / m[i]).sum() < 1e-12
            dens_i = pi_i / (mu_i[:, None] * nuf[None, :])          # dpi_i / d(mu_i (x) nu)
            cond = G / (mu_j / m[j])[None, :]                       # (gamma)_x(x') over x'
            dens = (cond.T @ dens_i) / m[j]
            assert np.allclose(cand, dens * mu_j[:, None] * nuf[None, :], rtol=1e-11, atol=1e-18)
    _ = C


def test_glued_flow_update_on_full_plan_and_box_version():
    """Flow update with gluing candidates from entropic gamma_ij (eps_gamma =
    (h/2)^2) on a full plan: marginals kept (Lemma 3.5), the transport-cost change
    equals the optimal value (Eq. total-cost-update), the entropy term does not
    increase (Lemma 3.9 (3)) and so the objective decreases (Prop. 3.10). The
    box version (OracleDD with eps_gamma) has the same edge costs, value and new
    basic marginals."""
    from oracle.flow import gluing_plans

    N, s = 8, 2
    mu = synth.four_bumps(N)
    eps = 1.0 / N ** 2
    g = Geometry(N, N, s)
    C = dense.cost_matrix(N, N, 1.0 / N)
    pi = np.zeros((N * N, N * N))
    x, y, mm = synth.rotation_coupling(mu)
    pi[x, y] = mm
    pi, _ = dense.domdec_iter(pi, g, 0, mu, C, eps, tol=1e-12)
    gam = gluing_plans(g, mu, 1.0 / N, (0.5 / N) ** 2)
    new, w, cbar, value = dense.flow_update(pi, g, mu, C, gammas=gam)
    assert value < -1e-6
    assert np.abs(new.sum(axis=0) - pi.sum(axis=0)).sum() < 1e-14
    assert np.abs(new.sum(axis=1) - pi.sum(axis=1)).sum() < 1e-12
    ref = np.outer(mu.reshape(-1), mu.reshape(-1))
    assert float((C * new).sum() - (C * pi).sum()) == pytest.approx(value, rel=1e-12, abs=1e-16)
    assert dense.kl(new, ref) <= dense.kl(pi, ref) + 1e-14
    assert dense.objective(new, mu, mu, C, eps) < dense.objective(pi, mu, mu, C, eps)
    # the product candidates give a different (weaker or equal) flow value here
    _, _, cbar_p, value_p = dense.flow_update(pi, g, mu, C)
    assert not np.allclose(cbar[~np.isnan(cbar)], cbar_p[~np.isnan(cbar_p)])
    # box version
    boxes = synth.boxes_from_coupling(mu.shape, s, x, y, mm)
    o = OracleDD(mu, mu, eps, s, boxes=boxes, tol=1e-12, eps_gamma=(0.5 / N) ** 2)
    o.iterate(0)
    f = o.flow_update()
    assert np.allclose(f["cbar"][~np.isnan(cbar)], cbar[~np.isnan(cbar)], rtol=1e-8, atol=1e-14)
    assert f["value"] == pytest.approx(value, rel=1e-9)
    for i in range(g.nb):
        ref_i = new[dense.cell_rows(g, i)].sum(axis=0).reshape(N, N)
        assert np.abs(embed(o.boxes[i], 0, 0, N, N) - ref_i).sum() < 1e-10


def test_glued_costs_with_product_gamma_equal_product_costs():
    """eps_gamma = inf: edge_costs_glued (matrix product of the plan) equals the
    product-candidate edge_costs (moments of the basic marginals) on the same
    pre-balance plan, to 1e-12 relative."""
    from oracle.domdec import Box
    from oracle.flow import edge_costs, edge_costs_glued, gluing_plans

    N, s = 16, 4
    mu, nu, eps, p = synth.workload("dd32", 0, N=N)
    o = OracleDD(mu, nu, eps, s, tol=1e-10, eps_gamma=1e30)
    o.iterate(0)
    g = o.geom
    gam = gluing_plans(g, mu, 1.0 / N, np.inf)
    cg = edge_costs_glued(g, mu, o.basic_plans, o.D, 1.0 / N, gam)
    pre = []
    for i in range(g.nb):
        Y, pi_i = o.basic_plans[i]
        a = np.zeros((N, N))
        np.add.at(a, (Y[:, 0], Y[:, 1]), pi_i.sum(axis=0))
        pre.append(Box(0, 0, a))
    cp = edge_costs(g, mu, pre, o.D, 1.0 / N)
    ok = ~np.isnan(cp)
    assert np.allclose(cg[ok], cp[ok], rtol=1e-12, atol=1e-15 * np.abs(cp[ok]).max())
