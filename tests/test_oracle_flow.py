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
