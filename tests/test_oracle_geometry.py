"""Pins for oracle.geometry: partitions (Def. 2.2, Fig. 3) and neighbourhoods (Def. 3.1)."""

import numpy as np
import pytest

from oracle.geometry import Geometry


def test_partitions_hand_written_8x8_s2():
    # n = 4 basic cells per axis; basic index = bi * 4 + bj.
    g = Geometry(8, 8, 2)
    assert g.partition(0) == [[0, 1, 4, 5], [2, 3, 6, 7], [8, 9, 12, 13], [10, 11, 14, 15]]
    assert g.partition(1) == [
        [0], [1, 2], [3],
        [4, 8], [5, 6, 9, 10], [7, 11],
        [12], [13, 14], [15],
    ]


@pytest.mark.parametrize("N,s", [(8, 2), (16, 4), (32, 4), (64, 4), (24, 4)])
def test_partitions_cover_once_and_connected(N, s):
    g = Geometry(N, N, s)
    for part in (0, 1):
        flat = sorted(i for c in g.partition(part) for i in c)
        assert flat == list(range(g.nb))
        for c in g.partition(part):
            assert c == sorted(c)  # members row-major
    assert len(g.partition(0)) == (g.n1 // 2) * (g.n2 // 2)
    assert len(g.partition(1)) == (g.n1 // 2 + 1) * (g.n2 // 2 + 1)
    assert g.partition_graph_connected()  # Def. 3.11, needed by Prop. 3.12


def test_composite_cells_are_rectangles():
    g = Geometry(32, 32, 4)
    for part in (0, 1):
        for c in g.partition(part):
            X = g.composite_pixels(c)
            r0, r1 = X[:, 0].min(), X[:, 0].max() + 1
            c0, c1 = X[:, 1].min(), X[:, 1].max() + 1
            assert (r1 - r0) * (c1 - c0) == len(X) == len(set(map(tuple, X)))


def test_neighbourhood_definition():
    g = Geometry(16, 24, 4)
    nbr = g.neighbours()
    for i in range(g.nb):
        assert nbr[i, 0] == i  # (i, i) in N
        bi, bj = divmod(i, g.n2)
        for k, (di, dj) in enumerate([(-1, 0), (1, 0), (0, -1), (0, 1)], start=1):
            ok = 0 <= bi + di < g.n1 and 0 <= bj + dj < g.n2
            assert (nbr[i, k] >= 0) == ok
            if ok:
                j = nbr[i, k]
                assert j == (bi + di) * g.n2 + bj + dj
                assert i in nbr[j]  # symmetry (Def. 3.1)
    assert (nbr >= 0).sum() == g.nb + 2 * (g.n1 - 1) * g.n2 + 2 * g.n1 * (g.n2 - 1)


def test_basic_masses():
    rng = np.random.default_rng(0)
    mu = rng.random((8, 16))
    g = Geometry(8, 16, 4)
    m = g.basic_masses(mu)
    for i in range(g.nb):
        X = g.cell_pixels(i)
        assert m[i] == pytest.approx(mu[X[:, 0], X[:, 1]].sum(), rel=1e-15)


@pytest.mark.parametrize("rebalance", ["project", "ipf"])
def test_prolongated_plan_is_feasible(rebalance):
    """Input recipe of the 1024 x 1024 configuration, at 64 x 64: a plan of the
    coarsened measures, prolongated with 1 % noise and rebalanced (noise
    projected to zero block marginals, or iterative proportional fitting), has
    both marginals of the fine measures (X to 1e-12 per basic cell, Y to 1e-12 in
    L1), and every child box lies inside the refinement of its parent's."""
    import numpy as np

    import synth

    from oracle.hybrid import OracleDD

    mu, nu, eps, p = synth.workload("dd1024", 0, N=64)
    muc, nuc = synth.coarsen(mu), synth.coarsen(nu)
    dd = OracleDD(muc, nuc, 4 * eps, 4, tol=1e-7)
    dd.step()
    coarse = [(b.o1, b.o2, b.a) for b in dd.boxes]
    fine = synth.prolongate(coarse, mu, nu, 4, noise=0.01, seed=0, rebalance=rebalance)
    m = mu.reshape(16, 4, 16, 4).sum(axis=(1, 3)).reshape(-1)
    assert len(fine) == 256
    Y = np.zeros_like(nu)
    for i, (o1, o2, a) in enumerate(fine):
        assert abs(a.sum() - m[i]) <= 1e-12 * m[i]
        Y[o1:o1 + a.shape[0], o2:o2 + a.shape[1]] += a
        bi, bj = divmod(i, 16)
        co1, co2, ca = coarse[(bi // 2) * 8 + bj // 2]
        assert 2 * co1 <= o1 and o1 + a.shape[0] <= 2 * (co1 + ca.shape[0])
        assert 2 * co2 <= o2 and o2 + a.shape[1] <= 2 * (co2 + ca.shape[1])
    # projection: the fine Y marginal inherits the coarse plan's Y error (its
    # truncation at 1e-15 per entry, ~1.5e-12 here); IPF fits it exactly
    assert np.abs(Y - nu).sum() <= (1e-11 if rebalance == "project" else 1e-12)
    if rebalance == "project":  # the noise: within 4 % of the noise-free plan, and not zero
        clean = synth.prolongate(coarse, mu, nu, 4, noise=0.0, seed=0)
        rel = [np.abs(a - c[2]).max() / c[2].max() for (_, _, a), c in zip(fine, clean) if a.shape == c[2].shape]
        assert max(rel) <= 0.04 and max(rel) > 1e-4
