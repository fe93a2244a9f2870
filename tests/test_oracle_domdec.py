"""Pins for the oracle's half-iteration on boxes (oracle.domdec).

Brute force for the box bookkeeping, invariants for balancing, the full-plan
Alg. 1 (oracle.dense) for the box version, and the single-cell case against
the global problem.
"""

import numpy as np
import pytest

import synth
from oracle import dense
from oracle.domdec import Box, balance, basic_to_composite, half_iteration, truncate_box, embed, l1_y_error
from oracle.geometry import Geometry
from oracle.hybrid import OracleDD


def test_basic_to_composite_brute_force():
    rng = np.random.default_rng(0)
    boxes = []
    for _ in range(4):
        o1, o2 = rng.integers(0, 20, 2)
        h, w = rng.integers(1, 9, 2)
        boxes.append(Box(int(o1), int(o2), rng.random((h, w))))
    J = basic_to_composite(boxes, [0, 1, 2, 3])
    dense_sum = np.zeros((40, 40))
    for b in boxes:
        dense_sum[b.o1:b.o1 + b.h, b.o2:b.o2 + b.w] += b.a
    rows = np.nonzero(dense_sum.any(axis=1))[0]
    cols = np.nonzero(dense_sum.any(axis=0))[0]
    assert (J.o1, J.o2, J.h, J.w) == (rows[0], cols[0], rows[-1] - rows[0] + 1, cols[-1] - cols[0] + 1)
    assert np.array_equal(embed(J, 0, 0, 40, 40), dense_sum)


def test_truncate_box_brute_force():
    rng = np.random.default_rng(1)
    for _ in range(50):
        a = rng.random((7, 9)) * (rng.random((7, 9)) < 0.3)
        a[rng.random((7, 9)) < 0.2] = 5e-16          # below the threshold
        b = truncate_box(a, 3, 4, 1e-15)
        keep = np.where(a < 1e-15, 0.0, a)
        if not keep.any():
            assert b.h == 0
            continue
        r, c = np.nonzero(keep)
        assert (b.o1, b.o2) == (3 + r.min(), 4 + c.min())
        assert (b.h, b.w) == (r.max() - r.min() + 1, c.max() - c.min() + 1)
        assert np.array_equal(embed(b, 3, 4, 7, 9), keep)


@pytest.mark.parametrize("seed", range(5))
def test_balance_invariants(seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 5))
    arrs = [rng.random((5, 6)) * (rng.random((5, 6)) < 0.7) + 1e-3 for _ in range(k)]
    tot = sum(a.sum() for a in arrs)
    m = rng.random(k) + 0.1
    m *= tot / m.sum()                                # |nu_J| = m_J
    out = balance(arrs, list(m))
    assert np.allclose(sum(out), sum(arrs), rtol=0, atol=1e-14)   # pointwise sum kept
    assert all((o >= 0).all() for o in out)
    assert np.allclose([o.sum() for o in out], m, rtol=1e-13, atol=0)


def test_balance_two_members_closed_form():
    a0 = np.array([[1.0, 3.0]])
    a1 = np.array([[2.0, 2.0]])
    out = balance([a0, a1], [3.0, 5.0])             # member 0 gives 1 unit, shaped like a0
    assert np.allclose(out[0], a0 * 0.75)
    assert np.allclose(out[1], a1 + a0 * 0.25)


def _small_problem(N=8, s=2, seed=10):
    mu = synth.gaussian_mixture(N, 2, (0.1, 0.3), 1e-2, seed=seed)
    nu = synth.gaussian_mixture(N, 2, (0.1, 0.3), 1e-2, seed=seed + 1)
    return mu, nu, 2.0 / N ** 2


def test_single_cell_equals_global_problem():
    """cell_size = N/2: partition A is one cell, so one A half-iteration is the global problem."""
    N = 8
    mu, nu, eps = _small_problem(N)
    pistar, _ = dense.global_sinkhorn(mu, nu, eps, 1.0 / N, tol=1e-13)
    o = OracleDD(mu, nu, eps, N // 2, tol=1e-13)     # product init
    info = o.iterate(0)
    assert len(o.geom.partition(0)) == 1
    g = o.geom
    for i in range(g.nb):
        ref = pistar[dense.cell_rows(g, i)].sum(axis=0).reshape(N, N)
        assert np.abs(embed(o.boxes[i], 0, 0, N, N) - ref).sum() < 1e-10
    C = dense.cost_matrix(N, N, 1.0 / N)
    assert info["E"] == pytest.approx(dense.objective(pistar, mu, nu, C, eps), rel=1e-11)


def test_box_half_iterations_match_full_plan_alg1():
    N, s = 8, 2
    mu, nu, eps = _small_problem(N)
    g = Geometry(N, N, s)
    C = dense.cost_matrix(N, N, 1.0 / N)
    boxes = synth.boxes_from_coupling(mu.shape, s, *synth.knothe_rosenblatt(mu, nu))
    pi = np.zeros((N * N, N * N))
    x, y, m = synth.knothe_rosenblatt(mu, nu)
    np.add.at(pi, (x, y), m)
    o = OracleDD(mu, nu, eps, s, boxes=boxes, tol=1e-11)
    for part in (0, 1, 0):
        info = o.iterate(part)
        pi, _ = dense.domdec_iter(pi, g, part, mu, C, eps, tol=1e-11)
        for i in range(g.nb):
            ref = pi[dense.cell_rows(g, i)].sum(axis=0).reshape(N, N)
            assert np.abs(embed(o.boxes[i], 0, 0, N, N) - ref).sum() < 1e-9
        assert info["E"] == pytest.approx(dense.objective(pi, mu, nu, C, eps), rel=1e-9)


def test_half_iteration_invariants():
    mu, nu, eps, p = synth.workload("dd32", 0, N=16)
    o = OracleDD(mu, nu, eps, 4, tol=1e-6)
    prev_E = np.inf
    m = o.geom.basic_masses(mu)
    for part in (0, 1, 0, 1):
        info = o.iterate(part)
        # Y-marginal preserved (Sinkhorn is Y-exact, balancing keeps sums); truncation only.
        assert l1_y_error(o.boxes, nu) < 1e-11
        # every basic cell holds its mass m_i (balancing, then the rescale after truncation)
        assert np.allclose([b.a.sum() for b in o.boxes], m, rtol=1e-13, atol=0)
        # X error of the stitched Gibbs plan within the cell tolerance
        assert info["l1_x"] <= 1e-6 * 1.0 + 1e-15
        assert all(e <= 1e-6 * mc for e, mc in zip(info["err"], [m[c].sum() for c in o.geom.partition(part)]))
        # block coordinate descent: the objective does not increase
        assert info["E"] <= prev_E + 1e-12
        prev_E = info["E"]
