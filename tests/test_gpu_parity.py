"""GPU parity: the CUDA library against the FP64 oracle, through the C ABI.

Tolerances (each derived below from the FP32 and FP64 arithmetic of the two sides):
* indexing (partitions, neighbours, box headers given identical values): bit-exact;
* fixed Sinkhorn iteration counts, same start: both sides run the same
  iteration; the GPU's FP32 log-sum-exp carries relative errors of a few 1e-7 per
  term and the FP32 duals of magnitude <= ~100 (base-2 units) round at ~6e-6, so
  the basic marginals agree to L1 <= 1e-5 (total mass 1) and the objective to
  1e-6 relative;
* tolerance mode: the GPU's exported duals, re-evaluated in FP64, give an L1 X
  error <= tol + 3e-5 per unit cell mass and a Y error <= 3e-5: the FP32 duals
  (magnitudes up to ~200 in base-2 units after the kernel's change of gauge)
  round at ~1.2e-5, and a pair of them enters each exponent. The library's own
  state is Y-exact up to FP32 storage (L1 Y error <= 1e-6) and X-exact per basic
  cell (rescaled to m_i);
* flow update: edge costs computed from the same state agree to 5e-7 of the
  largest |c_bar|: both terms of c_bar (candidate cost and D_i / m_i, each up to
  max|c_bar|) come from FP32-stored marginals summed in FP64 (relative ~2e-7,
  and the GPU takes its moments before the final FP32 rounding); the optimal
  values of the library's network simplex and the oracle's LP to 1e-9 relative.
"""

import numpy as np
import pytest

import synth
from oracle.cell import sq_cost
from oracle.domdec import Box, balance, basic_to_composite, box_pixels, embed, truncate_box, l1_y_error
from oracle.flow import edge_costs, exchange, min_cost_flow
from oracle.geometry import Geometry
from oracle.hybrid import OracleDD

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd(lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib


def as_boxes(lst):
    return [Box(o1, o2, np.asarray(a, dtype=np.float64)) for o1, o2, a in lst]


def plan_l1(a, b, shape):
    return sum(np.abs(embed(x, 0, 0, *shape) - embed(y, 0, 0, *shape)).sum() for x, y in zip(a, b))


def gpu_cell_errors(g, part, mu, nu, eps, geom, cells=None):
    """FP64 evaluation of the GPU's exported duals: per-cell L1 X error / m_J and Y error."""
    alpha, betas = g.duals(part)
    comp = g.composite(part)
    N = mu.shape[0]
    m = geom.basic_masses(mu)
    out = []
    parts = geom.partition(part)
    for J in (range(len(parts)) if cells is None else cells):
        members = parts[J]
        X = geom.composite_pixels(members)
        o1, o2, nuJ = comp[J]
        _, _, beta = betas[J]
        Y = box_pixels(o1, o2, nuJ.shape[0], nuJ.shape[1])
        supp = nuJ.reshape(-1) > 0
        C = sq_cost(X, Y[supp], 1.0 / N)
        a = alpha[X[:, 0], X[:, 1]]
        b = beta.reshape(-1)[supp]
        pi = np.exp((a[:, None] + b[None, :] - C) / eps) * mu[X[:, 0], X[:, 1]][:, None] * nu[Y[supp][:, 0], Y[supp][:, 1]][None, :]
        xe = np.abs(pi.sum(axis=1) - mu[X[:, 0], X[:, 1]]).sum() / m[members].sum()
        ye = np.abs(pi.sum(axis=0) - nuJ.reshape(-1)[supp]).sum() / nuJ.sum()
        out.append((J, xe, ye))
    return out


@pytest.mark.parametrize("N,s", [(16, 4), (32, 4), (64, 4), (32, 2), (48, 4)])
def test_partition_and_neighbours_bit_exact(dd, N, s):
    mu, nu, eps, _ = synth.workload("dd32", 0, N=N)
    g = dd.DomDec(mu, nu, eps, s)
    geom = Geometry(N, N, s)
    for part in (0, 1):
        mem = g.partition(part)
        ref = geom.partition(part)
        assert len(mem) == len(ref)
        for row, cell in zip(mem, ref):
            assert list(row[: len(cell)]) == cell and (row[len(cell):] == -1).all()
    assert np.array_equal(g.neighbours(), geom.neighbours())
    g.close()


@pytest.mark.parametrize("N,K", [(16, 30), (32, 40)])
def test_fixed_iterations_half_iterations_match_oracle(dd, N, K):
    mu, nu, eps, _ = synth.workload("dd32", 0, N=N)
    g = dd.DomDec(mu, nu, eps, 4, fixed_iters=K)
    o = OracleDD(mu, nu, eps, 4, fixed_iters=K)
    for part in (0, 1, 0):
        before = as_boxes(g.plan())
        sg = g.iterate(part)
        so = o.iterate(part)
        # BasicToComposite: headers bit-exact, values = FP32 sums of the same inputs
        comp = as_boxes(g.composite(part))
        for J, members in enumerate(o.geom.partition(part)):
            ref = basic_to_composite(before, members)
            assert (comp[J].o1, comp[J].o2, comp[J].h, comp[J].w) == (ref.o1, ref.o2, ref.h, ref.w)
            assert np.allclose(comp[J].a, ref.a, rtol=1e-6, atol=1e-15)
        assert abs(sg["objective"] - so["E"]) <= 1e-6 * abs(so["E"])
        assert plan_l1(as_boxes(g.plan()), o.boxes, mu.shape) <= 1e-5
        assert sg["iters_max"] == K
    g.close()


def test_composite_to_basic_D_and_balancing_from_gpu_duals(dd):
    N = 32
    mu, nu, eps, _ = synth.workload("dd32", 0, N=N)
    geom = Geometry(N, N, 4)
    m = geom.basic_masses(mu)
    g = dd.DomDec(mu, nu, eps, 4, tol=1e-6, flags=dd.DD_FLAG_KEEP_PREBALANCE)
    g.iterate(0)
    g.iterate(1)
    alpha, betas = g.duals(1)
    comp = as_boxes(g.composite(1))
    pre = as_boxes(g.prebalance())
    out = as_boxes(g.plan())
    mom = g.basic_moments()
    for J, members in enumerate(geom.partition(1)):
        X = geom.composite_pixels(members)
        nuJ = comp[J]
        Y = box_pixels(nuJ.o1, nuJ.o2, nuJ.h, nuJ.w)
        supp = nuJ.a.reshape(-1) > 0
        C = sq_cost(X, Y[supp], 1.0 / N)
        b = betas[J][2].reshape(-1)[supp]
        a = alpha[X[:, 0], X[:, 1]]
        pi = np.exp((a[:, None] + b[None, :] - C) / eps) * mu[X[:, 0], X[:, 1]][:, None] * nu[Y[supp][:, 0], Y[supp][:, 1]][None, :]
        ss = 16
        arrs = []
        for k, i in enumerate(members):
            ref = np.zeros(nuJ.h * nuJ.w)
            ref[supp] = pi[k * ss:(k + 1) * ss].sum(axis=0)
            # CompositeToBasic (Section A.1, partial log-sum-exp) = row sums of the Gibbs plan
            assert pre[i].o1 == nuJ.o1 and pre[i].a.shape == nuJ.a.shape
            assert np.abs(pre[i].a.reshape(-1) - ref).sum() <= 2e-5 * m[i]
            Dref = float((C[k * ss:(k + 1) * ss] * pi[k * ss:(k + 1) * ss]).sum())
            assert mom["D"][i] == pytest.approx(Dref, rel=1e-5)
            arrs.append(pre[i].a)
        # balancing + truncation applied by the oracle to the GPU's pre-balance values
        bal = balance(arrs, [m[i] for i in members])
        for k, i in enumerate(members):
            ref = truncate_box(bal[k], nuJ.o1, nuJ.o2, 1e-15, m[i])
            got = out[i]
            # headers bit-exact unless an entry sits within FP32 rounding of the threshold
            if (got.o1, got.o2, got.h, got.w) != (ref.o1, ref.o2, ref.h, ref.w):
                diff = np.abs(embed(got, 0, 0, N, N) - embed(ref, 0, 0, N, N))
                assert diff.max() < 2e-15
            assert np.abs(embed(got, 0, 0, N, N) - embed(ref, 0, 0, N, N)).sum() <= 1e-6 * m[i]
            assert got.a.sum() == pytest.approx(m[i], rel=1e-6)
    g.close()


@pytest.mark.parametrize("workload,N,init,levels,aa", [("dd32", 32, "product", 0, 0), ("dd256", 64, "kr", 0, 0),
                                                        ("dd32", 32, "product", 2, 0), ("dd256", 64, "kr", 2, 0),
                                                        ("dd32", 32, "product", 0, 4), ("dd256", 64, "kr", 2, 4),
                                                        ("dd256", 64, "kr", 2, 1)])
def test_tolerance_mode_marginal_errors(dd, workload, N, init, levels, aa):
    """levels > 0: eps-scaling inside each solve (coarser eps first); aa > 0:
    Anderson acceleration of the X-dual iteration. The stop and the solution are
    those of the target eps and of plain Sinkhorn (same fixed point, same
    stopping pair), so the same bounds hold."""
    mu, nu, eps, p = synth.workload(workload, 0, N=N)
    tol = 1e-5
    boxes = None if init == "product" else synth.boxes_from_coupling(mu.shape, 4, *synth.knothe_rosenblatt(mu, nu))
    g = dd.DomDec(mu, nu, eps, 4, boxes=boxes, tol=tol, max_iter=20000, eps_levels=levels, eps_factor=4.0,
                  anderson=aa)
    geom = Geometry(N, N, 4)
    for part in (0, 1, 0):
        st = g.iterate(part)
        assert st["n_maxiter"] == 0
        errs = gpu_cell_errors(g, part, mu, nu, eps, geom)
        assert max(e[1] for e in errs) <= tol + 3e-5
        assert max(e[2] for e in errs) <= 3e-5
        E, l1x, l1y = g.objective()
        assert l1x <= tol * 1.0 + 1e-12          # the kernel's own FP32 error estimate
        assert l1y <= 1e-6
    g.close()


@pytest.mark.parametrize("share,omega,gamma,aa", [(1.0, 1.0, 0.0, 0), (0.5, 1.4, 0.0, 0), (1.0, 1.4, 1.0, 0),
                                                   (1.0, 1.0, 1.0, 4)])
def test_tolerance_mode_batch_budget(dd, share, omega, gamma, aa):
    """dd_options.tol_share = s: cell J stops at L1 X error <= tol ((1 - s) m_J +
    s mean(m)), budgets that sum to tol |mu| (the paper's batch criterion over
    all cells of the half-iteration). FP64 re-evaluation of the exported duals:
    each cell within its budget (+ the FP32 slack of the per-cell test), the
    kernel's own total within tol; with over-relaxation (omega) or Anderson
    acceleration (aa) the same holds.
    tol_gamma > 0 reweights the budgets by the previous iteration counts (still
    summing to tol |mu|): the per-cell bound is then the total one."""
    mu, nu, eps, p = synth.workload("dd256", 0, N=64)
    tol = 1e-5
    boxes = synth.boxes_from_coupling(mu.shape, 4, *synth.knothe_rosenblatt(mu, nu))
    g = dd.DomDec(mu, nu, eps, 4, boxes=boxes, tol=tol, max_iter=20000, eps_levels=2, eps_factor=4.0,
                  tol_share=share, omega=omega, tol_gamma=gamma, anderson=aa)
    geom = Geometry(64, 64, 4)
    m = geom.basic_masses(mu)
    for part in (0, 1, 0):
        st = g.iterate(part)
        assert st["n_maxiter"] == 0 and st["n_stalled"] == 0
        parts = geom.partition(part)
        mJ = np.array([m[c].sum() for c in parts])
        budget = tol * ((1 - share) * mJ + share * mJ.mean()) if gamma == 0 else np.full(len(mJ), tol * mJ.sum())
        total = 0.0
        for J, xe, ye in gpu_cell_errors(g, part, mu, nu, eps, geom):
            assert xe * mJ[J] <= budget[J] + 3e-5 * mJ[J], (J, xe * mJ[J], budget[J])
            assert ye <= 3e-5
            total += xe * mJ[J]
        assert total <= tol * mJ.sum() + 3e-5 * mJ.sum()
        assert st["l1_x"] <= tol * mJ.sum() + 1e-12
    g.close()


def test_flow_update_matches_oracle_on_gpu_state(dd):
    N, s = 32, 4
    mu, nu, eps, _ = synth.workload("dd32", 0, N=N)
    geom = Geometry(N, N, s)
    m = geom.basic_masses(mu)
    nbr = geom.neighbours()
    g = dd.DomDec(mu, nu, eps, s, tol=1e-6)
    g.iterate(0)
    g.iterate(1)
    state = as_boxes(g.plan())
    D = g.basic_moments()["D"]
    f = g.flow_update()
    cbar, w = g.flow()
    ref = edge_costs(geom, mu, state, D, 1.0 / N)
    ok = ~np.isnan(ref)
    scale = np.abs(ref[ok]).max()
    assert np.abs(cbar[ok] - ref[ok]).max() <= 5e-7 * scale
    _, val_ref, _ = min_cost_flow(nbr, cbar, m)
    assert f["value"] == pytest.approx(val_ref, rel=1e-9, abs=1e-18)
    assert f["value"] < 0
    new_ref = exchange(geom, state, w, nbr, m, 1e-15)
    new = as_boxes(g.plan())
    assert plan_l1(new, new_ref, mu.shape) <= 1e-6
    assert l1_y_error(new, nu) <= 1e-5
    assert np.allclose([b.a.sum() for b in new], m, rtol=1e-6)
    g.close()


def test_flow_update_large_union_boxes_match_oracle(dd):
    """The exchange when the union box of a target exceeds the 4096 entries its
    kernel keeps in shared memory (the second gather for the compact write): a
    wide blur (eps = 0.5) keeps every basic box at the whole 72 x 72 grid."""
    N, s = 72, 4
    mu, nu, _, _ = synth.workload("dd32", 0, N=N)
    geom = Geometry(N, N, s)
    m = geom.basic_masses(mu)
    nbr = geom.neighbours()
    g = dd.DomDec(mu, nu, 0.5, s, tol=1e-6)
    g.iterate(0)
    g.iterate(1)
    state = as_boxes(g.plan())
    assert max(b.a.size for b in state) > 4096
    g.flow_update()
    _, w = g.flow()
    new_ref = exchange(geom, state, w, nbr, m, 1e-15)
    new = as_boxes(g.plan())
    assert max(b.a.size for b in new) > 4096
    assert plan_l1(new, new_ref, mu.shape) <= 1e-6
    assert np.allclose([b.a.sum() for b in new], m, rtol=1e-6)
    g.close()


@pytest.mark.parametrize("m,small_threads", [(8, 64), (32, 64), (32, None), (128, None)])
def test_cell_lse_box_sweep_cells_match_oracle(dd, m, small_threads):
    """The cell-LSE microbenchmark's inputs (synth.cell_lse_sweep: (2048/m)^2
    cells, 8 x 8 X blocks, m x m Gaussian boxes, cold start, 30 fixed iterations):
    sampled cells' pre-balance basic marginals and D_i against the FP64 oracle,
    with the default launch configuration or the small-box class on 64-thread CTAs.
    Bound 1e-5 (L1 per unit basic mass, relative D_i), the fixed-iteration bound
    above; measured <= 7.8e-7 at every box size from 8 to 128."""
    from oracle.domdec import composite_to_basic, solve_cell

    K = 30
    mu, nu, eps, s, (hdr, data) = synth.cell_lse_sweep(m, 0)
    N = mu.shape[0]
    g = dd.DomDec(mu, nu, eps, s, boxes=(hdr, data), fixed_iters=K, warm=dd.DD_WARM_COLD,
                  flags=dd.DD_FLAG_NO_GRAPH | dd.DD_FLAG_KEEP_PREBALANCE | dd.DD_FLAG_TRACE)
    if small_threads:
        g.set_tuning([512, small_threads, 512], 3072, 96, cl_size=1, cl_cells=0)
    st = g.iterate(0)
    assert st["ncell"] == (2048 // m) ** 2 and st["iters_max"] == K
    if small_threads:
        assert (g.trace(0)[:, 3] == small_threads).all()  # every cell ran on the small class
    pre = g.prebalance()
    D = g.basic_moments()["D"]
    g.close()
    geom = Geometry(N, N, s)
    mi = geom.basic_masses(mu)
    bx = [Box(o1, o2, np.asarray(a)) for o1, o2, a in dd.arrays_to_boxes(hdr, data)]
    cells = geom.partition(0)
    for J in np.random.default_rng(5).choice(len(cells), 3, replace=False):
        members = cells[J]
        nuJ = basic_to_composite(bx, members)
        assert (nuJ.h, nuJ.w) == (m, m)
        res = solve_cell(geom, mu, eps, 1.0 / N, members, nuJ, None, 1e-5, 100000, fixed_iters=K)
        arrs, Dref = composite_to_basic(geom, members, nuJ, res)
        for k, i in enumerate(members):
            o1, o2, got = pre[i]
            assert (o1, o2, got.shape) == (nuJ.o1, nuJ.o2, nuJ.a.shape)
            assert np.abs(got - arrs[k]).sum() <= 1e-5 * mi[i], (m, J, i)
            assert abs(D[i] - Dref[k]) <= 1e-5 * abs(Dref[k]), (m, J, i)


def _basic_plans_from_gpu_duals(g, part, mu, nu, eps, geom):
    """The Gibbs cell plans of the GPU's exported duals (FP64), split into the
    basic cells' rows: per basic cell (Y pixels, pi_i), and D_i = <c, pi_i>."""
    alpha, betas = g.duals(part)
    comp = g.composite(part)
    N = mu.shape[0]
    ss = geom.s * geom.s
    plans, D = [None] * geom.nb, np.zeros(geom.nb)
    for J, members in enumerate(geom.partition(part)):
        X = geom.composite_pixels(members)
        o1, o2, nuJ = comp[J]
        _, _, beta = betas[J]
        Y = box_pixels(o1, o2, nuJ.shape[0], nuJ.shape[1])
        supp = nuJ.reshape(-1) > 0
        C = sq_cost(X, Y[supp], 1.0 / N)
        a = alpha[X[:, 0], X[:, 1]]
        b = beta.reshape(-1)[supp]
        pi = np.exp((a[:, None] + b[None, :] - C) / eps) * mu[X[:, 0], X[:, 1]][:, None] * nu[Y[supp][:, 0], Y[supp][:, 1]][None, :]
        for k, i in enumerate(members):
            plans[i] = (Y[supp], pi[k * ss:(k + 1) * ss])
            D[i] = float((C[k * ss:(k + 1) * ss] * pi[k * ss:(k + 1) * ss]).sum())
    return plans, D


def test_glued_edge_costs_match_oracle_on_gpu_state(dd):
    """Gluing candidates from entropic gamma_ij (eps_gamma = (h/2)^2, Def. 3.7,
    Remark 3.8): the library's edge costs (gamma_ij by its FP64 device solve,
    the per-pixel mass and mean displacement of each cell plan from the FP32
    duals) against the oracle's explicit sums <c, pi_hat_ij> - D_i / m_i over the
    matrix-product candidate of Eq. (glued-plan), built from the same exported
    duals in FP64 with the oracle's own gamma_ij. Both terms of c_bar come from
    FP32 plan moments summed in FP32 per pixel (relative ~1e-6 each, the terms up
    to max |c_bar|): within 2e-6 of max |c_bar|; then the flow value equals the
    oracle LP's on those costs (1e-9) and the exchange matches."""
    from oracle.flow import edge_costs_glued, gluing_plans

    N, s = 32, 4
    mu, nu, eps, _ = synth.workload("dd32", 0, N=N)
    geom = Geometry(N, N, s)
    m = geom.basic_masses(mu)
    nbr = geom.neighbours()
    eg = (0.5 / N) ** 2
    g = dd.DomDec(mu, nu, eps, s, tol=1e-6, eps_gamma=eg)
    g.iterate(0)
    g.iterate(1)
    state = as_boxes(g.plan())
    f = g.flow_update()
    cbar, w = g.flow()
    plans, D = _basic_plans_from_gpu_duals(g, 1, mu, nu, eps, geom)
    ref = edge_costs_glued(geom, mu, plans, D, 1.0 / N, gluing_plans(geom, mu, 1.0 / N, eg))
    ok = ~np.isnan(ref)
    scale = np.abs(ref[ok]).max()
    assert np.abs(cbar[ok] - ref[ok]).max() <= 2e-6 * scale, np.abs(cbar[ok] - ref[ok]).max() / scale
    _, val_ref, _ = min_cost_flow(nbr, cbar, m)
    assert f["value"] == pytest.approx(val_ref, rel=1e-9, abs=1e-18)
    assert f["value"] < 0
    new_ref = exchange(geom, state, w, nbr, m, 1e-15)
    assert plan_l1(as_boxes(g.plan()), new_ref, mu.shape) <= 1e-6
    g.close()
