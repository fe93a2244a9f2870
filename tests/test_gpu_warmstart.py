"""The learned warm start on the GPU against the FP64 reference (oracle/mlp.py,
oracle/warmstart.py), through the C ABI.

Tolerances:
* network forward pass and gradient: both sides get the same BF16-rounded
  weights and inputs; the GPU rounds every hidden activation and every
  back-propagated gradient to BF16 (relative 2^-9) between layers and
  accumulates in FP32, so outputs and per-tensor gradients agree to 1e-2 in
  relative Frobenius norm (the precision the design states for BF16 paths);
* one Adam step from a known gradient: first step, m_hat = g and v_hat = g^2,
  so the update is lr g / (|g| + 1e-8) to FP32 rounding (rel 1e-5);
* features: BF16 outputs of FP32/FP64 arithmetic, |diff| <= 2^-8 |ref| + 2e-3;
* targets: same fixed iteration count on both sides from a cold start; the
  FP32 duals of the kernel (magnitudes up to a few hundred in base-2 units after
  its change of gauge) differ from the FP64 ones by ~1e-4, the r values and the
  auxiliary log duals to <= 2e-3 absolute.
"""

import os

import numpy as np
import pytest

import synth
from oracle import mlp as omlp
from oracle import warmstart as ows
from oracle.cell import cell_sinkhorn, sq_cost
from oracle.domdec import Box, basic_to_composite, box_pixels
from oracle.geometry import Geometry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd(lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib


def bf16(a):
    import torch

    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)


def rand_net(seed):
    from paper_2405_09400_gb300 import warmstart as ws

    rng = np.random.default_rng(seed)
    p = ws.init_params(seed)
    for _, bsl, _, _ in ws.layer_slices():
        p[bsl] = rng.normal(0, 0.1, bsl.stop - bsl.start).astype(np.float32)
    last_w = ws.layer_slices()[-1][0]
    p[last_w] *= 10.0
    q = p.copy()
    for wsl, _, _, _ in ws.layer_slices():
        q[wsl] = ws.round_bf16(q[wsl])
    return q


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("M", [1, 77, 200])
def test_mlp_forward_and_gradient_match_fp64_reference(dd, M):
    import torch

    p = rand_net(M)
    rng = np.random.default_rng(10 + M)
    Xh = bf16(rng.normal(0, 1, (M, 336)))
    X64 = Xh.float().numpy().astype(np.float64)
    T = rng.normal(0, 1, (M, 320)).astype(np.float32)
    w = rng.uniform(0.1, 1.0, 320).astype(np.float32)
    net = dd.MLP(256)
    net.set_params(p)
    y = net.forward(Xh.cuda()).cpu().numpy()
    yref, _ = omlp.forward(p.astype(np.float64), X64)
    assert rel(y, yref) <= 1e-2
    L, g = net.loss_grad(Xh.cuda(), torch.tensor(T).cuda(), torch.tensor(w).cuda())
    Lref, gref = omlp.loss_and_grad(p.astype(np.float64), X64, T.astype(np.float64), w.astype(np.float64))
    assert L == pytest.approx(Lref, rel=1e-2)
    from paper_2405_09400_gb300 import warmstart as ws

    for wsl, bsl, _, _ in ws.layer_slices():
        assert rel(g[wsl], gref[wsl]) <= 1e-2
        assert rel(g[bsl], gref[bsl]) <= 1e-2
    net.close()


@pytest.mark.parametrize("M", [1, 128, 129, 1089, 4500])
def test_mlp_forward_tcgen05_matches_mma_sync(dd, M):
    """The forward layer products on the tcgen05 kernel (TMA-staged operands,
    TMEM accumulator; one 128 x 64 tile per CTA, ragged M tails zero-filled by
    the tensor maps) against the warp-level mma.sync kernel on the same BF16
    weights and inputs. Both sum the same BF16 products in FP32 and round each
    hidden layer to BF16, so they differ only through the summation order and
    the few BF16 roundings it flips: relative Frobenius norm <= 2e-3, and a
    layout or descriptor error would give an O(1) difference."""
    p = rand_net(5)
    rng = np.random.default_rng(20 + M)
    X = bf16(rng.normal(0, 1, (M, 336))).cuda()
    net = dd.MLP(M)
    net.set_params(p)
    y_tc = net.forward(X).cpu().numpy()
    net.set_gemm(dd.DD_MLP_GEMM_MMA)
    y_ref = net.forward(X).cpu().numpy()
    net.set_gemm(dd.DD_MLP_GEMM_UMMA)
    y_tc2 = net.forward(X).cpu().numpy()
    net.get_params()  # synchronises and reports a timed-out wait, if any
    net.close()
    assert np.isfinite(y_tc).all()
    assert np.array_equal(y_tc, y_tc2)  # deterministic
    assert rel(y_tc, y_ref) <= 2e-3
    yref64, _ = omlp.forward(p.astype(np.float64), X.cpu().float().numpy().astype(np.float64))
    assert rel(y_tc, yref64) <= 1e-2


def test_mlp_set_gemm_rejects_unknown_kind(dd):
    net = dd.MLP(8)
    with pytest.raises(dd.DDError):
        net.set_gemm(7)
    net.close()


def test_adam_first_step(dd):
    import torch

    p = rand_net(3)
    rng = np.random.default_rng(4)
    M = 64
    X = bf16(rng.normal(0, 1, (M, 336))).cuda()
    T = torch.tensor(rng.normal(0, 1, (M, 320)).astype(np.float32)).cuda()
    w = torch.ones(320, device="cuda")
    net = dd.MLP(M)
    net.set_params(p)
    p0 = net.get_params()
    L0, g = net.loss_grad(X, T, w)
    idx = torch.arange(M, dtype=torch.int32, device="cuda")
    lr = 1e-3
    Lb = net.train_step(X, T, idx, w, lr, want_loss=True)
    assert Lb == pytest.approx(L0, rel=1e-6)
    p1 = net.get_params().astype(np.float64)
    g = g.astype(np.float64)
    expect = p0.astype(np.float64) - lr * g / (np.abs(g) + 1e-8)
    assert np.abs(p1 - expect).max() <= 1e-5 * lr + 1e-7
    # a few more steps on the same batch lower the loss
    for _ in range(20):
        net.train_step(X, T, idx, w, lr)
    L2, _ = net.loss_grad(X, T, w)
    assert L2 < 0.9 * L0
    net.close()


def _cold_run(dd, K, N=64):
    mu, nu, eps, p = synth.workload("dd256", 0, N=N)
    boxes = synth.boxes_from_coupling(mu.shape, 4, *synth.knothe_rosenblatt(mu, nu))
    g = dd.DomDec(mu, nu, eps, 4, boxes=boxes, fixed_iters=K, warm=dd.DD_WARM_COLD, flags=dd.DD_FLAG_COLLECT)
    return mu, nu, eps, boxes, g


def test_features_and_targets_match_reference(dd):
    K = 40
    N = 64
    mu, nu, eps, boxes, g = _cold_run(dd, K, N)
    g.iterate(0)
    feat, targ = g.collect(0)
    feat = feat.float().cpu().numpy()
    targ = targ.cpu().numpy()
    geom = Geometry(N, N, 4)
    cells = geom.partition(0)
    assert feat.shape == (len(cells), 336) and targ.shape == (len(cells), 320)
    h = 1.0 / N
    k2 = h * h / (eps * np.log(2.0))
    bx = [Box(o1, o2, np.asarray(a)) for o1, o2, a in boxes]
    rng = np.random.default_rng(0)
    for J in rng.choice(len(cells), 10, replace=False):
        members = cells[J]
        r0, c0, hx, wx, perm = ows.block_of(geom, members)
        nuJ = basic_to_composite(bx, members)
        mu_blk = mu[r0:r0 + 8, c0:c0 + 8]
        fref = ows.cell_features(mu_blk, r0, c0, nuJ.a, nuJ.o1, nuJ.o2, k2)
        assert np.all(np.abs(feat[J] - fref) <= 2.0 ** -8 * np.abs(fref) + 2e-3), J
        # the oracle's own solve of the same cell, same iteration count, cold
        X = geom.composite_pixels(members)
        Y = box_pixels(nuJ.o1, nuJ.o2, nuJ.h, nuJ.w)
        flat = nuJ.a.reshape(-1)
        supp = flat > 0
        C = sq_cost(X, Y[supp], h)
        res = cell_sinkhorn(mu[X[:, 0], X[:, 1]], flat[supp], C, eps, np.zeros(len(X)), fixed_iters=K)
        alpha_blk = res["alpha"][perm].reshape(8, 8)
        tref = ows.cell_targets(alpha_blk, mu_blk, nuJ.a, r0, c0, nuJ.o1, nuJ.o2, eps, k2)
        assert np.abs(targ[J, :64] - tref[:64]).max() <= 2e-3, J
        assert np.abs(targ[J, 64:] - tref[64:]).max() <= 2e-3, J
    g.close()


@pytest.mark.parametrize("warm", ["affine", "mlp"])
def test_warm_started_solves_reach_tolerance(dd, warm):
    """Any warm start gives the same tolerance; a random network only changes
    iteration counts."""
    N = 64
    mu, nu, eps, p = synth.workload("dd256", 0, N=N)
    boxes = synth.boxes_from_coupling(mu.shape, 4, *synth.knothe_rosenblatt(mu, nu))
    tol = 1e-5
    ref = dd.DomDec(mu, nu, eps, 4, boxes=boxes, tol=tol, max_iter=20000)
    kw = dict(warm=dd.DD_WARM_AFFINE) if warm == "affine" else dict(warm=dd.DD_WARM_MLP, weights=rand_net(7) * 0.01)
    g = dd.DomDec(mu, nu, eps, 4, boxes=boxes, tol=tol, max_iter=20000, **kw)
    for part in (0, 1, 0):
        a = ref.iterate(part)
        b = g.iterate(part)
        assert b["n_maxiter"] == 0
        assert abs(a["objective"] - b["objective"]) <= 1e-4 * abs(a["objective"])
        E, l1x, l1y = g.objective()
        assert l1x <= tol and l1y <= 1e-6
    ref.close()
    g.close()


def test_mlp_warm_start_requires_weights(dd):
    mu, nu, eps, p = synth.workload("dd32", 0, N=16)
    g = dd.DomDec(mu, nu, eps, 4, warm=dd.DD_WARM_MLP)
    with pytest.raises(dd.DDError) as e:
        g.iterate(0)
    assert e.value.code == dd.DD_ERR_STATE
    g.close()


WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2405_09400_gb300", "weights",
                       "warm_mlp_dd256.npz")


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained weights in the package")
def test_trained_network_lowers_iterations_on_unseen_seeds(dd):
    """The committed network, trained on seeds 100-124, on unseen seeds 0-2,
    three hybrid iterations from the Knothe-Rosenblatt coupling (tol 1e-5):
    the method's own initialisation (previous-iterate duals, cold on the first
    solve), the analytic affine start, and the network (its prediction on the
    first solve of a partition, the previous dual afterwards; with
    DD_FLAG_MLP_EVERY_SOLVE the previous dual plus the network's predicted change).
    Same tolerance everywhere. On the first iteration the network needs the fewest
    Sinkhorn iterations; over the run it never needs more than the method without
    it (2 % slack; 5 % for the every-solve variant)."""
    from paper_2405_09400_gb300 import warmstart as ws

    params, _ = ws.load_params(WEIGHTS)
    for k in range(3):
        mu, nu, eps, p = synth.workload("dd256", k)
        boxes = synth.boxes_from_coupling(mu.shape, 4, *synth.knothe_rosenblatt(mu, nu))
        first, total = {}, {}
        for name, kw in (("prev", dict(warm=dd.DD_WARM_PREV)), ("affine", dict(warm=dd.DD_WARM_AFFINE)),
                         ("mlp", dict(warm=dd.DD_WARM_MLP, weights=params)),
                         ("mlp_every", dict(warm=dd.DD_WARM_MLP, weights=params, flags=dd.DD_FLAG_MLP_EVERY_SOLVE))):
            g = dd.DomDec(mu, nu, eps, 4, boxes=boxes, tol=1e-5, max_iter=20000, **kw)
            tot = []
            for _ in range(3):
                a = g.iterate(0)
                b = g.iterate(1)
                assert a["n_maxiter"] == 0 and b["n_maxiter"] == 0
                E, l1x, l1y = g.objective()
                assert l1x <= 1e-5
                tot.append(a["iters_mean"] + b["iters_mean"])
                g.flow_update()
            first[name], total[name] = tot[0], sum(tot)
            g.close()
        assert first["mlp"] <= 0.75 * first["prev"], (k, first)
        assert first["mlp"] < first["affine"], (k, first)
        assert total["mlp"] <= 1.02 * total["prev"], (k, total)
        # same first solves; the network inputs are resampled with float atomics
        # (summation order varies), so a few cells may differ by an iteration
        assert abs(first["mlp_every"] - first["mlp"]) <= 0.01 * first["mlp"], (k, first)
        assert total["mlp_every"] <= 1.05 * total["prev"], (k, total)
