"""Pins of the FP64 warm-start reference (oracle/mlp.py, oracle/warmstart.py)
against independent facts: automatic differentiation and finite differences for
the network gradient; exact resampling identities; translation invariance of the
dual target (a shift of nu_J changes the exact dual by a linear function, which
the target removes); the auxiliary Y target against the Sinkhorn Y-update."""

import numpy as np
import pytest
import torch

import synth
from oracle import mlp
from oracle import warmstart as ws
from oracle.cell import cell_sinkhorn, sq_cost, y_update
from oracle.domdec import box_pixels

SMALL = (7, 6, 5, 4)


def rand_problem(dims, B, seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.5, mlp.n_params(dims))
    X = rng.normal(0, 1, (B, dims[0]))
    T = rng.normal(0, 1, (B, dims[-1]))
    w = rng.uniform(0.5, 2.0, dims[-1])
    return p, X, T, w


@pytest.mark.parametrize("dims", [SMALL, (12, 9, 3)])
def test_mlp_gradient_matches_autograd(dims):
    p, X, T, w = rand_problem(dims, 5, 1)
    L, g = mlp.loss_and_grad(p, X, T, w, dims)
    pt = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    h = torch.tensor(X)
    o = 0
    n_layers = len(dims) - 1
    for l in range(n_layers):
        k, n = dims[l], dims[l + 1]
        W = pt[o:o + n * k].reshape(n, k)
        o += n * k
        b = pt[o:o + n]
        o += n
        z = h @ W.T + b
        h = torch.nn.functional.silu(z) if l < n_layers - 1 else z
    Lt = (torch.tensor(w)[None, :] * (h - torch.tensor(T)) ** 2).sum() / X.shape[0]
    Lt.backward()
    assert L == pytest.approx(Lt.item(), rel=1e-13)
    assert np.abs(g - pt.grad.numpy()).max() <= 1e-12 * np.abs(g).max()


def test_mlp_gradient_central_differences():
    p, X, T, w = rand_problem(SMALL, 4, 2)
    _, g = mlp.loss_and_grad(p, X, T, w, SMALL)
    rng = np.random.default_rng(0)
    for k in rng.choice(len(p), 25, replace=False):
        e = np.zeros_like(p)
        e[k] = 1e-5
        fd = (mlp.loss(p + e, X, T, w, SMALL) - mlp.loss(p - e, X, T, w, SMALL)) / 2e-5
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k]))


def test_mlp_full_size_shapes_and_silu():
    assert mlp.n_params() == 336 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 320 + 320
    z = np.array([0.0, 50.0, -50.0])
    assert np.allclose(mlp.silu(z), [0.0, 50.0, 0.0], atol=1e-18)
    assert np.allclose(mlp.silu_grad(z), [0.5, 1.0, 0.0], atol=1e-18)
    # a network whose weights are all zero outputs its last bias
    p = np.zeros(mlp.n_params())
    p[-320:] = np.arange(320)
    y, _ = mlp.forward(p, np.ones((2, 336)))
    assert np.array_equal(y, np.tile(np.arange(320.0), (2, 1)))


@pytest.mark.parametrize("n", [3, 8, 16, 23, 32, 57])
def test_resample_overlap_is_mass_preserving(n):
    R = ws.overlap_matrix(n)
    assert np.allclose(R.sum(axis=0), 1.0, atol=1e-14)          # every pixel fully distributed
    assert np.allclose(R.sum(axis=1), n / 16.0, atol=1e-14)     # every output covers n/16 pixels
    a = np.random.default_rng(n).uniform(0, 1, (n, 16))
    rs = ws.resample16(a)
    assert rs.sum() == pytest.approx(a.sum(), rel=1e-14)


def test_resample_special_sizes():
    a = np.random.default_rng(0).uniform(0, 1, (16, 16))
    assert np.allclose(ws.resample16(a), a, atol=1e-15)
    b = np.random.default_rng(1).uniform(0, 1, (32, 32))
    assert np.allclose(ws.resample16(b), b.reshape(16, 2, 16, 2).sum(axis=(1, 3)), atol=1e-14)
    c = np.random.default_rng(2).uniform(0, 1, (8, 8))
    assert np.allclose(ws.resample16(c), np.kron(c, np.ones((2, 2))) / 4, atol=1e-15)


def test_gauge_of_uniform_block():
    mu = np.full((8, 8), 1 / 64)
    nu = np.zeros((16, 8))
    nu[:, :] = 1 / 128
    g = ws.cell_gauge(mu, 0, 0, nu, 4, 0)
    assert np.allclose(g["uc"], [3.5, 3.5]) and np.allclose(g["vc"], [7.5, 3.5])
    assert np.allclose(g["vu"], [63 / 12, 63 / 12]) and np.allclose(g["vv"], [255 / 12, 63 / 12])
    assert np.allclose(g["l"], [np.sqrt(255 / 63), 1.0])
    assert np.allclose(g["d"], [-4 + 3.5 - 7.5, 0.0])
    # product measures: the Gaussian map is the per-axis stretch
    assert np.allclose(g["A"], np.diag(g["l"]), atol=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_gaussian_map_pushes_covariance(seed):
    """A is symmetric positive semidefinite and A S A = T: the linear map that
    carries the covariance of mu_J onto that of nu_J (the defining property of
    the quadratic-cost transport map between Gaussians)."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.2, 1.0, (8, 8))
    nu = rng.uniform(0.0, 1.0, (11 + seed, 17 - seed)) ** 3
    g = ws.cell_gauge(mu, 0, 0, nu, 2, 3)
    A, S, T = g["A"], g["S"], g["T"]
    assert np.allclose(A, A.T, atol=1e-12)
    assert np.linalg.eigvalsh(A).min() >= -1e-12
    assert np.allclose(A @ S @ A, T, atol=1e-10 * np.abs(T).max())


def _solve(mu_blk, r0, c0, nu_arr, o1, o2, eps, h):
    X = box_pixels(r0, c0, 8, 8)
    Y = box_pixels(o1, o2, *nu_arr.shape)
    C = sq_cost(X, Y, h)
    res = cell_sinkhorn(mu_blk.reshape(-1), nu_arr.reshape(-1), C, eps, np.zeros(64), tol=1e-13, max_iter=200000)
    return res, C


@pytest.mark.parametrize("shift", [(0, 0), (3, -2), (-5, 4)])
def test_alpha_target_is_translation_invariant(shift):
    """nu_J = mu_J translated by t: the exact dual is the t = 0 dual minus
    2 h^2 t.x (the cost's cross term), so the target does not depend on t."""
    N, eps = 64, 2.0 / 64 ** 2
    h = 1.0 / N
    k2 = h * h / (eps * np.log(2.0))
    mu_full, _, _, _ = synth.workload("dd32", 3, N=N)
    mu_blk = mu_full[20:28, 20:28] / mu_full[20:28, 20:28].sum() * 0.01
    nu_arr = mu_blk.copy()
    t = np.array(shift)
    base = None
    res, _ = _solve(mu_blk, 20, 20, nu_arr, 20 + t[0], 20 + t[1], eps, h)
    r = ws.cell_targets(res["alpha"].reshape(8, 8), mu_blk, nu_arr, 20, 20, 20 + t[0], 20 + t[1], eps, k2)
    res0, _ = _solve(mu_blk, 20, 20, nu_arr, 20, 20, eps, h)
    base = ws.cell_targets(res0["alpha"].reshape(8, 8), mu_blk, nu_arr, 20, 20, 20, 20, eps, k2)
    assert np.abs(r - base).max() <= 1e-8
    # zero shift and equal shapes: d = 0, l = 1, r is the centred dual in base-2 units
    a = res0["alpha"] / (eps * np.log(2.0))
    a = a - (mu_blk.reshape(-1) * a).sum() / mu_blk.sum()
    assert np.abs(base[:64] - a).max() <= 1e-10


def test_alpha_target_round_trip():
    rng = np.random.default_rng(5)
    mu_blk = rng.uniform(0.5, 1.5, (8, 8))
    nu = rng.uniform(0, 1, (13, 21))
    eps, k2 = 2e-4, 0.7
    g = ws.cell_gauge(mu_blk, 40, 60, nu, 37, 50)
    alpha = rng.normal(0, 1e-3, (8, 8))
    r = ws.alpha_target(alpha, mu_blk, eps, k2, g)
    back = ws.alpha_from_prediction(r, mu_blk, eps, k2, g)
    diff = back - alpha
    assert np.abs(diff - diff.mean()).max() <= 1e-15


def test_beta_aux_target_matches_sinkhorn_y_update():
    """G is the Sinkhorn Y-update of the cell (beta_t / (eps ln 2)) plus the
    separable gauge term -k2 sum_k (1 - 1/l_k) vb_k^2 + 2 k2 d.vb, up to a
    constant (expand k2 |d + ub - vb|^2 against K and the subtracted base)."""
    N = 64
    h = 1.0 / N
    eps = 2 * h * h
    k2 = h * h / (eps * np.log(2.0))
    mu_full, nu_full, _, _ = synth.workload("dd32", 1, N=N)
    r0, c0, o1, o2 = 16, 24, 12, 26
    mu_blk = mu_full[r0:r0 + 8, c0:c0 + 8]
    nu_arr = nu_full[o1:o1 + 19, o2:o2 + 11] * 0.3
    nu_arr = nu_arr / nu_arr.sum() * mu_blk.sum()
    res, C = _solve(mu_blk, r0, c0, nu_arr, o1, o2, eps, h)
    tgt = ws.cell_targets(res["alpha"].reshape(8, 8), mu_blk, nu_arr, r0, c0, o1, o2, eps, k2)
    g = ws.cell_gauge(mu_blk, r0, c0, nu_arr, o1, o2)
    bt = y_update(res["alpha"], mu_blk.reshape(-1), C, eps).reshape(nu_arr.shape) / (eps * np.log(2.0))
    p1, p2 = ws.sample_pixels(*nu_arr.shape)
    vb1 = p1[:, None] - g["vc"][0]
    vb2 = p2[None, :] - g["vc"][1]
    ref = (bt[np.ix_(p1, p2)] - k2 * ((1 - 1 / g["l"][0]) * vb1 ** 2 + (1 - 1 / g["l"][1]) * vb2 ** 2)
           + 2 * k2 * (g["d"][0] * vb1 + g["d"][1] * vb2))
    ref = (ref - ref.mean()).reshape(-1)
    assert np.abs(tgt[64:] - ref).max() <= 1e-9


def test_features_of_a_known_cell():
    mu_blk = np.full((8, 8), 0.5)
    nu_arr = np.zeros((32, 16))
    nu_arr[8:24, :] = 1.0
    f = ws.cell_features(mu_blk, 100, 100, nu_arr, 90, 96, 0.5)
    assert np.allclose(f[:64], 0.0)
    rs = 2.0 ** (4 * f[64:320].reshape(16, 16)) - 1.0 / 256
    assert np.allclose(rs[4:12], 2.0) and np.allclose(rs[:4], 0.0) and np.allclose(rs[12:], 0.0)
    assert np.allclose(f[320:336], [1.0, 0.5, (10 + 3.5 - 15.5) / 8, (4 + 3.5 - 7.5) / 8, np.log2(np.sqrt((255 / 12) / (63 / 12))),
                                    np.log2(np.sqrt((255 / 12) / (63 / 12))), 0.0, 0.0, 0.0, 0.0, -1.0,
                                    np.sqrt(63 / 12) / 4, np.sqrt(63 / 12) / 4, np.sqrt(255 / 12) / 16,
                                    np.sqrt(255 / 12) / 16, 0.0])


def test_affine_dual_is_exact_for_a_linear_image():
    """nu_J the image of mu_J under x -> A0 x + t on a fine enough grid that the
    moments match: the map A recovered from the moments equals A0, and the
    target r of the exact unregularised dual vanishes."""
    rng = np.random.default_rng(3)
    A0 = np.array([[1.6, 0.4], [0.4, 0.9]])
    mu = rng.uniform(0.5, 1.5, (8, 8))
    # the moments of nu_J = the pushforward of mu_J
    g = ws.cell_gauge(mu, 0, 0, mu, 0, 0)
    S = g["S"]
    T = A0 @ S @ A0
    g2 = dict(g)
    g2["T"] = T
    Sh = np.real(ws.sqrtm(S))
    Shi = np.linalg.inv(Sh)
    A = Shi @ np.real(ws.sqrtm(Sh @ T @ Sh)) @ Shi
    assert np.allclose(A, A0, atol=1e-10)
    g2["A"] = A
    g2["d"] = np.array([1.5, -2.0])
    eps, k2 = 1e-3, 0.9
    ub1, ub2 = ws._ub(g2, 8, 8)
    # Brenier potential of T(x) = A0 x + t in centred coordinates, in base-2 units
    alpha = eps * np.log(2.0) * k2 * (ub1 ** 2 + ub2 ** 2 - (A0[0, 0] * ub1 ** 2 + 2 * A0[0, 1] * ub1 * ub2
                                                             + A0[1, 1] * ub2 ** 2) + 2 * (1.5 * ub1 - 2.0 * ub2))
    r = ws.alpha_target(alpha, mu, eps, k2, g2)
    assert np.abs(r).max() <= 1e-9
