"""Pins for the oracle's cell solver (oracle.cell).

Independent checks: the 2x2 closed form of the entropic problem, the Dirac
special case, the Gibbs optimality certificate of Prop. 2.1 (iii), and an
independent optimiser (scipy L-BFGS on the smooth dual) on a small problem.
"""

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle.cell import cell_sinkhorn, gibbs_plan, sq_cost


def _solve(mu_x, nu_y, C, eps, tol=1e-14):
    r = cell_sinkhorn(mu_x, nu_y, C, eps, np.zeros(len(mu_x)), tol=tol, max_iter=200000)
    return gibbs_plan(r["alpha"], r["beta_t"], mu_x, nu_y, C, eps), r


@pytest.mark.parametrize("p,q,eps", [(0.3, 0.6, 0.5), (0.5, 0.5, 1.0), (0.2, 0.9, 2.0), (0.7, 0.25, 0.4)])
def test_two_point_closed_form(p, q, eps):
    # X = {0, 1}, Y = {0, 2} on a line (pixel units, h = 1).
    X = np.array([[0, 0], [1, 0]])
    Y = np.array([[0, 0], [2, 0]])
    C = sq_cost(X, Y, 1.0)
    mu_x = np.array([p, 1 - p])
    nu_y = np.array([q, 1 - q])
    pi, _ = _solve(mu_x, nu_y, C, eps)
    # Gibbs form => pi11 pi22 / (pi12 pi21) = K = exp(-(c11 + c22 - c12 - c21) / eps).
    # With pi11 = a: (1 - K) a^2 + (1 - p - q + K (p + q)) a - K p q = 0.
    K = np.exp(-(C[0, 0] + C[1, 1] - C[0, 1] - C[1, 0]) / eps)
    A, B, Cq = 1 - K, 1 - p - q + K * (p + q), -K * p * q
    roots = np.roots([A, B, Cq])
    lo, hi = max(0.0, p + q - 1), min(p, q)
    a = [r.real for r in roots if lo - 1e-12 <= r.real <= hi + 1e-12][0]
    expect = np.array([[a, p - a], [q - a, 1 - p - q + a]])
    assert np.allclose(pi, expect, atol=1e-12, rtol=0)


def test_dirac_target():
    rng = np.random.default_rng(1)
    X = rng.integers(0, 10, size=(9, 2))
    mu_x = rng.random(9)
    mu_x /= mu_x.sum()
    Y = np.array([[4, 5]])
    pi, r = _solve(mu_x, np.array([1.0]), sq_cost(X, Y, 0.1), 0.01)
    assert np.allclose(pi[:, 0], mu_x, atol=1e-15)
    assert r["iters"] <= 2


def _random_cell(seed, nx=12, ny=17):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 6, size=(nx, 2))
    Y = rng.integers(2, 9, size=(ny, 2))
    mu_x = rng.random(nx) + 0.05
    nu_y = rng.random(ny) + 0.05
    mu_x /= mu_x.sum()
    nu_y /= nu_y.sum()
    return X, Y, mu_x, nu_y


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gibbs_certificate(seed):
    """Prop. 2.1 (iii): Gibbs form + exact marginals => optimal. Check both parts."""
    X, Y, mu_x, nu_y = _random_cell(seed)
    eps = 0.3
    C = sq_cost(X, Y, 0.5)
    pi, r = _solve(mu_x, nu_y, C, eps, tol=1e-13)
    assert np.abs(pi.sum(axis=0) - nu_y).sum() < 1e-14       # Y-exact
    assert np.abs(pi.sum(axis=1) - mu_x).sum() < 1e-12       # X within tol
    L = np.log(pi / np.outer(mu_x, nu_y)) + C / eps          # must be alpha(x) + beta(y)
    cross = L[:, None, :, None] + L[None, :, None, :] - L[:, None, None, :] - L[None, :, :, None]
    assert np.abs(cross).max() < 1e-9


def test_matches_independent_dual_optimiser():
    """L-BFGS on the smooth entropic dual reaches the same plan as the Sinkhorn solve."""
    X, Y, mu_x, nu_y = _random_cell(7, nx=6, ny=7)
    eps = 0.5
    C = sq_cost(X, Y, 0.5)
    nx = len(mu_x)

    def negdual(z):
        a, b = z[:nx], z[nx:]
        P = np.exp((a[:, None] + b[None, :] - C) / eps) * np.outer(mu_x, nu_y)
        f = a @ mu_x + b @ nu_y - eps * P.sum()
        g = np.concatenate([mu_x - P.sum(axis=1), nu_y - P.sum(axis=0)])
        return -f, -g

    z = minimize(negdual, np.zeros(nx + len(nu_y)), jac=True, method="L-BFGS-B",
                 options=dict(maxiter=20000, gtol=1e-14, ftol=1e-16)).x
    P_dual = np.exp((z[:nx, None] + z[None, nx:] - C) / eps) * np.outer(mu_x, nu_y)
    pi, _ = _solve(mu_x, nu_y, C, eps, tol=1e-14)
    assert np.abs(P_dual - pi).sum() < 1e-7


def test_stopping_rule_and_fixed_iterations():
    X, Y, mu_x, nu_y = _random_cell(3)
    C = sq_cost(X, Y, 0.5)
    eps = 0.05
    r = cell_sinkhorn(mu_x, nu_y, C, eps, np.zeros(len(mu_x)), tol=1e-6)
    pi = gibbs_plan(r["alpha"], r["beta_t"], mu_x, nu_y, C, eps)
    xerr = np.abs(pi.sum(axis=1) - mu_x).sum()
    assert xerr == pytest.approx(r["err"], rel=1e-9)        # err is the L1 X error of the returned pair
    assert xerr <= 1e-6 * mu_x.sum()
    r5 = cell_sinkhorn(mu_x, nu_y, C, eps, np.zeros(len(mu_x)), fixed_iters=5)
    assert r5["iters"] == 5
    r4 = cell_sinkhorn(mu_x, nu_y, C, eps, np.zeros(len(mu_x)), fixed_iters=4)
    assert not np.allclose(r4["alpha"], r5["alpha"])


def test_gauge_and_translation_invariance():
    X, Y, mu_x, nu_y = _random_cell(4)
    eps = 0.2
    pi0, _ = _solve(mu_x, nu_y, sq_cost(X, Y, 0.5), eps)
    pi1, _ = _solve(mu_x, nu_y, sq_cost(X + 7, Y + 7, 0.5), eps)   # common shift
    assert np.abs(pi0 - pi1).sum() < 1e-12
    r = cell_sinkhorn(mu_x, nu_y, sq_cost(X, Y, 0.5), eps, np.full(len(mu_x), 3.0), tol=1e-14)
    pi2 = gibbs_plan(r["alpha"], r["beta_t"], mu_x, nu_y, sq_cost(X, Y, 0.5), eps)
    assert np.abs(pi0 - pi2).sum() < 1e-12                         # (alpha + C, beta - C)
