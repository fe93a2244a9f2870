"""The composite-cell entropic transport problem and its log-domain Sinkhorn solve.

Alg. 1 (cell problem) asks for argmin <c, pi> + eps KL(pi | mu_J (x) nu) over
Pi(mu_J, nu_J). Since nu_J <= nu, the reference measure mu_J (x) nu_J gives the
same minimiser (the two objectives differ by a constant, Section 2.3), so the
solve uses mu_J (x) nu_J and a Gibbs plan

    pi(x, y) = exp((alpha(x) + beta_t(y) - c(x, y)) / eps) mu(x) nu_J(y)

(Prop. 2.1 (ii)). Sinkhorn alternates, in the log domain (Section A.1, "Custom
CUDA Sinkhorn"), a Y-update that makes the Y-marginal exactly nu_J and an
X-update; the sums are DENSE double sums over X_J x Y (no separable
factorisation).

Readings (Section A.2, "Stopping criterion"):
* one iteration = Y-update beta_t <- Y(alpha), then X-update alpha' <- X(beta_t);
* its error is the L1 X-marginal error of the pair (alpha, beta_t), i.e. after
  the Y-iteration: err = sum_x mu(x) |exp((alpha(x) - alpha'(x)) / eps) - 1|;
* stop as soon as err <= tol * mu(X_J) and return (alpha, beta_t), which is
  exactly Y-feasible; otherwise alpha <- alpha' and repeat;
* with `fixed_iters = K` the tolerance is ignored and the pair of iteration K
  is returned.
"""

from __future__ import annotations

import numpy as np


def logsumexp(a, b, axis):
    """log sum_k b_k exp(a_k) along `axis` (terms with b_k = 0 drop out)."""
    with np.errstate(divide="ignore"):
        t = a + np.log(b)
    m = np.max(t, axis=axis, keepdims=True)
    return np.squeeze(m, axis=axis) + np.log(np.sum(np.exp(t - m), axis=axis))


def sq_cost(xp: np.ndarray, yp: np.ndarray, h: float) -> np.ndarray:
    """c(x, y) = |x - y|^2 for pixel coordinates xp (nx, 2), yp (ny, 2), spacing h."""
    d = xp[:, None, :].astype(np.float64) - yp[None, :, :].astype(np.float64)
    return (h * h) * (d * d).sum(axis=-1)


def y_update(alpha, mu_x, C, eps):
    """beta_t(y) = -eps log sum_x exp((alpha(x) - c(x, y)) / eps) mu(x)."""
    return -eps * logsumexp((alpha[:, None] - C) / eps, b=mu_x[:, None], axis=0)


def x_update(beta_t, nu_y, C, eps):
    """alpha(x) = -eps log sum_y exp((beta_t(y) - c(x, y)) / eps) nu_J(y)."""
    return -eps * logsumexp((beta_t[None, :] - C) / eps, b=nu_y[None, :], axis=1)


def cell_sinkhorn(mu_x, nu_y, C, eps, alpha0, tol=1e-5, max_iter=100000, fixed_iters=None):
    """Solve one composite-cell problem.

    mu_x (nx,), nu_y (ny,) with nu_y > 0, C (nx, ny) the cost, alpha0 (nx,).
    Returns dict(alpha, beta_t, iters, err, converged).
    """
    m = float(mu_x.sum())
    alpha = np.array(alpha0, dtype=np.float64)
    k = 0
    while True:
        k += 1
        beta_t = y_update(alpha, mu_x, C, eps)
        alpha_new = x_update(beta_t, nu_y, C, eps)
        err = float(np.sum(mu_x * np.abs(np.expm1((alpha - alpha_new) / eps))))
        if fixed_iters is not None:
            if k >= fixed_iters:
                return dict(alpha=alpha, beta_t=beta_t, iters=k, err=err, converged=True)
        elif err <= tol * m:
            return dict(alpha=alpha, beta_t=beta_t, iters=k, err=err, converged=True)
        elif k >= max_iter:
            return dict(alpha=alpha, beta_t=beta_t, iters=k, err=err, converged=False)
        alpha = alpha_new


def gibbs_plan(alpha, beta_t, mu_x, nu_y, C, eps):
    """pi(x, y) = exp((alpha + beta_t - c) / eps) mu(x) nu_J(y) (Prop. 2.1 (ii))."""
    return np.exp((alpha[:, None] + beta_t[None, :] - C) / eps) * mu_x[:, None] * nu_y[None, :]
