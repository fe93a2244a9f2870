"""Seeded grid measures.

All measures live on an N x N pixel grid; pixel (p, q) has its centre at
((p + 1/2) h, (q + 1/2) h) with h = 1/N on [0, 1]^2 (the squared-Euclidean cost
is translation invariant, so only h matters). Arrays are float64, row-major,
shape (N, N), summing to 1.

The Gaussian-mixture recipe stands in for the paper's test images (Section A.2,
"Test data": mixtures with random variances, means and magnitudes):
  * means  ~ U[0.15, 0.85]^2
  * per-axis standard deviations ~ U[sigma_min, sigma_max], rotated by an
    angle ~ U[0, pi)
  * magnitudes ~ U[0.5, 1.5]
  * the mixture density is evaluated at pixel centres, scaled to peak 1, a
    constant floor is added, and the result is normalised to total mass 1.
numpy.random.default_rng(seed) draws everything, in the order listed.
"""

from __future__ import annotations

import math

import numpy as np


def pixel_centres(N: int) -> np.ndarray:
    return (np.arange(N, dtype=np.float64) + 0.5) / N


def gaussian_mixture(N: int, K: int, sigma_range=(0.05, 0.2), floor=1e-3,
                     seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    means = rng.uniform(0.15, 0.85, size=(K, 2))
    sig = rng.uniform(sigma_range[0], sigma_range[1], size=(K, 2))
    theta = rng.uniform(0.0, math.pi, size=K)
    mags = rng.uniform(0.5, 1.5, size=K)
    t = pixel_centres(N)
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    dens = np.zeros((N, N))
    for k in range(K):
        c, s = math.cos(theta[k]), math.sin(theta[k])
        d1 = X1 - means[k, 0]
        d2 = X2 - means[k, 1]
        r1 = c * d1 + s * d2
        r2 = -s * d1 + c * d2
        dens += mags[k] * np.exp(-0.5 * ((r1 / sig[k, 0]) ** 2 + (r2 / sig[k, 1]) ** 2))
    dens /= dens.max()
    dens += floor
    return dens / dens.sum()


def uniform_measure(N: int) -> np.ndarray:
    return np.full((N, N), 1.0 / (N * N))


def four_bumps(N: int, sigma=0.12, floor=1e-3) -> np.ndarray:
    """A measure with exact 4-fold rotational symmetry on the pixel grid.

    Stands in for the "four symmetrical bumps" test measure of Section 5.2
    (the image itself is not printed). One anisotropic bump is placed off
    centre and the pixel array is symmetrised under the quarter turn, so that
    the pixel permutation of the rotation T0 (Eq. T0) maps mu onto itself.
    """
    t = 2.0 * pixel_centres(N) - 1.0  # [-1, 1]^2 as in Section 5.2
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    g = np.exp(-0.5 * (((X1 - 0.45) / sigma) ** 2 + ((X2 - 0.3) / (1.6 * sigma)) ** 2))
    f = g + np.rot90(g, 1) + np.rot90(g, 2) + np.rot90(g, 3)
    f /= f.max()
    f += floor
    return f / f.sum()


# Named workloads. eps is the entropic regularisation of Eq. (entropic-transport),
# s the basic-cell edge in pixels, tol the cell Sinkhorn stopping tolerance
# (L1 X-marginal error <= tol * cell mass, Section A.2 "Stopping criterion").
WORKLOADS = {
    # 32x32, 3-component mixtures, floor 1e-3, eps = (1/32)^2, product init.
    "dd32": dict(N=32, K=3, sigma=(0.05, 0.2), floor=1e-3, eps_h2=1.0, s=4,
                 init="product", tol=1e-7, iters=20),
    # 256x256, 5-component mixtures, floor 1e-4, eps = 2 (1/256)^2, KR init.
    "dd256": dict(N=256, K=5, sigma=(0.05, 0.2), floor=1e-4, eps_h2=2.0, s=4,
                  init="kr", tol=1e-5, iters=None),
    # 512x512, mu uniform, nu 8 narrow Gaussians (sigma 0.01-0.03), floor 1e-5,
    # eps = (1/512)^2, KR init: widely varying bounding-box sizes.
    "uneven512": dict(N=512, K=8, sigma=(0.01, 0.03), floor=1e-5, eps_h2=1.0, s=4,
                      init="kr", tol=1e-5, iters=None, mu_uniform=True),
    # 1024x1024, 6-component mixtures, floor 1e-5, eps = 2 (1/1024)^2; initial
    # plan prolongated from a converged plan of the 2x2-coarsened measures
    # (couplings.prolongate).
    "dd1024": dict(N=1024, K=6, sigma=(0.05, 0.2), floor=1e-5, eps_h2=2.0, s=4,
                   init="prolongated", tol=1e-5, iters=None),
}


def workload(name: str, k: int = 0, N: int | None = None):
    """Return (mu, nu, eps, params) for workload `name` and seed pair k.

    mu uses seed 2k and nu seed 2k+1. N overrides the grid size (the same
    recipe at another resolution, used for small parity cases).
    """
    p = dict(WORKLOADS[name])
    if N is not None:
        p["N"] = N
    n = p["N"]
    if p.get("mu_uniform"):
        mu = uniform_measure(n)
    else:
        mu = gaussian_mixture(n, p["K"], p["sigma"], p["floor"], seed=2 * k)
    nu = gaussian_mixture(n, p["K"], p["sigma"], p["floor"], seed=2 * k + 1)
    eps = p["eps_h2"] / (n * n)
    return mu, nu, eps, p
