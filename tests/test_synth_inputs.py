"""Input generators (no method arithmetic): the cell-LSE sweep's plan is feasible."""

import numpy as np
import pytest

import synth
from oracle.geometry import Geometry


@pytest.mark.parametrize("m", [8, 16, 128])
def test_cell_lse_sweep_plan_is_feasible(m):
    mu, nu, eps, s, (hdr, data) = synth.cell_lse_sweep(m, 0)
    N = mu.shape[0]
    assert N == 16384 // m and s == 4 and eps == 2.0 / N ** 2
    geom = Geometry(N, N, s)
    assert len(geom.partition(0)) == (2048 // m) ** 2
    assert hdr.shape == (geom.nb, 4) and (hdr[:, 2:] == m).all()
    assert (hdr[:, :2] >= 0).all() and (hdr[:, :2] + m <= N).all()
    assert data.size == geom.nb * m * m and (data > 0).all()
    masses = data.reshape(geom.nb, m * m).sum(axis=1)
    assert np.allclose(masses, geom.basic_masses(mu), rtol=1e-12, atol=0)
    acc = np.zeros_like(nu)
    for i, (o1, o2, h, w) in enumerate(hdr):
        acc[o1:o1 + h, o2:o2 + w] += data[i * m * m:(i + 1) * m * m].reshape(h, w)
    assert np.abs(acc - nu).sum() <= 1e-13
    assert abs(nu.sum() - 1.0) <= 1e-12 and abs(mu.sum() - 1.0) <= 1e-12
    # the four members of an A-cell share one box
    for i in (0, geom.nb // 2 + 3):
        r, c = divmod(i, N // s)
        j = (r ^ 1) * (N // s) + c
        assert (hdr[i] == hdr[j]).all()


def test_cell_lse_sweep_rejects_other_sides():
    with pytest.raises(ValueError):
        synth.cell_lse_sweep(12)


@pytest.mark.parametrize("theta", [5.0, 20.0])
def test_rotation_contraction_coupling_is_feasible(theta):
    """Section 5.3's initial plan (id, T)_# mu, T = c R_theta: both marginals of
    the returned coupling are mu and nu exactly; the contracted image stays inside
    the grid (no mass on the clipped border pixels beyond bilinear rounding); the
    map is not the identity (the plan is not optimal)."""
    N = 32
    mu = synth.four_bumps(N)
    x, y, mass, nu = synth.rotation_contraction_coupling(mu, theta)
    assert (mass > 0).all()
    assert np.allclose(np.bincount(x, weights=mass, minlength=N * N).reshape(N, N), mu, rtol=1e-12, atol=0)
    assert abs(nu.sum() - 1.0) <= 1e-12
    th = np.deg2rad(theta)
    c = 1.0 / (np.cos(th) + np.sin(th))
    # the image of the grid's centre-of-mass is the rotated, contracted centre of mass
    t = 2.0 * (np.arange(N) + 0.5) / N - 1.0
    cm_mu = np.array([(mu.sum(axis=1) * t).sum(), (mu.sum(axis=0) * t).sum()])
    cm_nu = np.array([(nu.sum(axis=1) * t).sum(), (nu.sum(axis=0) * t).sum()])
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    assert np.allclose(cm_nu, c * R @ cm_mu, atol=2.0 / N)
    # second moments contract by c^2 (bilinear splatting adds at most a pixel^2 / 4 per axis)
    var = lambda a: (a.sum(axis=1) * t ** 2).sum() + (a.sum(axis=0) * t ** 2).sum()
    assert abs(var(nu) - c ** 2 * var(mu)) <= 2 * (2.0 / N) ** 2
    moved = np.abs(np.bincount(x, weights=mass) - np.bincount(y, weights=mass, minlength=N * N)).sum()
    assert moved > 0.1
