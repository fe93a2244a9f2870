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
