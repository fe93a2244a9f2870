"""CPU checks of the C ABI: the library loads, exports every declared entry point,
and its host-side min-cost flow (no GPU involved) matches the oracle's LP."""

import os
import re

import numpy as np
import pytest

from oracle.flow import min_cost_flow as oracle_mcf
from oracle.geometry import Geometry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "ddflow.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dd_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(lib):
    import ctypes

    so = ctypes.CDLL(lib.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(so, name), name
    assert set(declared) == set(lib.EXPORTS)


def test_strerror_and_defaults(lib):
    o = lib.default_options()
    assert o.tol == 1e-5 and o.trunc == 1e-15 and o.max_iter == 100000
    assert lib.strerror(lib.DD_ERR_STATE) == "call order violated"


def _flow_instance(N, s, seed):
    g = Geometry(N, N, s)
    rng = np.random.default_rng(seed)
    nbr = g.neighbours()
    phi = rng.normal(size=g.nb)
    cbar = np.where(nbr >= 0, phi[np.maximum(nbr, 0)] - phi[:, None] + 0.3 * rng.normal(size=nbr.shape), np.nan)
    cbar[:, 0] = 0.0
    m = rng.random(g.nb) + 0.1
    return nbr, cbar, m / m.sum()


@pytest.mark.parametrize("N,s,seed", [(8, 2, 0), (16, 2, 1), (32, 2, 2), (64, 2, 3), (64, 4, 4), (256, 2, 5)])
def test_host_min_cost_flow_matches_oracle_lp(lib, N, s, seed):
    # (256, 2): 16384 basic cells, 81920 arcs, a pricing list longer than the minimum
    nbr, cbar, m = _flow_instance(N, s, seed)
    w, val, piv = lib.dd_min_cost_flow(nbr, cbar, m)
    _, ref, _ = oracle_mcf(nbr, cbar, m)
    assert val == pytest.approx(ref, rel=1e-9, abs=1e-15)
    assert val <= 1e-15
    assert (w >= 0).all()
    assert np.allclose(w.sum(axis=1), m, rtol=1e-14, atol=0)            # outflow exact by construction
    ii, kk = np.nonzero(nbr >= 0)
    inflow = np.zeros(len(m))
    np.add.at(inflow, nbr[ii, kk], w[ii, kk])
    assert np.allclose(inflow, m, rtol=1e-12, atol=0)
    assert (w[nbr < 0] == 0).all()


def test_host_min_cost_flow_zero_costs_keeps_stationary_flow(lib):
    g = Geometry(8, 8, 2)
    nbr = g.neighbours()
    m = np.full(g.nb, 1.0 / g.nb)
    w, val, piv = lib.dd_min_cost_flow(nbr, np.zeros(nbr.shape), m)
    assert val == 0.0 and piv == 0
    assert np.allclose(w[:, 0], m) and (w[:, 1:] == 0).all()


def test_host_min_cost_flow_rejects_bad_input(lib):
    g = Geometry(8, 8, 2)
    nbr = g.neighbours()
    with pytest.raises(lib.DDError):
        lib.dd_min_cost_flow(nbr, np.zeros(nbr.shape), -np.ones(g.nb))
