"""The allocation-free entry point dd_l1_y_error_static against dd_get_objective.

dd_l1_y_error_static serves callers that cannot allocate device memory (inside
stream capture, or with all device memory reserved up front): it takes its
scratch from a fixed array inside the library. It must give the same L1 Y
error as the context's own reduction, call after call (the array is shared and
must be cleared each time). Both sum the same FP32 entries per pixel in FP64
with atomic additions in different orders: each pixel's sum of at most a few
entries differs by <= ~1e-15 nu(y), so the two L1 errors differ by at most
1e-15 * sum_y nu(y) = 1e-15 (absolute).
"""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_static_scratch_l1_y_matches_context(lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd = lib
    mu, nu, eps, p = synth.workload("dd256", 0, N=64)
    boxes = synth.boxes_from_coupling(mu.shape, 4, *synth.knothe_rosenblatt(mu, nu))
    g = dd.DomDec(mu, nu, eps, 4, boxes=boxes, tol=1e-5)
    nu_d = torch.from_numpy(nu.reshape(-1)).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(2):  # two calls in a row, each on a new state
        g.step(1, stats=False)
        _, _, l1y = g.objective()
        hdr, data = dd.dd_get_plan(g.ctx, g.nbasic)
        hdr_d = torch.from_numpy(hdr.copy()).cuda()
        data_d = torch.from_numpy(data.astype(np.float32)).cuda()  # the state's own FP32 values
        rc = dd.dd_l1_y_error_static(64, 64, g.nbasic, hdr_d.data_ptr(), data_d.data_ptr(), nu_d.data_ptr(),
                                     out.data_ptr())
        assert rc == dd.DD_OK
        torch.cuda.synchronize()
        got = float(out.item())
        assert l1y > 0
        assert abs(got - l1y) <= 1e-15, (got, l1y)
    # sizes beyond the static limit are rejected before any GPU work
    assert dd.dd_l1_y_error_static(2048, 2048, 10, hdr_d.data_ptr(), data_d.data_ptr(), nu_d.data_ptr(),
                                   out.data_ptr()) == dd.DD_ERR_ARG
    g.close()
