"""The allocation-free entry point dd_l1_y_error_static.

dd_l1_y_error_static serves callers that cannot allocate device memory
(pipelines that reserve all device memory up front, host frameworks whose own
allocator owns the GPU): it takes its scratch from a fixed array inside the
library. Checked, call after call (the array is shared and must be cleared each
time), against two references:
* the context's own reduction (dd_get_objective): both sum the same FP32 entries
  per pixel in FP64 with atomic additions in different orders, so each pixel's
  sum of at most a few entries differs by <= ~1e-15 nu(y) and the two L1 errors
  by at most 1e-15 * sum_y nu(y) = 1e-15 (absolute);
* an FP64 numpy sum of the exported plan (the same FP32 values, embedded on the
  grid on the host): within the same 1e-15.
The limits are rejected with DD_ERR_ARG before any GPU work.
"""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _numpy_l1_y(hdr, data32, nu):
    """sum_y |sum_i nu_i(y) - nu(y)| in FP64 on the host."""
    N1, N2 = nu.shape
    acc = np.zeros((N1, N2))
    off = 0
    for o1, o2, h, w in hdr:
        if h <= 0 or w <= 0:
            continue
        box = data32[off:off + h * w].astype(np.float64).reshape(h, w)
        off += h * w
        acc[o1:o1 + h, o2:o2 + w] += box
    return float(np.abs(acc - nu).sum())


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
        data32 = data.astype(np.float32)  # the state's own FP32 values
        hdr_d = torch.from_numpy(hdr.copy()).cuda()
        data_d = torch.from_numpy(data32).cuda()
        rc = dd.dd_l1_y_error_static(64, 64, g.nbasic, hdr_d.data_ptr(), data_d.data_ptr(), nu_d.data_ptr(),
                                     out.data_ptr())
        assert rc == dd.DD_OK
        torch.cuda.synchronize()
        got = float(out.item())
        assert l1y > 0
        assert abs(got - l1y) <= 1e-15, (got, l1y)
        ref = _numpy_l1_y(hdr, data32, nu)
        assert abs(got - ref) <= 1e-15, (got, ref)
    g.close()


def test_static_scratch_limits(lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd = lib
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    hdr_d = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    data_d = torch.zeros(16, dtype=torch.float32, device="cuda")
    nu_d = torch.zeros(16, dtype=torch.float64, device="cuda")
    args = (hdr_d.data_ptr(), data_d.data_ptr(), nu_d.data_ptr(), out.data_ptr())
    # beyond the static limits, or not positive: rejected before any GPU work
    assert dd.dd_l1_y_error_static(2048, 2048, 10, *args) == dd.DD_ERR_ARG
    assert dd.dd_l1_y_error_static(1024, 1025, 10, *args) == dd.DD_ERR_ARG
    assert dd.dd_l1_y_error_static(64, 64, dd.DD_STATIC_MAX_CELLS + 1, *args) == dd.DD_ERR_ARG
    assert dd.dd_l1_y_error_static(0, 64, 4, *args) == dd.DD_ERR_ARG
    assert dd.dd_l1_y_error_static(64, 64, 0, *args) == dd.DD_ERR_ARG
    torch.cuda.synchronize()
    assert float(out.item()) == -1.0  # untouched
    # exactly at the limits: a 1024 x 1024 grid and 65536 boxes (4 x 4 cells),
    # one unit mass on a single pixel, every other box empty or with a
    # non-positive extent (empty), nu the same unit mass one pixel further
    N = 1024
    nb = dd.DD_STATIC_MAX_CELLS
    hdr = np.zeros((nb, 4), dtype=np.int32)
    hdr[0] = (5, 7, 1, 1)
    hdr[1] = (0, 0, -3, 2)
    hdr[2] = (0, 0, 2, -1)
    nu = np.zeros((N, N))
    nu[5, 8] = 1.0
    hdr_d = torch.from_numpy(hdr).cuda()
    data_d = torch.ones(1, dtype=torch.float32, device="cuda")
    nu_d = torch.from_numpy(nu.reshape(-1)).cuda()
    for _ in range(2):
        assert dd.dd_l1_y_error_static(N, N, nb, hdr_d.data_ptr(), data_d.data_ptr(), nu_d.data_ptr(),
                                       out.data_ptr()) == dd.DD_OK
        torch.cuda.synchronize()
        assert float(out.item()) == 2.0
