"""The benchmark's CPU baseline leg (the FP64 oracle on several spawned
processes), run on the 32 x 32 workload: both the one-process and the pool path
return a positive time per hybrid iteration built from whole cell solves."""

import pytest

import synth


@pytest.mark.parametrize("workers", [1, 2])
def test_oracle_sample_runs(workers):
    import bench

    mu, nu, eps, p = synth.workload("dd32", 0)
    boxes = synth.boxes_from_coupling(mu.shape, p["s"], *synth.knothe_rosenblatt(mu, nu))
    ms, n, t_cell, t_cost, t_lp = bench._oracle_sample(mu, nu, eps, p, boxes, 0.5, workers)
    assert n >= 1 and t_cell > 0 and t_cost >= 0 and t_lp >= 0
    assert ms > 0
