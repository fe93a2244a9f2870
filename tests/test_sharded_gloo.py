"""The band-sharded hybrid iteration (paper_2405_09400_gb300/shard.py) on two
CPU ranks (gloo), with the FP64 oracle doing the per-cell compute: two hybrid
iterations must give exactly the boxes of the single-process oracle (every cell
problem, edge cost and the min-cost flow see identical inputs)."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from oracle.domdec import Box, balance, basic_to_composite, composite_to_basic, solve_cell, truncate_box
from oracle.flow import edge_costs, exchange, min_cost_flow
from oracle.geometry import Geometry
from oracle.hybrid import OracleDD
from paper_2405_09400_gb300 import shard

N, S, ITERS, TOL = 32, 4, 2, 1e-6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mu, nu, eps, _ = synth.workload("dd32", 0, N=N)
    geom = Geometry(N, N, S)
    n1 = n2 = N // S
    nb = geom.nb
    m = geom.basic_masses(mu)
    nbr = geom.neighbours()
    h = 1.0 / N
    boxes = [truncate_box(m[i] * nu, 0, 0, 1e-15) for i in range(nb)]
    make = lambda o1, o2, a: Box(o1, o2, a)  # noqa: E731
    r0, r1 = shard.band(n1, world, rank)
    own = [i for i in range(nb) if r0 <= i // n2 < r1]
    alpha = {0: {}, 1: {}}
    values = []
    for _ in range(ITERS):
        for part in (0, 1):
            D = np.zeros(nb)  # D_i = <c, pi_i> of the latest half-iteration only
            halo = shard.halo_rows(part, n1, world, rank)
            shard.share_rows(dist, boxes, halo, n1, n2, world, rank, make)
            cells = geom.partition(part)
            for J in shard.owned_cells(part, n1, n2, world, rank):
                members = cells[J]
                nuJ = basic_to_composite(boxes, members)
                res = solve_cell(geom, mu, eps, h, members, nuJ, alpha[part].get(J), TOL, 100000)
                arrs, Dm = composite_to_basic(geom, members, nuJ, res)
                bal = balance(arrs, [m[i] for i in members])
                for k, i in enumerate(members):
                    boxes[i] = truncate_box(bal[k], nuJ.o1, nuJ.o2, 1e-15, m[i])
                    D[i] = Dm[k]
                alpha[part][J] = res["alpha"]
            shard.return_rows(dist, boxes, halo, n1, n2, world, rank, make)
        # D_i of the last half-iteration comes from whichever rank solved the cell
        mine = [i for J in shard.owned_cells(1, n1, n2, world, rank) for i in geom.partition(1)[J]]
        D = shard.all_gather_rows(dist, D, mine, world)
        shard.share_rows(dist, boxes, shard.exchange_rows(n1, world, rank), n1, n2, world, rank, make)
        cb = edge_costs(geom, mu, boxes, D, h)
        cbar = shard.all_gather_rows(dist, np.nan_to_num(cb), own, world)
        cbar[nbr < 0] = np.nan
        w, value, _ = min_cost_flow(nbr, cbar, m)
        values.append(value)
        new = exchange(geom, boxes, w, nbr, m, 1e-15)
        for i in own:
            boxes[i] = new[i]
    # collect every rank's rows on rank 0
    for r in range(1, world):
        rr0, rr1 = shard.band(n1, world, r)
        cells_r = [i for i in range(nb) if rr0 <= i // n2 < rr1]
        if rank == r:
            shard.send_boxes(dist, boxes, cells_r, 0)
        elif rank == 0:
            shard.recv_boxes(dist, boxes, cells_r, r, make)
    if rank == 0:
        hdr, data = shard.pack(boxes, list(range(nb)))
        np.savez(out, hdr=hdr, data=data, values=np.array(values))
    dist.barrier()
    dist.destroy_process_group()


def test_band_layout_covers_every_cell_once():
    for n1, world in ((8, 2), (16, 3), (64, 4), (6, 4)):
        rows = [r for k in range(world) for r in range(*shard.band(n1, world, k))]
        assert rows == list(range(n1))
        for k in range(world):
            r0, r1 = shard.band(n1, world, k)
            assert r0 % 2 == 0 and r1 % 2 == 0
        for part in (0, 1):
            owned = sorted(J for k in range(world) for J in shard.owned_cells(part, n1, 6, world, k))
            ncell = (n1 // 2) * 3 if part == 0 else (n1 // 2 + 1) * 4
            assert owned == list(range(ncell))


def test_two_gloo_ranks_reproduce_the_single_process_oracle(tmp_path):
    out = str(tmp_path / "sharded.npz")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    z = np.load(out)
    mu, nu, eps, _ = synth.workload("dd32", 0, N=N)
    ref = OracleDD(mu, nu, eps, S, tol=TOL)
    vals = []
    for _ in range(ITERS):
        _, _, f = ref.step()
        vals.append(f["value"])
    hdr_ref, data_ref = shard.pack(ref.boxes, list(range(len(ref.boxes))))
    assert np.array_equal(z["hdr"], hdr_ref)
    assert np.array_equal(z["data"], data_ref)
    assert np.array_equal(z["values"], np.array(vals))
