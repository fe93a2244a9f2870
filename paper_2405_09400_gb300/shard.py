"""Band sharding of the hybrid iteration (Alg. 3) across ranks: host logic only.

Composite cells of one half-iteration are independent (Alg. 1), so the method
shards by cells. Ranks own horizontal bands of basic-cell rows; band edges sit
on even basic rows, so every A-cell (rows 2a, 2a+1) lies in one band. A B-cell
(rows 2a-1, 2a) straddles the edge at row 2a = r0 of a band: its owner is the
rank of row 2a (the last B row, a = n1/2, belongs to the rank of row n1-1), and
before a B half-iteration it receives basic row r0-1 from the rank above (the
halo) and returns the new boxes of that row afterwards. The flow update needs
each basic cell's own box for its edge costs (Eq. edge-cost), a gather of all
edge costs for the one min-cost flow (Eq. MinCostFlow, solved identically on
every rank), and the boxes of rows r0-1 and r1 for the exchange
(Eq. flow-update-cell-marginals). Scalars are summed across ranks.

This module decides who owns what and moves boxes between ranks with
torch.distributed point-to-point messages (sizes first, then the data); the
per-cell compute is the caller's. With one GPU per run the library itself runs
replicas only; this is the layout a multi-GPU run of the path uses, exercised
with CPU (gloo) ranks.
"""

from __future__ import annotations

import numpy as np


def band(n1: int, world: int, rank: int):
    """Basic-cell rows [r0, r1) of `rank`: near-equal bands with even edges."""
    pairs = n1 // 2
    lo = (pairs * rank) // world
    hi = (pairs * (rank + 1)) // world
    return 2 * lo, 2 * hi


def owner_of_row(n1: int, world: int, row: int) -> int:
    for r in range(world):
        r0, r1 = band(n1, world, r)
        if r0 <= row < r1:
            return r
    raise ValueError("row outside the grid")


def cell_rows(part: int, a: int, n1: int):
    """Basic rows of composite row a of partition part (0 = A, 1 = B)."""
    rows = [2 * a, 2 * a + 1] if part == 0 else [2 * a - 1, 2 * a]
    return [r for r in rows if 0 <= r < n1]


def owned_cells(part: int, n1: int, n2: int, world: int, rank: int):
    """Indices (row-major in (a, b), as the partitions list them) of the composite
    cells `rank` solves."""
    na = n1 // 2 if part == 0 else n1 // 2 + 1
    nb = n2 // 2 if part == 0 else n2 // 2 + 1
    out = []
    for a in range(na):
        rows = cell_rows(part, a, n1)
        if owner_of_row(n1, world, max(rows)) == rank:
            out.extend(a * nb + b for b in range(nb))
    return out


def halo_rows(part: int, n1: int, world: int, rank: int):
    """Basic rows `rank` needs from other ranks for the cells it owns (B: the row
    above its band; A: none)."""
    r0, r1 = band(n1, world, rank)
    if part == 1 and r0 > 0 and r0 < n1:
        return [r0 - 1]
    return []


def exchange_rows(n1: int, world: int, rank: int):
    """Basic rows needed by the flow exchange of the band's cells (4-neighbourhood)."""
    r0, r1 = band(n1, world, rank)
    return [r for r in (r0 - 1, r1) if 0 <= r < n1]


def row_cells(row: int, n2: int):
    return list(range(row * n2, (row + 1) * n2))


def _parts(b):
    return (b.o1, b.o2, b.a) if hasattr(b, "a") else b


def pack(boxes, cells):
    """Boxes of `cells` ((o1, o2, array) or objects with o1, o2, a) -> (int64
    header (len, 4), float64 data)."""
    hdr = np.zeros((len(cells), 4), dtype=np.int64)
    parts = []
    for k, i in enumerate(cells):
        o1, o2, a = _parts(boxes[i])
        a = np.asarray(a, dtype=np.float64)
        hdr[k] = (o1, o2, a.shape[0], a.shape[1])
        parts.append(a.reshape(-1))
    data = np.concatenate(parts) if parts else np.zeros(0)
    return hdr, data


def unpack(hdr, data, cells, boxes, make=None):
    """Store the received boxes; `make(o1, o2, array)` builds the stored object
    (default: a tuple)."""
    make = make or (lambda o1, o2, a: (o1, o2, a))
    k0 = 0
    for k, i in enumerate(cells):
        o1, o2, h, w = (int(x) for x in hdr[k])
        boxes[i] = make(o1, o2, np.array(data[k0:k0 + h * w]).reshape(h, w))
        k0 += h * w


def send_boxes(dist, boxes, cells, dst):
    """Sizes first (header length, data length), then header and data."""
    import torch

    hdr, data = pack(boxes, cells)
    dist.send(torch.tensor([hdr.shape[0], data.size], dtype=torch.int64), dst)
    dist.send(torch.from_numpy(hdr.reshape(-1).copy()), dst)
    dist.send(torch.from_numpy(data.copy()), dst)


def recv_boxes(dist, boxes, cells, src, make=None):
    import torch

    n = torch.zeros(2, dtype=torch.int64)
    dist.recv(n, src)
    hdr = torch.zeros(int(n[0]) * 4, dtype=torch.int64)
    dist.recv(hdr, src)
    data = torch.zeros(int(n[1]), dtype=torch.float64)
    dist.recv(data, src)
    unpack(hdr.numpy().reshape(-1, 4), data.numpy(), cells, boxes, make)


def share_rows(dist, boxes, rows_needed, n1, n2, world, rank, make=None):
    """Every rank receives the basic rows it lists from their owners. Pairwise
    exchanges in rank order (sends before receives on the lower rank), so the
    blocking point-to-point calls cannot deadlock."""
    need = {r: rows for r, rows in enumerate(_all_gather_obj(dist, rows_needed, world))}
    for a in range(world):
        for b in range(a + 1, world):
            # rows b needs from a, then rows a needs from b
            ab = [row for row in need[b] if owner_of_row(n1, world, row) == a]
            ba = [row for row in need[a] if owner_of_row(n1, world, row) == b]
            cab = [i for row in ab for i in row_cells(row, n2)]
            cba = [i for row in ba for i in row_cells(row, n2)]
            if rank == a:
                if cab:
                    send_boxes(dist, boxes, cab, b)
                if cba:
                    recv_boxes(dist, boxes, cba, b, make)
            elif rank == b:
                if cab:
                    recv_boxes(dist, boxes, cab, a, make)
                if cba:
                    send_boxes(dist, boxes, cba, a)


def return_rows(dist, boxes, rows, n1, n2, world, rank, make=None):
    """The inverse of share_rows for rows a rank updated on behalf of their owner
    (the B halo): each rank sends the boxes of `rows` back to their owners."""
    back = {r: rows_r for r, rows_r in enumerate(_all_gather_obj(dist, rows, world))}
    for a in range(world):
        for b in range(a + 1, world):
            ab = [row for row in back[a] if owner_of_row(n1, world, row) == b]  # a returns to b
            ba = [row for row in back[b] if owner_of_row(n1, world, row) == a]
            cab = [i for row in ab for i in row_cells(row, n2)]
            cba = [i for row in ba for i in row_cells(row, n2)]
            if rank == a:
                if cab:
                    send_boxes(dist, boxes, cab, b)
                if cba:
                    recv_boxes(dist, boxes, cba, b, make)
            elif rank == b:
                if cab:
                    recv_boxes(dist, boxes, cab, a, make)
                if cba:
                    send_boxes(dist, boxes, cba, a)


def all_gather_rows(dist, values, own, world):
    """values: (nbasic, ...) array valid on the rows `own` of this rank; returns
    the array with every rank's rows filled in."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(values))
    mask = np.zeros(values.shape[0], dtype=bool)
    mask[own] = True
    t = t * torch.from_numpy(mask.reshape((-1,) + (1,) * (values.ndim - 1)).astype(values.dtype))
    dist.all_reduce(t)  # disjoint rows: the sum is a gather
    return t.numpy()


def all_sum(dist, x: float) -> float:
    import torch

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t)
    return float(t.item())


def _all_gather_obj(dist, obj, world):
    out = [None] * world
    dist.all_gather_object(out, obj)
    return out
