"""Basic cells, composite partitions and the neighbourhood set.

Def. 2.2 (basic / composite partitions), Fig. 3 (2x2 groups of basic cells, the
B partition offset by one basic cell), Def. 3.1 (neighbourhood set), and the
4-neighbourhood used in Section 4/5.

Readings:
* Basic cell i = (bi, bj) is the s x s pixel block with top-left pixel
  (bi*s, bj*s); i = bi * n2 + bj (row-major).
* A-cell (a, b), a < n1/2, b < n2/2, holds basic cells {2a, 2a+1} x {2b, 2b+1}.
* B-cell (a, b), a <= n1/2, b <= n2/2, holds {2a-1, 2a} x {2b-1, 2b}
  intersected with the grid: at the border B-cells are truncated (1 or 2
  basic cells) instead of padding the image as the paper's GPU code does
  (Section A.2, Fig. 12), which would change the problem.
* Cells are listed row-major in (a, b); members within a cell row-major.
* Neighbours of i: (i, -axis1, +axis1, -axis2, +axis2), -1 where the grid ends.
"""

from __future__ import annotations

import numpy as np


class Geometry:
    def __init__(self, N1: int, N2: int, s: int):
        if N1 % s or N2 % s:
            raise ValueError("cell size must divide the grid")
        self.N1, self.N2, self.s = N1, N2, s
        self.n1, self.n2 = N1 // s, N2 // s
        if self.n1 % 2 or self.n2 % 2:
            raise ValueError("need an even number of basic cells per axis")
        self.nb = self.n1 * self.n2
        self._parts = {0: self._part_a(), 1: self._part_b()}

    # basic cells -----------------------------------------------------------
    def cell_origin(self, i: int):
        bi, bj = divmod(i, self.n2)
        return bi * self.s, bj * self.s

    def cell_pixels(self, i: int) -> np.ndarray:
        """(s*s, 2) integer pixel coordinates of X_i, row-major."""
        r0, c0 = self.cell_origin(i)
        r, c = np.meshgrid(np.arange(r0, r0 + self.s), np.arange(c0, c0 + self.s), indexing="ij")
        return np.stack([r.reshape(-1), c.reshape(-1)], axis=1)

    def basic_masses(self, mu: np.ndarray) -> np.ndarray:
        s = self.s
        return mu.reshape(self.n1, s, self.n2, s).sum(axis=(1, 3)).reshape(-1)

    # composite partitions -------------------------------------------------
    def _part_a(self):
        cells = []
        for a in range(self.n1 // 2):
            for b in range(self.n2 // 2):
                cells.append([bi * self.n2 + bj for bi in (2 * a, 2 * a + 1)
                              for bj in (2 * b, 2 * b + 1)])
        return cells

    def _part_b(self):
        cells = []
        for a in range(self.n1 // 2 + 1):
            for b in range(self.n2 // 2 + 1):
                rows = [r for r in (2 * a - 1, 2 * a) if 0 <= r < self.n1]
                cols = [c for c in (2 * b - 1, 2 * b) if 0 <= c < self.n2]
                cells.append([r * self.n2 + c for r in rows for c in cols])
        return cells

    def partition(self, part: int):
        """List of composite cells (each a list of basic indices) of part 0=A, 1=B."""
        return self._parts[part]

    def composite_pixels(self, members) -> np.ndarray:
        return np.concatenate([self.cell_pixels(i) for i in members], axis=0)

    # neighbourhood ----------------------------------------------------------
    def neighbours(self) -> np.ndarray:
        nbr = -np.ones((self.nb, 5), dtype=np.int64)
        for i in range(self.nb):
            bi, bj = divmod(i, self.n2)
            nbr[i, 0] = i
            if bi > 0:
                nbr[i, 1] = i - self.n2
            if bi < self.n1 - 1:
                nbr[i, 2] = i + self.n2
            if bj > 0:
                nbr[i, 3] = i - 1
            if bj < self.n2 - 1:
                nbr[i, 4] = i + 1
        return nbr

    def partition_graph_connected(self) -> bool:
        """Def. 3.11: vertices A u B, edges between intersecting cells."""
        cells = [set(c) for c in self.partition(0)] + [set(c) for c in self.partition(1)]
        seen = {0}
        stack = [0]
        while stack:
            u = stack.pop()
            for v in range(len(cells)):
                if v not in seen and cells[u] & cells[v]:
                    seen.add(v)
                    stack.append(v)
        return len(seen) == len(cells)
