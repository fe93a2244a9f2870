"""One domain-decomposition half-iteration on the basic-cell bounding-box state.

The state is the list of basic-cell Y-marginals nu_i (Eq. basic-cell-Y-marginal),
each on its bounding box (Section A.1, "Bounding box representation"). One
half-iteration on partition P follows Alg. 1, in the order of its restatement
Alg. 4:

  1. BasicToComposite: nu_J = sum_{i in J} nu_i on the union box
     (Eq. get-composite-cell-marginal);
  2. the cell problem of Alg. 1 with X-marginal mu restricted to X_J and
     Y-marginal nu_J, solved by `cell.cell_sinkhorn`;
  3. CompositeToBasic: nu_i(y) = sum_{x in X_i} pi_J(x, y), here by its
     definition on the explicit cell plan (the paper's partial log-sum-exp
     route, Section A.1 "Online reduction", is what the library does);
  4. balancing (Alg. 4, BalanceGPU) and
  5. truncation at 1e-15 with the minimal bounding box (Alg. 4, TruncateGPU;
     Section A.2).

Readings:
* Balancing is only named in the paper. Reading: per composite cell, excess
  e_i = |nu_i| - m_i; donors (e_i > 0) and receivers (e_i < 0) are each taken
  in member order and a two-pointer walk moves d = min(remaining donor excess,
  remaining receiver deficit) from donor i to receiver j in proportion to nu_i:
  nu_i -= d nu_i / |nu_i|, nu_j += d nu_i / |nu_i|. This keeps sum_i nu_i
  pointwise, keeps every entry >= 0 and ends with |nu_i| = m_i whenever
  |nu_J| = m_J.
* Truncation sets entries < 1e-15 to zero and the box becomes the minimal box
  of the remaining entries; the basic marginal is then rescaled to its mass
  m_i. The paper is silent on the removed mass. Without the rescale the
  absolute threshold removes a relative share of ~1e-6 per step from the
  lightest cells (mass ~1e-7 on the 256 x 256 workload), the composite masses
  drift away from mu(X_J), and the cell problems become unbalanced, so that no
  Sinkhorn solve can reach its tolerance there. The rescale keeps every basic
  X-marginal exact and moves the (1e-15-sized) removed mass into the Y error.
* D_i = <c, pi_i> (needed by the flow update) is taken from the Gibbs plan of
  the half-iteration, before balancing.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .cell import cell_sinkhorn, gibbs_plan, sq_cost


@dataclass
class Box:
    o1: int
    o2: int
    a: np.ndarray  # (h, w) float64

    @property
    def h(self):
        return self.a.shape[0]

    @property
    def w(self):
        return self.a.shape[1]


def union_header(boxes):
    """Smallest box (o1, o2, h, w) containing every non-empty box."""
    nz = [b for b in boxes if b.h > 0 and b.w > 0]
    o1 = min(b.o1 for b in nz)
    o2 = min(b.o2 for b in nz)
    e1 = max(b.o1 + b.h for b in nz)
    e2 = max(b.o2 + b.w for b in nz)
    return o1, o2, e1 - o1, e2 - o2


def embed(box: Box, o1, o2, h, w) -> np.ndarray:
    out = np.zeros((h, w))
    if box.h and box.w:
        out[box.o1 - o1: box.o1 - o1 + box.h, box.o2 - o2: box.o2 - o2 + box.w] = box.a
    return out


def basic_to_composite(boxes, members) -> Box:
    """nu_J = sum_{i in J} nu_i on the union of the member boxes (Eq. get-composite-cell-marginal)."""
    o1, o2, h, w = union_header([boxes[i] for i in members])
    acc = np.zeros((h, w))
    for i in members:
        acc += embed(boxes[i], o1, o2, h, w)
    return Box(o1, o2, acc)


def balance(arrs, m):
    """Balancing walk (see module docstring). arrs: member arrays on one box."""
    out = [a.copy() for a in arrs]
    mass = [float(a.sum()) for a in arrs]
    e = [mass[k] - m[k] for k in range(len(arrs))]
    pos = [k for k in range(len(arrs)) if e[k] > 0]
    neg = [k for k in range(len(arrs)) if e[k] < 0]
    p = q = 0
    rp = e[pos[0]] if pos else 0.0
    rq = -e[neg[0]] if neg else 0.0
    while p < len(pos) and q < len(neg):
        i, j = pos[p], neg[q]
        d = min(rp, rq)
        moved = (d / mass[i]) * arrs[i]
        out[i] -= moved
        out[j] += moved
        rp -= d
        rq -= d
        if rp <= 0.0:
            p += 1
            rp = e[pos[p]] if p < len(pos) else 0.0
        if rq <= 0.0:
            q += 1
            rq = -e[neg[q]] if q < len(neg) else 0.0
    return out


def truncate_box(a: np.ndarray, o1: int, o2: int, thr: float = 1e-15, mass=None) -> Box:
    """Drop entries < thr, shrink to the minimal bounding box, rescale to `mass` if given."""
    a = np.where(a < thr, 0.0, a)
    if mass is not None and a.sum() > 0:
        a = a * (mass / a.sum())
    rows = np.nonzero(a.any(axis=1))[0]
    cols = np.nonzero(a.any(axis=0))[0]
    if len(rows) == 0:
        return Box(o1, o2, np.zeros((0, 0)))
    r0, r1, c0, c1 = rows[0], rows[-1] + 1, cols[0], cols[-1] + 1
    return Box(o1 + int(r0), o2 + int(c0), a[r0:r1, c0:c1].copy())


def box_pixels(o1, o2, h, w) -> np.ndarray:
    r, c = np.meshgrid(np.arange(o1, o1 + h), np.arange(o2, o2 + w), indexing="ij")
    return np.stack([r.reshape(-1), c.reshape(-1)], axis=1)


def solve_cell(geom, mu, eps, hgrid, members, nuJ: Box, alpha0, tol, max_iter, fixed_iters=None):
    """Steps 2-3 for one composite cell: the Sinkhorn solve and the cell plan.

    Returns dict with alpha (over the member pixels, member-major), beta_t on the
    support of nu_J, the support mask, the plan pi (nx, ny_support), the
    X-marginal r, the member row ranges and the solve statistics.
    """
    X = geom.composite_pixels(members)
    mu_x = mu[X[:, 0], X[:, 1]]
    Y = box_pixels(nuJ.o1, nuJ.o2, nuJ.h, nuJ.w)
    flat = nuJ.a.reshape(-1)
    supp = flat > 0
    C = sq_cost(X, Y[supp], hgrid)
    if alpha0 is None:
        alpha0 = np.zeros(len(mu_x))
    res = cell_sinkhorn(mu_x, flat[supp], C, eps, alpha0, tol, max_iter, fixed_iters)
    pi = gibbs_plan(res["alpha"], res["beta_t"], mu_x, flat[supp], C, eps)
    res.update(X=X, mu_x=mu_x, supp=supp, C=C, pi=pi, r=pi.sum(axis=1))
    return res


def composite_to_basic(geom, members, nuJ: Box, cellres):
    """nu_i(y) = sum_{x in X_i} pi_J(x, y) on the composite box, and D_i = <c, pi_i>."""
    ss = geom.s * geom.s
    pi, C, supp = cellres["pi"], cellres["C"], cellres["supp"]
    arrs, D = [], []
    for k, _ in enumerate(members):
        rows = slice(k * ss, (k + 1) * ss)
        flat = np.zeros(nuJ.h * nuJ.w)
        flat[supp] = pi[rows].sum(axis=0)
        arrs.append(flat.reshape(nuJ.h, nuJ.w))
        D.append(float((C[rows] * pi[rows]).sum()))
    return arrs, D


def cell_objective(cellres, nuJ: Box, nu, eps):
    """sum_x alpha r + sum_y beta nu_J with beta = beta_t + eps log(nu_J / nu) (mu (x) nu convention)."""
    Y = box_pixels(nuJ.o1, nuJ.o2, nuJ.h, nuJ.w)[cellres["supp"]]
    nuJ_s = nuJ.a.reshape(-1)[cellres["supp"]]
    beta = cellres["beta_t"] + eps * np.log(nuJ_s / nu[Y[:, 0], Y[:, 1]])
    return float(np.dot(cellres["alpha"], cellres["r"]) + np.dot(beta, nuJ_s))


def half_iteration(geom, mu, nu, eps, hgrid, boxes, part, alpha_prev=None, tol=1e-5,
                   max_iter=100000, fixed_iters=None, thr=1e-15, keep_plans=False):
    """One DomDecIter (Alg. 1 / Alg. 4) on partition `part` (0 = A, 1 = B).

    Returns (new_boxes, info). info holds per-cell alpha (for the next warm
    start), iterations, errors, nu_J, the objective E and the L1 X-marginal
    error of the stitched Gibbs plans, and per-basic-cell D_i and masses.
    """
    m = geom.basic_masses(mu)
    cells = geom.partition(part)
    new_boxes = list(boxes)
    info = dict(alpha=[], iters=[], err=[], converged=[], nuJ=[], beta_t=[], supp=[],
                D=np.zeros(geom.nb), prebal={}, E=0.0, l1_x=0.0)
    if keep_plans:
        info["plans"] = []
    for J, members in enumerate(cells):
        nuJ = basic_to_composite(boxes, members)
        a0 = None if alpha_prev is None else alpha_prev[J]
        res = solve_cell(geom, mu, eps, hgrid, members, nuJ, a0, tol, max_iter, fixed_iters)
        arrs, D = composite_to_basic(geom, members, nuJ, res)
        for k, i in enumerate(members):
            info["D"][i] = D[k]
            info["prebal"][i] = (nuJ.o1, nuJ.o2, arrs[k])
        bal = balance(arrs, [m[i] for i in members])
        for k, i in enumerate(members):
            new_boxes[i] = truncate_box(bal[k], nuJ.o1, nuJ.o2, thr, m[i])
        info["alpha"].append(res["alpha"])
        info["beta_t"].append(res["beta_t"])
        info["supp"].append(res["supp"])
        info["iters"].append(res["iters"])
        info["err"].append(res["err"])
        info["converged"].append(res["converged"])
        info["nuJ"].append(nuJ)
        info["E"] += cell_objective(res, nuJ, nu, eps)
        info["l1_x"] += float(np.abs(res["r"] - res["mu_x"]).sum())
        if keep_plans:
            info["plans"].append((res["X"], box_pixels(nuJ.o1, nuJ.o2, nuJ.h, nuJ.w)[res["supp"]], res["pi"]))
    return new_boxes, info


def y_marginal(boxes, shape) -> np.ndarray:
    acc = np.zeros(shape)
    for b in boxes:
        if b.h and b.w:
            acc[b.o1:b.o1 + b.h, b.o2:b.o2 + b.w] += b.a
    return acc


def l1_y_error(boxes, nu) -> float:
    """sum_y |sum_i nu_i(y) - nu(y)| (Table 1, Y-marginal error)."""
    return float(np.abs(y_marginal(boxes, nu.shape) - nu).sum())
