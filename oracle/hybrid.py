"""The hybrid scheme (Alg. 3) on the box state, with the objective and errors.

Schedule (Alg. 3): k % 3 == 1 -> DomDecIter on A, 2 -> on B, 0 -> FlowUpdate.
The flow update needs <c, pi_i> of a Gibbs plan, so it is only valid directly
after a half-iteration (the paper counts it at the end of the B iteration,
Section 5.2).

Warm start (Alg. 4 input alpha_init): the previous alpha of the same partition;
the very first solve of each partition starts from alpha = 0.
"""

from __future__ import annotations

import numpy as np

from .domdec import Box, half_iteration, l1_y_error, truncate_box
from .flow import edge_costs, edge_costs_glued, exchange, gluing_plans, min_cost_flow
from .geometry import Geometry


class OracleDD:
    def __init__(self, mu, nu, eps, s, boxes=None, tol=1e-5, max_iter=100000,
                 fixed_iters=None, thr=1e-15, hgrid=None, eps_gamma=None):
        """eps_gamma: None (or inf) for product gluing candidates, else the
        regularisation of the entropic gamma_ij of the gluing candidates
        (Def. 3.7, Remark 3.8)."""
        self.mu = np.asarray(mu, dtype=np.float64)
        self.nu = np.asarray(nu, dtype=np.float64)
        self.eps = float(eps)
        N1, N2 = self.mu.shape
        self.geom = Geometry(N1, N2, s)
        self.hgrid = 1.0 / N1 if hgrid is None else hgrid
        self.m = self.geom.basic_masses(self.mu)
        self.tol, self.max_iter, self.fixed_iters, self.thr = tol, max_iter, fixed_iters, thr
        if boxes is None:  # product coupling mu (x) nu: nu_i = m_i nu
            boxes = [truncate_box(self.m[i] * self.nu, 0, 0, thr) for i in range(self.geom.nb)]
        self.boxes = [b if isinstance(b, Box) else Box(int(b[0]), int(b[1]), np.asarray(b[2], np.float64))
                      for b in boxes]
        self.alpha = {0: None, 1: None}
        self.D = None
        self.eps_gamma = None if eps_gamma is None or not np.isfinite(eps_gamma) else float(eps_gamma)
        self.gammas = None
        self.basic_plans = None  # per basic cell (Y pixels, pi_i) of the latest half-iteration
        self.k = 0
        self.history = []

    def set_eps(self, eps):
        """Change eps between hybrid iterations: the eps schedule of the paper's
        solvers (Section 5, "Multi-scale and eps-scaling"; here without the
        multiscale layers). The plan is kept, and so are the dual potentials
        alpha of both partitions in cost units: they only warm-start the next
        cell solves, which then solve the cell problems at the new eps."""
        if not (eps > 0.0 and np.isfinite(eps)):
            raise ValueError("eps must be positive and finite")
        self.eps = float(eps)

    def iterate(self, part: int, keep_plans=False):
        glued = self.eps_gamma is not None
        self.boxes, info = half_iteration(
            self.geom, self.mu, self.nu, self.eps, self.hgrid, self.boxes, part,
            self.alpha[part], self.tol, self.max_iter, self.fixed_iters, self.thr, keep_plans or glued)
        self.alpha[part] = info["alpha"]
        self.D = info["D"]
        if glued:  # the basic cells' rows of the Gibbs cell plans (member-major)
            ss = self.geom.s * self.geom.s
            self.basic_plans = [None] * self.geom.nb
            for members, (X, Y, pi) in zip(self.geom.partition(part), info["plans"]):
                for k, i in enumerate(members):
                    self.basic_plans[i] = (Y, pi[k * ss:(k + 1) * ss])
        info["l1_y"] = l1_y_error(self.boxes, self.nu)
        self.history.append(("A" if part == 0 else "B", info["E"], info["l1_x"], info["l1_y"]))
        return info

    def flow_update(self):
        if self.D is None:
            raise RuntimeError("flow update needs a preceding half-iteration")
        nbr = self.geom.neighbours()
        if self.eps_gamma is None:
            cbar = edge_costs(self.geom, self.mu, self.boxes, self.D, self.hgrid)
        else:
            if self.gammas is None:
                self.gammas = gluing_plans(self.geom, self.mu, self.hgrid, self.eps_gamma)
            cbar = edge_costs_glued(self.geom, self.mu, self.basic_plans, self.D, self.hgrid, self.gammas)
        w, value, _ = min_cost_flow(nbr, cbar, self.m)
        self.boxes = exchange(self.geom, self.boxes, w, nbr, self.m, self.thr)
        self.D = None
        info = dict(cbar=cbar, w=w, value=value, l1_y=l1_y_error(self.boxes, self.nu))
        self.history.append(("F", value, None, info["l1_y"]))
        return info

    def step(self):
        """One hybrid iteration of Alg. 3: A, B, then the flow update."""
        a = self.iterate(0)
        b = self.iterate(1)
        f = self.flow_update()
        self.k += 1
        return a, b, f
