"""Inputs and training targets of the learned warm start (test infrastructure only).

Not in the paper: the library can initialise the X dual of each composite-cell
Sinkhorn solve (alpha_init of Alg. 1 / Alg. 4) from a small network. This
module defines, in plain FP64, what that network sees and what it is trained
to predict, for cells whose X block is the full 2s x 2s = 8 x 8 pixels.

Change of gauge of a cell (the same one the GPU solver uses; any choice is
exact, this one makes the duals small): with block coordinates u of X_J and box
coordinates v of nu_J,
  uc, vc      barycentres of mu_J and nu_J (per axis),
  l_k         clamp(sqrt(Var_nu,k / Var_mu,k), 1/8, 8), or 1 when Var_mu,k <= 1e-3,
  d           (block origin - box origin) + uc - vc, the barycentre offset in pixels,
  k2          h^2 / (eps ln 2) (the cost in base-2 units per squared pixel).
With ub = u - uc and vb = v - vc the cell's cost in that gauge is
  K(u, v) = k2 sum_k l_k (ub_k - vb_k / l_k)^2.

Affine dual. With S and T the 2 x 2 covariances of mu_J and nu_J (pixels), the
map x -> m_nu + A (x - m_mu) with the symmetric positive semidefinite
  A = S^(-1/2) (S^(1/2) T S^(1/2))^(1/2) S^(-1/2)
is the optimal (unregularised) transport between Gaussians of those moments,
and its Kantorovich dual for the cost |x - y|^2 is, in base-2 units,
  base(u) = k2 (ub' (I - A) ub + 2 d.ub).
(When det S <= 1e-6 the per-axis map A = diag(l) stands in.)

Features (336 values):
  [0, 64)     log2(mu_J / its mean) / 4 on the 8 x 8 block;
  [64, 320)   nu_J resampled to 16 x 16 by exact area overlap (output row i
              covers [i h / 16, (i + 1) h / 16) of the box rows, likewise the
              columns): log2(value / mean + 1/256) / 4;
  [320, 336)  h/32, w/32, d_1/8, d_2/8, log2 l_1, log2 l_2, (uc_1 - 3.5)/4,
              (uc_2 - 3.5)/4, (vc_1 + 0.5)/h - 0.5, (vc_2 + 0.5)/w - 0.5, log2 k2,
              sqrt(S_11)/4, sqrt(S_22)/4, sqrt(T_11)/16, sqrt(T_22)/16,
              T_12 / sqrt(T_11 T_22) (0 if either is 0).

Targets (320 values), from the converged dual alpha of the cell:
  [0, 64)     r(u) = alpha(u) / (eps ln 2) - base(u), shifted to a mu-weighted
              mean of zero (duals are defined up to a constant). The solver
              starts from alpha_init = eps ln 2 (base + r_pred).
  [64, 320)   an auxiliary output, trained but not used by the solver: the
              Y-side log dual of the cell's dual a(u) = log2 mu(u) + q(u) + r(u)
              in the gauge, q(u) = k2 ub' (diag(l) - A) ub,
                G(v) = -log2 sum_u 2^(a(u) - K(u, v)),
              at the 16 x 16 box pixels v_p = (((2i + 1) h) div 32,
              ((2j + 1) w) div 32), shifted to a plain mean of zero.
"""

from __future__ import annotations

import numpy as np
from scipy.linalg import sqrtm

LN2 = np.log(2.0)
NF, NT = 336, 320


def block_of(geom, members):
    """Block origin and shape (r0, c0, hx, wx) of composite cell `members`, and for
    each block pixel (row-major) its index in the member-major pixel order."""
    px = geom.composite_pixels(members)
    r0, c0 = px[:, 0].min(), px[:, 1].min()
    hx, wx = px[:, 0].max() - r0 + 1, px[:, 1].max() - c0 + 1
    perm = np.empty(hx * wx, dtype=np.int64)
    for k, (r, c) in enumerate(px):
        perm[(r - r0) * wx + (c - c0)] = k
    return int(r0), int(c0), int(hx), int(wx), perm


def cell_gauge(mu_blk, r0, c0, nu_arr, o1, o2):
    """uc, vc, variances, covariances S and T, l, d and the map A (module docstring)."""
    hx, wx = mu_blk.shape
    h, w = nu_arr.shape
    mx = mu_blk.sum()
    u1 = np.arange(hx)[:, None] * np.ones((1, wx))
    u2 = np.ones((hx, 1)) * np.arange(wx)[None, :]
    v1 = np.arange(h)[:, None] * np.ones((1, w))
    v2 = np.ones((h, 1)) * np.arange(w)[None, :]
    my = nu_arr.sum()
    uc = np.array([(mu_blk * u1).sum() / mx, (mu_blk * u2).sum() / mx])
    vc = np.array([(nu_arr * v1).sum() / my, (nu_arr * v2).sum() / my])
    vu = np.maximum(np.array([(mu_blk * u1 * u1).sum() / mx, (mu_blk * u2 * u2).sum() / mx]) - uc * uc, 0.0)
    vv = np.maximum(np.array([(nu_arr * v1 * v1).sum() / my, (nu_arr * v2 * v2).sum() / my]) - vc * vc, 0.0)
    cu = (mu_blk * u1 * u2).sum() / mx - uc[0] * uc[1]
    cv = (nu_arr * v1 * v2).sum() / my - vc[0] * vc[1]
    lam = np.where(vu > 1e-3, np.clip(np.sqrt(vv / np.where(vu > 0, vu, 1.0)), 0.125, 8.0), 1.0)
    d = np.array([r0 - o1, c0 - o2], dtype=np.float64) + uc - vc
    S = np.array([[vu[0], cu], [cu, vu[1]]])
    T = np.array([[vv[0], cv], [cv, vv[1]]])
    if np.linalg.det(S) > 1e-6:
        Sh = np.real(sqrtm(S))
        Shi = np.linalg.inv(Sh)
        A = Shi @ np.real(sqrtm(Sh @ T @ Sh)) @ Shi
        A = 0.5 * (A + A.T)
    else:
        A = np.diag(lam)
    return dict(uc=uc, vc=vc, vu=vu, vv=vv, S=S, T=T, l=lam, d=d, A=A)


def overlap_matrix(n: int, m: int = 16) -> np.ndarray:
    """R[i, v] = length of [i n / m, (i + 1) n / m) intersected with [v, v + 1)."""
    R = np.zeros((m, n))
    for i in range(m):
        lo, hi = i * n / m, (i + 1) * n / m
        for v in range(n):
            R[i, v] = max(0.0, min(v + 1.0, hi) - max(float(v), lo))
    return R


def resample16(arr) -> np.ndarray:
    h, w = arr.shape
    return overlap_matrix(h) @ arr @ overlap_matrix(w).T


def cell_features(mu_blk, r0, c0, nu_arr, o1, o2, k2) -> np.ndarray:
    g = cell_gauge(mu_blk, r0, c0, nu_arr, o1, o2)
    h, w = nu_arr.shape
    f = np.zeros(NF)
    f[:64] = np.log2(mu_blk / mu_blk.mean()).reshape(-1) / 4
    rs = resample16(nu_arr)
    f[64:320] = np.log2(rs / rs.mean() + 1.0 / 256).reshape(-1) / 4
    T = g["T"]
    rho = T[0, 1] / np.sqrt(T[0, 0] * T[1, 1]) if T[0, 0] > 0 and T[1, 1] > 0 else 0.0
    f[320:336] = [h / 32, w / 32, g["d"][0] / 8, g["d"][1] / 8, np.log2(g["l"][0]), np.log2(g["l"][1]),
                  (g["uc"][0] - 3.5) / 4, (g["uc"][1] - 3.5) / 4, (g["vc"][0] + 0.5) / h - 0.5,
                  (g["vc"][1] + 0.5) / w - 0.5, np.log2(k2), np.sqrt(g["vu"][0]) / 4, np.sqrt(g["vu"][1]) / 4,
                  np.sqrt(g["vv"][0]) / 16, np.sqrt(g["vv"][1]) / 16, rho]
    return f


def _ub(g, hx, wx):
    ub1 = np.arange(hx)[:, None] - g["uc"][0] + np.zeros((1, wx))
    ub2 = np.arange(wx)[None, :] - g["uc"][1] + np.zeros((hx, 1))
    return ub1, ub2


def _quad(M, ub1, ub2):
    return M[0, 0] * ub1 ** 2 + 2 * M[0, 1] * ub1 * ub2 + M[1, 1] * ub2 ** 2


def affine_dual(mu_blk, k2, g) -> np.ndarray:
    """base(u) = k2 (ub' (I - A) ub + 2 d.ub) on the block."""
    hx, wx = mu_blk.shape
    ub1, ub2 = _ub(g, hx, wx)
    return k2 * (_quad(np.eye(2) - g["A"], ub1, ub2) + 2.0 * (g["d"][0] * ub1 + g["d"][1] * ub2))


def alpha_target(alpha_blk, mu_blk, eps, k2, g) -> np.ndarray:
    """r on the block (row-major, 64 values), mu-weighted mean zero."""
    r = alpha_blk / (eps * LN2) - affine_dual(mu_blk, k2, g)
    r = r - (mu_blk * r).sum() / mu_blk.sum()
    return r.reshape(-1)


def alpha_from_prediction(r_pred, mu_blk, eps, k2, g) -> np.ndarray:
    """The warm start the solver builds from a predicted r (inverse of alpha_target
    up to the free constant)."""
    hx, wx = mu_blk.shape
    return eps * LN2 * (affine_dual(mu_blk, k2, g) + np.asarray(r_pred).reshape(hx, wx))


def sample_pixels(h, w):
    i = np.arange(16)
    return ((2 * i + 1) * h) // 32, ((2 * i + 1) * w) // 32


def beta_aux_target(r, mu_blk, h, w, k2, g) -> np.ndarray:
    """G at the 16 x 16 sample pixels (row-major, 256 values), plain mean zero."""
    hx, wx = mu_blk.shape
    ub1, ub2 = _ub(g, hx, wx)
    q = k2 * _quad(np.diag(g["l"]) - g["A"], ub1, ub2)
    a = (np.log2(mu_blk) + q + np.asarray(r).reshape(hx, wx)).reshape(-1)
    p1, p2 = sample_pixels(h, w)
    out = np.zeros((16, 16))
    for i in range(16):
        for j in range(16):
            vb1, vb2 = p1[i] - g["vc"][0], p2[j] - g["vc"][1]
            K = k2 * (g["l"][0] * (ub1 - vb1 / g["l"][0]) ** 2 + g["l"][1] * (ub2 - vb2 / g["l"][1]) ** 2)
            t = a - K.reshape(-1)
            m = t.max()
            out[i, j] = -(m + np.log2(np.sum(np.exp2(t - m))))
    return (out - out.mean()).reshape(-1)


def cell_targets(alpha_blk, mu_blk, nu_arr, r0, c0, o1, o2, eps, k2) -> np.ndarray:
    g = cell_gauge(mu_blk, r0, c0, nu_arr, o1, o2)
    r = alpha_target(alpha_blk, mu_blk, eps, k2, g)
    t = np.zeros(NT)
    t[:64] = r
    t[64:] = beta_aux_target(r, mu_blk, nu_arr.shape[0], nu_arr.shape[1], k2, g)
    return t
