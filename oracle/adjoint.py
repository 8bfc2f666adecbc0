"""Reverse-mode derivative of SG-WLS in FP64 (test infrastructure only).

The paper has no backward pass; this is the chain rule through its forward
definition (Eq. 2 weights, Eq. 4 form of A_s, Eq. 5 subsystem, the four
steps of Sec. 2.3):

* step 4 (averaging) transposed:      Vbar / count
* step 3 (inverse construction)^T:    ubar = gather of Vbar/count along the vector
* step 2 (u = A_s^{-1} f):            v = A_s^{-1} ubar   (A_s is symmetric),
                                      fbar = v,  Abar = -v u^T
* step 1 (construction)^T:            scatter fbar back onto the pixels
* A_s = I + lambda L(w):  dLoss/dw_pq = -lambda (v_p - v_q).(u_p - u_q),
                          dLoss/dlambda = -sum_pq w_pq (v_p - v_q).(u_p - u_q)
  (the dot runs over channels, which share A_s)
* Eq. 2 weights:  exp:  dw/dG_p = -w (G_p - G_q) / sigma_r^2
                  frac: dw/dG_p = -S h^2 alpha_r |G_p-G_q|^(alpha_r-1) sign(G_p-G_q),
                        with S the spatial factor and h the range factor
  and dw/dG_q = -dw/dG_p.  The frac derivative needs alpha_r >= 1.

TEST INFRASTRUCTURE ONLY.
"""
from __future__ import annotations

import numpy as np

from .sgwls import (
    COLUMN,
    Params,
    centre_indices,
    coverage_counts,
    guidance_weight,
    neighbourhood_construction,
    pass_directions,
    sgwls,
    solve_subsystem,
    subsystem_band,
)


def _weight_and_grad(rp, cp, rq, cq, G, prm: Params):
    """w_pq (Eq. 2) and dw_pq / dG_p."""
    G = np.asarray(G, dtype=np.float64)
    w = guidance_weight(rp, cp, rq, cq, G, prm)
    dg = G[rp, cp] - G[rq, cq]
    if prm.weight == "exp":
        dw = -w * dg / (prm.sigma_r ** 2)
    else:
        if prm.alpha_r < 1.0:
            raise ValueError("frac-weight gradient needs alpha_r >= 1")
        d = np.sqrt((rp - rq).astype(np.float64) ** 2 + (cp - cq).astype(np.float64) ** 2)
        spatial = 1.0 / (d ** prm.alpha_s + prm.eps)
        h = 1.0 / (np.abs(dg) ** prm.alpha_r + prm.eps)
        dw = -spatial * h * h * prm.alpha_r * np.abs(dg) ** (prm.alpha_r - 1.0) * np.sign(dg)
    return w, dw


def sgwls_pass_vjp(U_in, G, lam: float, prm: Params, direction: int, V_bar):
    """Vector-Jacobian product of one pass ``sgwls_pass(U_in) -> V``.

    Returns (U_in_bar, G_bar, lam_bar)."""
    U_in = np.asarray(U_in, dtype=np.float64)
    C, H, W = U_in.shape
    r = prm.r
    cnt = coverage_counts(direction, H, W, prm)
    Vb = np.asarray(V_bar, dtype=np.float64) / cnt
    U_bar = np.zeros_like(U_in)
    G_bar = np.zeros((H, W))
    lam_bar = 0.0
    dim = W if direction == COLUMN else H
    for k in centre_indices(dim, r, prm.step):
        rows, cols = neighbourhood_construction(direction, k, r, H, W)
        s = len(rows)
        ab = subsystem_band(rows, cols, G, lam, prm)
        u = solve_subsystem(ab, U_in[:, rows, cols].T, r)      # (s, C)
        ubar = Vb[:, rows, cols].T
        v = solve_subsystem(ab, ubar, r)
        U_bar[:, rows, cols] += v.T
        for t in range(1, r + 1):
            if t >= s:
                break
            p = np.arange(0, s - t)
            q = p + t
            w, dw = _weight_and_grad(rows[p], cols[p], rows[q], cols[q], G, prm)
            dvu = np.sum((v[p] - v[q]) * (u[p] - u[q]), axis=1)
            w_bar = -lam * dvu
            lam_bar += float(np.sum(-w * dvu))
            np.add.at(G_bar, (rows[p], cols[p]), w_bar * dw)
            np.add.at(G_bar, (rows[q], cols[q]), -w_bar * dw)
    return U_bar, G_bar, lam_bar


def sgwls_vjp(F, G, lam: float, prm: Params, U_bar):
    """Gradients of <U_bar, sgwls(F, G, lam)> with respect to F, G, lambda.

    The forward inputs of every pass are kept (per-pass checkpoints) and the
    passes are walked in reverse order.  Returns (F_bar, G_bar, lam_bar)."""
    F = np.asarray(F, dtype=np.float64)
    squeeze = F.ndim == 2
    if squeeze:
        F = F[None]
    _, inputs = sgwls(F, G, lam, prm, return_inputs=True)
    dirs = pass_directions(prm)
    V_bar = np.asarray(U_bar, dtype=np.float64).reshape(F.shape)
    G_bar = np.zeros(np.asarray(G).shape)
    lam_bar = 0.0
    for t in range(len(dirs) - 1, -1, -1):
        V_bar, g, l = sgwls_pass_vjp(inputs[t], G, lam, prm, dirs[t], V_bar)
        G_bar += g
        lam_bar += l
    return (V_bar[0] if squeeze else V_bar), G_bar, lam_bar
