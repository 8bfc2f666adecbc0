"""Line relaxation of the 2D WLS model, FP64 on the CPU.

TEST INFRASTRUCTURE ONLY (see the package docstring).

This is not the paper's SG-WLS subsystem (Sec. 2.1 solves the whole
(2r+1)-line zig-zag strip exactly).  It is the alternative reading of the
task's wording in which each pass solves one 1D system per image line with
the off-line neighbours at their current estimates: a block-Jacobi
iteration on the dense 2D WLS system of Eqs. 1-4 (A = I + lambda L over the
(2r+1) x (2r+1) square neighbourhood, Eq. 4's convention), the blocks being
the image rows (row pass) or columns (column pass).

For pixel p on line y of the pass, with N(p) the square neighbourhood and
w_pq the Eq. 2 weight, the line system is

    (1 + lambda sum_{q in N(p)} w_pq) u_p - lambda sum_{q in N(p), on the line} w_pq u_q
        = F_p + lambda sum_{q in N(p), off the line} w_pq U_q,

where F is the filter's input (the data term of Eq. 1) and U the estimate
the pass starts from (U = F before the first pass).  Each line matrix is
symmetric, banded with half-bandwidth r and strictly diagonally dominant;
the splitting of A into these line blocks is a regular splitting of an
M-matrix, so alternating row and column passes converge to the 2D WLS
solution A^-1 F, which pins the iteration (tests/test_oracle_line_relax.py).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_banded

from .sgwls import COLUMN, ROW, Params, guidance_weight, pass_directions


def line_relax_pass(U: np.ndarray, F: np.ndarray, G: np.ndarray, lam: float, prm: Params,
                    direction: int) -> np.ndarray:
    """One pass: every row (direction ROW) or column (COLUMN) solved as one
    banded system, the other lines at the estimate U.  U, F: (C, H, W);
    G: (H, W) or (Cg, H, W)."""
    U = np.asarray(U, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    C, H, W = U.shape
    r = prm.r
    out = np.empty_like(U)
    nlines, n = (H, W) if direction == ROW else (W, H)
    for k in range(nlines):
        # pixel coordinates of the line's entries, in order along the line
        idx = np.arange(n)
        ys, xs = (np.full(n, k), idx) if direction == ROW else (idx, np.full(n, k))
        ab = np.zeros((2 * r + 1, n))
        ab[r, :] = 1.0
        rhs = F[:, ys, xs].T.copy()                      # (n, C)
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                if dy == 0 and dx == 0:
                    continue
                qy, qx = ys + dy, xs + dx
                ok = (qy >= 0) & (qy < H) & (qx >= 0) & (qx < W)
                p = np.nonzero(ok)[0]
                w = lam * guidance_weight(ys[p], xs[p], qy[p], qx[p], G, prm)
                ab[r, p] += w                             # every neighbour on the diagonal
                along = dx if direction == ROW else dy    # offset along the line
                across = dy if direction == ROW else dx   # offset across the lines
                if across == 0:
                    # on the line: a matrix entry A[p, p + along] (LAPACK band storage)
                    ab[r - along, p + along] -= w
                else:
                    # off the line: its current estimate moves to the right-hand side
                    rhs[p] += w[:, None] * U[:, qy[p], qx[p]].T
        out[:, ys, xs] = solve_banded((r, r), ab, rhs).T
    return out


def line_relax(F: np.ndarray, G: np.ndarray, lam: float, prm: Params, U0: np.ndarray | None = None) -> np.ndarray:
    """prm.iters iterations of (first direction, second direction) passes
    in the order of Sec. 2.3 (column direction first unless
    prm.axis_order = 1), starting from U0 (default: F)."""
    F = np.asarray(F, dtype=np.float64)
    squeeze = F.ndim == 2
    if squeeze:
        F = F[None]
    U = F.copy() if U0 is None else np.asarray(U0, dtype=np.float64).reshape(F.shape).copy()
    for d in pass_directions(prm):
        U = line_relax_pass(U, F, G, lam, prm, d)
    return U[0] if squeeze else U


__all__ = ["line_relax_pass", "line_relax", "COLUMN", "ROW"]
