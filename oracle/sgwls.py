"""SG-WLS in FP64 on the CPU, step by step in the paper's order.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation follows the paper: an M x N image (here H x W), a (2r+1) x (2r+1)
neighbourhood, the formed 1D vector f of length s, the subsystem A_s u = f
(Eq. 5), the sliding step tau (Sec. 2.3) and T alternating iterations.
Indices are 0-based internally; the paper's 1-based row number i + 1 is
spelled out where parity matters.

Readings of points the paper leaves open:

* |i - j| in Eq. 2 is the Euclidean distance between the two pixels'
  image coordinates (snake neighbours are 2D neighbours, Sec. 2.1).
* A_s is "formed in a way similar to Eq. 4": A_s = I + lambda * L, where L is
  the weighted Laplacian of the 1D neighbourhood {q : 0 < |p - q| <= r} on
  the formed vector (Eq. 4's convention, not the factor 2 that the normal
  equations of Eq. 1 would give).
* Centres are k = r .. dim-1-r (0-based, Sec. 2.1); with a sliding step
  tau > 1 the last centre dim-1-r is appended if the stride misses it, so
  every line is covered (tau <= 2r + 1 is required for full coverage).
* The guidance G is fixed for all passes; the multi-channel input is
  filtered channel by channel with the same A_s (A_s depends on G and lambda
  only).
* For a vector guidance (a colour image), |G_i - G_j| in Eq. 2 is the
  Euclidean norm of the difference of the two guidance vectors.
* The default pass order is column direction first, then row direction
  (Sec. 2.3: "along column direction and row direction alternatively");
  axis_order=1 runs the row direction first.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.linalg import solve_banded

COLUMN = 0  # neighbourhood construction along column direction (centres are columns)
ROW = 1     # neighbourhood construction along row direction (centres are rows)


@dataclass(frozen=True)
class Params:
    """User constants of the method (Eq. 2, Sec. 2.1, Sec. 2.3)."""

    r: int = 1                 # neighbourhood radius: (2r+1) x (2r+1) system
    iters: int = 1             # T: number of (column, row) pass pairs
    step: int = 1              # tau: sliding step between subsystem centres
    axis_order: int = 0        # 0: column direction first (paper); 1: row first
    weight: str = "exp"        # "exp" or "frac" (Eq. 2)
    sigma_s: float = 1.0       # exp weight: spatial scale
    sigma_r: float = 0.1       # exp weight: range scale
    alpha_s: float = 1.2       # frac weight: spatial exponent
    alpha_r: float = 1.2       # frac weight: range exponent
    eps: float = 1e-4          # frac weight: epsilon (Sec. 1: 0.0001)


def centre_indices(dim: int, r: int, step: int = 1) -> list[int]:
    """Centres of the subsystems along one direction.

    Sec. 2.1: the k-th column, k = r+1, ..., N-r (1-based), i.e. 0-based
    k = r .. dim-1-r.  Sec. 2.3: the construction slides with step tau.
    Reading: with tau > 1 the last centre is appended when the stride misses
    it."""
    if dim < 2 * r + 1:
        raise ValueError("image dimension smaller than 2r+1")
    ks = list(range(r, dim - r, step))
    if ks[-1] != dim - 1 - r:
        ks.append(dim - 1 - r)
    return ks


def neighbourhood_construction(direction: int, k: int, r: int, H: int, W: int):
    """Sec. 2.1, step 1 of Sec. 2.3: the formed 1D vector as pixel coordinates.

    Column direction: take the 2r+1 columns k-r .. k+r; the image has M row
    vectors of size 2r+1 over them; the i-th row vector (1-based i) is
    reversed when i is even; the row vectors are joined head to end, giving a
    (2r+1)M vector.  Row direction is the same construction along the rows
    k-r .. k+r, giving a (2r+1)N vector whose j-th column segment (1-based j)
    is reversed when j is even.

    Returns (rows, cols), integer arrays of length s = (2r+1) * lines."""
    seg = np.arange(k - r, k + r + 1)
    rows, cols = [], []
    if direction == COLUMN:
        for i in range(H):
            piece = seg[::-1] if (i + 1) % 2 == 0 else seg
            rows.append(np.full(2 * r + 1, i))
            cols.append(piece)
    elif direction == ROW:
        for j in range(W):
            piece = seg[::-1] if (j + 1) % 2 == 0 else seg
            rows.append(piece)
            cols.append(np.full(2 * r + 1, j))
    else:
        raise ValueError("direction must be COLUMN or ROW")
    return np.concatenate(rows), np.concatenate(cols)


def guidance_weight(rows_i, cols_i, rows_j, cols_j, G: np.ndarray, prm: Params) -> np.ndarray:
    """Eq. 2: the guidance weight between pixels i and j (vectorised).

    exp:  exp(-|i-j|^2 / (2 sigma_s^2)) * exp(-|G_i-G_j|^2 / (2 sigma_r^2))
    frac: 1 / (|i-j|^alpha_s + eps) * 1 / (|G_i-G_j|^alpha_r + eps)
    |i - j| is the Euclidean distance of the image coordinates.  G is (H, W)
    or, for a vector guidance (a colour image), (Cg, H, W); |G_i - G_j| is
    then the Euclidean norm of the difference of the two guidance vectors."""
    G = np.asarray(G, dtype=np.float64)
    d2 = (rows_i - rows_j).astype(np.float64) ** 2 + (cols_i - cols_j).astype(np.float64) ** 2
    if G.ndim == 3:
        diff = G[:, rows_i, cols_i] - G[:, rows_j, cols_j]          # (Cg, pairs)
        dg = np.sqrt(np.sum(diff * diff, axis=0))
    else:
        dg = G[rows_i, cols_i] - G[rows_j, cols_j]
    if prm.weight == "exp":
        return np.exp(-d2 / (2.0 * prm.sigma_s ** 2)) * np.exp(-(dg ** 2) / (2.0 * prm.sigma_r ** 2))
    if prm.weight == "frac":
        d = np.sqrt(d2)
        return 1.0 / (d ** prm.alpha_s + prm.eps) * 1.0 / (np.abs(dg) ** prm.alpha_r + prm.eps)
    raise ValueError("weight must be 'exp' or 'frac'")


def subsystem_band(rows, cols, G, lam: float, prm: Params) -> np.ndarray:
    """Eq. 5: A_s of the formed vector, formed like Eq. 4 on the 1D
    neighbourhood of 2r+1 entries (Sec. 2.2).

    A_s[p, p] = 1 + lambda * sum_{q in N(p)} w_pq,  A_s[p, q] = -lambda * w_pq
    for 0 < |p - q| <= r.  Returned in LAPACK band storage for
    ``scipy.linalg.solve_banded((r, r), ...)``: ab[r + p - q, q] = A_s[p, q]."""
    r = prm.r
    s = len(rows)
    ab = np.zeros((2 * r + 1, s))
    ab[r, :] = 1.0
    for t in range(1, r + 1):
        if t >= s:
            break
        p = np.arange(0, s - t)
        q = p + t
        w = guidance_weight(rows[p], cols[p], rows[q], cols[q], G, prm)
        ab[r - t, q] = -lam * w      # upper: A_s[p, p+t]
        ab[r + t, p] = -lam * w      # lower: A_s[p+t, p]
        ab[r, p] += lam * w
        ab[r, q] += lam * w
    return ab


def solve_subsystem(ab: np.ndarray, f: np.ndarray, r: int) -> np.ndarray:
    """Step 2 of Sec. 2.3: solve A_s u = f exactly (Eq. 5).  A generic banded
    LU with partial pivoting (LAPACK gbsv) serves as this step; f may hold
    several channels as columns."""
    return solve_banded((r, r), ab, f)


def coverage_counts(direction: int, H: int, W: int, prm: Params) -> np.ndarray:
    """How many subsystems contain each pixel (the divisor of step 4)."""
    cnt = np.zeros((H, W))
    dim = W if direction == COLUMN else H
    for k in centre_indices(dim, prm.r, prm.step):
        lo, hi = k - prm.r, k + prm.r + 1
        if direction == COLUMN:
            cnt[:, lo:hi] += 1
        else:
            cnt[lo:hi, :] += 1
    return cnt


def sgwls_pass(U: np.ndarray, G: np.ndarray, lam: float, prm: Params, direction: int) -> np.ndarray:
    """One direction of Sec. 2.3: for every centre, (1) construct the 1D
    vector, (2) solve its subsystem, (3) put the solution back into the
    (2r+1)-line patch, and (4) average the values each pixel received.

    U: (C, H, W) current estimate; G: (H, W) or (Cg, H, W) guidance."""
    U = np.asarray(U, dtype=np.float64)
    C, H, W = U.shape
    acc = np.zeros_like(U)
    cnt = np.zeros((H, W))
    dim = W if direction == COLUMN else H
    for k in centre_indices(dim, prm.r, prm.step):
        rows, cols = neighbourhood_construction(direction, k, prm.r, H, W)   # step 1
        f = U[:, rows, cols].T                                              # (s, C)
        ab = subsystem_band(rows, cols, G, lam, prm)
        u = solve_subsystem(ab, f, prm.r)                                   # step 2
        acc[:, rows, cols] += u.T                                           # step 3 (each pixel once per vector)
        cnt[rows, cols] += 1.0
    return acc / cnt                                                        # step 4


def pass_directions(prm: Params) -> list[int]:
    """The order of the 2T passes (Sec. 2.3)."""
    first = [COLUMN, ROW] if prm.axis_order == 0 else [ROW, COLUMN]
    return first * prm.iters


def sgwls(F: np.ndarray, G: np.ndarray, lam: float, prm: Params, return_inputs: bool = False):
    """SG-WLS smoothing (Sec. 2.3): the four steps performed T times along
    the column direction and the row direction alternately.

    F: (C, H, W) or (H, W) input; G: (H, W) or (Cg, H, W) guidance (fixed
    for all passes).
    Returns the (C, H, W) float64 result (and, if ``return_inputs``, the
    list of each pass's input estimate)."""
    U = np.asarray(F, dtype=np.float64)
    if U.ndim == 2:
        U = U[None]
    inputs = []
    for direction in pass_directions(prm):
        inputs.append(U)
        U = sgwls_pass(U, G, lam, prm, direction)
    return (U, inputs) if return_inputs else U


def sgwls_interpolate(F: np.ndarray, Hm: np.ndarray, G: np.ndarray, lam: float, prm: Params,
                      return_parts: bool = False):
    """Guided sparse interpolation (Sec. 2.3, Eq. 21): the SG-WLS smoothing
    applied to the sparse input F and to its index map Hm (1 where F holds
    data, 0 elsewhere), and their ratio per pixel.  Reading: a pixel that no
    data reaches (smoothed index map exactly 0) is 0.

    F: (C, H, W) or (H, W), zero where Hm is zero; Hm: (H, W); G: (H, W) or
    (Cg, H, W)."""
    N = sgwls(F, G, lam, prm)
    D = sgwls(np.asarray(Hm, dtype=np.float64), G, lam, prm)[0]
    U = np.where(D > 0, N / np.where(D > 0, D, 1.0), 0.0)
    return (U, N, D) if return_parts else U
