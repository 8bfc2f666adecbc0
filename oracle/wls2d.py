"""The full two-dimensional WLS model (Sec. 1, Eqs. 1-4), solved densely.

TEST INFRASTRUCTURE ONLY.  O((HW)^3): for images of at most 16 x 16.

A (S x S, S = M N) has A[i, i] = 1 + lambda * sum_{j in N(i)} w_ij and
A[i, j] = -lambda * w_ij for j in N(i), the (2r+1) x (2r+1) square patch
centred at i (Eq. 4); U = A^{-1} F (Eq. 3), channel by channel.  Weights
are Eq. 2 on image coordinates.
"""
from __future__ import annotations

import numpy as np

from .sgwls import Params, guidance_weight


def wls2d_matrix(G: np.ndarray, lam: float, prm: Params) -> np.ndarray:
    H, W = G.shape
    S = H * W
    A = np.eye(S)
    r = prm.r
    for i in range(H):
        for j in range(W):
            a = i * W + j
            for di in range(-r, r + 1):
                for dj in range(-r, r + 1):
                    if di == 0 and dj == 0:
                        continue
                    ii, jj = i + di, j + dj
                    if 0 <= ii < H and 0 <= jj < W:
                        w = guidance_weight(np.array([i]), np.array([j]),
                                            np.array([ii]), np.array([jj]), G, prm)[0]
                        A[a, ii * W + jj] = -lam * w
                        A[a, a] += lam * w
    return A


def wls2d(F: np.ndarray, G: np.ndarray, lam: float, prm: Params) -> np.ndarray:
    """Eq. 3: U = A^{-1} F for every channel of F (C, H, W)."""
    F = np.asarray(F, dtype=np.float64)
    if F.ndim == 2:
        F = F[None]
    C, H, W = F.shape
    A = wls2d_matrix(G, lam, prm)
    U = np.linalg.solve(A, F.reshape(C, H * W).T).T
    return U.reshape(C, H, W)
