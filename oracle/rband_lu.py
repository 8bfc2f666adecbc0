"""The paper's r-band LU decomposition (Sec. 2.2, Eqs. 6-20), in its notation.

TEST INFRASTRUCTURE ONLY.  Pure-Python loops: use on small systems.

A_s has diagonal a_k, upper bands b_{k,i} = A_s[k, k+i] and lower bands
c_{k,i} = A_s[k+i, k] (1-based k, i = 1..r).  A_s = P Q (Eq. 6) with P lower
triangular (diagonal alpha_k, bands gamma_{k,i} = P[k+i, k]) and Q unit upper
triangular (bands beta_{k,i} = Q[k, k+i]).  P y = f (Eq. 7) and Q u = y
(Eq. 8) are then solved by forward and back substitution.

The recurrences below are Eqs. 9-14 (decomposition), 15-17 (forward) and
18-20 (backward).  The summation ranges are the ones the products P Q
require: gamma_{k,i} and beta_{k,i} sum over t = 1 .. min(k-1, r-i), which
is k-1 in Eq. 10 and r-i in Eqs. 11 and 13; alpha_k sums over
t = 1 .. min(k-1, r) (Eqs. 10 and 12); Eq. 14 is the empty sum at i = r.
"""
from __future__ import annotations

import numpy as np


def band_from_dense(A: np.ndarray, r: int):
    """Read a_k, b_{k,i}, c_{k,i} (1-based dicts) out of a dense matrix."""
    s = A.shape[0]
    a = {k: A[k - 1, k - 1] for k in range(1, s + 1)}
    b, c = {}, {}
    for k in range(1, s + 1):
        for i in range(1, r + 1):
            if k + i <= s:
                b[k, i] = A[k - 1, k + i - 1]
                c[k, i] = A[k + i - 1, k - 1]
    return a, b, c


def rband_lu(a, b, c, r: int, s: int):
    """Eqs. 9-14: alpha_k, gamma_{k,i}, beta_{k,i} of A_s = P Q."""
    alpha, gamma, beta = {}, {}, {}
    for k in range(1, s + 1):
        # alpha_k (Eq. 9 for k = 1, Eq. 10 for k <= r, Eq. 12 for k > r)
        acc = a[k]
        for t in range(1, min(k - 1, r) + 1):
            acc -= gamma[k - t, t] * beta[k - t, t]
        alpha[k] = acc
        # gamma_{k,i}, beta_{k,i} (Eqs. 9, 10, 11, 13, 14) for entries inside A_s
        for i in range(1, r + 1):
            if k + i > s:
                break
            g = c[k, i]
            bb = b[k, i]
            for t in range(1, min(k - 1, r - i) + 1):
                g -= gamma[k - t, i + t] * beta[k - t, t]
                bb -= beta[k - t, i + t] * gamma[k - t, t]
            gamma[k, i] = g
            beta[k, i] = bb / alpha[k]
    return alpha, gamma, beta


def rband_solve(alpha, gamma, beta, f, r: int, s: int):
    """Eqs. 15-17 (P y = f) then Eqs. 18-20 (Q u = y).  f: length-s array
    (0-based storage, 1-based formulas)."""
    y = np.zeros(s + 1)
    for k in range(1, s + 1):
        acc = f[k - 1]
        for t in range(1, min(k - 1, r) + 1):
            acc -= gamma[k - t, t] * y[k - t]
        y[k] = acc / alpha[k]
    u = np.zeros(s + 2)
    for k in range(s, 0, -1):
        acc = y[k]
        for t in range(1, min(s - k, r) + 1):
            acc -= beta[k, t] * u[k + t]
        u[k] = acc
    return u[1:s + 1]


def solve_dense_rband(A: np.ndarray, f: np.ndarray, r: int) -> np.ndarray:
    """Solve A u = f for a dense matrix of half-bandwidth r with Eqs. 9-20."""
    s = A.shape[0]
    a, b, c = band_from_dense(A, r)
    alpha, gamma, beta = rband_lu(a, b, c, r, s)
    return rband_solve(alpha, gamma, beta, np.asarray(f, dtype=np.float64), r, s)
