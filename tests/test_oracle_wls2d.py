"""Pins of the dense 2D WLS oracle (oracle/wls2d.py, Eqs. 1-4).

Each check follows from the model, not from the oracle's own code:

* Eq. 4: A = I + lambda L with L a weighted graph Laplacian, so A is
  symmetric, A 1 = 1 (unit row sums), and diagonal minus the sum of the
  off-diagonal magnitudes is exactly 1 in every row; the off-diagonals are
  -lambda w_ij on the (2r+1) x (2r+1) square patch (Sec. 1), so a pixel has
  (min(y+r, H-1) - max(y-r, 0) + 1) (the same across) - 1 neighbours.
* lambda = 0 returns F; a constant image stays constant.
* An image one row high: the square patch reduces to the r nearest pixels
  on each side along the row, so U must equal the solve of a 1D banded
  system built here from Eq. 2's closed form and solved with
  scipy.linalg.solve_banded.
* Eq. 1 and the factor-2 reading: U minimises
  E(U) = sum (U - F)^2 + lambda sum_{unordered pairs} w (U_i - U_j)^2,
  whose normal equations are (I + lambda L) U = F; the gradient of E, summed
  here pair by pair, vanishes at U, and E grows along random directions.
A planted mistake (a dropped diagonal term, a sign flip, a doubled
lambda, a patch clipped one pixel short) fails at least one of these.
"""
import numpy as np
import pytest
from scipy.linalg import solve_banded

from oracle import Params
from oracle.wls2d import wls2d, wls2d_matrix


def _img(H, W, seed):
    rng = np.random.default_rng(seed)
    return rng.random((H, W))


def _w_exp(dy, dx, g1, g2, prm):
    return np.exp(-(dy * dy + dx * dx) / (2 * prm.sigma_s ** 2)) * np.exp(-(g1 - g2) ** 2 / (2 * prm.sigma_r ** 2))


@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("weight", ["exp", "frac"])
def test_matrix_structure(r, weight):
    G = _img(6, 7, 1)
    prm = Params(r=r, sigma_s=float(r), sigma_r=0.2, weight=weight)
    lam = 1.7
    A = wls2d_matrix(G, lam, prm)
    assert np.allclose(A, A.T, atol=0, rtol=1e-15)
    assert np.allclose(A.sum(axis=1), 1.0, atol=1e-12)
    off = A - np.diag(np.diag(A))
    assert (off <= 0).all()
    assert np.allclose(np.diag(A) - np.abs(off).sum(axis=1), 1.0, atol=1e-12)
    # neighbour count of every pixel: the square patch clipped at the border
    H, W = G.shape
    for y in range(H):
        for x in range(W):
            ny = min(y + r, H - 1) - max(y - r, 0) + 1
            nx = min(x + r, W - 1) - max(x - r, 0) + 1
            assert np.count_nonzero(off[y * W + x]) == ny * nx - 1, (y, x)


def test_matrix_entries_closed_form():
    """Two hand-picked pairs of Eq. 2 with exp weights: a horizontal and a
    diagonal neighbour."""
    G = _img(5, 5, 2)
    prm = Params(r=2, sigma_s=2.0, sigma_r=0.15)
    lam = 0.9
    A = wls2d_matrix(G, lam, prm)
    W = 5
    for (y, x), (yy, xx) in [((2, 2), (2, 3)), ((1, 1), (3, 2))]:
        want = -lam * _w_exp(yy - y, xx - x, G[y, x], G[yy, xx], prm)
        assert A[y * W + x, yy * W + xx] == pytest.approx(want, rel=1e-13)


def test_lambda_zero_and_constant():
    F = _img(8, 9, 3)[None].repeat(2, axis=0)
    G = _img(8, 9, 4)
    prm = Params(r=1, sigma_s=1.0, sigma_r=0.1)
    assert np.allclose(wls2d(F, G, 0.0, prm), F, atol=1e-14)
    c = np.full((1, 8, 9), 0.37)
    assert np.allclose(wls2d(c, G, 5.0, prm), c, atol=1e-12)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_single_row_equals_1d_banded_solve(r):
    W = 14
    rng = np.random.default_rng(10 + r)
    g = rng.random(W)
    f = rng.random(W)
    prm = Params(r=r, sigma_s=float(r), sigma_r=0.2)
    lam = 2.3
    # 1D system I + lambda L over pairs at distance 1..r along the row,
    # in LAPACK band storage (ab[r + i - j, j] = A[i, j])
    ab = np.zeros((2 * r + 1, W))
    ab[r] = 1.0
    for i in range(W):
        for t in range(1, r + 1):
            j = i + t
            if j < W:
                w = lam * _w_exp(0, t, g[i], g[j], prm)
                ab[r + i - j, j] -= w   # A[i, j]
                ab[r + j - i, i] -= w   # A[j, i]
                ab[r, i] += w
                ab[r, j] += w
    want = solve_banded((r, r), ab, f)
    got = wls2d(f[None, None, :], g[None, :], lam, prm)[0, 0]
    assert np.allclose(got, want, atol=1e-12, rtol=0)


def test_minimises_eq1_energy():
    H, W = 6, 6
    F = _img(H, W, 5)
    G = _img(H, W, 6)
    prm = Params(r=1, sigma_s=1.0, sigma_r=0.3)
    lam = 1.3
    U = wls2d(F, G, lam, prm)[0]

    pairs = []
    for y in range(H):
        for x in range(W):
            for dy in range(-1, 2):
                for dx in range(-1, 2):
                    yy, xx = y + dy, x + dx
                    if (dy, dx) != (0, 0) and 0 <= yy < H and 0 <= xx < W and (yy, xx) > (y, x):
                        pairs.append((y, x, yy, xx, _w_exp(dy, dx, G[y, x], G[yy, xx], prm)))

    def energy(V):
        e = ((V - F) ** 2).sum()
        for y, x, yy, xx, w in pairs:
            e += lam * w * (V[y, x] - V[yy, xx]) ** 2
        return e

    grad = 2 * (U - F)
    for y, x, yy, xx, w in pairs:
        d = 2 * lam * w * (U[y, x] - U[yy, xx])
        grad[y, x] += d
        grad[yy, xx] -= d
    assert np.abs(grad).max() < 1e-12
    e0 = energy(U)
    rng = np.random.default_rng(7)
    for _ in range(5):
        D = rng.standard_normal((H, W))
        assert energy(U + 1e-3 * D) > e0
