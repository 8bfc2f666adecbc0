"""Pins of the line-relaxation oracle (oracle/line_relax.py), the
block-Jacobi reading of "one 1D system per line, off-line neighbours at
their current estimates" on the dense 2D WLS of Eqs. 1-4.

* One pass equals the dense block-Jacobi step built from the pinned 2D WLS
  matrix (oracle/wls2d.py): for every line L, u_L = A_LL^-1 (F_L - A_L,rest
  U_rest), A the (2r+1) x (2r+1)-neighbourhood matrix of Eq. 4.
* Alternating passes converge to the dense 2D WLS solution A^-1 F (the
  fixed point of the splitting).
* lambda = 0 returns F; a constant image stays constant; on an image one
  row high the row pass has no off-line neighbours and is the exact 2D WLS
  solution in one pass.
A planted mistake (an off-line weight left out of the diagonal, the data
term taken from U instead of F, a sign flip) fails the first two."""
import numpy as np
import pytest

from oracle import COLUMN, ROW, Params
from oracle.line_relax import line_relax, line_relax_pass
from oracle.wls2d import wls2d, wls2d_matrix


def _img(C, H, W, seed):
    return np.random.default_rng(seed).random((C, H, W))


@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("direction", [COLUMN, ROW])
@pytest.mark.parametrize("weight", ["exp", "frac"])
def test_pass_equals_dense_block_jacobi(r, direction, weight):
    C, H, W = 2, 7, 9
    F = _img(C, H, W, 1)
    U = _img(C, H, W, 2)
    G = _img(1, H, W, 3)[0]
    prm = Params(r=r, sigma_s=float(r), sigma_r=0.2, weight=weight)
    lam = 1.7
    A = wls2d_matrix(G, lam, prm)
    want = np.empty_like(U)
    nlines = H if direction == ROW else W
    for k in range(nlines):
        if direction == ROW:
            idx = [k * W + x for x in range(W)]
        else:
            idx = [y * W + k for y in range(H)]
        rest = [i for i in range(H * W) if i not in set(idx)]
        ALL = A[np.ix_(idx, idx)]
        ALR = A[np.ix_(idx, rest)]
        for c in range(C):
            f = F[c].reshape(-1)
            u = U[c].reshape(-1)
            sol = np.linalg.solve(ALL, f[idx] - ALR @ u[rest])
            want[c].reshape(-1)[idx] = sol
    got = line_relax_pass(U, F, G, lam, prm, direction)
    assert np.allclose(got, want, atol=1e-12, rtol=0)


@pytest.mark.parametrize("r", [1, 2])
def test_converges_to_dense_2d_wls(r):
    C, H, W = 1, 9, 11
    F = _img(C, H, W, 4)
    G = _img(1, H, W, 5)[0]
    prm = Params(r=r, iters=60, sigma_s=float(r), sigma_r=0.3)
    lam = 0.8
    got = line_relax(F, G, lam, prm)
    assert np.abs(got - wls2d(F, G, lam, prm)).max() < 1e-9


def test_lambda_zero_constant_and_single_row():
    F = _img(3, 6, 8, 6)
    G = _img(1, 6, 8, 7)[0]
    prm = Params(r=2, iters=2, sigma_s=2.0, sigma_r=0.1)
    assert np.allclose(line_relax(F, G, 0.0, prm), F, atol=1e-14)
    c = np.full((1, 6, 8), 0.42)
    assert np.allclose(line_relax(c, G, 3.0, prm), c, atol=1e-12)
    row = _img(1, 1, 13, 8)
    grow = _img(1, 1, 13, 9)[0]
    one = line_relax_pass(row, row, grow, 2.0, Params(r=2, sigma_s=2.0, sigma_r=0.2), ROW)
    assert np.allclose(one, wls2d(row, grow, 2.0, Params(r=2, sigma_s=2.0, sigma_r=0.2)), atol=1e-12)
