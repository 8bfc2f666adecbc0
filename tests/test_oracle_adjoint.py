"""Pins of the oracle's reverse-mode derivative (FP64).

The paper has no backward pass; the derivative is checked against FP64
central finite differences of the oracle's forward map, the adjoint identity
of the linear map F -> U, and the closed form dU/dlambda = -A_s^{-1} L u of a
single subsystem.
"""
import numpy as np
import pytest

from oracle import COLUMN, ROW, Params, neighbourhood_construction, sgwls, sgwls_pass, solve_subsystem, subsystem_band
from oracle.adjoint import sgwls_pass_vjp, sgwls_vjp


def _loss(F, G, lam, prm, Ubar):
    return float(np.sum(sgwls(F, G, lam, prm) * Ubar))


@pytest.mark.parametrize("prm", [
    Params(r=1, iters=1, sigma_s=1.0, sigma_r=0.3),
    Params(r=2, iters=2, sigma_s=2.0, sigma_r=0.4, axis_order=1),
    Params(r=1, iters=1, weight="frac", alpha_s=1.2, alpha_r=1.2),
])
def test_vjp_matches_central_differences(prm):
    rng = np.random.default_rng(3)
    C, H, W = 2, 7, 6
    F = rng.uniform(0, 1, size=(C, H, W))
    G = rng.uniform(0, 1, size=(H, W))
    lam = 1.5 if prm.weight == "exp" else 0.01
    Ubar = rng.normal(size=(C, H, W))
    Fb, Gb, lb = sgwls_vjp(F, G, lam, prm, Ubar)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 3, 2), (0, 6, 5), (1, 2, 4)]:
        Fp, Fm = F.copy(), F.copy()
        Fp[idx] += h
        Fm[idx] -= h
        fd = (_loss(Fp, G, lam, prm, Ubar) - _loss(Fm, G, lam, prm, Ubar)) / (2 * h)
        assert Fb[idx] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    for idx in [(0, 0), (3, 3), (6, 1), (2, 5)]:
        Gp, Gm = G.copy(), G.copy()
        Gp[idx] += h
        Gm[idx] -= h
        fd = (_loss(F, Gp, lam, prm, Ubar) - _loss(F, Gm, lam, prm, Ubar)) / (2 * h)
        assert Gb[idx] == pytest.approx(fd, rel=1e-5, abs=1e-7)
    hl = 1e-6 * max(lam, 1e-3)
    fd = (_loss(F, G, lam + hl, prm, Ubar) - _loss(F, G, lam - hl, prm, Ubar)) / (2 * hl)
    assert lb == pytest.approx(fd, rel=1e-5)


@pytest.mark.parametrize("direction", [COLUMN, ROW])
def test_pass_adjoint_identity(direction):
    """<P x, y> = <x, P^T y> for the pass as a linear map of its input."""
    rng = np.random.default_rng(11)
    C, H, W = 3, 8, 9
    G = rng.uniform(0, 1, size=(H, W))
    prm = Params(r=2, sigma_s=2.0, sigma_r=0.2)
    x = rng.normal(size=(C, H, W))
    y = rng.normal(size=(C, H, W))
    Px = sgwls_pass(x, G, 2.0, prm, direction)
    PTy, _, _ = sgwls_pass_vjp(x, G, 2.0, prm, direction, y)
    assert np.sum(Px * y) == pytest.approx(np.sum(x * PTy), rel=1e-12)


def test_subsystem_dlambda_closed_form():
    """d u / d lambda = -A_s^{-1} L u for u = A_s^{-1} f, A_s = I + lambda L."""
    rng = np.random.default_rng(5)
    H, W, r = 6, 5, 1
    G = rng.uniform(0, 1, size=(H, W))
    prm = Params(r=r, sigma_r=0.3)
    rows, cols = neighbourhood_construction(COLUMN, 2, r, H, W)
    f = rng.uniform(0, 1, size=len(rows))
    lam = 0.7
    ab = subsystem_band(rows, cols, G, lam, prm)
    u = solve_subsystem(ab, f, r)
    L_ab = (subsystem_band(rows, cols, G, 1.0, prm) - subsystem_band(rows, cols, G, 0.0, prm))
    s = len(rows)
    L = np.zeros((s, s))
    for p in range(s):
        for q in range(max(0, p - r), min(s, p + r + 1)):
            L[p, q] = L_ab[r + p - q, q]
    du = -solve_subsystem(ab, L @ u, r)
    h = 1e-6
    fd = (solve_subsystem(subsystem_band(rows, cols, G, lam + h, prm), f, r)
          - solve_subsystem(subsystem_band(rows, cols, G, lam - h, prm), f, r)) / (2 * h)
    np.testing.assert_allclose(du, fd, atol=1e-8)
    # the oracle pass VJP reproduces <ubar, du/dlambda> for this one subsystem
    # (a single-centre image: W = 3 columns, r = 1)
    G3 = rng.uniform(0, 1, size=(H, 3))
    U3 = rng.uniform(0, 1, size=(1, H, 3))
    Vb = rng.normal(size=(1, H, 3))
    _, _, lb = sgwls_pass_vjp(U3, G3, lam, prm, COLUMN, Vb)
    rows, cols = neighbourhood_construction(COLUMN, 1, r, H, 3)
    ab = subsystem_band(rows, cols, G3, lam, prm)
    L_ab = subsystem_band(rows, cols, G3, 1.0, prm) - subsystem_band(rows, cols, G3, 0.0, prm)
    L = np.zeros((len(rows), len(rows)))
    for p in range(len(rows)):
        for q in range(max(0, p - r), min(len(rows), p + r + 1)):
            L[p, q] = L_ab[r + p - q, q]
    u = solve_subsystem(ab, U3[0, rows, cols], r)
    du = -solve_subsystem(ab, L @ u, r)
    assert lb == pytest.approx(float(np.sum(Vb[0, rows, cols] * du)), rel=1e-10)
