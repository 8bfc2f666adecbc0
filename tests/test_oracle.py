"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
paper's worked construction example, its structural statements (Sec. 2.1,
Sec. 2.2), the paper's own r-band LU (Eqs. 9-20) as an independent solver,
closed forms, invariants, and brute force on tiny inputs.
"""
import os

import numpy as np
import pytest

import synth
from oracle import (
    COLUMN,
    ROW,
    Params,
    centre_indices,
    coverage_counts,
    guidance_weight,
    neighbourhood_construction,
    sgwls,
    sgwls_pass,
    solve_subsystem,
    subsystem_band,
)
from oracle.rband_lu import solve_dense_rband
from oracle.wls2d import wls2d
from scipy.linalg import solve_banded

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _band_to_dense(ab, r):
    s = ab.shape[1]
    A = np.zeros((s, s))
    for p in range(s):
        for q in range(max(0, p - r), min(s, p + r + 1)):
            A[p, q] = ab[r + p - q, q]
    return A


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [int(v) for v in vals]
    return out


# ---------------------------------------------------------------- Sec. 2.1

def test_snake_matches_worked_example():
    gold = _read_golden("snake_3x3_r1.txt")
    num = np.arange(1, 10).reshape(3, 3)
    rows, cols = neighbourhood_construction(COLUMN, 1, 1, 3, 3)
    seq = list(num[rows, cols])
    assert seq == gold["column"]
    i5 = seq.index(5)
    assert sorted([seq[i5 - 1], seq[i5 + 1]]) == gold["neighbours_of_5_column"]
    rows, cols = neighbourhood_construction(ROW, 1, 1, 3, 3)
    seq = list(num[rows, cols])
    assert seq == gold["row"]
    i5 = seq.index(5)
    assert sorted([seq[i5 - 1], seq[i5 + 1]]) == gold["neighbours_of_5_row"]


@pytest.mark.parametrize("r", [1, 2, 3, 5])
@pytest.mark.parametrize("direction", [COLUMN, ROW])
def test_snake_neighbours_are_2d_neighbours(r, direction):
    """Sec. 2.1: any 2r+1 neighbouring entries of the formed vector are
    neighbours in the (2r+1) x (2r+1) system."""
    H, W = 9 + r, 8 + 2 * r
    dim = W if direction == COLUMN else H
    for k in centre_indices(dim, r):
        rows, cols = neighbourhood_construction(direction, k, r, H, W)
        s = len(rows)
        assert s == (2 * r + 1) * (H if direction == COLUMN else W)
        for t in range(1, r + 1):
            assert np.all(np.abs(rows[t:] - rows[:-t]) <= r)
            assert np.all(np.abs(cols[t:] - cols[:-t]) <= r)
        # a permutation of the (2r+1)-line strip
        flat = rows * W + cols
        assert len(np.unique(flat)) == s
        if direction == COLUMN:
            assert set(np.unique(cols)) == set(range(k - r, k + r + 1))
        else:
            assert set(np.unique(rows)) == set(range(k - r, k + r + 1))


def test_snake_structure_independent_build():
    """Independent construction from a strip array with numpy slicing."""
    r, H, W, k = 2, 6, 9, 4
    num = np.arange(H * W).reshape(H, W)
    strip = num[:, k - r:k + r + 1].copy()
    strip[1::2] = strip[1::2, ::-1]          # 1-based even rows reversed
    rows, cols = neighbourhood_construction(COLUMN, k, r, H, W)
    assert np.array_equal(num[rows, cols], strip.reshape(-1))
    k = 3
    strip = num[k - r:k + r + 1, :].T.copy()  # one segment per column
    strip[1::2] = strip[1::2, ::-1]
    rows, cols = neighbourhood_construction(ROW, k, r, H, W)
    assert np.array_equal(num[rows, cols], strip.reshape(-1))


def test_centres_and_coverage():
    assert centre_indices(10, 1) == list(range(1, 9))
    assert centre_indices(10, 2, step=2) == [2, 4, 6, 7]
    assert centre_indices(5, 2) == [2]
    with pytest.raises(ValueError):
        centre_indices(4, 2)
    prm = Params(r=2)
    cnt = coverage_counts(COLUMN, 3, 12, prm)
    # column c is covered by centres k in [max(r, c-r), min(W-1-r, c+r)]
    expect = [len([k for k in range(2, 10) if abs(k - c) <= 2]) for c in range(12)]
    assert np.array_equal(cnt[0], expect)
    assert expect[:3] == [1, 2, 3] and expect[5] == 5
    prm = Params(r=1, step=3)
    cnt = coverage_counts(ROW, 11, 4, prm)
    assert np.all(cnt >= 1)


# ------------------------------------------------------------------ Eq. 2

def test_weight_closed_forms():
    G = np.array([[0.3, 0.4], [0.3, 0.9]])
    prm = Params(weight="exp", sigma_s=1.0, sigma_r=0.1)
    # horizontal neighbours, |dG| = 0.1: exp(-1/2) exp(-0.01/0.02)
    w = guidance_weight(np.array([0]), np.array([0]), np.array([0]), np.array([1]), G, prm)[0]
    assert w == pytest.approx(np.exp(-0.5) * np.exp(-0.5), rel=1e-14)
    # vertical neighbours with equal guidance: spatial factor only
    w = guidance_weight(np.array([0]), np.array([0]), np.array([1]), np.array([0]), G, prm)[0]
    assert w == pytest.approx(np.exp(-0.5), rel=1e-14)
    # diagonal neighbours: |i-j|^2 = 2, |dG| = 0.6
    prm2 = Params(weight="exp", sigma_s=2.0, sigma_r=0.5)
    w = guidance_weight(np.array([0]), np.array([0]), np.array([1]), np.array([1]), G, prm2)[0]
    assert w == pytest.approx(np.exp(-2 / 8.0) * np.exp(-0.36 / 0.5), rel=1e-14)
    prmf = Params(weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)
    w = guidance_weight(np.array([0]), np.array([0]), np.array([1]), np.array([1]), G, prmf)[0]
    assert w == pytest.approx(1 / (2 ** 0.6 + 1e-4) / (0.6 ** 1.2 + 1e-4), rel=1e-14)
    # equal guidance: frac range factor is 1/eps (Eq. 2 with eps = 0.0001)
    w = guidance_weight(np.array([0]), np.array([0]), np.array([1]), np.array([0]), G, prmf)[0]
    assert w == pytest.approx(1 / (1 + 1e-4) / 1e-4, rel=1e-14)


# ----------------------------------------------------------- Eqs. 4 and 5

def _bruteforce_dense(rows, cols, G, lam, r, sigma_s, sigma_r):
    """Independent dense builder: every pair of entries at vector distance
    1..r, weight from the pixel coordinates."""
    s = len(rows)
    A = np.eye(s)
    for p in range(s):
        for q in range(s):
            if p != q and abs(p - q) <= r:
                d2 = float((rows[p] - rows[q]) ** 2 + (cols[p] - cols[q]) ** 2)
                dg = float(G[rows[p], cols[p]] - G[rows[q], cols[q]])
                w = np.exp(-d2 / (2 * sigma_s ** 2)) * np.exp(-dg * dg / (2 * sigma_r ** 2))
                A[p, q] = -lam * w
                A[p, p] += lam * w
    return A


@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("direction", [COLUMN, ROW])
def test_subsystem_matrix_bruteforce_and_structure(r, direction):
    rng = np.random.default_rng(10 + r)
    H, W = 2 * r + 3, 2 * r + 4
    G = rng.uniform(0, 1, size=(H, W))
    lam = 1.7
    prm = Params(r=r, sigma_s=float(r), sigma_r=0.3)
    k = r + 1
    rows, cols = neighbourhood_construction(direction, k, r, H, W)
    A = _band_to_dense(subsystem_band(rows, cols, G, lam, prm), r)
    B = _bruteforce_dense(rows, cols, G, lam, r, prm.sigma_s, prm.sigma_r)
    np.testing.assert_allclose(A, B, rtol=1e-13, atol=1e-15)
    # symmetric, unit row sums, strictly diagonally dominant with margin 1
    np.testing.assert_allclose(A, A.T, atol=0)
    np.testing.assert_allclose(A.sum(axis=1), 1.0, atol=1e-12)
    margin = np.diag(A) - (np.abs(A).sum(axis=1) - np.abs(np.diag(A)))
    np.testing.assert_allclose(margin, 1.0, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(A) > 0.999)


# --------------------------------------------------- Eqs. 6-20 and Eq. 5

@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_paper_rband_lu_solves_subsystem(r):
    """The paper's r-band LU (Eqs. 9-20) and the oracle's banded solve agree
    on subsystem matrices, and both reproduce a dense solve."""
    rng = np.random.default_rng(r)
    H, W = 2 * r + 2, 2 * r + 2
    G = rng.uniform(0, 1, size=(H, W))
    prm = Params(r=r, sigma_s=float(r), sigma_r=0.2)
    rows, cols = neighbourhood_construction(COLUMN, r, r, H, W)
    ab = subsystem_band(rows, cols, G, 3.0, prm)
    A = _band_to_dense(ab, r)
    f = rng.uniform(0, 1, size=len(rows))
    u_lapack = solve_subsystem(ab, f, r)
    u_paper = solve_dense_rband(A, f, r)
    u_dense = np.linalg.solve(A, f)
    np.testing.assert_allclose(u_paper, u_dense, rtol=0, atol=1e-12)
    np.testing.assert_allclose(u_lapack, u_dense, rtol=0, atol=1e-12)


@pytest.mark.parametrize("r", [1, 2, 4])
def test_paper_rband_lu_general_band(r):
    """Eqs. 9-20 on a random banded diagonally dominant (nonsymmetric) matrix."""
    rng = np.random.default_rng(100 + r)
    s = 6 * r + 5
    A = np.zeros((s, s))
    for p in range(s):
        for q in range(max(0, p - r), min(s, p + r + 1)):
            A[p, q] = rng.uniform(-1, 1)
        A[p, p] = 2 * r + 1 + rng.uniform(0, 1)
    f = rng.uniform(-1, 1, size=s)
    np.testing.assert_allclose(solve_dense_rband(A, f, r), np.linalg.solve(A, f), atol=1e-12)


def test_r1_is_textbook_thomas():
    """For r = 1 the subsystem is tridiagonal (Sec. 2.2); compare with the
    textbook Thomas algorithm."""
    rng = np.random.default_rng(7)
    H, W = 7, 5
    G = rng.uniform(0, 1, size=(H, W))
    prm = Params(r=1)
    rows, cols = neighbourhood_construction(COLUMN, 2, 1, H, W)
    ab = subsystem_band(rows, cols, G, 2.0, prm)
    a, b, c = ab[2, :-1].copy(), ab[1].copy(), ab[0, 1:].copy()  # sub, diag, super
    d = rng.uniform(0, 1, size=len(rows))
    n = len(d)
    cp, dp = np.zeros(n), np.zeros(n)
    cp[0], dp[0] = c[0] / b[0], d[0] / b[0]
    for i in range(1, n):
        den = b[i] - a[i - 1] * cp[i - 1]
        cp[i] = c[i] / den if i < n - 1 else 0.0
        dp[i] = (d[i] - a[i - 1] * dp[i - 1]) / den
    x = np.zeros(n)
    x[-1] = dp[-1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    np.testing.assert_allclose(solve_subsystem(ab, d, 1), x, atol=1e-13)


@pytest.mark.parametrize("r", [1, 3])
def test_subsystem_solution_invariants(r):
    rng = np.random.default_rng(20 + r)
    H, W = 12, 2 * r + 3
    G = rng.uniform(0, 1, size=(H, W))
    prm = Params(r=r, sigma_s=float(r), sigma_r=0.1)
    rows, cols = neighbourhood_construction(COLUMN, r + 1, r, H, W)
    f = rng.uniform(0, 1, size=len(rows))
    # lambda = 0: u = f
    u0 = solve_subsystem(subsystem_band(rows, cols, G, 0.0, prm), f, r)
    np.testing.assert_allclose(u0, f, atol=1e-15)
    ab = subsystem_band(rows, cols, G, 2.5, prm)
    u = solve_subsystem(ab, f, r)
    # sum preserved (A_s symmetric with A_s 1 = 1), bounded by min/max of f
    assert u.sum() == pytest.approx(f.sum(), rel=1e-12)
    assert u.min() >= f.min() - 1e-12 and u.max() <= f.max() + 1e-12
    # constant vector is a fixed point (L 1 = 0)
    np.testing.assert_allclose(solve_subsystem(ab, np.full(len(f), 0.37), r), 0.37, atol=1e-13)
    # lambda -> infinity: u -> mean(f), error O(1/lambda)
    Gc = np.full((H, W), 0.5)
    e = []
    for lam in (1e4, 1e5):
        uu = solve_subsystem(subsystem_band(rows, cols, Gc, lam, prm), f, r)
        e.append(np.abs(uu - f.mean()).max())
    assert e[1] < e[0] / 5 and e[1] < 0.05


# ------------------------------------------------- Sec. 2.3, whole passes

def _bruteforce_pass(U, G, lam, r, sigma_s, sigma_r, direction, centres=None):
    """Independent pass: explicit strip arrays, dense matrices, dense solve;
    `centres` (default: every r .. dim-1-r) lists the strips' centres."""
    C, H, W = U.shape
    acc = np.zeros_like(U)
    cnt = np.zeros((H, W))
    dim = W if direction == COLUMN else H
    for k in (range(r, dim - r) if centres is None else centres):
        if direction == COLUMN:
            rr, cc = np.mgrid[0:H, k - r:k + r + 1]
        else:
            cc, rr = np.mgrid[0:W, k - r:k + r + 1]
        rr, cc = rr.copy(), cc.copy()
        rr[1::2] = rr[1::2, ::-1]
        cc[1::2] = cc[1::2, ::-1]
        rows, cols = rr.reshape(-1), cc.reshape(-1)
        A = _bruteforce_dense(rows, cols, G, lam, r, sigma_s, sigma_r)
        u = np.linalg.solve(A, U[:, rows, cols].T)
        for p in range(len(rows)):
            acc[:, rows[p], cols[p]] += u[p]
            cnt[rows[p], cols[p]] += 1
    return acc / cnt


@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("direction", [COLUMN, ROW])
def test_pass_bruteforce_tiny(r, direction):
    rng = np.random.default_rng(30 + r)
    H, W = 2 * r + 4, 2 * r + 3
    U = rng.uniform(0, 1, size=(2, H, W))
    G = rng.uniform(0, 1, size=(H, W))
    prm = Params(r=r, sigma_s=float(r), sigma_r=0.25)
    got = sgwls_pass(U, G, 1.3, prm, direction)
    ref = _bruteforce_pass(U, G, 1.3, r, prm.sigma_s, prm.sigma_r, direction)
    np.testing.assert_allclose(got, ref, atol=1e-13)


@pytest.mark.parametrize("r,step,dim", [(1, 2, 8), (1, 3, 9), (2, 3, 12), (2, 5, 13)])
@pytest.mark.parametrize("direction", [COLUMN, ROW])
def test_sliding_step_pass_bruteforce(r, step, dim, direction):
    """Sec. 2.3 with a sliding step: the centres r, r + tau, ... (and the
    last centre dim-1-r when the stride misses it, so every line is
    covered); each pixel averages the strips that contain it.  Checked
    against the explicit brute-force pass on that centre list."""
    rng = np.random.default_rng(50 + 10 * r + step)
    H, W = (7, dim) if direction == COLUMN else (dim, 7)
    U = rng.uniform(0, 1, size=(2, H, W))
    G = rng.uniform(0, 1, size=(H, W))
    prm = Params(r=r, step=step, sigma_s=float(r), sigma_r=0.25)
    centres = list(range(r, dim - r, step))
    if centres[-1] != dim - 1 - r:
        centres.append(dim - 1 - r)
    assert centre_indices(dim, r, step) == centres
    got = sgwls_pass(U, G, 1.3, prm, direction)
    ref = _bruteforce_pass(U, G, 1.3, r, prm.sigma_s, prm.sigma_r, direction, centres)
    np.testing.assert_allclose(got, ref, atol=1e-13)
    # invariants survive the sparser centre set: constants, the range, lambda = 0
    np.testing.assert_allclose(sgwls_pass(np.full_like(U, 0.4), G, 1.3, prm, direction), 0.4, atol=1e-13)
    assert got.min() >= U.min() - 1e-12 and got.max() <= U.max() + 1e-12
    np.testing.assert_allclose(sgwls_pass(U, G, 0.0, prm, direction), U, atol=1e-14)


@pytest.mark.parametrize("r", [1, 2])
def test_row_pass_is_transposed_column_pass(r):
    rng = np.random.default_rng(40 + r)
    U = rng.uniform(0, 1, size=(3, 9, 13))
    G = rng.uniform(0, 1, size=(9, 13))
    prm = Params(r=r, sigma_s=float(r))
    a = sgwls_pass(U, G, 0.8, prm, ROW)
    b = sgwls_pass(U.transpose(0, 2, 1), G.T, 0.8, prm, COLUMN).transpose(0, 2, 1)
    np.testing.assert_allclose(a, b, atol=1e-14)


def test_filter_invariants_and_pass_order():
    F = synth.rgb_scene(20, 23, seed=3, n_rect=6, n_disk=2).astype(np.float64)
    G = synth.luminance(F.astype(np.float32)).astype(np.float64)
    prm = Params(r=1, iters=2)
    np.testing.assert_allclose(sgwls(F, G, 0.0, prm), F, atol=1e-15)
    const = np.full_like(F, 0.42)
    np.testing.assert_allclose(sgwls(const, G, 5.0, prm), 0.42, atol=1e-12)
    U = sgwls(F, G, 2.0, prm)
    for c in range(3):
        assert U[c].min() >= F[c].min() - 1e-12 and U[c].max() <= F[c].max() + 1e-12
    # axis_order 1 runs the row direction first
    p1 = Params(r=1, iters=1, axis_order=1)
    expect = sgwls_pass(sgwls_pass(F, G, 2.0, p1, ROW), G, 2.0, p1, COLUMN)
    np.testing.assert_allclose(sgwls(F, G, 2.0, p1), expect, atol=1e-15)
    # smoothing: total variation decreases
    tv = lambda X: np.abs(np.diff(X, axis=1)).sum() + np.abs(np.diff(X, axis=2)).sum()
    assert tv(U) < 0.8 * tv(F)


def test_close_to_full_wls_2d():
    """Sec. 2.1/2.3 claim SG-WLS approximates the 2D WLS model: on a 16x16
    image the SG-WLS result is much closer to the dense 2D solution than the
    input is (soft check; the paper gives no number)."""
    F = synth.rect_gray(16, 16, seed=1, n_rect=3)[0].astype(np.float64)
    rms = lambda X: float(np.sqrt(np.mean(X ** 2)))
    for r, lam, T in ((1, 2.0, 2), (2, 8.0, 3)):
        prm = Params(r=r, iters=T, sigma_s=float(r), sigma_r=0.2)
        ref = wls2d(F, F, lam, prm)[0]
        U = sgwls(F, F, lam, prm)[0]
        assert rms(U - ref) < 0.6 * rms(F - ref)


def test_sampled_pass_offsets_match_whole_pass():
    """The per-offset pass oracle used by the full-size GPU tests equals the
    whole-image pass at every offset of a small image, both directions."""
    from sampled_pass import oracle_pass_offsets
    F = synth.rgb_scene(23, 29, seed=12, n_rect=6, n_disk=2)
    G = synth.luminance(F)
    for r in (1, 2):
        prm = Params(r=r, iters=1, sigma_s=float(r), sigma_r=0.1)
        for d, dim in ((COLUMN, 29), (ROW, 23)):
            whole = sgwls_pass(F.astype(np.float64), G.astype(np.float64), 1.3, prm, d)
            offs = list(range(dim))
            got = oracle_pass_offsets(F, G, 1.3, prm, d, offs)
            ref = whole if d == ROW else whole.transpose(0, 2, 1)
            assert np.abs(got - ref).max() < 1e-12


# --------------------------------- the BF16 tolerance's premise (reading D14)

@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("weight", ["exp", "frac"])
def test_pass_is_max_norm_nonexpansive(r, weight):
    """A_s^-1 is entrywise non-negative with unit row sums (A_s is an
    M-matrix with A_s 1 = 1), so every subsystem solve and hence every pass
    (a convex average of solves) is non-expansive in the max norm: a
    rounding of the stored estimate by e moves the next pass's output by at
    most e.  The BF16 storage bound rests on this."""
    rng = np.random.default_rng(7 * r + (weight == "frac"))
    H, W = 9, 4 * r + 3
    G = rng.uniform(0, 1, size=(H, W))
    lam = 3.0 if weight == "exp" else 0.01
    prm = Params(r=r, sigma_s=float(r), sigma_r=0.1, weight=weight)
    rows, cols = neighbourhood_construction(COLUMN, r + 1, r, H, W)
    Ainv = np.linalg.inv(_band_to_dense(subsystem_band(rows, cols, G, lam, prm), r))
    assert Ainv.min() >= -1e-12
    np.testing.assert_allclose(Ainv.sum(axis=1), 1.0, atol=1e-10)
    for direction in (COLUMN, ROW):
        for _ in range(3):
            X = rng.uniform(0, 1, size=(2, H, W))
            Y = X + rng.uniform(-1e-3, 1e-3, size=X.shape)
            dx = np.abs(sgwls_pass(X, G, lam, prm, direction) - sgwls_pass(Y, G, lam, prm, direction)).max()
            assert dx <= np.abs(X - Y).max() * (1 + 1e-9)


@pytest.mark.parametrize("r", [1, 2])
def test_frac_settings_fp32_sensitivity_is_the_diagonal(r):
    """At the frac-weight application settings (Sec. 3: alpha = 1.2,
    eps = 1e-4, lambda = 900) lambda w reaches ~1e7.  Rounding only the
    off-diagonals -lambda w to FP32, with every row's diagonal-dominance
    margin kept at exactly 1 (Eq. 4: A = I + lambda L), moves the exact
    subsystem solution by less than 1e-7; rounding the diagonal
    1 + lambda sum w to FP32 as well moves it by more than 1e-4.  This is
    why the FP32 residual of the refinement applies A as u + lambda L u
    (the identity kept apart) instead of forming A's diagonal."""
    F = synth.rgb_scene(96, 64, seed=11, n_rect=20, n_disk=5)
    G = synth.luminance(F)
    prm = Params(r=r, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)
    lam = 900.0
    worst_off = worst_all = 0.0
    for k in range(r, 64 - r, 9):
        rows, cols = neighbourhood_construction(COLUMN, k, r, 96, 64)
        ab = subsystem_band(rows, cols, G, lam, prm)
        f = F[0, rows, cols]
        exact = solve_banded((r, r), ab, f)
        s = ab.shape[1]
        ab_off = np.zeros_like(ab)
        ab_off[r] = 1.0
        for t in range(1, r + 1):
            w = (-ab[r - t, t:]).astype(np.float32).astype(np.float64)   # lambda w(p, p+t), FP32-rounded
            ab_off[r - t, t:] = -w
            ab_off[r + t, :s - t] = -w
            ab_off[r, :s - t] += w
            ab_off[r, t:] += w
        worst_off = max(worst_off, float(np.abs(solve_banded((r, r), ab_off, f) - exact).max()))
        ab_all = ab.astype(np.float32).astype(np.float64)
        worst_all = max(worst_all, float(np.abs(solve_banded((r, r), ab_all, f) - exact).max()))
    assert worst_off < 1e-7, worst_off
    assert worst_all > 1e-4, worst_all


@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("weight", ["exp", "frac"])
def test_schur_complements_keep_margin_form(r, weight):
    """The fact the subtraction-free pivots rest on, checked in FP64 on the
    oracle's A_s (Eq. 4): eliminating any leading block I of A_s leaves a
    Schur complement S on the rest whose off-diagonals are <= 0 and whose
    rows sum to 1 plus the margin the eliminated entries pass on,
    1 + |A_RI| A_II^-1 1 (so >= 1); hence each diagonal entry of S equals
    its row's margin plus the magnitudes of its off-diagonals.  A sign error
    (a Laplacian with +lambda w off the diagonal) breaks all three."""
    F = synth.rgb_scene(24, 30, seed=21, n_rect=6, n_disk=2)
    G = synth.luminance(F)
    prm = Params(r=r, weight=weight, sigma_s=float(r), sigma_r=0.1, alpha_s=1.2, alpha_r=1.2, eps=1e-4)
    lam = 900.0 if weight == "frac" else 1.0
    rows, cols = neighbourhood_construction(COLUMN, 12, r, 24, 30)
    A = _band_to_dense(subsystem_band(rows, cols, G, lam, prm), r)
    s = A.shape[0]
    assert np.allclose(A.sum(axis=1), 1.0, rtol=0, atol=1e-9 * np.abs(A).max())
    for cut in (1, r, 2 * r + 1, s // 3, s // 2):
        I, Rr = slice(0, cut), slice(cut, s)
        Aii_inv = np.linalg.inv(A[I, I])
        S = A[Rr, Rr] - A[Rr, I] @ Aii_inv @ A[I, Rr]
        off = S - np.diag(np.diag(S))
        scale = np.abs(A).max()
        assert off.max() <= 1e-12 * scale
        margin = 1.0 + np.abs(A[Rr, I]) @ (Aii_inv @ np.ones(cut))
        assert np.all(margin >= 1.0 - 1e-12)
        assert np.allclose(S.sum(axis=1), margin, rtol=1e-9, atol=1e-9 * scale)
        assert np.allclose(np.diag(S), margin + np.abs(off).sum(axis=1), rtol=1e-12, atol=1e-9 * scale)
