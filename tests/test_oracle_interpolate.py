"""Pins of the oracle's guided sparse interpolation (Sec. 2.3, Eq. 21):
U = SGWLS(F) / SGWLS(Hm).  Each pin follows from the linearity and
positivity of a pass (Eq. 4 systems are M-matrices with unit row sums,
averaging is convex) and is checked on data the oracle never saw."""
import numpy as np

import synth
from oracle import Params, sgwls, sgwls_interpolate

PRM = Params(r=2, iters=2, sigma_s=2.0, sigma_r=0.1)


def _guide(H, W, seed):
    return synth.luminance(synth.rgb_scene(H, W, seed=seed, n_rect=8, n_disk=2)).astype(np.float64)


def test_dense_index_map_reduces_to_the_filter():
    """Hm = 1 everywhere: SGWLS(1) = 1 (constants are preserved), so the
    interpolation is the plain filter."""
    G = _guide(21, 26, 3)
    F = synth.rgb_scene(21, 26, seed=4, n_rect=5, n_disk=1)[:2].astype(np.float64)
    U = sgwls_interpolate(F, np.ones((21, 26)), G, 1.7, PRM)
    assert np.abs(U - sgwls(F, G, 1.7, PRM)).max() < 1e-12


def test_constant_data_is_reproduced_everywhere_it_reaches():
    """F = c Hm: SGWLS(F) = c SGWLS(Hm) by linearity, so U = c wherever the
    data reaches (every pixel here)."""
    G = _guide(25, 31, 5)
    _, Hm, _ = synth.sparse_depth(25, 31, factor=4, seed=8)
    Hm = Hm.astype(np.float64)
    U, N, D = sgwls_interpolate(0.37 * Hm, Hm, G, 3.0, PRM, return_parts=True)
    assert (D > 0).all()
    assert np.abs(U - 0.37).max() < 1e-12


def test_interpolation_stays_inside_the_data_range():
    """Positivity of every pass: min(data) Hm <= F <= max(data) Hm implies
    min(data) <= U <= max(data) wherever D > 0."""
    G = _guide(24, 33, 9)
    F, Hm = synth.scribbles(24, 33, n=6, C=2, seed=10)
    F, Hm = F.astype(np.float64), Hm.astype(np.float64)
    U, N, D = sgwls_interpolate(F, Hm, G, 2.0, PRM, return_parts=True)
    for c in range(2):
        vals = F[c][Hm > 0]
        m = D > 1e-12
        assert U[c][m].min() >= vals.min() - 1e-9
        assert U[c][m].max() <= vals.max() + 1e-9


def test_no_data_gives_zero():
    """An empty index map reaches no pixel: U = 0 (the reading for 0 / 0)."""
    G = _guide(12, 14, 2)
    U = sgwls_interpolate(np.zeros((1, 12, 14)), np.zeros((12, 14)), G, 1.0, PRM)
    assert (U == 0).all()
