"""Pins of the oracle's vector guidance (a colour guidance image, Eq. 2 with
|G_i - G_j| the Euclidean norm of the difference of the guidance vectors).

Each pin fails for a plausible wrong norm: three equal channels must act as
one channel scaled by sqrt(3) (an L1 norm gives 3, a max norm 1); constant
extra channels must change nothing (a channel average would); and any
orthogonal mixing of the channels must leave the result unchanged, which
the Euclidean norm alone of the usual norms satisfies.
"""
import numpy as np
import pytest

import synth
from oracle import Params, guidance_weight, sgwls, sgwls_interpolate

PRMS = [Params(r=1, iters=1), Params(r=2, iters=1, sigma_s=2.0, sigma_r=0.2),
        Params(r=1, iters=1, weight="frac", alpha_r=1.2, eps=1e-4)]


def _scene(H, W, seed):
    rgb = synth.rgb_scene(H, W, seed=seed, n_rect=6, n_disk=2)
    return rgb.astype(np.float64)


@pytest.mark.parametrize("prm", PRMS)
def test_equal_channels_are_one_scaled_channel(prm):
    rgb = _scene(11, 13, 3)
    g = rgb[0]
    F = rgb[1:]
    got = sgwls(F, np.stack([g, g, g]), 2.0, prm)
    ref = sgwls(F, np.sqrt(3.0) * g, 2.0, prm)
    assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("prm", PRMS)
def test_constant_channels_change_nothing(prm):
    rgb = _scene(12, 9, 4)
    g = rgb[0]
    G = np.stack([np.full_like(g, 0.3), g, np.full_like(g, -2.0)])
    assert np.abs(sgwls(rgb, G, 3.0, prm) - sgwls(rgb, g, 3.0, prm)).max() < 1e-12
    # a one-plane vector guidance is the plain guidance
    assert np.abs(sgwls(rgb, g[None], 3.0, prm) - sgwls(rgb, g, 3.0, prm)).max() < 1e-12


@pytest.mark.parametrize("prm", PRMS)
def test_orthogonal_channel_mixing_is_invariant(prm):
    rgb = _scene(10, 14, 5)
    Q, _ = np.linalg.qr(np.random.default_rng(9).standard_normal((3, 3)))
    G2 = np.einsum("kc,chw->khw", Q, rgb)
    F = rgb[:2]
    a = sgwls(F, rgb, 1.5, prm)
    b = sgwls(F, G2, 1.5, prm)
    assert np.abs(a - b).max() < 1e-12
    # the mixing changes the channels themselves (the pin is not vacuous)
    assert np.abs(G2 - rgb).max() > 0.1


def test_pair_weight_of_a_vector_guidance():
    """Two neighbouring pixels whose guidance vectors differ by (0.03,
    0.04): |G_i - G_j| = 0.05 (the 3-4-5 triangle), in both weight forms."""
    G = np.zeros((2, 1, 2))
    G[0, 0, 1] = 0.03
    G[1, 0, 1] = 0.04          # |G_i - G_j| = 0.05
    r0, c0, r1, c1 = np.array([0]), np.array([0]), np.array([0]), np.array([1])
    prm = Params(r=1, sigma_s=1.0, sigma_r=0.1)
    w = guidance_weight(r0, c0, r1, c1, G, prm)[0]
    assert w == pytest.approx(np.exp(-0.5) * np.exp(-0.25 / 2.0), rel=1e-14)
    prm = Params(r=1, weight="frac", alpha_s=1.0, alpha_r=2.0, eps=1e-4)
    w = guidance_weight(r0, c0, r1, c1, G, prm)[0]
    assert w == pytest.approx(1.0 / (1.0 + 1e-4) / (0.0025 + 1e-4), rel=1e-12)


def test_interpolation_with_vector_guidance():
    """Eq. 21 with a colour guidance: a dense index map reproduces the
    filter; a constant input stays constant wherever data reaches."""
    rgb = _scene(12, 12, 6)
    prm = Params(r=1, iters=1)
    F = rgb[:1]
    Hm = np.ones((12, 12))
    assert np.abs(sgwls_interpolate(F, Hm, rgb, 2.0, prm) - sgwls(F, rgb, 2.0, prm)).max() < 1e-12
    Hm = (np.random.default_rng(2).random((12, 12)) < 0.2).astype(np.float64)
    U = sgwls_interpolate(0.7 * Hm[None], Hm, rgb, 2.0, prm)
    _, _, D = sgwls_interpolate(0.7 * Hm[None], Hm, rgb, 2.0, prm, return_parts=True)
    assert np.abs(U[0][D > 0] - 0.7).max() < 1e-12
