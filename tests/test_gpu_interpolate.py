"""GPU parity of guided sparse interpolation (Eq. 21) with the FP64 oracle.

U = N / D with N = SGWLS(F) and D = SGWLS(Hm): an FP32 error e in N and D
becomes at most e (1 + |U|) / D in U, so the bound is 2e-4 (1 + |U|) / D on
pixels with D >= 1e-3 (all pixels of these inputs but the far corners of
sparse scribbles), and U = 0 exactly where D = 0."""
import numpy as np
import pytest

import synth
from oracle import Params, sgwls_interpolate

pytestmark = pytest.mark.gpu

TOL = 2e-4


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01674_gb300 import build
    build.build()
    import paper_1705_01674_gb300 as m
    return m


def _check(api, F, Hm, G, lam, **kw):
    import torch
    u = api.sgwls_interpolate(torch.from_numpy(F).cuda(), torch.from_numpy(Hm).cuda(),
                              torch.from_numpy(G).cuda(), lam, **kw)
    torch.cuda.synchronize()
    prm = Params(r=kw["r"], iters=kw["iters"], step=kw.get("step", 1), sigma_s=float(kw["r"]), sigma_r=kw["sigma_r"])
    U, N, D = sgwls_interpolate(F.astype(np.float64), Hm.astype(np.float64), G.astype(np.float64), lam, prm,
                                return_parts=True)
    got = u.cpu().numpy().astype(np.float64).reshape(U.shape)
    ok = D >= 1e-3
    bound = TOL * (1.0 + np.abs(U)) / np.maximum(D, 1e-3)
    assert (np.abs(got - U)[:, ok] <= bound[:, ok]).all(), float((np.abs(got - U)[:, ok] / bound[:, ok]).max())
    assert (got[:, D == 0] == 0).all()
    assert np.isfinite(got).all()


@pytest.mark.parametrize("r", [1, 2, 4])
def test_guided_depth_upsampling(api, r):
    """4x upsampling pattern: depth on every 4th row and column, guidance =
    luminance of a scene (61 x 75, ragged bands and chunks)."""
    F, Hm, _ = synth.sparse_depth(61, 75, factor=4, seed=20 + r)
    G = synth.luminance(synth.rgb_scene(61, 75, seed=20 + r, n_rect=12, n_disk=3))
    _check(api, F, Hm, G, 4.0, r=r, iters=2, sigma_r=0.1)


@pytest.mark.parametrize("C", [1, 2, 3])
def test_colourisation_scribbles(api, C):
    """Random chrominance strokes in C channels (C + 1 right-hand sides of
    one factorisation), 57 x 83."""
    F, Hm = synth.scribbles(57, 83, n=14, C=C, seed=30 + C)
    G = synth.luminance(synth.rgb_scene(57, 83, seed=30 + C, n_rect=12, n_disk=3))
    _check(api, F, Hm, G, 20.0, r=2, iters=3, sigma_r=0.05)


def test_depth_upsampling_with_sliding_step(api):
    """The paper's depth-upsampling setting r = 4 with sliding step 4
    (Sec. 2.3), 4x grid, 73 x 90."""
    F, Hm, _ = synth.sparse_depth(73, 90, factor=4, seed=44)
    G = synth.luminance(synth.rgb_scene(73, 90, seed=44, n_rect=12, n_disk=3))
    _check(api, F, Hm, G, 4.0, r=4, step=4, iters=2, sigma_r=0.1)
