"""The paper's frac-weight application settings (Sec. 3: detail enhancement
r = 1, alpha_s = alpha_r = 1.2, lambda = 900; HDR tone mapping lambda = 5 /
40 / 320; eps = 1e-4).  There lambda * w reaches ~1e7 (the range factor is
1 / eps on flat guidance), so a diagonal formed as 1 + lambda sum w in FP32
loses the identity's 1: rounding A_s's entries to FP32 alone moves the exact
FP64 solution by up to ~5e-3 (measured below by the oracle itself).  The
kernels form every pivot as a margin plus coupling magnitudes (no
subtraction), which keeps the represented matrix's unit row sums, so the
plain FP32 filter -- kept factors, recomputed factors, a single chunk, both
pass orders -- stays within 2e-4 of the FP64 oracle without refinement."""
import importlib

import numpy as np
import pytest

import synth
from oracle import Params, sgwls

pytestmark = pytest.mark.gpu

osg = importlib.import_module("oracle.sgwls")

TOL = 2e-4
FRAC = dict(weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01674_gb300 import build
    build.build()
    import paper_1705_01674_gb300 as m
    return m


def _run(api, F, G, lam, **kw):
    import torch
    u = api.sgwls_filter(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(), lam, **kw)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64).reshape(F.shape)


@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("lam", [5.0, 40.0, 320.0, 900.0])
def test_frac_application_settings(api, lam, r, monkeypatch):
    F = synth.rgb_scene(64, 80, seed=11, n_rect=20, n_disk=5)
    G = synth.luminance(F)
    prm = Params(r=r, iters=2, **FRAC)
    ref = sgwls(F.astype(np.float64), G.astype(np.float64), lam, prm)
    # the oracle with A_s rounded to FP32: how much the naive FP32 matrix moves
    band = osg.subsystem_band
    monkeypatch.setattr(osg, "subsystem_band",
                        lambda *a, **k: band(*a, **k).astype(np.float32).astype(np.float64))
    ref32 = sgwls(F.astype(np.float64), G.astype(np.float64), lam, prm)
    monkeypatch.undo()
    sens = float(np.abs(ref32 - ref).max())
    err = float(np.abs(_run(api, F, G, lam, r=r, iters=2, **FRAC) - ref).max())
    assert err <= TOL, (err, sens)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_frac_settings_every_solve_path(api, r):
    """lambda = 900: factors kept (two chunk kernels), recomputed
    (factor_cache = 2), one chunk per subsystem (the recompute kernel alone),
    short chunks (long reduced chains), both pass orders."""
    F = synth.rgb_scene(41, 57, seed=12, n_rect=12, n_disk=4)
    G = synth.luminance(F)
    lam = 900.0
    for axis_order in (0, 1):
        ref = sgwls(F.astype(np.float64), G.astype(np.float64), lam,
                    Params(r=r, iters=1, axis_order=axis_order, **FRAC))
        for extra in (dict(), dict(factor_cache=2), dict(chunk_lines=64), dict(chunk_lines=1),
                      dict(chunk_lines=2, factor_cache=2)):
            u = _run(api, F, G, lam, r=r, iters=1, axis_order=axis_order, **FRAC, **extra)
            err = float(np.abs(u - ref).max())
            assert err <= TOL, (axis_order, extra, err)


def test_frac_settings_batched(api):
    """The batched filter at lambda = 320 and 900 (one launch per kernel per
    pass over images of different sizes)."""
    import torch
    imgs = [synth.rgb_scene(h, w, seed=20 + h, n_rect=10, n_disk=3) for h, w in ((37, 52), (61, 44), (48, 48))]
    lams = [320.0, 900.0, 900.0]
    fs = [torch.from_numpy(x).cuda() for x in imgs]
    gs = [torch.from_numpy(synth.luminance(x)).cuda() for x in imgs]
    us = api.sgwls_filter_batched(fs, gs, lams, r=1, iters=2, **FRAC)
    torch.cuda.synchronize()
    for x, lam, u in zip(imgs, lams, us):
        ref = sgwls(x.astype(np.float64), synth.luminance(x).astype(np.float64), lam, Params(r=1, iters=2, **FRAC))
        err = float(np.abs(u.cpu().numpy().astype(np.float64) - ref).max())
        assert err <= TOL, (x.shape, lam, err)
