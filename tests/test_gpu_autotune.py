"""The autotuner on the GPU: tuning a filter, a batched call and a
backward stores an entry in the cache file named by $SGWLS_TUNE_CACHE;
calls with autotune="cache" then run with the tuned knobs, and their
results still match the FP64 oracle (forward) or the untuned call
(batched, backward)."""
import numpy as np
import pytest

import synth
from oracle import Params, sgwls

pytestmark = pytest.mark.gpu

TOL = 2e-4


@pytest.fixture()
def api(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    monkeypatch.setenv("SGWLS_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.delenv("SGWLS_AUTOTUNE", raising=False)
    from paper_1705_01674_gb300 import build
    build.build()
    import paper_1705_01674_gb300 as m
    return m


def test_tuned_filter_parity(api):
    import torch
    F = synth.rgb_scene(200, 330, seed=41, n_rect=30, n_disk=6)
    G = synth.luminance(F)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(G).cuda()
    kw = dict(r=2, iters=2, sigma_r=0.1)
    entry = api.autotune_mod.tune_filter(f, g, 1.0, steps=2, warmup=1, **kw)
    assert entry["ms"] <= entry["default_ms"] and entry["trials"] > 5
    key = api.autotune_mod.filter_key(f, g, dict(kw, storage="f32"))
    assert api.autotune_mod.lookup(key) == entry["knobs"]
    u = api.sgwls_filter(f, g, 1.0, autotune="cache", **kw)
    torch.cuda.synchronize()
    ref = sgwls(F.astype(np.float64), G.astype(np.float64), 1.0, Params(r=2, iters=2, sigma_s=2.0, sigma_r=0.1))
    assert float(np.abs(u.cpu().numpy() - ref).max()) <= TOL
    # "search" on a new workload tunes once, then finds its entry
    n0 = len(api.autotune_mod.load_cache())
    api.sgwls_filter(f[:1].contiguous(), g, 1.0, autotune="search", **kw)
    assert len(api.autotune_mod.load_cache()) == n0 + 1
    assert api.device_flag() == 0


def test_tuned_batched_and_backward(api):
    import torch
    imgs = [synth.rect_gray(H, W, seed=50 + i) for i, (H, W) in enumerate([(90, 140), (160, 75), (64, 64)])]
    fs = [torch.from_numpy(x).cuda() for x in imgs]
    gs = [x[0] for x in fs]
    lams = [0.7, 1.5, 3.0]
    kw = dict(r=2, iters=2, sigma_r=0.1)
    ref = api.sgwls_filter_batched(fs, gs, lams, **kw)
    api.autotune_mod.tune_batched(fs, gs, lams, steps=2, warmup=1, **kw)
    got = api.sgwls_filter_batched(fs, gs, lams, autotune="cache", **kw)
    torch.cuda.synchronize()
    for a, b in zip(ref, got):
        assert float((a - b).abs().max()) <= TOL

    F = synth.rgb_scene(70, 90, seed=52, n_rect=10, n_disk=2)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(synth.luminance(F)).cuda()
    kwb = dict(r=1, iters=2, sigma_r=0.1)
    saved = torch.empty((4,) + tuple(f.shape), device="cuda")
    u = api.sgwls_filter(f, g, 1.0, saved=saved, **kwb)
    gu = (2.0 * (u - 0.5)).contiguous()
    gf0, gg0, gl0 = api.sgwls_filter_backward(gu, g, saved, 1.0, **kwb)
    api.autotune_mod.tune_backward(gu, g, saved, 1.0, steps=2, warmup=1, **kwb)
    gf1, gg1, gl1 = api.sgwls_filter_backward(gu, g, saved, 1.0, autotune="cache", **kwb)
    torch.cuda.synchronize()
    assert float((gf0 - gf1).abs().max()) <= 1e-4 * max(1.0, float(gf0.abs().max()))
    assert float((gg0 - gg1).abs().max()) <= 1e-3 * max(1.0, float(gg0.abs().max()))
