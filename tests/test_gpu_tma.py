"""Tensor-copy (TMA) staging of the column direction's tiles.

Column-direction passes over FP32 images whose rows start on 16-byte
boundaries stage their tiles with cp.async.bulk.tensor boxes completed on an
mbarrier; the same image at an address 4 bytes off that boundary takes the
asynchronous-copy staging instead.  The two fill the tile with the same
values, so the passes must agree bit for bit; both are checked against the
FP64 oracle.  Covered: factors kept (k_summary) and recomputed (k_summary +
k_recover, whose first block starts its tile left of the image), several
chunk lengths, RGB and five channels (two channel groups), the refinement's
three tile-staging kernels, and the whole filter."""
import numpy as np
import pytest

import synth
from oracle import COLUMN, Params, sgwls, sgwls_pass

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


def _aligned_and_not(torch, x):
    """x on the device twice: 256-byte aligned, and 4 bytes past a 16-byte
    boundary (a view one float into a larger buffer)."""
    a = torch.from_numpy(x).cuda()
    buf = torch.empty(x.size + 1, dtype=torch.float32, device="cuda")
    b = buf[1:].view(x.shape)
    b.copy_(a)
    assert a.data_ptr() % 16 == 0 and b.data_ptr() % 16 == 4
    return a, b


@pytest.mark.parametrize("r", [1, 2, 3, 5])
@pytest.mark.parametrize("kw", [dict(), dict(factor_cache=2), dict(chunk_lines=3), dict(chunk_lines=16)])
def test_tma_pass_equals_async_staging(api, r, kw):
    import torch
    C, H, W = 3, 90, 200   # W a multiple of 4: rows 16-byte aligned when the base is
    F = synth.rgb_scene(H, W, seed=500 + r, n_rect=20, n_disk=4)
    G = synth.luminance(F)
    fa, fb = _aligned_and_not(torch, F)
    ga, gb = _aligned_and_not(torch, G)
    ua = api.sgwls_filter_pass(fa, ga, 1.2, 0, r=r, sigma_r=0.1, **kw)
    ub = api.sgwls_filter_pass(fb, gb, 1.2, 0, r=r, sigma_r=0.1, **kw)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub), kw
    ref = sgwls_pass(F.astype(np.float64), G.astype(np.float64), 1.2, Params(r=r, sigma_s=float(r), sigma_r=0.1), COLUMN)
    assert float(np.abs(ua.cpu().numpy() - ref).max()) <= TOL
    assert api.device_flag() == 0


def test_tma_filter_five_channels_and_refinement(api):
    import torch
    rgb = synth.rgb_scene(64, 128, seed=520, n_rect=15, n_disk=3)
    F = np.concatenate([rgb, rgb[::-1]])[:5].copy()
    G = synth.luminance(rgb)
    fa, fb = _aligned_and_not(torch, F)
    ga, gb = _aligned_and_not(torch, G)
    kw = dict(r=2, iters=2, sigma_r=0.1)
    ua = api.sgwls_filter(fa, ga, 0.9, **kw)
    ub = api.sgwls_filter(fb, gb, 0.9, **kw)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)
    ref = sgwls(F.astype(np.float64), G.astype(np.float64), 0.9, Params(r=2, iters=2, sigma_s=2.0, sigma_r=0.1))
    assert float(np.abs(ua.cpu().numpy() - ref).max()) <= TOL
    kwr = dict(r=1, iters=1, refine=1, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)
    ra = api.sgwls_filter(fa[:3].contiguous(), ga, 40.0, **kwr)
    rb = api.sgwls_filter(fb[:3].contiguous(), gb, 40.0, **kwr) if fb[:3].data_ptr() % 16 else None
    torch.cuda.synchronize()
    if rb is not None:
        assert torch.equal(ra, rb)
    refr = sgwls(F[:3].astype(np.float64), G.astype(np.float64), 40.0,
                 Params(r=1, iters=1, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4))
    assert float(np.abs(ra.cpu().numpy() - refr).max()) <= TOL
    assert api.device_flag() == 0


@pytest.mark.parametrize("r,step", [(2, 2), (3, 2), (3, 3), (4, 4), (5, 3)])
def test_tma_sliding_step_tile(api, r, step):
    """The sliding step's wider band tile (31 step + 2r + 1 columns) staged
    by tensor copies equals the per-element staging bit for bit."""
    import torch
    from oracle import Params as P
    F = synth.rgb_scene(72, 260, seed=540 + r, n_rect=20, n_disk=4)
    G = synth.luminance(F)
    fa, fb = _aligned_and_not(torch, F)
    ga, gb = _aligned_and_not(torch, G)
    kw = dict(r=r, step=step, sigma_r=0.1)
    ua = api.sgwls_filter_pass(fa, ga, 1.1, 0, **kw)
    ub = api.sgwls_filter_pass(fb, gb, 1.1, 0, **kw)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)
    ref = sgwls_pass(F.astype(np.float64), G.astype(np.float64), 1.1, P(r=r, step=step, sigma_s=float(r), sigma_r=0.1),
                     COLUMN)
    assert float(np.abs(ua.cpu().numpy() - ref).max()) <= TOL
    assert api.device_flag() == 0
