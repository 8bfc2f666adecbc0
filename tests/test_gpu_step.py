"""GPU parity of the sliding construction with step tau > 1 (Sec. 2.3):
centres r, r + tau, ... and the last centre D-1-r appended when the stride
misses it (so every line stays covered); each pixel averages the subsystems whose strips
cover it.  Against the FP64 oracle, same tolerance as step 1."""
import numpy as np
import pytest

import synth
from oracle import Params, sgwls

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


def _run(api, F, G, lam, **kw):
    import torch
    u = api.sgwls_filter(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(), lam, **kw)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64)


def _ref(F, G, lam, r, step, iters, axis_order=0, sigma_r=0.1):
    prm = Params(r=r, iters=iters, step=step, axis_order=axis_order, sigma_s=float(r), sigma_r=sigma_r)
    return sgwls(F.astype(np.float64), G.astype(np.float64), lam, prm)


CASES = sorted({(r, t) for r in (1, 2, 3, 4) for t in (2, r, r + 1, 2 * r + 1) if 2 <= t <= 2 * r + 1})


@pytest.mark.parametrize("r,step", CASES)
@pytest.mark.parametrize("C", [1, 3])
def test_step_small_ragged(api, r, step, C):
    """53 x 71 (and 71 x 53 for the other pass order): several bands, ragged
    last band, the appended last centre whenever the stride misses it."""
    F = synth.rgb_scene(53, 71, seed=40 + r + step, n_rect=15, n_disk=4)[:C]
    G = synth.luminance(synth.rgb_scene(53, 71, seed=40 + r + step, n_rect=15, n_disk=4))
    for axis_order in (0, 1):
        got = _run(api, F, G, 2.0, r=r, step=step, iters=2, axis_order=axis_order, sigma_r=0.1)
        err = float(np.abs(got.reshape(F.shape) - _ref(F, G, 2.0, r, step, 2, axis_order)).max())
        assert err <= TOL, (axis_order, err)


@pytest.mark.parametrize("chunk_lines", [1, 3, 0])
def test_step_chunkings(api, chunk_lines):
    """r = 4, tau = 4 (the paper's depth-upsampling setting) with 1- and
    3-line chunks and the automatic plan, 97 x 130."""
    F = synth.rgb_scene(97, 130, seed=77, n_rect=20, n_disk=5)
    G = synth.luminance(F)
    got = _run(api, F, G, 3.0, r=4, step=4, iters=1, chunk_lines=chunk_lines, sigma_r=0.1)
    err = float(np.abs(got - _ref(F, G, 3.0, 4, 4, 1)).max())
    assert err <= TOL, err


def test_step_pass_entry_and_bf16(api):
    """One pass through sgwls_filter_pass (both directions) and BF16 storage
    (bound: one BF16 rounding of the stored estimate per pass plus the FP32
    bound)."""
    import torch
    from oracle import sgwls_pass
    F = synth.rgb_scene(45, 66, seed=8, n_rect=10, n_disk=3)
    G = synth.luminance(F)
    prm = Params(r=2, iters=1, step=3, sigma_s=2.0, sigma_r=0.1)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(G).cuda()
    for d in (0, 1):
        u = api.sgwls_filter_pass(f, g, 1.5, d, r=2, step=3, sigma_r=0.1)
        torch.cuda.synchronize()
        ref = sgwls_pass(F.astype(np.float64), G.astype(np.float64), 1.5, prm, d)
        assert float(np.abs(u.cpu().numpy() - ref).max()) <= TOL
    fb = f.to(torch.bfloat16)
    gb = g.to(torch.bfloat16)
    u = api.sgwls_filter(fb, gb, 1.5, r=2, step=3, iters=1, sigma_r=0.1, inter_storage="f32")
    torch.cuda.synchronize()
    Fb = fb.float().cpu().numpy().astype(np.float64)
    Gb = gb.float().cpu().numpy().astype(np.float64)
    ref = sgwls(Fb, Gb, 1.5, prm)
    assert float(np.abs(u.float().cpu().numpy() - ref).max()) <= 2.0 ** -9 + TOL


def test_step_unsupported_paths(api):
    """The sliding step runs on kept factors only: recomputation, batched
    calls and the backward say so before any launch."""
    import torch
    F = synth.rgb_scene(30, 40, seed=3, n_rect=5, n_disk=1)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(synth.luminance(F)).cuda()
    with pytest.raises(api.SgwlsError) as e:
        api.sgwls_filter(f, g, 1.0, r=2, step=2, factor_cache=2)
    assert e.value.status == -7
    with pytest.raises(api.SgwlsError):
        api.sgwls_filter_batched([f], [g], [1.0], r=2, step=2)
