"""GPU parity of a vector guidance (Eq. 2 with |G_i - G_j| the Euclidean norm
of the difference of the two pixels' guidance vectors: an RGB guidance
image, or 2 and 4 planes) against the FP64 oracle; same FP32 tolerance as
the single-plane guidance."""
import numpy as np
import pytest

import synth
from oracle import COLUMN, Params, sgwls, sgwls_interpolate

from sampled_pass import oracle_pass_offsets

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


def _gpu(api, F, G, lam, **kw):
    import torch
    u = api.sgwls_filter(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(), lam, **kw)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64).reshape(F.shape)


def _prm(**kw):
    kw = dict(kw)
    kw.setdefault("sigma_s", float(kw.get("r", 1)))
    return Params(**kw)


@pytest.mark.parametrize("r", [1, 2, 3, 5])
@pytest.mark.parametrize("C", [1, 3])
def test_rgb_guidance_small_ragged(api, r, C):
    """53 x 71 with its own RGB image as guidance (the joint filter of a
    colour image), both pass orders: ragged bands and chunks."""
    rgb = synth.rgb_scene(53, 71, seed=60 + r, n_rect=15, n_disk=4)
    F = rgb[:C].copy()
    for axis_order in (0, 1):
        kw = dict(r=r, iters=2, axis_order=axis_order, sigma_r=0.2)
        err = float(np.abs(_gpu(api, F, rgb, 2.0, **kw) - sgwls(F, rgb, 2.0, _prm(**kw))).max())
        assert err <= TOL, (axis_order, err)


@pytest.mark.parametrize("Cg", [2, 4])
def test_two_and_four_guidance_planes(api, Cg):
    rgb = synth.rgb_scene(47, 66, seed=70 + Cg, n_rect=12, n_disk=3)
    G = np.concatenate([rgb, synth.luminance(rgb)[None]])[:Cg].copy()
    F = rgb.copy()
    kw = dict(r=2, iters=1, sigma_r=0.2)
    err = float(np.abs(_gpu(api, F, G, 3.0, **kw) - sgwls(F, G, 3.0, _prm(**kw))).max())
    assert err <= TOL, err


def test_equal_planes_match_scaled_gray_on_gpu(api):
    """Three equal guidance planes give the filter of sqrt(3) times that
    plane (the norm's scaling), here through two different kernels."""
    rgb = synth.rgb_scene(40, 58, seed=81, n_rect=10, n_disk=2)
    g = synth.luminance(rgb)
    kw = dict(r=2, iters=1, sigma_r=0.2)
    a = _gpu(api, rgb, np.stack([g, g, g]), 2.0, **kw)
    b = _gpu(api, rgb, (np.sqrt(3.0) * g).astype(np.float32), 2.0, **kw)
    assert float(np.abs(a - b).max()) <= TOL


def test_frac_weights_rgb_guidance(api):
    """Fractional weights (alpha = 1.2, eps = 1e-4) with a small lambda."""
    rgb = synth.rgb_scene(37, 52, seed=84, n_rect=10, n_disk=2)
    for r in (1, 2):
        kw = dict(r=r, iters=1, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)
        err = float(np.abs(_gpu(api, rgb, rgb, 0.002, **kw) - sgwls(rgb, rgb, 0.002, _prm(**kw))).max())
        assert err <= TOL, (r, err)


@pytest.mark.parametrize("r,step", [(2, 2), (2, 5), (3, 3)])
def test_rgb_guidance_with_sliding_step(api, r, step):
    rgb = synth.rgb_scene(53, 71, seed=90 + r + step, n_rect=15, n_disk=4)
    kw = dict(r=r, step=step, iters=2, sigma_r=0.2)
    err = float(np.abs(_gpu(api, rgb, rgb, 2.0, **kw) - sgwls(rgb, rgb, 2.0, _prm(**kw))).max())
    assert err <= TOL, err


def test_rgb_guidance_chunkings(api):
    """One-line and three-line chunks and the automatic plan."""
    rgb = synth.rgb_scene(61, 45, seed=95, n_rect=12, n_disk=3)
    ref = sgwls(rgb, rgb, 4.0, _prm(r=1, iters=1, sigma_r=0.2))
    for chunk_lines in (1, 3, 0):
        got = _gpu(api, rgb, rgb, 4.0, r=1, iters=1, sigma_r=0.2, chunk_lines=chunk_lines)
        assert float(np.abs(got - ref).max()) <= TOL, chunk_lines


def test_rgb_guidance_bf16_storage(api):
    """BF16 input, guidance and output (FP32 arithmetic and intermediate
    estimate): against the oracle on the same BF16-rounded planes, one BF16
    rounding of the result (2^-9 for values in [0, 1]) plus the FP32 bound."""
    import torch
    rgb = synth.rgb_scene(45, 60, seed=97, n_rect=12, n_disk=3)
    f = torch.from_numpy(rgb).cuda().to(torch.bfloat16)
    u = api.sgwls_filter(f, f, 2.0, r=2, iters=1, sigma_r=0.2, inter_storage="f32")
    torch.cuda.synchronize()
    Fb = f.float().cpu().numpy().astype(np.float64)
    ref = sgwls(Fb, Fb, 2.0, _prm(r=2, iters=1, sigma_r=0.2))
    assert float(np.abs(u.float().cpu().numpy() - ref).max()) <= 2.0 ** -9 + TOL


def test_rgb_guidance_unsupported_paths(api):
    """A vector guidance runs on kept factors only; the refinement's FP64
    residual reads one plane: both say so before any launch."""
    import torch
    f = torch.from_numpy(synth.rgb_scene(30, 40, seed=3, n_rect=5, n_disk=1)).cuda()
    for kw in (dict(factor_cache=2), dict(refine=1)):
        with pytest.raises(api.SgwlsError) as e:
            api.sgwls_filter(f, f, 1.0, r=1, **kw)
        assert e.value.status == -7


def test_depth_upsampling_with_rgb_guidance(api):
    """Eq. 21 guided by the colour image (the paper's depth upsampling
    setting: depth samples on every 4th row and column)."""
    import torch
    F, Hm, _ = synth.sparse_depth(61, 75, factor=4, seed=33)
    rgb = synth.rgb_scene(61, 75, seed=33, n_rect=12, n_disk=3)
    u = api.sgwls_interpolate(torch.from_numpy(F).cuda(), torch.from_numpy(Hm).cuda(), torch.from_numpy(rgb).cuda(),
                              4.0, r=2, iters=2, sigma_r=0.2)
    torch.cuda.synchronize()
    U, N, D = sgwls_interpolate(F.astype(np.float64), Hm.astype(np.float64), rgb.astype(np.float64), 4.0,
                                _prm(r=2, iters=2, sigma_r=0.2), return_parts=True)
    got = u.cpu().numpy().astype(np.float64).reshape(U.shape)
    ok = D >= 1e-3
    bound = TOL * (1.0 + np.abs(U)) / np.maximum(D, 1e-3)
    assert (np.abs(got - U)[:, ok] <= bound[:, ok]).all()
    assert (got[:, D == 0] == 0).all()


@pytest.mark.parametrize("direction", [0, 1])
def test_rgb_guidance_fullsize_pass_sampled(api, direction):
    """The 1024 x 768 RGB workload with its own RGB guidance: one pass,
    sampled offsets against the oracle."""
    import torch
    F = synth.rgb_scene(768, 1024, seed=2)
    f = torch.from_numpy(F).cuda()
    u = api.sgwls_filter_pass(f, f, 1.0, direction, r=1, sigma_r=0.2)
    torch.cuda.synchronize()
    C, H, W = F.shape
    dim = W if direction == COLUMN else H
    offsets = [0, 1, 2, 31, 32, 33, dim // 2, dim - 3, dim - 2, dim - 1]
    ref = oracle_pass_offsets(F, F, 1.0, _prm(r=1, iters=1, sigma_r=0.2), direction, offsets)
    U = u.cpu().numpy().astype(np.float64)
    got = U[:, :, offsets].transpose(0, 2, 1) if direction == COLUMN else U[:, offsets, :]
    assert float(np.abs(got - ref).max()) <= TOL
