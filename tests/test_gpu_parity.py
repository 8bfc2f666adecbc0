"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: max |GPU - oracle| <= 2e-4 on [0, 1]-valued FP32 images for
r <= 3 and T <= 3 (the stated target).  The same bound is applied to r = 4, 5
(all elimination is FP32 on strictly diagonally dominant systems, so the
error does not grow with r beyond FP32 rounding).  BF16 storage bounds
follow from each pass being a convex averaging of exact solves
(non-expansive in the max norm): each BF16 store adds at most 2^-9 for
values in [0, 1].
"""
import numpy as np
import pytest

import synth
from oracle import COLUMN, ROW, Params, sgwls, sgwls_pass

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
    dev = torch.device("cuda:0")
    f = torch.from_numpy(np.ascontiguousarray(F)).to(dev)
    g = torch.from_numpy(np.ascontiguousarray(G)).to(dev)
    u = api.sgwls_filter(f, g, lam, **kw)
    torch.cuda.synchronize()
    return u.float().cpu().numpy().astype(np.float64)


def _oracle(F, G, lam, r=1, iters=1, axis_order=0, weight="exp", sigma_s=None, sigma_r=0.1,
            alpha_s=1.2, alpha_r=1.2, eps=1e-4, **_):
    prm = Params(r=r, iters=iters, axis_order=axis_order, weight=weight,
                 sigma_s=float(r if sigma_s is None else sigma_s), sigma_r=sigma_r,
                 alpha_s=alpha_s, alpha_r=alpha_r, eps=eps)
    return sgwls(F.astype(np.float64), G.astype(np.float64), lam, prm)


def _maxerr(a, b):
    return float(np.abs(a.reshape(b.shape) - b).max())


def test_config_gray64(api):
    """64x64 grayscale, 8 rectangles + noise, guidance = input, r = 1, T = 1,
    lambda = 1, range parameter 0.1."""
    F = synth.rect_gray(64, 64, seed=0)
    kw = dict(r=1, iters=1, sigma_r=0.1)
    err = _maxerr(_gpu(api, F, F[0], 1.0, **kw), _oracle(F, F[0], 1.0, **kw))
    assert err <= TOL, err


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("C", [1, 3])
@pytest.mark.parametrize("axis_order", [0, 1])
@pytest.mark.parametrize("chunk_lines", [0, 1, 3, 1000])
def test_parity_small_ragged(api, r, C, axis_order, chunk_lines):
    """53 x 71 images: several warp bands with a ragged last band, several
    chunks with a ragged last chunk (or one chunk), both pass orders."""
    F = synth.rgb_scene(53, 71, seed=10 + r, n_rect=15, n_disk=4)[:C]
    G = synth.luminance(synth.rgb_scene(53, 71, seed=10 + r, n_rect=15, n_disk=4))
    kw = dict(r=r, iters=2, axis_order=axis_order, sigma_r=0.1)
    got = _gpu(api, F, G, 2.0, chunk_lines=chunk_lines, **kw)
    err = _maxerr(got, _oracle(F, G, 2.0, **kw))
    assert err <= TOL, err


@pytest.mark.parametrize("r", [1, 2, 3, 5])
@pytest.mark.parametrize("C", [1, 3, 4])
@pytest.mark.parametrize("factor_cache", [1, 2])
def test_parity_factor_cache_modes(api, r, C, factor_cache):
    """Both sources of the chunk factors in the second kernel of a pass:
    kept by the first kernel (1) or recomputed from the staged tile (2),
    with 1- and 3-line chunks (many chunks, ragged last chunk and group)."""
    F = synth.rgb_scene(61, 75, seed=30 + r, n_rect=15, n_disk=4)
    F = np.concatenate([F, F[:1]])[:C]
    G = synth.luminance(synth.rgb_scene(61, 75, seed=30 + r, n_rect=15, n_disk=4))
    kw = dict(r=r, iters=2, sigma_r=0.1)
    ref = _oracle(F, G, 1.5, **kw)
    for chunk_lines in (1, 3):
        got = _gpu(api, F, G, 1.5, chunk_lines=chunk_lines, factor_cache=factor_cache, **kw)
        err = _maxerr(got, ref)
        assert err <= TOL, (chunk_lines, err)


@pytest.mark.parametrize("chunk_lines", [1, 2, 5])
def test_parity_long_reduced_chain(api, chunk_lines):
    """A tall strip cut into many chunks: 900 x 40 with 1-, 2- and 5-line
    chunks gives 113, 57 and 23 chunk groups per column subsystem (the
    band's reduced chain in global memory, and split into segments in
    shared memory)."""
    F = synth.rgb_scene(900, 40, seed=77, n_rect=30, n_disk=5)
    G = synth.luminance(F)
    for r in (1, 2):
        kw = dict(r=r, iters=1, sigma_r=0.1)
        err = _maxerr(_gpu(api, F, G, 3.0, chunk_lines=chunk_lines, **kw), _oracle(F, G, 3.0, **kw))
        assert err <= TOL, (r, err)


@pytest.mark.parametrize("shape", [(3, 3), (3, 40), (40, 3), (5, 130), (130, 5), (33, 31)])
def test_edge_shapes(api, shape):
    """Minimum sizes (a single centre), very thin images, sizes one past a
    warp band."""
    H, W = shape
    r = 1 if min(H, W) < 5 else 2
    rng = np.random.default_rng(H * 1000 + W)
    F = rng.uniform(0, 1, size=(2, H, W)).astype(np.float32)
    G = rng.uniform(0, 1, size=(H, W)).astype(np.float32)
    kw = dict(r=r, iters=2, sigma_r=0.3)
    assert _maxerr(_gpu(api, F, G, 1.5, **kw), _oracle(F, G, 1.5, **kw)) <= TOL


def test_many_channels_and_alias(api):
    """C = 6 (channel groups of 4 + 2 against one guidance), and C = 1 with
    the guidance tensor being the input tensor itself."""
    import torch
    F = np.concatenate([synth.rgb_scene(40, 45, seed=s, n_rect=8, n_disk=2) for s in (1, 2)])
    G = synth.luminance(F[:3])
    kw = dict(r=2, iters=1, sigma_r=0.1)
    assert _maxerr(_gpu(api, F, G, 1.0, **kw), _oracle(F, G, 1.0, **kw)) <= TOL
    f = torch.from_numpy(F[1]).cuda()
    u = api.sgwls_filter(f, f, 1.0, **kw)
    torch.cuda.synchronize()
    assert _maxerr(u.cpu().numpy().astype(np.float64), _oracle(F[1:2], F[1], 1.0, **kw)) <= TOL


def test_frac_weights(api):
    """Eq. 2 fractional weights (alpha_s = alpha_r = 1.2, eps = 1e-4) with a
    small lambda (the 1/eps range factor makes lambda * w large)."""
    F = synth.rgb_scene(37, 52, seed=4, n_rect=10, n_disk=2)
    G = synth.luminance(F)
    for r in (1, 2):
        kw = dict(r=r, iters=1, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)
        err = _maxerr(_gpu(api, F, G, 0.002, **kw), _oracle(F, G, 0.002, **kw))
        assert err <= TOL, (r, err)


def test_single_pass_entry(api):
    import torch
    F = synth.rgb_scene(29, 47, seed=6, n_rect=6, n_disk=2)
    G = synth.luminance(F)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(G).cuda()
    for direction, d in ((0, COLUMN), (1, ROW)):
        u = api.sgwls_filter_pass(f, g, 3.0, direction, r=2, sigma_r=0.2)
        torch.cuda.synchronize()
        ref = sgwls_pass(F.astype(np.float64), G.astype(np.float64), 3.0, Params(r=2, sigma_s=2.0, sigma_r=0.2), d)
        assert _maxerr(u.cpu().numpy().astype(np.float64), ref) <= TOL


def test_saved_checkpoints_and_iters0(api):
    import torch
    F = synth.rgb_scene(31, 36, seed=8, n_rect=6, n_disk=2)
    G = synth.luminance(F)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(G).cuda()
    T = 2
    saved = torch.empty((2 * T,) + tuple(f.shape), device="cuda")
    u = api.sgwls_filter(f, g, 1.0, r=1, iters=T, saved=saved)
    torch.cuda.synchronize()
    _, inputs = sgwls(F, G, 1.0, Params(r=1, iters=T), return_inputs=True)
    for t in range(2 * T):
        assert _maxerr(saved[t].cpu().numpy().astype(np.float64), inputs[t]) <= TOL
    u0 = api.sgwls_filter(f, g, 1.0, r=1, iters=0)
    torch.cuda.synchronize()
    assert torch.equal(u0, f)


@pytest.mark.parametrize("inter", ["f32", "bf16"])
def test_bf16_storage(api, inter):
    """BF16 input/guidance/output (FP32 elimination).  The oracle filters the
    same BF16-rounded inputs; bound: one BF16 rounding of the output per
    store (2^-9 on [0, 1]) per BF16 store, plus the FP32 tolerance."""
    import torch
    F = synth.rgb_scene(64, 80, seed=9, n_rect=12, n_disk=3)
    G = synth.luminance(F)
    fb = torch.from_numpy(F).to(torch.bfloat16)
    gb = torch.from_numpy(G).to(torch.bfloat16)
    T = 2
    u = api.sgwls_filter(fb.cuda(), gb.cuda(), 1.0, r=2, iters=T, inter_storage=inter)
    torch.cuda.synchronize()
    ref = _oracle(fb.float().numpy(), gb.float().numpy(), 1.0, r=2, iters=T)
    stores = 1 if inter == "f32" else 2 * T
    bound = stores * 2.0 ** -9 + TOL
    err = _maxerr(u.float().cpu().numpy().astype(np.float64), ref)
    assert err <= bound, (err, bound)


_FULL_REF = {}


@pytest.mark.parametrize("factor_cache", [0, 2])
@pytest.mark.parametrize("lam", [0.5, 2.0])
def test_config_rgb_1024x768_full(api, lam, factor_cache):
    """Full size: 1024 x 768 RGB scene (200 rectangles, 50 disks, texture,
    noise), guidance = luminance, r = 1, T = 3, range parameter 0.1; every
    output pixel compared with the FP64 oracle, with the chunk factors kept
    between the kernels (the automatic choice at this size) and recomputed."""
    F = synth.rgb_scene(768, 1024, seed=2)
    G = synth.luminance(F)
    kw = dict(r=1, iters=3, sigma_r=0.1)
    if lam not in _FULL_REF:
        _FULL_REF[lam] = _oracle(F, G, lam, **kw)
    err = _maxerr(_gpu(api, F, G, lam, factor_cache=factor_cache, **kw), _FULL_REF[lam])
    assert err <= TOL, err


def test_binding_rejects_mis_sized_buffers(api):
    """The binding checks every buffer the library writes or reads by size
    before the call: an output of the wrong shape or dtype, a checkpoint
    buffer that is too small, a vector guidance for the backward."""
    import torch
    f = torch.from_numpy(synth.rgb_scene(20, 24, seed=1, n_rect=3, n_disk=1)).cuda()
    g = f[0].contiguous()
    with pytest.raises(ValueError):
        api.sgwls_filter(f, g, 1.0, out=torch.empty((3, 20, 23), device="cuda"))
    with pytest.raises(ValueError):
        api.sgwls_filter(f, g, 1.0, out=torch.empty((3, 20, 24), device="cuda", dtype=torch.bfloat16))
    with pytest.raises(ValueError):
        api.sgwls_filter_pass(f, g, 1.0, 0, out=torch.empty((2, 20, 24), device="cuda"))
    with pytest.raises(ValueError):
        api.sgwls_filter(f, g, 1.0, iters=2, saved=torch.empty((3, 3, 20, 24), device="cuda"))
    saved = torch.empty((2, 3, 20, 24), device="cuda")
    api.sgwls_filter(f, g, 1.0, iters=1, saved=saved)
    with pytest.raises(ValueError):
        api.sgwls_filter_backward(torch.ones_like(f), f, saved, 1.0, iters=1)
    with pytest.raises(ValueError):
        api.sgwls_filter_backward(torch.ones_like(f), g, saved[:1], 1.0, iters=1)
    with pytest.raises(ValueError):
        api.sgwls_filter_batched([f], [g], [1.0], outs=[torch.empty((3, 20, 20), device="cuda")])
