"""GPU parity of the batched entry point (many images of uneven sizes, one
launch per kernel per pass) against the FP64 oracle, and its equality with
single-image calls; CUDA-graph capture of a whole batched filter."""
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


def _batch(n, seed, lo, hi, C=1):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=(n, 2))
    lams = rng.uniform(0.5, 4.0, size=n)
    if C == 1:
        imgs = [synth.rect_gray(int(h), int(w), seed=1000 * seed + b) for b, (h, w) in enumerate(sizes)]
        guides = [im[0] for im in imgs]
    else:
        imgs = [synth.rgb_scene(int(h), int(w), seed=1000 * seed + b, n_rect=10, n_disk=2)
                for b, (h, w) in enumerate(sizes)]
        guides = [synth.luminance(im) for im in imgs]
    return imgs, guides, [float(x) for x in lams]


@pytest.mark.parametrize("factor_cache", [0, 2])
@pytest.mark.parametrize("r,C", [(2, 1), (1, 3), (3, 1)])
def test_batched_uneven_matches_oracle(api, r, C, factor_cache):
    """7 images, sides 2r+1 .. 90 (single-chunk images beside multi-group
    ones), chunk factors kept (automatic at these sizes) and recomputed."""
    import torch
    imgs, guides, lams = _batch(7, seed=40 + r, lo=2 * r + 1, hi=90, C=C)
    kw = dict(r=r, iters=2, sigma_r=0.1, factor_cache=factor_cache)
    fs = [torch.from_numpy(x).cuda() for x in imgs]
    gs = [torch.from_numpy(x).cuda() for x in guides]
    outs = api.sgwls_filter_batched(fs, gs, lams, **kw)
    torch.cuda.synchronize()
    prm = Params(r=r, iters=2, sigma_s=float(r), sigma_r=0.1)
    for x, g, lam, u in zip(imgs, guides, lams, outs):
        ref = sgwls(x.astype(np.float64), g.astype(np.float64), lam, prm)
        err = float(np.abs(u.cpu().numpy().astype(np.float64) - ref).max())
        assert err <= TOL, (x.shape, err)


def test_batched_equals_single_calls_many_images(api):
    """70 images (two launches per pass: 64 + 6) of sides 64..300."""
    import torch
    imgs, guides, lams = _batch(70, seed=4, lo=64, hi=300)
    kw = dict(r=2, iters=2, sigma_r=0.1)
    fs = [torch.from_numpy(x).cuda() for x in imgs]
    gs = [torch.from_numpy(x).cuda() for x in guides]
    outs = api.sgwls_filter_batched(fs, gs, lams, **kw)
    singles = [api.sgwls_filter(f, g, lam, **kw) for f, g, lam in zip(fs, gs, lams)]
    torch.cuda.synchronize()
    for u, v in zip(outs, singles):
        assert float((u - v).abs().max()) <= TOL


def test_batched_cuda_graph(api):
    """The whole batched filter (all passes) captured in a CUDA graph and
    replayed on new inputs."""
    import torch
    imgs, guides, lams = _batch(5, seed=11, lo=40, hi=200)
    kw = dict(r=2, iters=2, sigma_r=0.1)
    fs = [torch.from_numpy(x).cuda() for x in imgs]
    gs = [torch.from_numpy(x).cuda() for x in guides]
    outs = [torch.empty_like(f) for f in fs]
    nws = api.batched_workspace_bytes(fs, gs, lams, **kw)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.sgwls_filter_batched(fs, gs, lams, outs=outs, workspace=ws, stream=s, **kw)   # warm-up
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        api.sgwls_filter_batched(fs, gs, lams, outs=outs, workspace=ws, stream=s, **kw)
    new = [synth.rect_gray(x.shape[1], x.shape[2], seed=999 + i) for i, x in enumerate(imgs)]
    for f, g, x in zip(fs, gs, new):
        f.copy_(torch.from_numpy(x))
        g.copy_(torch.from_numpy(x[0]))
    graph.replay()
    torch.cuda.synchronize()
    prm = Params(r=2, iters=2, sigma_s=2.0, sigma_r=0.1)
    for x, lam, u in zip(new, lams, outs):
        ref = sgwls(x.astype(np.float64), x[0].astype(np.float64), lam, prm)
        assert float(np.abs(u.cpu().numpy().astype(np.float64) - ref).max()) <= TOL


@pytest.mark.parametrize("inter", ["f32", "bf16"])
def test_batched_bf16_storage(api, inter):
    """BF16 inputs, guidance and outputs (FP32 elimination) in one batched
    call: against the oracle on the same BF16-rounded planes, with one BF16
    rounding per stored estimate (2^-9 for values in [0, 1]) per pass that
    stores BF16, plus the FP32 bound."""
    import torch
    imgs, guides, lams = _batch(5, seed=61, lo=20, hi=80, C=3)
    kw = dict(r=1, iters=2, sigma_r=0.1, inter_storage=inter)
    fs = [torch.from_numpy(x).cuda().to(torch.bfloat16) for x in imgs]
    gs = [torch.from_numpy(x).cuda().to(torch.bfloat16) for x in guides]
    outs = api.sgwls_filter_batched(fs, gs, lams, **kw)
    torch.cuda.synchronize()
    stores = 1 if inter == "f32" else 4
    prm = Params(r=1, iters=2, sigma_s=1.0, sigma_r=0.1)
    for f, g, lam, u in zip(fs, gs, lams, outs):
        ref = sgwls(f.float().cpu().numpy().astype(np.float64), g.float().cpu().numpy().astype(np.float64), lam, prm)
        err = float(np.abs(u.float().cpu().numpy().astype(np.float64) - ref).max())
        assert err <= stores * 2.0 ** -9 + TOL, (tuple(f.shape), err)


def test_batched_full_uneven_workload(api):
    """The full uneven workload (64 gray images, sides U[256, 2048], r = 2,
    T = 2, lambda U[0.5, 4], guidance = input): the batched call equals the
    single-image calls for every image, and the two smallest images match
    the FP64 oracle over every pixel."""
    import torch
    imgs, lams = synth.batch_uneven_gray(n=64, seed=4)
    kw = dict(r=2, iters=2, sigma_r=0.1)
    fs = [torch.from_numpy(x).cuda() for x in imgs]
    gs = [f[0] for f in fs]
    outs = api.sgwls_filter_batched(fs, gs, lams, **kw)
    torch.cuda.synchronize()
    for f, g, lam, u in zip(fs, gs, lams, outs):
        v = api.sgwls_filter(f, g, lam, **kw)
        torch.cuda.synchronize()
        assert float((u - v).abs().max()) <= TOL, tuple(f.shape)
    prm = Params(r=2, iters=2, sigma_s=2.0, sigma_r=0.1)
    for b in sorted(range(len(imgs)), key=lambda i: imgs[i].size)[:2]:
        x = imgs[b].astype(np.float64)
        ref = sgwls(x, x[0], lams[b], prm)
        assert float(np.abs(outs[b].cpu().numpy().astype(np.float64) - ref).max()) <= TOL, x.shape


@pytest.mark.parametrize("r", [1, 2])
def test_batched_mixed_channel_counts(api, r):
    """Images of 1, 3, 5 and 6 channels (channel groups of 1, 3, 4 + 1 and
    4 + 2) of uneven sizes in one call: every image against the oracle, and
    the launch count: one uniform batch per channel-group size present
    (sizes 1, 2, 3, 4), each two launches per pass."""
    import torch
    rng = np.random.default_rng(70 + r)
    imgs, guides, lams = [], [], []
    for b, C in enumerate([1, 3, 5, 6, 3, 1]):
        H, W = (int(x) for x in rng.integers(2 * r + 5, 80, size=2))
        rgb = synth.rgb_scene(H, W, seed=700 + b, n_rect=8, n_disk=2)
        x = np.concatenate([rgb, rgb[::-1], rgb])[:C].copy()
        imgs.append(x)
        guides.append(synth.luminance(rgb))
        lams.append(float(rng.uniform(0.5, 3.0)))
    fs = [torch.from_numpy(x).cuda() for x in imgs]
    gs = [torch.from_numpy(x).cuda() for x in guides]
    kw = dict(r=r, iters=2, sigma_r=0.1)
    n0 = api.launch_count()
    outs = api.sgwls_filter_batched(fs, gs, lams, **kw)
    torch.cuda.synchronize()
    n1 = api.launch_count()
    assert n1 - n0 <= 4 * 2 * 2 * 2   # 4 group sizes x 4 passes x at most 2 kernels
    prm = Params(r=r, iters=2, sigma_s=float(r), sigma_r=0.1)
    for x, g, lam, u in zip(imgs, guides, lams, outs):
        ref = sgwls(x.astype(np.float64), g.astype(np.float64), lam, prm)
        err = float(np.abs(u.cpu().numpy().astype(np.float64) - ref).max())
        assert err <= TOL, (x.shape, err)
