"""GPU parity of the backward (adjoint) against the FP64 oracle.

The oracle's adjoint is pinned by FP64 central differences on the CPU
(tests/test_oracle_adjoint.py).  Here the GPU gradients with respect to f,
g and lambda must match it to 1e-3 relative (max error over the max
magnitude of the reference), and FP64 central differences of the oracle's
forward map directly on a 32x32 crop.
"""
import numpy as np
import pytest

import synth
from oracle import Params, sgwls
from oracle.adjoint import sgwls_vjp

pytestmark = pytest.mark.gpu

REL = 1e-3


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01674_gb300 import build
    build.build()
    import paper_1705_01674_gb300 as m
    return m


def _prm(r=1, iters=1, axis_order=0, weight="exp", sigma_r=0.1, alpha_s=1.2, alpha_r=1.2, eps=1e-4, **_):
    return Params(r=r, iters=iters, axis_order=axis_order, weight=weight, sigma_s=float(r), sigma_r=sigma_r,
                  alpha_s=alpha_s, alpha_r=alpha_r, eps=eps)


def _gpu_grads(api, F, G, lam, Ubar, **kw):
    import torch
    f = torch.from_numpy(np.ascontiguousarray(F, dtype=np.float32)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(G, dtype=np.float32)).cuda()
    T = kw.get("iters", 1)
    saved = torch.empty((2 * T,) + tuple(f.shape), device="cuda")
    api.sgwls_filter(f, g, lam, saved=saved, **kw)
    gu = torch.from_numpy(np.ascontiguousarray(Ubar, dtype=np.float32)).cuda()
    gf, gg, gl = api.sgwls_filter_backward(gu, g, saved, lam, **kw)
    torch.cuda.synchronize()
    return gf.cpu().numpy().astype(np.float64), gg.cpu().numpy().astype(np.float64), float(gl.item())


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-30))


@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("C", [1, 3])
@pytest.mark.parametrize("axis_order", [0, 1])
@pytest.mark.parametrize("chunk_lines", [0, 1, 3])
@pytest.mark.parametrize("factor_cache", [0, 2])
def test_backward_matches_oracle_adjoint(api, r, C, axis_order, chunk_lines, factor_cache):
    """factor_cache 0: the adjoint passes keep their chunk factors (k_summary,
    then k_backsub's adjoint mode); 2: k_recover recomputes them."""
    rng = np.random.default_rng(100 * r + 10 * C + axis_order)
    F3 = synth.rgb_scene(37, 45, seed=50 + r, n_rect=10, n_disk=2)
    F = F3[:C].astype(np.float32)
    G = synth.luminance(F3)
    Ubar = rng.normal(size=F.shape).astype(np.float32)
    kw = dict(r=r, iters=2, axis_order=axis_order, sigma_r=0.2)
    gf, gg, gl = _gpu_grads(api, F, G, 1.5, Ubar, chunk_lines=chunk_lines, factor_cache=factor_cache, **kw)
    rf, rg, rl = sgwls_vjp(F.astype(np.float64), G.astype(np.float64), 1.5, _prm(**kw), Ubar.astype(np.float64))
    assert _rel(gf, rf) <= REL, ("f", _rel(gf, rf))
    assert _rel(gg, rg) <= REL, ("g", _rel(gg, rg))
    assert abs(gl - rl) <= REL * abs(rl), ("lambda", gl, rl)


def test_backward_frac_weights(api):
    rng = np.random.default_rng(7)
    F3 = synth.rgb_scene(30, 33, seed=77, n_rect=8, n_disk=2)
    G = synth.luminance(F3)
    Ubar = rng.normal(size=F3.shape).astype(np.float32)
    kw = dict(r=1, iters=1, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)
    gf, gg, gl = _gpu_grads(api, F3, G, 0.002, Ubar, **kw)
    rf, rg, rl = sgwls_vjp(F3.astype(np.float64), G.astype(np.float64), 0.002, _prm(**kw), Ubar.astype(np.float64))
    assert _rel(gf, rf) <= REL
    assert _rel(gg, rg) <= 2e-3  # |dG|^(alpha_r - 1) near equal guidance values is steep
    assert abs(gl - rl) <= REL * abs(rl)


def test_backward_frac_application_setting(api):
    """The adjoint at the frac weights' HDR setting (lambda = 320, lambda w
    up to ~3e6): the u and v solves run on the same margin-form pivots as
    the forward, so the f and lambda gradients keep their 1e-3 bound."""
    rng = np.random.default_rng(8)
    F3 = synth.rgb_scene(30, 33, seed=78, n_rect=8, n_disk=2)
    G = synth.luminance(F3)
    Ubar = rng.normal(size=F3.shape).astype(np.float32)
    kw = dict(r=1, iters=1, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)
    gf, gg, gl = _gpu_grads(api, F3, G, 320.0, Ubar, **kw)
    rf, rg, rl = sgwls_vjp(F3.astype(np.float64), G.astype(np.float64), 320.0, _prm(**kw), Ubar.astype(np.float64))
    assert _rel(gf, rf) <= REL, _rel(gf, rf)
    assert abs(gl - rl) <= REL * abs(rl), (gl, rl)


def test_backward_central_differences_32x32(api):
    """GPU gradients against FP64 central differences of the oracle's forward
    map on a 32x32 crop (loss = sum((U - target)^2))."""
    F3 = synth.rgb_scene(32, 32, seed=5, n_rect=6, n_disk=2).astype(np.float64)
    target = synth.rgb_scene(32, 32, seed=5000, n_rect=6, n_disk=2).astype(np.float64)
    G = synth.luminance(F3.astype(np.float32)).astype(np.float64)
    F3 = F3.astype(np.float32).astype(np.float64)
    kw = dict(r=1, iters=3, sigma_r=0.1)
    prm = _prm(**kw)
    lam = 1.0

    def loss(F, G, lam):
        return float(np.sum((sgwls(F, G, lam, prm) - target) ** 2))

    U = sgwls(F3, G, lam, prm)
    Ubar = 2.0 * (U - target)
    gf, gg, gl = _gpu_grads(api, F3, G, lam, Ubar, **kw)
    h = 1e-5
    for idx in [(0, 3, 4), (1, 16, 16), (2, 31, 0), (0, 10, 29)]:
        Fp, Fm = F3.copy(), F3.copy()
        Fp[idx] += h
        Fm[idx] -= h
        fd = (loss(Fp, G, lam) - loss(Fm, G, lam)) / (2 * h)
        assert gf[idx] == pytest.approx(fd, rel=REL, abs=1e-6)
    for idx in [(5, 5), (16, 20), (31, 31)]:
        Gp, Gm = G.copy(), G.copy()
        Gp[idx] += h
        Gm[idx] -= h
        fd = (loss(F3, Gp, lam) - loss(F3, Gm, lam)) / (2 * h)
        assert gg[idx] == pytest.approx(fd, rel=5 * REL, abs=1e-5)
    fd = (loss(F3, G, lam + h) - loss(F3, G, lam - h)) / (2 * h)
    assert gl == pytest.approx(fd, rel=REL)


def test_autograd_function(api):
    import torch
    F3 = synth.rgb_scene(24, 28, seed=9, n_rect=5, n_disk=1)
    G = synth.luminance(F3)
    f = torch.from_numpy(F3).cuda().requires_grad_(True)
    g = torch.from_numpy(G).cuda().requires_grad_(True)
    lam = torch.tensor(2.0, device="cuda", requires_grad=True)
    u = api.sgwls(f, g, lam, r=1, iters=2, sigma_r=0.1)
    (u * u).sum().backward()
    Ubar = 2.0 * u.detach().cpu().numpy().astype(np.float64)
    rf, rg, rl = sgwls_vjp(F3.astype(np.float64), G.astype(np.float64), 2.0, _prm(r=1, iters=2), Ubar)
    assert _rel(f.grad.cpu().numpy(), rf) <= REL
    assert _rel(g.grad.cpu().numpy(), rg) <= REL
    assert abs(float(lam.grad) - rl) <= REL * abs(rl)


def test_differentiation_workload_512(api):
    """One image of the differentiation workload: RGB 512x512 scene and a
    separate random target, loss = sum((SG-WLS(f, g; lambda) - target)^2),
    r = 1, T = 3; gradients against the oracle's adjoint."""
    import torch
    F3, T3 = synth.diff_batch(n=1, H=512, W=512, seed=5)
    F3, T3 = F3[0], T3[0]
    G = synth.luminance(F3)
    kw = dict(r=1, iters=3, sigma_r=0.1)
    f = torch.from_numpy(F3).cuda().requires_grad_(True)
    g = torch.from_numpy(G).cuda().requires_grad_(True)
    lam = torch.tensor(1.0, device="cuda", requires_grad=True)
    u = api.sgwls(f, g, lam, **kw)
    loss = ((u - torch.from_numpy(T3).cuda()) ** 2).sum()
    loss.backward()
    Ubar = 2.0 * (u.detach().cpu().numpy().astype(np.float64) - T3.astype(np.float64))
    rf, rg, rl = sgwls_vjp(F3.astype(np.float64), G.astype(np.float64), 1.0, _prm(**kw), Ubar)
    assert _rel(f.grad.cpu().numpy(), rf) <= REL
    assert _rel(g.grad.cpu().numpy(), rg) <= REL
    assert abs(float(lam.grad) - rl) <= REL * abs(rl)


@pytest.mark.parametrize("r", [1, 2])
def test_batched_backward_matches_oracle_and_single_calls(api, r):
    """A batched forward with per-image checkpoints and the batched backward
    over images of uneven sizes and channel counts (1, 3 and 5 channels:
    channel groups of 1, 3 / 2 + 1, 3 + 2 / 2 + 2 + 1): every image's
    gradients against the oracle's adjoint (1e-3 relative) and against the
    single-image backward on the same checkpoints."""
    import torch
    rng = np.random.default_rng(300 + r)
    specs = [(1, 33, 47), (3, 41, 29), (5, 26, 38), (3, 30, 30)]
    T = 2
    kw = dict(r=r, iters=T, sigma_r=0.1)
    Fs, Gs, lams, Ubs = [], [], [], []
    for b, (C, H, W) in enumerate(specs):
        rgb = synth.rgb_scene(H, W, seed=310 + b, n_rect=8, n_disk=2)
        Fs.append(np.concatenate([rgb, rgb[::-1]])[:C].copy())
        Gs.append(synth.luminance(rgb))
        lams.append(float(rng.uniform(0.5, 2.5)))
        Ubs.append(rng.standard_normal((C, H, W)).astype(np.float32))
    fs = [torch.from_numpy(x).cuda() for x in Fs]
    gs = [torch.from_numpy(x).cuda() for x in Gs]
    saveds = [torch.empty((2 * T,) + x.shape, device="cuda") for x in Fs]
    api.sgwls_filter_batched(fs, gs, lams, saveds=saveds, **kw)
    gus = [torch.from_numpy(x).cuda() for x in Ubs]
    n0 = api.launch_count()
    gfs, ggs, gls = api.sgwls_filter_backward_batched(gus, gs, saveds, lams, **kw)
    torch.cuda.synchronize()
    # per pass: one scale launch + at most two kernels per channel-group size
    assert api.launch_count() - n0 <= 2 * T * (1 + 2 * 3)
    prm = _prm(**kw)
    for b in range(len(specs)):
        # the checkpoints equal the single-image forward's
        sv1 = torch.empty_like(saveds[b])
        api.sgwls_filter(fs[b], gs[b], lams[b], saved=sv1, **kw)
        torch.cuda.synchronize()
        assert float((sv1 - saveds[b]).abs().max()) <= 1e-6
        Fb, Gb, lb = sgwls_vjp(Fs[b].astype(np.float64), Gs[b].astype(np.float64), lams[b], prm,
                               Ubs[b].astype(np.float64))
        assert _rel(gfs[b].cpu().numpy(), Fb) <= REL, b
        assert _rel(ggs[b].cpu().numpy(), Gb) <= REL, b
        assert abs(float(gls[b].item()) - lb) <= REL * max(abs(lb), 1e-30), b
        gf1, gg1, gl1 = api.sgwls_filter_backward(gus[b], gs[b], saveds[b], lams[b], **kw)
        torch.cuda.synchronize()
        assert _rel(gfs[b].cpu().numpy(), gf1.cpu().numpy()) <= 1e-5, b


@pytest.mark.parametrize("r", [1, 2, 4])
@pytest.mark.parametrize("C", [1, 2, 3])
def test_backward_kept_factors_many_bands_and_groups(api, r, C):
    """Kept-factor adjoint over several bands, several chunk groups (3-line
    chunks: up to 56 chunks, 7 groups of 8) and ragged tails in both
    directions: against the recomputing adjoint and the oracle's adjoint
    (1e-3 relative)."""
    rng = np.random.default_rng(400 + 10 * r + C)
    F3 = synth.rgb_scene(167, 109, seed=410 + r, n_rect=25, n_disk=5)
    F = np.concatenate([F3, F3[::-1]])[:C].astype(np.float32)
    G = synth.luminance(F3)
    Ubar = rng.normal(size=F.shape).astype(np.float32)
    kw = dict(r=r, iters=1, sigma_r=0.15, chunk_lines=3)
    gk = _gpu_grads(api, F, G, 1.3, Ubar, factor_cache=1, **kw)
    gr = _gpu_grads(api, F, G, 1.3, Ubar, factor_cache=2, **kw)
    # dLoss/df has no atomics: the two differ by the factors' FP32 rounding;
    # dLoss/dG and dLoss/dlambda are atomic sums of signed pair terms whose
    # cancellation amplifies the order-dependent rounding
    assert _rel(gk[0], gr[0]) <= 1e-5
    assert _rel(gk[1], gr[1]) <= 1e-4
    assert abs(gk[2] - gr[2]) <= 1e-4 * abs(gr[2])
    rf, rg, rl = sgwls_vjp(F.astype(np.float64), G.astype(np.float64), 1.3, _prm(**kw), Ubar.astype(np.float64))
    assert _rel(gk[0], rf) <= REL
    assert _rel(gk[1], rg) <= REL
    assert abs(gk[2] - rl) <= REL * abs(rl)
    assert api.device_flag() == 0
