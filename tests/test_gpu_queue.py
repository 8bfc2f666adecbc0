"""The queue-scheduled pass (schedule = 2, opt-in for a forward pass with
kept factors at sliding step 1): one persistent kernel whose blocks
take summary and back-substitution work items from a queue, with the
factor store a ring of band slots.

It runs the same per-item arithmetic as the two-kernel pass (schedule = 1);
the two kernels are compiled separately, so the compiler may fuse a multiply
and an add in one and not in the other: they must agree to FP32 rounding
(1e-6 on [0, 1] values), and both are compared with the FP64 oracle.
Small rings (ring_slots = 4, the minimum) make every band after the fourth
wait for the readers of the band whose slot it reuses.  After every case
the device error flag (set when a bounded wait gives up) must be clear."""
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
    assert m.device_flag(clear=True) == 0
    return m


def _run(api, f, g, lam, **kw):
    import torch
    u = api.sgwls_filter(f, g, lam, **kw)
    torch.cuda.synchronize()
    return u


@pytest.mark.parametrize("r", [1, 2, 3, 5])
@pytest.mark.parametrize("shape", [(70, 333), (257, 130), (41, 1000)])
def test_queue_matches_two_kernels_and_oracle(api, r, shape):
    import torch
    H, W = shape
    F = synth.rgb_scene(H, W, seed=80 + r, n_rect=25, n_disk=5)
    G = synth.luminance(F)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(G).cuda()
    kw = dict(r=r, iters=2, sigma_r=0.1, factor_cache=1)
    u1 = _run(api, f, g, 1.3, schedule=1, **kw)
    ref = sgwls(F.astype(np.float64), G.astype(np.float64), 1.3, Params(r=r, iters=2, sigma_s=float(r), sigma_r=0.1))
    for sched in (dict(schedule=2), dict(schedule=2, ring_slots=4), dict(schedule=2, ring_slots=5),
                  dict(schedule=2, chunk_lines=3), dict(schedule=2, lookahead=40)):
        u2 = _run(api, f, g, 1.3, **sched, **kw)
        if "chunk_lines" not in sched:
            # the same arithmetic, another order of work items
            d = float((u1 - u2).abs().max())
            assert d <= 1e-6, (sched, d)
        err = float(np.abs(u2.cpu().numpy().astype(np.float64) - ref).max())
        assert err <= TOL, (sched, err)
    assert api.device_flag() == 0


@pytest.mark.parametrize("C", [1, 2, 5])
def test_queue_channel_groups_and_pass_order(api, C):
    """More than four channels run as two channel groups (two launches per
    pass, each resetting its own queue); both pass orders; BF16 storage."""
    import torch
    F = synth.rgb_scene(150, 220, seed=90 + C, n_rect=20, n_disk=4)
    F = np.concatenate([F, F[::-1]])[:C].copy()
    G = synth.luminance(synth.rgb_scene(150, 220, seed=90 + C, n_rect=20, n_disk=4))
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(G).cuda()
    for axis_order in (0, 1):
        kw = dict(r=2, iters=2, sigma_r=0.1, axis_order=axis_order, ring_slots=4)
        u1 = _run(api, f, g, 0.8, schedule=1, **kw)
        u2 = _run(api, f, g, 0.8, schedule=2, **kw)
        assert torch.equal(u1, u2)
        ref = sgwls(F.astype(np.float64), G.astype(np.float64), 0.8,
                    Params(r=2, iters=2, sigma_s=2.0, sigma_r=0.1, axis_order=axis_order))
        assert float(np.abs(u2.cpu().numpy().astype(np.float64) - ref).max()) <= TOL
    fb, gb = f.to(torch.bfloat16), g.to(torch.bfloat16)
    kw = dict(r=2, iters=2, sigma_r=0.1, ring_slots=4)
    assert torch.equal(_run(api, fb, gb, 0.8, schedule=1, **kw), _run(api, fb, gb, 0.8, schedule=2, **kw))
    assert api.device_flag() == 0


def test_queue_fullsize_small_ring(api):
    """The headline image (1920 x 1080 RGB, r = 2, T = 2) with the smallest
    ring and with the automatic one: bitwise equal to the two-kernel pass."""
    import torch
    F = synth.rgb_scene(1080, 1920, seed=3)
    G = synth.luminance(F)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(G).cuda()
    kw = dict(r=2, iters=2, sigma_r=0.1)
    u1 = _run(api, f, g, 1.0, schedule=1, **kw)
    for rs in (4, 0):
        assert torch.equal(u1, _run(api, f, g, 1.0, schedule=2, ring_slots=rs, **kw)), rs
    assert api.device_flag() == 0


def test_queue_single_pass_entry_and_graph(api):
    """sgwls_filter_pass on the queue kernel, inside a captured CUDA graph
    replayed twice (the control words reset themselves between passes)."""
    import torch
    F = synth.rgb_scene(96, 300, seed=7, n_rect=15, n_disk=3)
    G = synth.luminance(F)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(G).cuda()
    kw = dict(r=1, sigma_r=0.1, ring_slots=4)
    ref = api.sgwls_filter_pass(f, g, 1.0, 0, schedule=1, **kw)
    out = torch.empty_like(f)
    ws = torch.empty(1 << 26, dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        api.sgwls_filter_pass(f, g, 1.0, 0, out=out, workspace=ws, stream=st, schedule=2, **kw)   # warm-up
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        api.sgwls_filter_pass(f, g, 1.0, 0, out=out, workspace=ws, stream=st, schedule=2, **kw)
    for _ in range(2):
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    assert api.device_flag() == 0
