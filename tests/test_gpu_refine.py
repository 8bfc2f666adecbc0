"""Refinement of every subsystem solve, all in FP32: u1 = A~^-1 f, the
residual rho = f - u1 - lambda L u1 (A = I + lambda L applied without
forming its diagonal, the pair weights recomputed from the guidance),
u = u1 + A~^-1 rho, then the averaging.  At the paper's frac-weight
application settings (alpha = 1.2, eps = 1e-4, lambda 5 .. 900), where a
diagonal formed as 1 + lambda sum w in FP32 would lose the identity, both
the plain solve (margin-form pivots) and the refined one stay within 2e-4
of the FP64 oracle."""
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
    return u.cpu().numpy().astype(np.float64).reshape(F.shape)


@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("lam", [5.0, 40.0, 320.0, 900.0])
def test_refine_frac_application_settings(api, lam, r):
    F = synth.rgb_scene(64, 80, seed=11, n_rect=20, n_disk=5)
    G = synth.luminance(F)
    kw = dict(r=r, iters=2, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)
    ref = sgwls(F.astype(np.float64), G.astype(np.float64), lam,
                Params(r=r, iters=2, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4))
    err0 = float(np.abs(_run(api, F, G, lam, **kw) - ref).max())
    err1 = float(np.abs(_run(api, F, G, lam, refine=1, **kw) - ref).max())
    assert err0 <= TOL, (err0, err1)
    assert err1 <= TOL, (err0, err1)


@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("C", [1, 3])
def test_refine_exp_weights(api, r, C):
    """The refined filter on the exp-weight workloads (already accurate):
    parity is kept, both pass orders, ragged sizes, 1- and 3-line chunks."""
    F = synth.rgb_scene(53, 71, seed=60 + r, n_rect=15, n_disk=4)[:C]
    G = synth.luminance(synth.rgb_scene(53, 71, seed=60 + r, n_rect=15, n_disk=4))
    for axis_order, chunk_lines in ((0, 0), (1, 1), (0, 3)):
        kw = dict(r=r, iters=2, axis_order=axis_order, sigma_r=0.1)
        ref = sgwls(F.astype(np.float64), G.astype(np.float64), 2.0,
                    Params(r=r, iters=2, axis_order=axis_order, sigma_s=float(r), sigma_r=0.1))
        err = float(np.abs(_run(api, F, G, 2.0, refine=1, chunk_lines=chunk_lines, **kw) - ref).max())
        assert err <= TOL, (axis_order, chunk_lines, err)


@pytest.mark.parametrize("r", [2, 3])
def test_refine_frac_larger_radius(api, r):
    """The frac-weight setting at r = 2, 3: the residual's pairs that cross
    the snake's turn (pixel offsets (d, 1) with |d| < r) in both pass
    orders."""
    F = synth.rgb_scene(45, 58, seed=70 + r, n_rect=15, n_disk=4)
    G = synth.luminance(F)
    for axis_order in (0, 1):
        kw = dict(r=r, iters=1, axis_order=axis_order, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)
        prm = Params(r=r, iters=1, axis_order=axis_order, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)
        ref = sgwls(F.astype(np.float64), G.astype(np.float64), 40.0, prm)
        err = float(np.abs(_run(api, F, G, 40.0, refine=1, **kw) - ref).max())
        assert err <= TOL, (axis_order, err)


def test_refine_single_pass_entry(api):
    """sgwls_filter_pass with refine = 1, both directions."""
    import torch
    from oracle import sgwls_pass, COLUMN, ROW
    F = synth.rgb_scene(41, 66, seed=77, n_rect=12, n_disk=3)
    G = synth.luminance(F)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(G).cuda()
    prm = Params(r=2, weight="frac", alpha_s=1.2, alpha_r=1.2, eps=1e-4)
    for direction, d in ((0, COLUMN), (1, ROW)):
        u = api.sgwls_filter_pass(f, g, 40.0, direction, r=2, refine=1, weight="frac", alpha_s=1.2,
                                  alpha_r=1.2, eps=1e-4)
        torch.cuda.synchronize()
        ref = sgwls_pass(F.astype(np.float64), G.astype(np.float64), 40.0, prm, d)
        assert float(np.abs(u.cpu().numpy() - ref).max()) <= TOL, direction


def test_refine_unsupported_paths(api):
    import torch
    F = synth.rgb_scene(30, 40, seed=3, n_rect=5, n_disk=1)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(synth.luminance(F)).cuda()
    for kw in (dict(step=2), dict(factor_cache=2)):
        with pytest.raises(api.SgwlsError) as e:
            api.sgwls_filter(f, g, 1.0, r=2, refine=1, **kw)
        assert e.value.status == -7
