"""GPU parity of the line-relaxation variant (sgwls_line_relax: one banded
system per image line per pass, the off-line neighbours of the (2r+1) x
(2r+1) square at their current estimates) against its FP64 oracle
(oracle/line_relax.py, pinned by the dense block-Jacobi step and by
convergence to the dense 2D WLS solution), and its convergence to the dense
2D WLS on a tiny image."""
import numpy as np
import pytest

import synth
from oracle import Params
from oracle.line_relax import line_relax
from oracle.wls2d import wls2d

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


@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("C", [1, 3, 5])
@pytest.mark.parametrize("axis_order", [0, 1])
def test_line_relax_matches_oracle(api, r, C, axis_order):
    import torch
    rgb = synth.rgb_scene(37, 52, seed=400 + r, n_rect=10, n_disk=2)
    F = np.concatenate([rgb, rgb[::-1]])[:C].copy()
    G = synth.luminance(rgb)
    for weight, lam in (("exp", 1.3), ("frac", 0.05)):
        kw = dict(r=r, iters=2, axis_order=axis_order, weight=weight, sigma_r=0.1, alpha_s=1.2, alpha_r=1.2, eps=1e-4)
        u = api.sgwls_line_relax(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(), lam, **kw)
        torch.cuda.synchronize()
        ref = line_relax(F.astype(np.float64), G.astype(np.float64), lam,
                         Params(r=r, iters=2, axis_order=axis_order, weight=weight, sigma_s=float(r), sigma_r=0.1,
                                alpha_s=1.2, alpha_r=1.2, eps=1e-4))
        err = float(np.abs(u.cpu().numpy().astype(np.float64) - ref).max())
        assert err <= TOL, (weight, err)


def test_line_relax_converges_to_2d_wls(api):
    import torch
    F = synth.rect_gray(12, 15, seed=3)
    G = F[0]
    kw = dict(r=1, iters=40, sigma_r=0.2)
    u = api.sgwls_line_relax(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(), 0.7, **kw)
    torch.cuda.synchronize()
    ref = wls2d(F.astype(np.float64), G.astype(np.float64), 0.7, Params(r=1, sigma_s=1.0, sigma_r=0.2))
    assert float(np.abs(u.cpu().numpy() - ref).max()) <= 1e-4


def test_line_relax_rejects_unsupported(api):
    import torch
    f = torch.zeros((1, 20, 20), device="cuda")
    with pytest.raises(api.SgwlsError) as e:
        api.sgwls_line_relax(f, f[0], 1.0, r=5)
    assert e.value.status == -7
    with pytest.raises(api.SgwlsError) as e:
        api.sgwls_line_relax(f, f[0], 1.0, r=1, step=2)
    assert e.value.status == -7
