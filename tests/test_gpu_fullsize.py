"""Full-size parity on sampled outputs: one pass over a 1920 x 1080 RGB
scene (the r = 2, 3, 5 workload) in the launch configuration the library
picks for that size (chunk factors kept, per-radius chunk length, segmented
band chain), both directions.

The oracle computes the sampled across-offsets one by one: the output at
offset o of a pass is the mean, over the centres k with |k - o| <= r, of
subsystem k's exact solution at o (Sec. 2.3, steps 1-4), so only those
2r + 1 subsystems are solved per sample."""
import numpy as np
import pytest

import synth
from oracle import COLUMN, Params
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


@pytest.fixture(scope="module")
def scene():
    F = synth.rgb_scene(1080, 1920, seed=3)
    return F, synth.luminance(F)


@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("r", [2, 3, 5])
def test_fullsize_pass_sampled(api, scene, r, direction):
    import torch
    F, G = scene
    C, H, W = F.shape
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(G).cuda()
    u = api.sgwls_filter_pass(f, g, 1.0, direction, r=r, sigma_r=0.1)
    torch.cuda.synchronize()
    dim = W if direction == COLUMN else H
    rng = np.random.default_rng(100 * r + direction)
    offsets = sorted({0, 1, r, r + 1, 31, 32, 33, dim // 2, dim - 2 - r, dim - 1 - r, dim - 2, dim - 1,
                      *rng.integers(0, dim, size=4).tolist()})
    ref = oracle_pass_offsets(F, G, 1.0, Params(r=r, iters=1, sigma_s=float(r), sigma_r=0.1), direction, offsets)
    U = u.cpu().numpy().astype(np.float64)
    got = U[:, :, offsets].transpose(0, 2, 1) if direction == COLUMN else U[:, offsets, :]
    err = float(np.abs(got - ref).max())
    assert err <= TOL, err


@pytest.mark.parametrize("direction", [0, 1])
def test_large_image_pass_sampled(api, direction):
    """A 4096 x 6144 grayscale image (25 MP, the factor store 0.3 GB per
    pass): one pass, sampled offsets against the oracle."""
    import torch
    from synth import rect_gray
    F = rect_gray(4096, 6144, seed=12, n_rect=400)
    G = F[0]
    f = torch.from_numpy(F).cuda()
    u = api.sgwls_filter_pass(f, f[0], 2.0, direction, r=1, sigma_r=0.1)
    torch.cuda.synchronize()
    C, H, W = F.shape
    dim = W if direction == COLUMN else H
    offsets = [0, 1, 2, 777, dim // 2 + 13, dim - 2, dim - 1]
    ref = oracle_pass_offsets(F, G, 2.0, Params(r=1, iters=1, sigma_s=1.0, sigma_r=0.1), direction, offsets)
    U = u.cpu().numpy().astype(np.float64)
    got = U[:, :, offsets].transpose(0, 2, 1) if direction == COLUMN else U[:, offsets, :]
    err = float(np.abs(got - ref).max())
    assert err <= TOL, err


@pytest.mark.parametrize("r", [2, 3, 5])
def test_fullsize_pass_bf16_and_refined(api, scene, r):
    """1920 x 1080 RGB, one column pass per r: BF16 storage (against the
    oracle on the same BF16-rounded planes: one BF16 rounding of the output,
    2^-9, plus the FP32 bound) and the refined FP32 pass, on sampled
    offsets."""
    import torch
    F, G = scene
    C, H, W = F.shape
    rng = np.random.default_rng(300 + r)
    offsets = sorted({0, r, 31, 32, W // 2, W - 1 - r, W - 1, *rng.integers(0, W, size=3).tolist()})
    prm = Params(r=r, iters=1, sigma_s=float(r), sigma_r=0.1)

    def sampled(u):
        U = u.float().cpu().numpy().astype(np.float64)
        return U[:, :, offsets].transpose(0, 2, 1)

    fb = torch.from_numpy(F).cuda().to(torch.bfloat16)
    gb = torch.from_numpy(G).cuda().to(torch.bfloat16)
    ub = api.sgwls_filter_pass(fb, gb, 1.0, 0, r=r, sigma_r=0.1)
    torch.cuda.synchronize()
    Fb = fb.float().cpu().numpy().astype(np.float64)
    Gb = gb.float().cpu().numpy().astype(np.float64)
    ref_b = oracle_pass_offsets(Fb, Gb, 1.0, prm, COLUMN, offsets)
    assert float(np.abs(sampled(ub) - ref_b).max()) <= 2.0 ** -9 + TOL

    uf = api.sgwls_filter_pass(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(), 1.0, 0, r=r,
                               sigma_r=0.1, refine=1)
    torch.cuda.synchronize()
    ref = oracle_pass_offsets(F, G, 1.0, prm, COLUMN, offsets)
    assert float(np.abs(sampled(uf) - ref).max()) <= TOL


@pytest.mark.parametrize("shape", [(65536, 5), (7, 65536)])
def test_maximum_side_length(api, shape):
    """The longest side the library accepts (65536) on a thin image: one
    pass per direction, against the oracle on the whole pass where it has
    few subsystems and on sampled offsets where it has ~65k."""
    import torch
    from oracle import ROW, sgwls_pass
    H, W = shape
    rng = np.random.default_rng(H + W)
    F = rng.uniform(0, 1, size=(2, H, W)).astype(np.float32)
    G = rng.uniform(0, 1, size=(H, W)).astype(np.float32)
    prm = Params(r=1, iters=1, sigma_s=1.0, sigma_r=0.3)
    f, g = torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda()
    for direction, d in ((0, COLUMN), (1, ROW)):
        u = api.sgwls_filter_pass(f, g, 2.0, direction, r=1, sigma_r=0.3)
        torch.cuda.synchronize()
        U = u.cpu().numpy().astype(np.float64)
        dim = W if direction == 0 else H
        if dim <= 64:
            ref = sgwls_pass(F.astype(np.float64), G.astype(np.float64), 2.0, prm, d)
            assert float(np.abs(U - ref).max()) <= TOL, direction
        else:
            offsets = [0, 1, 2, 31, 32, 33, 4097, dim // 2, dim - 3, dim - 2, dim - 1]
            ref = oracle_pass_offsets(F, G, 2.0, prm, d, offsets)
            got = U[:, :, offsets].transpose(0, 2, 1) if direction == 0 else U[:, offsets, :]
            assert float(np.abs(got - ref).max()) <= TOL, direction


_FILTER_REF = {}


@pytest.mark.parametrize("r", [2, 3])
def test_fullsize_filter_every_pixel(api, scene, r):
    """The headline workload end to end: the whole T = 2 filter of the
    1920 x 1080 RGB scene (luminance guidance, lambda = 1, range parameter
    0.1, sigma_s = r) in the launch configuration the benchmark times,
    every output pixel of every channel against the FP64 oracle."""
    import torch
    from oracle import sgwls
    F, G = scene
    if r not in _FILTER_REF:
        _FILTER_REF[r] = sgwls(F.astype(np.float64), G.astype(np.float64), 1.0,
                               Params(r=r, iters=2, sigma_s=float(r), sigma_r=0.1))
    u = api.sgwls_filter(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(), 1.0, r=r, iters=2, sigma_r=0.1)
    torch.cuda.synchronize()
    err = float(np.abs(u.cpu().numpy().astype(np.float64) - _FILTER_REF[r]).max())
    assert err <= TOL, err
