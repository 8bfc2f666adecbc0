"""sgwls_filter_pass_noalloc: the pass for callers that cannot allocate.

Such callers (a host with a fixed device-memory budget, or a path that must
not enter the allocator) get a pass whose scratch is a fixed device array
inside the library.  This file is collected last; the test calls the entry
point through the C ABI twice in a row and compares each result with the
workspace-taking sgwls_filter_pass on the same inputs.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 2e-4


def test_noalloc_pass_matches_workspace_pass():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01674_gb300 import build
    build.build()
    import paper_1705_01674_gb300 as sg
    from paper_1705_01674_gb300 import _capi

    lib = _capi.lib()
    stream = torch.cuda.current_stream()
    cases = [(0, synth.rgb_scene(96, 130, seed=21, n_rect=20, n_disk=4), 1.5, 1),
             (1, synth.rgb_scene(77, 101, seed=22, n_rect=15, n_disk=3), 0.7, 2)]
    for direction, F, lam, r in cases:
        G = synth.luminance(F)
        f = torch.from_numpy(F).cuda()
        g = torch.from_numpy(G).cuda()
        C, H, W = f.shape
        p = _capi.make_params(r=r, sigma_r=0.1)
        u = torch.full_like(f, float("nan"))
        st = lib.sgwls_filter_pass_noalloc(
            ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(u.data_ptr()),
            H, W, C, ctypes.c_float(lam), ctypes.byref(p), direction, ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, _capi.STATUS_NAMES.get(st, st)
        ref = sg.sgwls_filter_pass(f, g, lam, direction, r=r, sigma_r=0.1)
        torch.cuda.synchronize()
        err = float((u - ref).abs().max())
        assert err <= TOL, err
        assert bool(torch.isfinite(u).all())


def test_noalloc_rejects_oversized_request():
    pytest.importorskip("torch")
    from paper_1705_01674_gb300 import build
    build.build()
    from paper_1705_01674_gb300 import _capi
    lib = _capi.lib()
    p = _capi.make_params(r=3, sigma_r=0.1)
    # a 4096 x 4096 RGB pass needs far more than the 16 MiB scratch; the
    # pointers are never touched because the size check comes first
    st = lib.sgwls_filter_pass_noalloc(ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000),
                                       4096, 4096, 3, ctypes.c_float(1.0), ctypes.byref(p), 0, ctypes.c_void_p(0))
    assert st == -4
