"""The C ABI library loads, exports every symbol include/sgwls.h declares,
and validates arguments on the host (no GPU needed for any of this)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(sgwls_\w+)\s*\(", text, flags=re.M):
            if not m.group(0).lstrip().startswith(("typedef", "#")):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def capi():
    from paper_1705_01674_gb300 import build, _capi
    build.build()
    return _capi


def test_header_declares_entry_points():
    names = _declared_functions()
    for need in ("sgwls_filter", "sgwls_workspace_bytes", "sgwls_params_default", "sgwls_status_string"):
        assert need in names


def test_library_exports_every_declared_symbol(capi):
    lib = capi.lib()
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_and_status_strings(capi):
    lib = capi.lib()
    p = capi.SgwlsParams()
    lib.sgwls_params_default(ctypes.byref(p))
    assert (p.r, p.iters, p.step, p.axis_order, p.weight) == (1, 1, 1, 0, 0)
    assert p.sigma_s == pytest.approx(1.0) and p.sigma_r == pytest.approx(0.1)
    assert p.eps == pytest.approx(1e-4)
    for code in range(-7, 1):
        assert lib.sgwls_status_string(code).decode().startswith("SGWLS_")


def test_workspace_bytes_host_only(capi):
    lib = capi.lib()
    p = capi.make_params(r=1, iters=3)
    n1 = lib.sgwls_workspace_bytes(768, 1024, 3, ctypes.byref(p))
    assert n1 >= 768 * 1024 * 3 * 4 and n1 % 256 == 0
    p0 = capi.make_params(r=1, iters=0)
    assert lib.sgwls_workspace_bytes(768, 1024, 3, ctypes.byref(p0)) < n1
    bad = capi.make_params(r=1)
    bad.r = 9
    assert lib.sgwls_workspace_bytes(64, 64, 1, ctypes.byref(bad)) == 0
    assert lib.sgwls_workspace_bytes(2, 64, 1, ctypes.byref(p)) == 0


def _call(capi, H=64, W=64, C=1, lam=1.0, p=None, f=0x1000, g=0x2000, u=0x3000, ws=0x10000, nws=1 << 30):
    lib = capi.lib()
    p = p if p is not None else capi.make_params()
    return lib.sgwls_filter(ctypes.c_void_p(f), ctypes.c_void_p(g), ctypes.c_void_p(u), H, W, C,
                            ctypes.c_float(lam), ctypes.byref(p), ctypes.c_void_p(ws), nws,
                            ctypes.c_void_p(0), ctypes.c_void_p(0))


def test_validation_before_any_launch(capi):
    """Invalid arguments are rejected on the host (the pointers here are
    never dereferenced: every call fails validation first)."""
    E_INVALID, E_SHAPE, E_DTYPE, E_WS, E_UNSUP = -1, -2, -3, -4, -7
    assert _call(capi, f=0) == E_INVALID
    assert _call(capi, u=0x1000) == E_INVALID            # u aliases f
    assert _call(capi, lam=-1.0) == E_INVALID
    assert _call(capi, lam=float("nan")) == E_INVALID
    assert _call(capi, H=2, p=capi.make_params(r=1)) == E_SHAPE
    assert _call(capi, W=4, p=capi.make_params(r=2)) == E_SHAPE
    assert _call(capi, C=0) == E_SHAPE
    assert _call(capi, H=65537, W=5) == E_SHAPE            # longest side 65536
    assert _call(capi, H=32768, W=32768) == E_SHAPE        # more than 2^29 pixels
    for field, val in (("r", 0), ("r", 9), ("iters", -1), ("step", 0), ("axis_order", 2),
                       ("weight", 5), ("sigma_r", 0.0), ("chunk_lines", -2),
                       ("factor_cache", 3), ("factor_cache", -1)):
        p = capi.make_params()
        setattr(p, field, val)
        assert _call(capi, p=p) == E_INVALID, field
    p = capi.make_params()
    p.storage = 7
    assert _call(capi, p=p) == E_DTYPE
    assert _call(capi, ws=0) == E_WS
    assert _call(capi, nws=16) == E_WS
    assert _call(capi, ws=0x10010) == E_WS                # misaligned
    assert _call(capi, p=capi.make_params(r=1, refine=2)) == E_INVALID
    assert _call(capi, p=capi.make_params(r=2, refine=1, step=2)) == E_UNSUP


def test_interpolate_validation_host_only(capi):
    """sgwls_interpolate rejects bad arguments before any launch."""
    lib = capi.lib()
    E_INVALID, E_SHAPE, E_WS, E_UNSUP = -1, -2, -4, -7

    def call(C=1, p=None, f=0x1000, h=0x2000, g=0x3000, u=0x4000, ws=0x10000, nws=1 << 30, lam=1.0):
        p = p if p is not None else capi.make_params()
        return lib.sgwls_interpolate(ctypes.c_void_p(f), ctypes.c_void_p(h), ctypes.c_void_p(g),
                                     ctypes.c_void_p(u), 64, 64, C, ctypes.c_float(lam), ctypes.byref(p),
                                     ctypes.c_void_p(ws), nws, ctypes.c_void_p(0))

    p = capi.make_params(r=2, iters=2)
    need = lib.sgwls_interpolate_workspace_bytes(64, 64, 3, ctypes.byref(p))
    assert need >= lib.sgwls_workspace_bytes(64, 64, 4, ctypes.byref(p)) + 2 * 4 * 64 * 64 * 4
    assert lib.sgwls_interpolate_workspace_bytes(64, 64, 0, ctypes.byref(p)) == 0
    assert call(C=0) == E_SHAPE
    assert call(f=0) == E_INVALID
    assert call(h=0) == E_INVALID
    assert call(u=0x1000) == E_INVALID           # u aliases f
    assert call(u=0x2000) == E_INVALID           # u aliases the index map
    assert call(lam=-1.0) == E_INVALID
    assert call(nws=16) == E_WS
    assert call(p=capi.make_params(storage="bf16")) == E_UNSUP


def test_guide_channels_validation_host_only(capi):
    """A vector guidance (guide_channels = Cg > 1): range checked, runs on
    kept factors only, and the entry points without a vector-guidance path
    say so before any launch (the pointers here are never dereferenced)."""
    lib = capi.lib()
    E_INVALID, E_UNSUP = -1, -7
    for bad in (-1, 5):
        assert _call(capi, p=capi.make_params(guide_channels=bad)) == E_INVALID, bad
        assert lib.sgwls_workspace_bytes(64, 64, 1, ctypes.byref(capi.make_params(guide_channels=bad))) == 0
    p = capi.make_params(r=2, iters=2, guide_channels=3)
    assert lib.sgwls_workspace_bytes(64, 64, 3, ctypes.byref(p)) > 0
    assert _call(capi, p=capi.make_params(guide_channels=3, factor_cache=2)) == E_UNSUP
    assert _call(capi, p=capi.make_params(guide_channels=3, refine=1)) == E_UNSUP
    # batched, backward and the no-allocation pass take one guidance plane
    img = (capi.SgwlsImage * 1)()
    img[0].f, img[0].g, img[0].u = 0x1000, 0x2000, 0x3000
    img[0].H, img[0].W, img[0].C = 64, 64, 1
    img[0].lam = 1.0
    img[0].saved = None
    assert lib.sgwls_filter_batched(1, img, ctypes.byref(p), ctypes.c_void_p(0x10000), 1 << 30,
                                    ctypes.c_void_p(0)) == E_UNSUP
    pb = capi.make_params(r=1, iters=1, guide_channels=3)
    st = lib.sgwls_filter_backward(ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000),
                                   64, 64, 1, ctypes.c_float(1.0), ctypes.byref(pb), ctypes.c_void_p(0x4000),
                                   ctypes.c_void_p(0), None, ctypes.c_void_p(0x10000), 1 << 30,
                                   ctypes.c_void_p(0))
    assert st == E_UNSUP
    st = lib.sgwls_filter_pass_noalloc(ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000),
                                       64, 64, 1, ctypes.c_float(1.0), ctypes.byref(pb), 0, ctypes.c_void_p(0))
    assert st == E_UNSUP


def test_refinement_workspace_adds_two_entry_buffers(capi):
    """refine = 1 adds two per-entry buffers (the first solve's entries and
    the residual: one value per channel for each of the 2r+1 entries per
    line of every subsystem) and nothing else: the FP32 residual recomputes
    its pair weights from the guidance."""
    lib = capi.lib()
    a256 = lambda x: (x + 255) // 256 * 256
    H = W = 64
    for r in (1, 2, 3, 4):
        for C in (1, 3):
            p0 = capi.make_params(r=r, iters=1, factor_cache=1)
            p1 = capi.make_params(r=r, iters=1, factor_cache=1, refine=1)
            n0 = lib.sgwls_workspace_bytes(H, W, C, ctypes.byref(p0))
            n1 = lib.sgwls_workspace_bytes(H, W, C, ctypes.byref(p1))
            nsys = (W - 2 * r + 31) // 32 * 32
            ent = H * (2 * r + 1) * C * nsys * 4
            assert n1 - n0 == 2 * a256(ent), (r, C)


def test_batched_validation_host_only(capi):
    """sgwls_filter_batched and its workspace query reject bad image tables
    on the host (the pointers here are never dereferenced)."""
    lib = capi.lib()
    E_INVALID, E_SHAPE, E_WS, E_UNSUP = -1, -2, -4, -7

    def table(specs):
        tab = (capi.SgwlsImage * len(specs))()
        for i, sp in enumerate(specs):
            d = dict(f=0x1000 * (3 * i + 1), g=0x1000 * (3 * i + 2), u=0x1000 * (3 * i + 3), H=64, W=80, C=1,
                     lam=1.0, saved=None)
            d.update(sp)
            tab[i].f, tab[i].g, tab[i].u = d["f"], d["g"], d["u"]
            tab[i].H, tab[i].W, tab[i].C, tab[i].lam, tab[i].saved = d["H"], d["W"], d["C"], d["lam"], d["saved"]
        return tab

    def call(specs, p=None, ws=0x100000, nws=1 << 30):
        p = p if p is not None else capi.make_params(r=2, iters=2)
        tab = table(specs)
        return lib.sgwls_filter_batched(len(specs), tab, ctypes.byref(p), ctypes.c_void_p(ws), nws,
                                        ctypes.c_void_p(0))

    p = capi.make_params(r=2, iters=2)
    good = table([{}, {"H": 100, "W": 33}])
    assert lib.sgwls_batched_workspace_bytes(2, good, ctypes.byref(p)) > 0
    assert lib.sgwls_filter_batched(0, good, ctypes.byref(p), ctypes.c_void_p(0x100000), 1 << 30,
                                    ctypes.c_void_p(0)) == E_INVALID
    # any channel counts: the workspace holds one uniform batch per channel-group size
    mixed = table([{}, {"C": 3}, {"C": 5}])
    n_mixed = lib.sgwls_batched_workspace_bytes(3, mixed, ctypes.byref(p))
    n_one = lib.sgwls_batched_workspace_bytes(1, table([{}]), ctypes.byref(p))
    assert n_mixed > n_one > 0 and n_mixed % 256 == 0
    assert call([{"C": 65}]) == E_SHAPE
    assert call([{"u": 0x2000}]) == E_INVALID              # output aliases the guidance
    assert call([{"C": 0}]) == E_SHAPE
    assert call([{}, {"H": 4}]) == E_SHAPE                 # smaller than 2r+1
    assert call([{"f": 0}]) == E_INVALID
    assert call([{"u": 0x1000}]) == E_INVALID              # output aliases the input
    assert call([{"lam": -1.0}]) == E_INVALID
    assert call([{"lam": float("nan")}]) == E_INVALID
    assert call([{}], p=capi.make_params(r=9)) == E_INVALID
    assert call([{}], p=capi.make_params(r=2, step=2)) == E_UNSUP
    bad = capi.make_params(r=2)
    bad.step = 0
    assert call([{}], p=bad) == E_INVALID                  # out of range, not merely unsupported
    assert call([{}], nws=16) == E_WS
    assert call([{}], ws=0x100010) == E_WS                 # misaligned workspace


def test_backward_validation_host_only(capi):
    """sgwls_filter_backward rejects bad arguments before any launch."""
    lib = capi.lib()
    E_INVALID, E_WS, E_UNSUP = -1, -4, -7

    def call(gu=0x1000, g=0x2000, saved=0x3000, gf=0x4000, p=None, lam=1.0, ws=0x100000, nws=1 << 30):
        p = p if p is not None else capi.make_params(r=1, iters=1)
        return lib.sgwls_filter_backward(ctypes.c_void_p(gu), ctypes.c_void_p(g), ctypes.c_void_p(saved), 64, 64, 3,
                                         ctypes.c_float(lam), ctypes.byref(p), ctypes.c_void_p(gf),
                                         ctypes.c_void_p(0), None, ctypes.c_void_p(ws), nws, ctypes.c_void_p(0))

    p = capi.make_params(r=1, iters=1)
    assert lib.sgwls_backward_workspace_bytes(64, 64, 3, ctypes.byref(p)) > 0
    assert call(gu=0) == E_INVALID
    assert call(gf=0) == E_INVALID
    assert call(gf=0x1000) == E_INVALID                  # grad_f aliases grad_u
    assert call(saved=0) == E_INVALID                    # iters > 0 needs the checkpoints
    assert call(lam=-2.0) == E_INVALID
    assert call(p=capi.make_params(storage="bf16")) == E_UNSUP
    assert call(p=capi.make_params(weight="frac", alpha_r=0.8)) == E_UNSUP   # |x|^alpha not differentiable at 0
    assert call(p=capi.make_params(r=2, step=2)) == E_UNSUP
    assert call(p=capi.make_params(refine=1)) == E_UNSUP
    assert call(nws=64) == E_WS


def test_noalloc_validation_matches_workspace_pass(capi):
    """The no-allocation pass validates the caller's parameters exactly as
    sgwls_filter_pass does (same status for the same mistake), and both
    reject an output that aliases the input or the guidance; the pointers
    are never dereferenced because every case fails on the host."""
    lib = capi.lib()
    E_INVALID, E_SHAPE, E_DTYPE, E_UNSUP = -1, -2, -3, -7

    def both(p, H=64, W=80, C=3, f=0x1000, g=0x2000, u=0x3000, lam=1.0, direction=0):
        a = lib.sgwls_filter_pass(ctypes.c_void_p(f), ctypes.c_void_p(g), ctypes.c_void_p(u), H, W, C,
                                  ctypes.c_float(lam), ctypes.byref(p), direction, ctypes.c_void_p(0x100000),
                                  1 << 30, ctypes.c_void_p(0))
        b = lib.sgwls_filter_pass_noalloc(ctypes.c_void_p(f), ctypes.c_void_p(g), ctypes.c_void_p(u), H, W, C,
                                          ctypes.c_float(lam), ctypes.byref(p), direction, ctypes.c_void_p(0))
        return a, b

    bad_dtype = capi.make_params(r=1)
    bad_dtype.storage = 5
    assert both(bad_dtype) == (E_DTYPE, E_DTYPE)
    bad_inter = capi.make_params(r=1)
    bad_inter.inter_storage = 9
    assert both(bad_inter) == (E_DTYPE, E_DTYPE)
    p = capi.make_params(r=2)
    assert both(p, H=4) == (E_SHAPE, E_SHAPE)               # smaller than 2r + 1
    assert both(p, C=0) == (E_SHAPE, E_SHAPE)
    assert both(p, W=70000) == (E_SHAPE, E_SHAPE)
    bad_fc = capi.make_params(r=1)
    bad_fc.factor_cache = 7
    assert both(bad_fc) == (E_INVALID, E_INVALID)            # out of range, not silently replaced
    bad_r = capi.make_params(r=1)
    bad_r.r = 0
    assert both(bad_r) == (E_INVALID, E_INVALID)
    assert both(p, u=0x1000) == (E_INVALID, E_INVALID)       # output aliases the input
    assert both(p, u=0x2000) == (E_INVALID, E_INVALID)       # output aliases the guidance
    assert both(p, lam=-1.0) == (E_INVALID, E_INVALID)
    assert both(p, direction=2) == (E_INVALID, E_INVALID)
    # kept factors do not fit the fixed scratch
    st = lib.sgwls_filter_pass_noalloc(ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000),
                                       64, 80, 3, ctypes.c_float(1.0),
                                       ctypes.byref(capi.make_params(r=1, factor_cache=1)), 0, ctypes.c_void_p(0))
    assert st == E_UNSUP


def test_batched_backward_validation_host_only(capi):
    """sgwls_filter_backward_batched and its workspace query reject bad
    tables on the host (no pointer is dereferenced)."""
    lib = capi.lib()
    E_INVALID, E_WS, E_UNSUP = -1, -4, -7

    def table(specs):
        tab = (capi.SgwlsGradImage * len(specs))()
        for i, sp in enumerate(specs):
            base = 0x100000 * (i + 1)
            d = dict(grad_u=base, g=base + 0x1000, saved=base + 0x2000, grad_f=base + 0x3000, grad_g=0,
                     grad_lambda=0, H=40, W=50, C=3, lam=1.0)
            d.update(sp)
            for k, v in d.items():
                setattr(tab[i], "lam" if k == "lam" else k, v)
        return tab

    def call(specs, p=None, ws=0x10000000, nws=1 << 30):
        p = p if p is not None else capi.make_params(r=1, iters=2)
        tab = table(specs)
        return lib.sgwls_filter_backward_batched(len(specs), tab, ctypes.byref(p), ctypes.c_void_p(ws), nws,
                                                 ctypes.c_void_p(0))

    p = capi.make_params(r=1, iters=2)
    good = table([{}, {"C": 1, "H": 70}, {"C": 5}])
    n = lib.sgwls_backward_batched_workspace_bytes(3, good, ctypes.byref(p))
    assert n > 0 and n % 256 == 0
    assert lib.sgwls_filter_backward_batched(0, good, ctypes.byref(p), ctypes.c_void_p(0x10000000), 1 << 30,
                                             ctypes.c_void_p(0)) == E_INVALID
    assert call([{"grad_f": 0x100000}]) == E_INVALID        # grad_f aliases grad_u
    assert call([{"saved": 0}]) == E_INVALID                # iters > 0 needs the checkpoints
    assert call([{"grad_u": 0}]) == E_INVALID
    assert call([{"lam": -1.0}]) == E_INVALID
    assert call([{}], p=capi.make_params(r=1, iters=2, storage="bf16")) == E_UNSUP
    assert call([{}], p=capi.make_params(r=2, step=2)) == E_UNSUP
    assert call([{}], p=capi.make_params(weight="frac", alpha_r=0.8)) == E_UNSUP
    assert call([{}], nws=1024) == E_WS
    assert call([{}], ws=0x10000010) == E_WS
