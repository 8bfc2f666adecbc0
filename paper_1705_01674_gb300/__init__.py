"""GB300-native Semi-Global Weighted Least Squares (SG-WLS) filtering.

Python face of libsgwls.so (include/sgwls.h).  PyTorch supplies device
memory and the current CUDA stream; every step of the filter runs in the
library's CUDA kernels.  Tensors must be CUDA tensors: there is no CPU path.

    u = sgwls_filter(f, g, lam, r=1, iters=3)        # f: (C,H,W), g: (H,W)

Parameters follow Liu et al., ICCV 2017: ``r`` the neighbourhood radius of
the (2r+1)x(2r+1) system, ``iters`` the number T of (column, row) pass pairs
(Sec. 2.3), ``step`` the sliding step tau, Eq. 2 weights ``weight='exp'``
(``sigma_s``, default r, and ``sigma_r``) or ``'frac'`` (``alpha_s``,
``alpha_r``, ``eps``).
"""
from __future__ import annotations

import ctypes

import torch

from . import _capi
from . import autotune as autotune_mod
from ._capi import SgwlsError, make_params

__all__ = ["sgwls", "sgwls_filter", "sgwls_filter_pass", "sgwls_filter_backward", "sgwls_filter_batched",
           "sgwls_interpolate", "sgwls_filter_sharded",
           "batched_workspace_bytes", "SGWLSFunction",
           "workspace_bytes", "launch_count", "make_params", "SgwlsError"]

_DT = {torch.float32: _capi.F32, torch.bfloat16: _capi.BF16}


def _check_tensor(x: torch.Tensor, name: str):
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (the SG-WLS library has no CPU path)")
    if x.dtype not in _DT:
        raise TypeError(f"{name} must be float32 or bfloat16, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _check_like(x: torch.Tensor, ref: torch.Tensor, name: str):
    """x must be a contiguous CUDA tensor with ref's shape and dtype (the
    library writes exactly that many elements)."""
    _check_tensor(x, name)
    if x.shape != ref.shape or x.dtype != ref.dtype:
        raise ValueError(f"{name} must have shape {tuple(ref.shape)} and dtype {ref.dtype}")


def _chw(f: torch.Tensor):
    if f.dim() == 2:
        return 1, f.shape[0], f.shape[1]
    if f.dim() == 3:
        return f.shape[0], f.shape[1], f.shape[2]
    raise ValueError("f must be (H, W) or (C, H, W)")


def _guide(g: torch.Tensor, H: int, W: int) -> int:
    """Guidance planes of g: (H, W) -> 1, (Cg, H, W) -> Cg (a vector
    guidance, |G_i - G_j| of Eq. 2 the Euclidean norm)."""
    if tuple(g.shape) == (H, W):
        return 1
    if g.dim() == 3 and tuple(g.shape[1:]) == (H, W) and g.shape[0] >= 1:
        return int(g.shape[0])
    raise ValueError("g must be (H, W) or (Cg, H, W)")


def workspace_bytes(C: int, H: int, W: int, **kw) -> int:
    p = make_params(**kw)
    n = _capi.lib().sgwls_workspace_bytes(int(H), int(W), int(C), ctypes.byref(p))
    if n == 0 and p.iters > 0:
        raise SgwlsError(-1, "sgwls_workspace_bytes", "invalid arguments")
    return int(n)


def _tuned(kind: str, mode, key_fn, tune_fn, kw: dict) -> dict:
    """kw with the autotuner's cached knobs merged (``autotune`` mode
    "cache"), after tuning on a cache miss (mode "search")."""
    mode = autotune_mod.normalise_mode(mode)
    if mode == "off":
        return kw
    explicit = {k for k in autotune_mod.KNOBS if k in kw}
    knobs = autotune_mod.lookup(key_fn())
    if knobs is None and mode == "search":
        knobs = tune_fn()["knobs"]
    return autotune_mod.merge(kw, knobs, explicit)


def sgwls_filter(f: torch.Tensor, g: torch.Tensor, lam: float, *, out: torch.Tensor | None = None,
                 saved: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                 stream: torch.cuda.Stream | None = None, autotune=None, **kw) -> torch.Tensor:
    """SG-WLS filter of one image through ``sgwls_filter`` (C ABI).

    f: (C,H,W) or (H,W); g: (H,W), or (Cg,H,W) for a vector guidance (an
    RGB image, say), same dtype as f (float32 or bfloat16).
    ``saved`` (optional): a float tensor with 2*iters*C*H*W elements in the
    intermediate storage type that receives each pass's input estimate.
    Keyword parameters: see ``make_params``; ``autotune`` ("cache",
    "search", True, False or None for $SGWLS_AUTOTUNE): see ``autotune``."""
    _check_tensor(f, "f")
    _check_tensor(g, "g")
    C, H, W = _chw(f)
    kw["guide_channels"] = _guide(g, H, W)
    if g.dtype != f.dtype:
        raise TypeError("g must have the dtype of f")
    kw.setdefault("storage", "bf16" if f.dtype == torch.bfloat16 else "f32")
    kw = _tuned("filter", autotune, lambda: autotune_mod.filter_key(f, g, kw),
                lambda: autotune_mod.tune_filter(f, g, lam, **kw), kw)
    p = make_params(**kw)
    lib = _capi.lib()
    if out is None:
        out = torch.empty_like(f)
    else:
        _check_like(out, f, "out")
    if saved is not None:
        _check_tensor(saved, "saved")
        sdt = torch.bfloat16 if p.inter_storage == _capi.BF16 else torch.float32
        if saved.dtype != sdt or saved.numel() < 2 * p.iters * C * H * W:
            raise ValueError(f"saved must hold 2*iters*C*H*W = {2 * p.iters * C * H * W} elements of {sdt}")
    nws = lib.sgwls_workspace_bytes(H, W, C, ctypes.byref(p))
    if workspace is None or workspace.numel() < nws:
        workspace = torch.empty(max(nws, 1), dtype=torch.uint8, device=f.device)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    status = lib.sgwls_filter(
        ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        H, W, C, ctypes.c_float(float(lam)), ctypes.byref(p),
        ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()),
        ctypes.c_void_p(saved.data_ptr() if saved is not None else 0),
        ctypes.c_void_p(st.cuda_stream))
    _capi.check(status, "sgwls_filter")
    return out


def sgwls_interpolate(f: torch.Tensor, hmap: torch.Tensor, g: torch.Tensor, lam: float, *,
                      out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                      stream: torch.cuda.Stream | None = None, **kw) -> torch.Tensor:
    """Guided sparse interpolation (Eq. 21) through ``sgwls_interpolate``:
    SG-WLS(f) / SG-WLS(hmap) per pixel.  f: (C,H,W) or (H,W) float32, zero
    where hmap is zero; hmap: (H,W) float32; g: (H,W) or (Cg,H,W) float32.
    Keyword parameters: see ``make_params``."""
    _check_tensor(f, "f")
    _check_tensor(hmap, "hmap")
    _check_tensor(g, "g")
    C, H, W = _chw(f)
    if tuple(hmap.shape) != (H, W):
        raise ValueError("hmap must be (H, W)")
    kw["guide_channels"] = _guide(g, H, W)
    if not (f.dtype == hmap.dtype == g.dtype == torch.float32):
        raise TypeError("f, hmap and g must be float32")
    p = make_params(**kw)
    lib = _capi.lib()
    if out is None:
        out = torch.empty_like(f)
    else:
        _check_like(out, f, "out")
    nws = lib.sgwls_interpolate_workspace_bytes(H, W, C, ctypes.byref(p))
    if workspace is None or workspace.numel() < nws:
        workspace = torch.empty(max(nws, 1), dtype=torch.uint8, device=f.device)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    status = lib.sgwls_interpolate(
        ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(hmap.data_ptr()), ctypes.c_void_p(g.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), H, W, C, ctypes.c_float(float(lam)), ctypes.byref(p),
        ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()), ctypes.c_void_p(st.cuda_stream))
    _capi.check(status, "sgwls_interpolate")
    return out


def sgwls_filter_pass(f: torch.Tensor, g: torch.Tensor, lam: float, direction: int, *,
                      out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                      stream: torch.cuda.Stream | None = None, **kw) -> torch.Tensor:
    """One pass along ``direction`` (0: column direction, 1: row direction)
    through ``sgwls_filter_pass`` (C ABI)."""
    _check_tensor(f, "f")
    _check_tensor(g, "g")
    C, H, W = _chw(f)
    kw["guide_channels"] = _guide(g, H, W)
    if g.dtype != f.dtype:
        raise ValueError("g must have the dtype of f")
    kw.setdefault("storage", "bf16" if f.dtype == torch.bfloat16 else "f32")
    p = make_params(**kw)
    lib = _capi.lib()
    if out is None:
        out = torch.empty_like(f)
    else:
        _check_like(out, f, "out")
    nws = lib.sgwls_workspace_bytes(H, W, C, ctypes.byref(p))
    if workspace is None or workspace.numel() < nws:
        workspace = torch.empty(max(nws, 1), dtype=torch.uint8, device=f.device)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    status = lib.sgwls_filter_pass(
        ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        H, W, C, ctypes.c_float(float(lam)), ctypes.byref(p), int(direction),
        ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()),
        ctypes.c_void_p(st.cuda_stream))
    _capi.check(status, "sgwls_filter_pass")
    return out


def launch_count() -> int:
    """Kernels launched by libsgwls.so in this process so far."""
    return int(_capi.lib().sgwls_launch_count())


def device_flag(clear: bool = False) -> int:
    """Status of the current device's error flag through
    ``sgwls_device_flag``: 0 (clear) or -6 (a bounded wait of the
    queue-scheduled pass gave up).  Synchronises with the device."""
    return int(_capi.lib().sgwls_device_flag(1 if clear else 0))


def sgwls_filter_backward(grad_u: torch.Tensor, g: torch.Tensor, saved: torch.Tensor, lam: float, *,
                          stream: torch.cuda.Stream | None = None, autotune=None, **kw):
    """dLoss/df, dLoss/dg, dLoss/dlambda through ``sgwls_filter_backward``.

    grad_u: (C,H,W) FP32; g: (H,W) FP32; saved: the (2*iters, C, H, W)
    checkpoints written by ``sgwls_filter(..., saved=saved)``.
    Returns (grad_f, grad_g, grad_lambda) with grad_lambda a 0-d tensor."""
    for x, name in ((grad_u, "grad_u"), (g, "g"), (saved, "saved")):
        _check_tensor(x, name)
        if x.dtype != torch.float32:
            raise TypeError(f"{name} must be float32 for the backward")
    C, H, W = _chw(grad_u)
    if tuple(g.shape) != (H, W):
        raise ValueError("g must be (H, W): the backward takes a single guidance plane")
    kw = _tuned("backward", autotune, lambda: autotune_mod.backward_key(grad_u, kw),
                lambda: autotune_mod.tune_backward(grad_u, g, saved, lam, **kw), kw)
    p = make_params(**kw)
    if saved.numel() < 2 * p.iters * C * H * W:
        raise ValueError(f"saved must hold 2*iters*C*H*W = {2 * p.iters * C * H * W} elements")
    lib = _capi.lib()
    grad_f = torch.empty_like(grad_u)
    grad_g = torch.empty((H, W), dtype=torch.float32, device=grad_u.device)
    grad_lam = torch.empty((), dtype=torch.float32, device=grad_u.device)
    nws = lib.sgwls_backward_workspace_bytes(H, W, C, ctypes.byref(p))
    ws = torch.empty(max(nws, 1), dtype=torch.uint8, device=grad_u.device)
    st = stream if stream is not None else torch.cuda.current_stream(grad_u.device)
    status = lib.sgwls_filter_backward(
        ctypes.c_void_p(grad_u.data_ptr()), ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(saved.data_ptr()),
        H, W, C, ctypes.c_float(float(lam)), ctypes.byref(p), ctypes.c_void_p(grad_f.data_ptr()),
        ctypes.c_void_p(grad_g.data_ptr()), ctypes.c_void_p(grad_lam.data_ptr()),
        ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), ctypes.c_void_p(st.cuda_stream))
    _capi.check(status, "sgwls_filter_backward")
    return grad_f, grad_g, grad_lam


class SGWLSFunction(torch.autograd.Function):
    """Differentiable SG-WLS: forward through ``sgwls_filter`` with per-pass
    checkpoints (memory 2*iters images), backward through
    ``sgwls_filter_backward``.  Gradients for f, g and lambda."""

    @staticmethod
    def forward(ctx, f, g, lam, kw):
        lam_f = float(lam)
        T = int(kw.get("iters", 1))
        saved = torch.empty((2 * T,) + tuple(f.shape), dtype=torch.float32, device=f.device)
        u = sgwls_filter(f.contiguous(), g.contiguous(), lam_f, saved=saved, **kw)
        ctx.save_for_backward(g, saved)
        ctx.lam = lam_f
        ctx.kw = kw
        ctx.lam_is_tensor = isinstance(lam, torch.Tensor)
        ctx.f_shape = f.shape
        return u

    @staticmethod
    def backward(ctx, grad_u):
        g, saved = ctx.saved_tensors
        gu = grad_u.contiguous().reshape(saved.shape[1:]).to(torch.float32)
        grad_f, grad_g, grad_lam = sgwls_filter_backward(gu, g, saved, ctx.lam, **ctx.kw)
        gl = grad_lam if ctx.lam_is_tensor else None
        return grad_f.reshape(ctx.f_shape), grad_g, gl, None


def sgwls(f: torch.Tensor, g: torch.Tensor, lam, **kw) -> torch.Tensor:
    """SG-WLS filter; differentiable w.r.t. f, g and lam (if a tensor)."""
    needs = f.requires_grad or g.requires_grad or (isinstance(lam, torch.Tensor) and lam.requires_grad)
    if needs:
        return SGWLSFunction.apply(f, g, lam, kw)
    return sgwls_filter(f, g, float(lam), **kw)


def _image_table(fs, gs, lams, outs, saveds=None, iters=1, inter_bf16=False):
    n = len(fs)
    if not (len(gs) == n and len(lams) == n and len(outs) == n):
        raise ValueError("fs, gs, lams (and outs) must have the same length")
    if saveds is not None and len(saveds) != n:
        raise ValueError("saveds must have one entry per image")
    tab = (_capi.SgwlsImage * n)()
    for i, (f, g, lam, u) in enumerate(zip(fs, gs, lams, outs)):
        _check_tensor(f, f"fs[{i}]")
        _check_tensor(g, f"gs[{i}]")
        C, H, W = _chw(f)
        if tuple(g.shape) != (H, W) or g.dtype != f.dtype:
            raise ValueError(f"gs[{i}] must be (H, W) with the dtype of fs[{i}]")
        if u is not f:
            _check_like(u, f, f"outs[{i}]")
        tab[i].f, tab[i].g, tab[i].u = f.data_ptr(), g.data_ptr(), u.data_ptr()
        tab[i].H, tab[i].W, tab[i].C = H, W, C
        tab[i].lam = float(lam)
        tab[i].saved = None
        if saveds is not None and saveds[i] is not None:
            sv = saveds[i]
            _check_tensor(sv, f"saveds[{i}]")
            sdt = torch.bfloat16 if inter_bf16 else torch.float32
            if sv.dtype != sdt or sv.numel() < 2 * iters * C * H * W:
                raise ValueError(f"saveds[{i}] must hold 2*iters*C*H*W = {2 * iters * C * H * W} elements of {sdt}")
            tab[i].saved = sv.data_ptr()
    return tab


def batched_workspace_bytes(fs, gs, lams, **kw) -> int:
    tab = _image_table(fs, gs, lams, fs)
    p = make_params(**kw)
    return int(_capi.lib().sgwls_batched_workspace_bytes(len(fs), tab, ctypes.byref(p)))


def sgwls_filter_batched(fs, gs, lams, *, outs=None, saveds=None, workspace: torch.Tensor | None = None,
                         stream: torch.cuda.Stream | None = None, autotune=None, **kw):
    """SG-WLS of many images of uneven sizes and channel counts through
    ``sgwls_filter_batched`` (per pass one launch per kernel per
    channel-group size).  fs / gs / lams: sequences of (C,H,W) inputs, (H,W)
    guidance tensors and lambdas; ``saveds`` (optional): per image a tensor
    of 2*iters*C*H*W elements receiving the per-pass checkpoints that
    ``sgwls_filter_backward_batched`` reads."""
    if outs is None:
        outs = [torch.empty_like(f) for f in fs]
    kw.setdefault("storage", "bf16" if fs[0].dtype == torch.bfloat16 else "f32")
    kw = _tuned("batched", autotune, lambda: autotune_mod.batched_key(fs, kw),
                lambda: autotune_mod.tune_batched(fs, gs, lams, **kw), kw)
    p = make_params(**kw)
    tab = _image_table(fs, gs, lams, outs, saveds, p.iters, p.inter_storage == _capi.BF16)
    lib = _capi.lib()
    nws = lib.sgwls_batched_workspace_bytes(len(fs), tab, ctypes.byref(p))
    if workspace is None or workspace.numel() < nws:
        workspace = torch.empty(max(nws, 1), dtype=torch.uint8, device=fs[0].device)
    st = stream if stream is not None else torch.cuda.current_stream(fs[0].device)
    status = lib.sgwls_filter_batched(len(fs), tab, ctypes.byref(p), ctypes.c_void_p(workspace.data_ptr()),
                                      ctypes.c_size_t(workspace.numel()), ctypes.c_void_p(st.cuda_stream))
    _capi.check(status, "sgwls_filter_batched")
    return outs


def sgwls_line_relax(f: torch.Tensor, g: torch.Tensor, lam: float, *, out: torch.Tensor | None = None,
                     workspace: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None,
                     **kw) -> torch.Tensor:
    """Line relaxation of the 2D WLS model through ``sgwls_line_relax`` (an
    opt-in variant, not the paper's SG-WLS: one banded system per image line
    per pass, off-line neighbours at their current estimates).  f: (C,H,W)
    or (H,W) float32; g: (H,W) float32.  Keyword parameters: see
    ``make_params`` (r <= 4)."""
    _check_tensor(f, "f")
    _check_tensor(g, "g")
    C, H, W = _chw(f)
    if tuple(g.shape) != (H, W) or f.dtype != torch.float32 or g.dtype != torch.float32:
        raise ValueError("f must be float32 and g a float32 (H, W) guidance")
    p = make_params(**kw)
    lib = _capi.lib()
    if out is None:
        out = torch.empty_like(f)
    else:
        _check_like(out, f, "out")
    nws = lib.sgwls_line_relax_workspace_bytes(H, W, C, ctypes.byref(p))
    if workspace is None or workspace.numel() < nws:
        workspace = torch.empty(max(nws, 1), dtype=torch.uint8, device=f.device)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    status = lib.sgwls_line_relax(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), H, W, C, ctypes.c_float(float(lam)),
                                  ctypes.byref(p), ctypes.c_void_p(workspace.data_ptr()),
                                  ctypes.c_size_t(workspace.numel()), ctypes.c_void_p(st.cuda_stream))
    _capi.check(status, "sgwls_line_relax")
    return out


def sgwls_filter_backward_batched(grad_us, gs, saveds, lams, *, stream: torch.cuda.Stream | None = None,
                                  workspace: torch.Tensor | None = None, **kw):
    """dLoss/df, dLoss/dg, dLoss/dlambda of many images through
    ``sgwls_filter_backward_batched``: grad_us (C,H,W) FP32 per image, gs
    (H,W) FP32, saveds the per-image checkpoints written by
    ``sgwls_filter_batched(..., saveds=...)``, lams the forward lambdas.
    Returns three lists (grad_f, grad_g, grad_lambda as 0-d tensors)."""
    n = len(grad_us)
    if not (len(gs) == n and len(saveds) == n and len(lams) == n):
        raise ValueError("grad_us, gs, saveds and lams must have the same length")
    p = make_params(**kw)
    tab = (_capi.SgwlsGradImage * n)()
    gfs, ggs, gls = [], [], []
    for i, (gu, g, sv, lam) in enumerate(zip(grad_us, gs, saveds, lams)):
        for x, name in ((gu, "grad_us"), (g, "gs"), (sv, "saveds")):
            _check_tensor(x, f"{name}[{i}]")
            if x.dtype != torch.float32:
                raise TypeError(f"{name}[{i}] must be float32 for the backward")
        C, H, W = _chw(gu)
        if tuple(g.shape) != (H, W):
            raise ValueError(f"gs[{i}] must be (H, W)")
        if sv.numel() < 2 * p.iters * C * H * W:
            raise ValueError(f"saveds[{i}] must hold 2*iters*C*H*W elements")
        gf = torch.empty_like(gu)
        gg = torch.empty((H, W), dtype=torch.float32, device=gu.device)
        gl = torch.empty((), dtype=torch.float32, device=gu.device)
        gfs.append(gf)
        ggs.append(gg)
        gls.append(gl)
        tab[i].grad_u, tab[i].g, tab[i].saved = gu.data_ptr(), g.data_ptr(), sv.data_ptr()
        tab[i].grad_f, tab[i].grad_g, tab[i].grad_lambda = gf.data_ptr(), gg.data_ptr(), gl.data_ptr()
        tab[i].H, tab[i].W, tab[i].C = H, W, C
        tab[i].lam = float(lam)
    lib = _capi.lib()
    nws = lib.sgwls_backward_batched_workspace_bytes(n, tab, ctypes.byref(p))
    if workspace is None or workspace.numel() < nws:
        workspace = torch.empty(max(nws, 1), dtype=torch.uint8, device=grad_us[0].device)
    st = stream if stream is not None else torch.cuda.current_stream(grad_us[0].device)
    status = lib.sgwls_filter_backward_batched(n, tab, ctypes.byref(p), ctypes.c_void_p(workspace.data_ptr()),
                                               ctypes.c_size_t(workspace.numel()), ctypes.c_void_p(st.cuda_stream))
    _capi.check(status, "sgwls_filter_backward_batched")
    return gfs, ggs, gls


from .shard import sgwls_filter_sharded  # noqa: E402  (one image over several ranks)
