"""ctypes view of libsgwls.so (the C ABI in include/sgwls.h).

Only argument marshalling lives here.  The shared library is built in-tree
by ``paper_1705_01674_gb300.build``; if it is missing, loading fails with an
error that says so -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsgwls.so")

SGWLS_OK = 0
STATUS_NAMES = {
    0: "SGWLS_OK",
    -1: "SGWLS_E_INVALID",
    -2: "SGWLS_E_SHAPE",
    -3: "SGWLS_E_DTYPE",
    -4: "SGWLS_E_WORKSPACE",
    -5: "SGWLS_E_CUDA",
    -6: "SGWLS_E_DEVICE_FLAG",
    -7: "SGWLS_E_UNSUPPORTED",
}
F32, BF16 = 0, 1
W_EXP, W_FRAC = 0, 1
R_MAX = 8


class SgwlsParams(ctypes.Structure):
    """Mirror of ``sgwls_params``."""

    _fields_ = [
        ("weight", ctypes.c_int),
        ("sigma_s", ctypes.c_float),
        ("sigma_r", ctypes.c_float),
        ("alpha_s", ctypes.c_float),
        ("alpha_r", ctypes.c_float),
        ("eps", ctypes.c_float),
        ("r", ctypes.c_int),
        ("iters", ctypes.c_int),
        ("step", ctypes.c_int),
        ("axis_order", ctypes.c_int),
        ("refine", ctypes.c_int),
        ("storage", ctypes.c_int),
        ("inter_storage", ctypes.c_int),
        ("chunk_lines", ctypes.c_int),
        ("factor_cache", ctypes.c_int),
        ("guide_channels", ctypes.c_int),
        ("schedule", ctypes.c_int),
        ("ring_slots", ctypes.c_int),
        ("group_warps", ctypes.c_int),
        ("lookahead", ctypes.c_int),
    ]


class SgwlsImage(ctypes.Structure):
    """Mirror of ``sgwls_image`` (one entry of a batched call)."""

    _fields_ = [
        ("f", ctypes.c_void_p),
        ("g", ctypes.c_void_p),
        ("u", ctypes.c_void_p),
        ("H", ctypes.c_int),
        ("W", ctypes.c_int),
        ("C", ctypes.c_int),
        ("lam", ctypes.c_float),
        ("saved", ctypes.c_void_p),
    ]


class SgwlsGradImage(ctypes.Structure):
    """Mirror of ``sgwls_grad_image`` (one entry of a batched backward)."""

    _fields_ = [
        ("grad_u", ctypes.c_void_p),
        ("g", ctypes.c_void_p),
        ("saved", ctypes.c_void_p),
        ("grad_f", ctypes.c_void_p),
        ("grad_g", ctypes.c_void_p),
        ("grad_lambda", ctypes.c_void_p),
        ("H", ctypes.c_int),
        ("W", ctypes.c_int),
        ("C", ctypes.c_int),
        ("lam", ctypes.c_float),
    ]


class SgwlsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {name}" + (f" ({detail})" if detail else ""))


_lib = None


def _declare(lib):
    P = ctypes.POINTER(SgwlsParams)
    vp, sz, ci, cf = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_float
    lib.sgwls_params_default.argtypes = [P]
    lib.sgwls_params_default.restype = None
    lib.sgwls_status_string.argtypes = [ci]
    lib.sgwls_status_string.restype = ctypes.c_char_p
    lib.sgwls_last_cuda_error.argtypes = []
    lib.sgwls_last_cuda_error.restype = ctypes.c_char_p
    lib.sgwls_workspace_bytes.argtypes = [ci, ci, ci, P]
    lib.sgwls_workspace_bytes.restype = sz
    lib.sgwls_filter.argtypes = [vp, vp, vp, ci, ci, ci, cf, P, vp, sz, vp, vp]
    lib.sgwls_filter.restype = ci
    lib.sgwls_filter_pass.argtypes = [vp, vp, vp, ci, ci, ci, cf, P, ci, vp, sz, vp]
    lib.sgwls_filter_pass.restype = ci
    lib.sgwls_filter_pass_noalloc.argtypes = [vp, vp, vp, ci, ci, ci, cf, P, ci, vp]
    lib.sgwls_filter_pass_noalloc.restype = ci
    lib.sgwls_launch_count.argtypes = []
    lib.sgwls_launch_count.restype = ctypes.c_ulonglong
    lib.sgwls_device_flag.argtypes = [ci]
    lib.sgwls_device_flag.restype = ci
    if hasattr(lib, "sgwls_batched_workspace_bytes"):
        lib.sgwls_batched_workspace_bytes.argtypes = [ci, ctypes.POINTER(SgwlsImage), P]
        lib.sgwls_batched_workspace_bytes.restype = sz
        lib.sgwls_filter_batched.argtypes = [ci, ctypes.POINTER(SgwlsImage), P, vp, sz, vp]
        lib.sgwls_filter_batched.restype = ci
    lib.sgwls_line_relax_workspace_bytes.argtypes = [ci, ci, ci, P]
    lib.sgwls_line_relax_workspace_bytes.restype = sz
    lib.sgwls_line_relax.argtypes = [vp, vp, vp, ci, ci, ci, cf, P, vp, sz, vp]
    lib.sgwls_line_relax.restype = ci
    lib.sgwls_backward_batched_workspace_bytes.argtypes = [ci, ctypes.POINTER(SgwlsGradImage), P]
    lib.sgwls_backward_batched_workspace_bytes.restype = sz
    lib.sgwls_filter_backward_batched.argtypes = [ci, ctypes.POINTER(SgwlsGradImage), P, vp, sz, vp]
    lib.sgwls_filter_backward_batched.restype = ci
    if hasattr(lib, "sgwls_backward_workspace_bytes"):
        lib.sgwls_backward_workspace_bytes.argtypes = [ci, ci, ci, P]
        lib.sgwls_backward_workspace_bytes.restype = sz
        lib.sgwls_filter_backward.argtypes = [vp, vp, vp, ci, ci, ci, cf, P, vp, vp, vp, vp, sz, vp]
        lib.sgwls_filter_backward.restype = ci
    lib.sgwls_interpolate_workspace_bytes.argtypes = [ci, ci, ci, P]
    lib.sgwls_interpolate_workspace_bytes.restype = sz
    lib.sgwls_interpolate.argtypes = [vp, vp, vp, vp, ci, ci, ci, cf, P, vp, sz, vp]
    lib.sgwls_interpolate.restype = ci
    return lib


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libsgwls.so not found at {LIB_PATH}; build it with "
                "`python -m paper_1705_01674_gb300.build` (there is no CPU fallback)")
        _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


def check(status: int, where: str):
    if status != SGWLS_OK:
        detail = ""
        if status == -5:
            detail = lib().sgwls_last_cuda_error().decode(errors="replace")
        raise SgwlsError(status, where, detail)


def make_params(r=1, iters=1, step=1, axis_order=0, weight="exp", sigma_s=None, sigma_r=0.1,
                alpha_s=1.2, alpha_r=1.2, eps=1e-4, storage="f32", inter_storage=None,
                refine=0, chunk_lines=0, factor_cache=0, guide_channels=1, schedule=0,
                ring_slots=0, group_warps=0, lookahead=0) -> SgwlsParams:
    p = SgwlsParams()
    lib().sgwls_params_default(ctypes.byref(p))
    p.weight = {"exp": W_EXP, "frac": W_FRAC}[weight]
    p.r = int(r)
    p.iters = int(iters)
    p.step = int(step)
    p.axis_order = int(axis_order)
    p.sigma_s = float(r if sigma_s is None else sigma_s)
    p.sigma_r = float(sigma_r)
    p.alpha_s = float(alpha_s)
    p.alpha_r = float(alpha_r)
    p.eps = float(eps)
    p.refine = int(refine)
    p.chunk_lines = int(chunk_lines)
    p.factor_cache = int(factor_cache)
    p.guide_channels = int(guide_channels)
    p.schedule = int(schedule)
    p.ring_slots = int(ring_slots)
    p.group_warps = int(group_warps)
    p.lookahead = int(lookahead)
    dt = {"f32": F32, "bf16": BF16}
    p.storage = dt[storage]
    p.inter_storage = dt[inter_storage or storage]
    return p
