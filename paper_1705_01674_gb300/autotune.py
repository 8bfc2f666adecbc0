"""Autotuner of the SG-WLS launch knobs.

The filter's result does not depend on its launch knobs beyond FP32
rounding, but its speed does: the chunk length of the parallel subsystem
solve (``chunk_lines``), the chunk-warps per block (``group_warps``),
whether the chunk factors are kept or recomputed (``factor_cache``), the
pass schedule (two kernels, or one queue-scheduled persistent kernel:
``schedule``) and the size of that kernel's factor-store ring
(``ring_slots``).  Which setting is fastest depends on the image size,
channel count, radius and storage types, and on the GPU.

``tune_filter`` (and ``tune_batched``, ``tune_backward``) times candidate
settings on the caller's own workload with CUDA events, the L2 flushed
before every timed call, by coordinate descent from the library's
automatic choice: one knob at a time over its candidate values, keeping a
change only when it is faster by more than 2 %, two rounds.  A candidate
whose output differs from the automatic choice's by more than 1e-4 (or that
the library rejects) is skipped.  The winner is stored in a JSON cache at
``$SGWLS_TUNE_CACHE`` (default ``~/.cache/sgwls_gb300/tune.json``), keyed
by the device name and the workload; writes go through a temporary file
and a rename, so concurrent writers never leave a torn file.

The entry points use the cache when asked: ``sgwls_filter(...,
autotune=...)`` (likewise ``sgwls_filter_batched``,
``sgwls_filter_backward``) with ``"cache"`` (or ``True``) merges a cached
setting if one exists, ``"search"`` tunes on a cache miss first; the
default comes from ``$SGWLS_AUTOTUNE`` ("", "0": off).  Knobs the caller
passes explicitly always win over cached ones.
"""
from __future__ import annotations

import json
import os
import statistics
import tempfile

KNOBS = ("chunk_lines", "factor_cache", "schedule", "ring_slots", "group_warps", "lookahead")
CANDIDATES = {
    "chunk_lines": (0, 3, 4, 6, 8, 12, 16, 24),
    "group_warps": (0, 1, 2, 4),
    "factor_cache": (0, 1, 2),
    "schedule": (0, 2),
    "ring_slots": (0, 4, 6, 8, 12, 16, 24, 32, 48),
    "lookahead": (0, 2, 4, 8, 16, 32),
}
# knobs each entry point honours
KIND_KNOBS = {
    "filter": KNOBS,
    "batched": ("chunk_lines", "factor_cache"),
    "backward": ("chunk_lines", "group_warps", "factor_cache"),
}
MIN_GAIN = 0.02
AGREE = 1e-4


def cache_path() -> str:
    p = os.environ.get("SGWLS_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "sgwls_gb300", "tune.json")


def mode_from_env() -> str:
    v = os.environ.get("SGWLS_AUTOTUNE", "").strip().lower()
    if v in ("", "0", "off", "false", "no"):
        return "off"
    if v in ("search", "tune"):
        return "search"
    return "cache"


def normalise_mode(mode) -> str:
    if mode is None:
        return mode_from_env()
    if mode is True:
        return "cache"
    if mode is False:
        return "off"
    mode = str(mode).lower()
    if mode not in ("off", "cache", "search"):
        raise ValueError("autotune must be None, a bool, 'off', 'cache' or 'search'")
    return mode


WORK_FIELDS = ("r", "iters", "step", "storage", "inter_storage", "weight", "refine", "guide_channels",
               "axis_order")


def workload_key(kind: str, device: str, shape, params) -> str:
    """Cache key of a workload: the entry point, the device, the shape(s)
    and every parameter that changes the work (not the tuning knobs);
    `params` is the sgwls_params the call passes (an object with those
    attributes)."""
    fields = {k: int(getattr(params, k)) for k in WORK_FIELDS}
    return json.dumps({"kind": kind, "device": device, "shape": shape, **fields}, sort_keys=True)


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_entry(key: str, entry: dict, path: str | None = None) -> None:
    """Adds one entry to the cache file (read, update, atomic replace)."""
    path = path or cache_path()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    d = load_cache(path)
    d[key] = entry
    fd, tmp = tempfile.mkstemp(prefix=".tune.", dir=os.path.dirname(os.path.abspath(path)))
    try:
        with os.fdopen(fd, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def lookup(key: str, path: str | None = None) -> dict | None:
    e = load_cache(path).get(key)
    if not isinstance(e, dict) or not isinstance(e.get("knobs"), dict):
        return None
    return {k: int(v) for k, v in e["knobs"].items() if k in KNOBS}


def merge(kw: dict, knobs: dict | None, explicit: set) -> dict:
    """kw with the cached knobs added, except those the caller set."""
    if not knobs:
        return kw
    out = dict(kw)
    for k, v in knobs.items():
        if k not in explicit:
            out[k] = v
    return out


def coordinate_descent(run, kind: str, check=None, rounds: int = 2):
    """Minimises run(knobs) -> ms over the knobs of `kind`, one knob at a
    time from the automatic setting.  check(knobs) -> bool rejects a setting
    whose output disagrees.  Returns (best knobs, best ms, automatic ms,
    trials)."""
    best = {}
    base_ms = run(best)
    best_ms = base_ms
    trials = [({}, base_ms)]
    for _ in range(rounds):
        improved = False
        for knob in KIND_KNOBS[kind]:
            for v in CANDIDATES[knob]:
                cand = dict(best)
                if v == 0:   # 0: the library's automatic choice
                    cand.pop(knob, None)
                else:
                    cand[knob] = v
                if cand == best:
                    continue
                if knob in ("ring_slots", "lookahead") and cand.get("schedule") != 2:
                    continue
                try:
                    ms = run(cand)
                except Exception:
                    continue
                trials.append((cand, ms))
                if ms < best_ms * (1.0 - MIN_GAIN) and (check is None or check(cand)):
                    best, best_ms, improved = cand, ms, True
        if not improved:
            break
    return best, best_ms, base_ms, trials


def _timer(fn, steps: int, warmup: int, stream, device):
    """Median device ms of fn() over `steps` calls, L2 flushed before each."""
    import torch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
        evs = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
    torch.cuda.synchronize(device)
    return statistics.median(a.elapsed_time(b) for a, b in evs)


def _device_name(t) -> str:
    import torch
    return torch.cuda.get_device_name(t.device)


def _store(key, best, best_ms, base_ms, trials, save):
    entry = {"knobs": best, "ms": best_ms, "default_ms": base_ms, "trials": len(trials)}
    if save:
        save_entry(key, entry)
    return entry


def _params(kw):
    from ._capi import make_params
    return make_params(**{k: v for k, v in kw.items() if k not in KNOBS})


def filter_key(f, g, kw) -> str:
    C, H, W = (1,) + tuple(f.shape) if f.dim() == 2 else tuple(f.shape)
    kw = dict(kw)
    kw.setdefault("storage", "bf16" if str(f.dtype) == "torch.bfloat16" else "f32")
    kw["guide_channels"] = 1 if g.dim() == 2 else int(g.shape[0])
    return workload_key("filter", _device_name(f), [C, H, W], _params(kw))


def tune_filter(f, g, lam, *, steps: int = 3, warmup: int = 1, save: bool = True, **kw) -> dict:
    """Tunes the knobs of ``sgwls_filter`` for this input's shape and the
    parameters in kw.  Returns the cache entry ({"knobs", "ms",
    "default_ms", "trials"})."""
    import torch

    from . import sgwls_filter
    kw = {k: v for k, v in kw.items() if k not in KNOBS}
    st = torch.cuda.Stream(f.device)
    kw["autotune"] = "off"
    ref = sgwls_filter(f, g, lam, stream=st, **kw)
    out = torch.empty_like(ref)
    torch.cuda.synchronize(f.device)

    def run(knobs):
        return _timer(lambda: sgwls_filter(f, g, lam, out=out, stream=st, **kw, **knobs), steps, warmup, st, f.device)

    def check(knobs):
        with torch.cuda.stream(st):
            u = sgwls_filter(f, g, lam, stream=st, **kw, **knobs)
        torch.cuda.synchronize(f.device)
        return float((u.float() - ref.float()).abs().max()) <= AGREE

    best, best_ms, base_ms, trials = coordinate_descent(run, "filter", check)
    kw.pop("autotune")
    return _store(filter_key(f, g, kw), best, best_ms, base_ms, trials, save)


def batched_key(fs, kw) -> str:
    shapes = sorted([list(x.shape) for x in fs])
    kw = dict(kw)
    kw.setdefault("storage", "bf16" if str(fs[0].dtype) == "torch.bfloat16" else "f32")
    return workload_key("batched", _device_name(fs[0]), shapes, _params(kw))


def tune_batched(fs, gs, lams, *, steps: int = 3, warmup: int = 1, save: bool = True, **kw) -> dict:
    """Tunes the knobs of ``sgwls_filter_batched`` for these images."""
    import torch

    from . import sgwls_filter_batched
    kw = {k: v for k, v in kw.items() if k not in KNOBS}
    st = torch.cuda.Stream(fs[0].device)
    kw["autotune"] = "off"
    ref = sgwls_filter_batched(fs, gs, lams, stream=st, **kw)
    outs = [torch.empty_like(x) for x in ref]
    torch.cuda.synchronize(fs[0].device)

    def run(knobs):
        return _timer(lambda: sgwls_filter_batched(fs, gs, lams, outs=outs, stream=st, **kw, **knobs), steps, warmup,
                      st, fs[0].device)

    def check(knobs):
        us = sgwls_filter_batched(fs, gs, lams, stream=st, **kw, **knobs)
        torch.cuda.synchronize(fs[0].device)
        return all(float((u.float() - v.float()).abs().max()) <= AGREE for u, v in zip(us, ref))

    best, best_ms, base_ms, trials = coordinate_descent(run, "batched", check)
    kw.pop("autotune")
    return _store(batched_key(fs, kw), best, best_ms, base_ms, trials, save)


def backward_key(grad_u, kw) -> str:
    return workload_key("backward", _device_name(grad_u), list(grad_u.shape), _params(kw))


def tune_backward(grad_u, g, saved, lam, *, steps: int = 3, warmup: int = 1, save: bool = True, **kw) -> dict:
    """Tunes the knobs of ``sgwls_filter_backward`` for this shape."""
    import torch

    from . import sgwls_filter_backward
    kw = {k: v for k, v in kw.items() if k not in KNOBS}
    st = torch.cuda.Stream(grad_u.device)
    kw["autotune"] = "off"
    ref = sgwls_filter_backward(grad_u, g, saved, lam, stream=st, **kw)
    torch.cuda.synchronize(grad_u.device)

    def run(knobs):
        return _timer(lambda: sgwls_filter_backward(grad_u, g, saved, lam, stream=st, **kw, **knobs), steps, warmup,
                      st, grad_u.device)

    def check(knobs):
        got = sgwls_filter_backward(grad_u, g, saved, lam, stream=st, **kw, **knobs)
        torch.cuda.synchronize(grad_u.device)
        scale = max(1.0, float(ref[0].abs().max()))
        return float((got[0] - ref[0]).abs().max()) <= AGREE * scale

    best, best_ms, base_ms, trials = coordinate_descent(run, "backward", check)
    kw.pop("autotune")
    return _store(backward_key(grad_u, kw), best, best_ms, base_ms, trials, save)
