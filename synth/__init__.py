"""Seeded synthetic inputs shaped like the SG-WLS paper's workloads.

The paper evaluates on natural photographs (1-megapixel RGB smoothing,
Table 1), HDR images, a guided depth-upsampling dataset (Table 2) and
scribble images; none of them is available here.  These generators stand in
for them with the structure an edge-preserving smoother reacts to:
piecewise-constant regions with sharp edges (rectangles, disks), smooth
texture and i.i.d. noise, all in [0, 1].

This module is shared by the CUDA tests/bench and by the CPU oracle's tests.
It holds no arithmetic of the filtering method itself: it only draws images.
The luminance helper is input preparation (the guidance image), not part of
the method.

Every generator uses ``numpy.random.default_rng(seed)`` (PCG64) and returns
float32 arrays in planar C x H x W layout.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rect_gray",
    "rgb_scene",
    "luminance",
    "batch_uneven_gray",
    "diff_batch",
]


def _paste_rect(img: np.ndarray, rng: np.random.Generator, value) -> None:
    """Paste an axis-aligned rectangle whose two corners are integer points
    drawn uniformly over the image (sorted per axis)."""
    _, H, W = img.shape
    ys = np.sort(rng.integers(0, H, size=2))
    xs = np.sort(rng.integers(0, W, size=2))
    img[:, ys[0]:ys[1] + 1, xs[0]:xs[1] + 1] = np.asarray(value, dtype=np.float64)[:, None, None]


def rect_gray(H: int = 64, W: int = 64, seed: int = 0, n_rect: int = 8,
              noise: float = 0.05) -> np.ndarray:
    """Grayscale test image: U[0,1] background, ``n_rect`` rectangles with
    values U[0,1] pasted in draw order, N(0, noise^2) noise, clipped to [0,1].
    Returns float32 (1, H, W)."""
    rng = np.random.default_rng(seed)
    img = rng.uniform(0.0, 1.0, size=(1, H, W))
    for _ in range(n_rect):
        _paste_rect(img, rng, [rng.uniform(0.0, 1.0)])
    img += rng.normal(0.0, noise, size=img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def rgb_scene(H: int = 768, W: int = 1024, seed: int = 2, n_rect: int = 200,
              n_disk: int = 50, texture_amp: float = 0.1,
              noise: float = 0.03) -> np.ndarray:
    """RGB test image: U[0,1]^3 background; ``n_rect`` rectangles and
    ``n_disk`` filled disks (radius U[4, 96] px) with per-channel values
    U[0,1], drawn in a random interleaved order; per-channel sinusoidal
    texture ``amp*sin(2*pi*(x/px + y/py) + phi)`` with px, py ~ U[4, 64] and
    phi ~ U[0, 2*pi); N(0, noise^2) noise; clipped to [0, 1].
    Returns float32 (3, H, W)."""
    rng = np.random.default_rng(seed)
    img = rng.uniform(0.0, 1.0, size=(3, H, W))
    kinds = np.array([0] * n_rect + [1] * n_disk)
    rng.shuffle(kinds)
    yy, xx = np.mgrid[0:H, 0:W]
    for kind in kinds:
        value = rng.uniform(0.0, 1.0, size=3)
        if kind == 0:
            _paste_rect(img, rng, value)
        else:
            cy = rng.uniform(0, H)
            cx = rng.uniform(0, W)
            rad = rng.uniform(4.0, 96.0)
            y0, y1 = max(0, int(cy - rad) - 1), min(H, int(cy + rad) + 2)
            x0, x1 = max(0, int(cx - rad) - 1), min(W, int(cx + rad) + 2)
            sub = (yy[y0:y1, x0:x1] - cy) ** 2 + (xx[y0:y1, x0:x1] - cx) ** 2 <= rad * rad
            for ch in range(3):
                img[ch, y0:y1, x0:x1][sub] = value[ch]
    for ch in range(3):
        px = rng.uniform(4.0, 64.0)
        py = rng.uniform(4.0, 64.0)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        img[ch] += texture_amp * np.sin(2.0 * np.pi * (xx / px + yy / py) + phi)
    img += rng.normal(0.0, noise, size=img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def luminance(rgb: np.ndarray) -> np.ndarray:
    """Guidance image from an RGB image: 0.299 R + 0.587 G + 0.114 B,
    computed in float64 and rounded once to float32.  Returns (H, W)."""
    x = rgb.astype(np.float64)
    return (0.299 * x[0] + 0.587 * x[1] + 0.114 * x[2]).astype(np.float32)


def batch_uneven_gray(n: int = 64, seed: int = 4, lo: int = 256, hi: int = 2048,
                      lam_lo: float = 0.5, lam_hi: float = 4.0):
    """A batch of grayscale rectangle images of uneven sizes.

    Sizes and per-image lambda come from ``seed``; image ``b`` is drawn with
    seed ``1000*seed + b`` (so seed 4 gives 4000 + b).  The rectangle count
    is 8 as in the small grayscale case; rectangle corners are drawn over the
    whole image, so rectangle sizes scale with the image.
    Returns (list of float32 (1, H, W) arrays, list of float lambdas)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=(n, 2))
    lams = rng.uniform(lam_lo, lam_hi, size=n)
    imgs = [rect_gray(int(h), int(w), seed=1000 * seed + b) for b, (h, w) in enumerate(sizes)]
    return imgs, [float(x) for x in lams]


def diff_batch(n: int = 16, H: int = 512, W: int = 512, seed: int = 5):
    """Inputs and separate random targets for the differentiation workload:
    ``n`` RGB scenes, input ``b`` drawn with seed ``100*seed + b`` and target
    ``b`` with seed ``1000*seed + b`` (5000 + b for seed 5).
    Returns (f: float32 (n, 3, H, W), target: float32 (n, 3, H, W))."""
    f = np.stack([rgb_scene(H, W, seed=100 * seed + b) for b in range(n)])
    t = np.stack([rgb_scene(H, W, seed=1000 * seed + b) for b in range(n)])
    return f, t


def sparse_depth(H: int, W: int, factor: int = 4, seed: int = 6, noise: float = 0.01):
    """Guided-upsampling stand-in: a depth map of planar patches (a plane
    a + b y + c x per rectangle, pasted in draw order over a background
    plane), sampled on the regular grid of every ``factor``-th row and column
    (the low-resolution depth projected onto the high-resolution grid), with
    N(0, noise^2) noise.  Returns (F (1,H,W) float32, zero off the grid;
    Hm (H,W) float32 index map; dense depth (1,H,W) float32)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    y, x = yy / max(H - 1, 1), xx / max(W - 1, 1)

    def plane():
        a, b, c = rng.uniform(0.2, 0.8), rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3)
        return a + b * y + c * x

    depth = plane()
    for _ in range(max(4, H * W // 4000)):
        y0, y1 = np.sort(rng.integers(0, H + 1, size=2))
        x0, x1 = np.sort(rng.integers(0, W + 1, size=2))
        p = plane()
        depth[y0:y1, x0:x1] = p[y0:y1, x0:x1]
    depth = np.clip(depth, 0.0, 1.0)
    Hm = np.zeros((H, W))
    Hm[::factor, ::factor] = 1.0
    F = (depth + rng.normal(0.0, noise, size=depth.shape)) * Hm
    return F[None].astype(np.float32), Hm.astype(np.float32), depth[None].astype(np.float32)


def scribbles(H: int, W: int, n: int = 12, C: int = 2, seed: int = 7):
    """Colourisation stand-in: ``n`` random strokes (random walks of 3-pixel
    wide dots) carrying per-stroke chrominance values U[-0.5, 0.5] in C
    channels.  Returns (F (C,H,W) float32, zero off the strokes; Hm (H,W))."""
    rng = np.random.default_rng(seed)
    F = np.zeros((C, H, W))
    Hm = np.zeros((H, W))
    for _ in range(n):
        val = rng.uniform(-0.5, 0.5, size=C)
        py, px = rng.uniform(0, H), rng.uniform(0, W)
        ang = rng.uniform(0, 2 * np.pi)
        for _ in range(int(rng.integers(5, 40))):
            ang += rng.normal(0.0, 0.4)
            py = min(max(py + np.sin(ang), 0.0), H - 1.0)
            px = min(max(px + np.cos(ang), 0.0), W - 1.0)
            y0, x0 = int(py), int(px)
            F[:, max(y0 - 1, 0):y0 + 2, max(x0 - 1, 0):x0 + 2] = val[:, None, None]
            Hm[max(y0 - 1, 0):y0 + 2, max(x0 - 1, 0):x0 + 2] = 1.0
    return F.astype(np.float32), Hm.astype(np.float32)
