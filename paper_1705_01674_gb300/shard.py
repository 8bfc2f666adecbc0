"""One image filtered by several ranks (one GPU each): the image is split
into strips, and every pass runs on the owning ranks' strips plus a halo.

A pass along the column direction (Sec. 2.1: centres are columns) needs,
for the output columns [a, b), the subsystems centred on [a-r, b+r-1],
which read the columns [a-2r, b+2r).  So a rank that owns a column strip
runs the ordinary single-GPU pass on the strip widened by 2r columns on
each side (clipped at the image border) and keeps its own columns: the
result is exact, not an approximation, because every subsystem that
reaches an owned column lies inside the widened strip, and a border of the
widened strip is a border of the image wherever it cuts a subsystem's
coverage.  The row direction is the same with rows.  Between passes of
different directions the ranks exchange blocks so that each holds its
next strip (an all-to-all re-partition, point-to-point sends of the
intersections); the guidance, which is fixed, is re-partitioned once per
direction.

On entry and exit every rank holds its own column strip (all rows, columns
[a_i, b_i) of a balanced split).  The arithmetic of each pass is the
library's (``sgwls_filter_pass``); this module only moves data.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def split(n: int, parts: int) -> list[tuple[int, int]]:
    """Balanced ranges [lo, hi) covering 0..n-1, one per part."""
    q, m = divmod(n, parts)
    out, lo = [], 0
    for i in range(parts):
        hi = lo + q + (1 if i < m else 0)
        out.append((lo, hi))
        lo = hi
    return out


def _rect_owned(direction: int, rank: int, H: int, W: int, world: int):
    """The block rank owns after a pass along `direction` (0: column strips,
    1: row strips), as (row0, row1, col0, col1)."""
    if direction == 0:
        a, b = split(W, world)[rank]
        return (0, H, a, b)
    c, d = split(H, world)[rank]
    return (c, d, 0, W)


def _rect_needed(direction: int, rank: int, H: int, W: int, world: int, r: int):
    """The block rank reads for a pass along `direction`: its strip widened
    by 2r on both sides across the strips, clipped to the image."""
    r0, r1, c0, c1 = _rect_owned(direction, rank, H, W, world)
    if direction == 0:
        return (0, H, max(0, c0 - 2 * r), min(W, c1 + 2 * r))
    return (max(0, r0 - 2 * r), min(H, r1 + 2 * r), 0, W)


def _intersect(p, q):
    r0, r1 = max(p[0], q[0]), min(p[1], q[1])
    c0, c1 = max(p[2], q[2]), min(p[3], q[3])
    return (r0, r1, c0, c1) if r0 < r1 and c0 < c1 else None


def _crop(x: torch.Tensor, held, want):
    """The part `want` of tensor x (C, rows, cols) that holds block `held`."""
    return x[:, want[0] - held[0]:want[1] - held[0], want[2] - held[2]:want[3] - held[2]]


def redistribute(x: torch.Tensor, held, want_of, group=None) -> torch.Tensor:
    """Every rank holds a block of a (C, H, W) array (this rank: block
    `held`, in x); returns the block want_of(rank) for this rank, assembled
    from the intersections that the ranks holding parts of it send
    (point-to-point, all posted before any wait).  want_of(k) must give
    every rank's wanted block, the same on every rank."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    helds = [None] * world
    dist.all_gather_object(helds, held, group=group)
    mine = want_of(rank)
    out = x.new_empty((x.shape[0], mine[1] - mine[0], mine[3] - mine[2]))
    ops, recvs = [], []
    for peer in range(world):
        if peer == rank:
            continue
        part = _intersect(held, want_of(peer))
        if part is not None:
            ops.append(dist.P2POp(dist.isend, _crop(x, held, part).contiguous(), peer, group))
        part = _intersect(helds[peer], mine)
        if part is not None:
            buf = x.new_empty((x.shape[0], part[1] - part[0], part[3] - part[2]))
            ops.append(dist.P2POp(dist.irecv, buf, peer, group))
            recvs.append((part, buf))
    part = _intersect(held, mine)
    if part is not None:
        _crop(out, mine, part).copy_(_crop(x, held, part))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for part, buf in recvs:
        _crop(out, mine, part).copy_(buf)
    return out


def filter_sharded(f_strip: torch.Tensor, g_strip: torch.Tensor, lam: float, H: int, W: int, pass_fn, *,
                   r: int, iters: int, axis_order: int = 0, group=None) -> torch.Tensor:
    """The SG-WLS filter (Sec. 2.3) of an H x W image split into column
    strips across the ranks of `group`.  f_strip: this rank's (C, H, w)
    strip of the input; g_strip: its (H, w) or (Cg, H, w) strip of the
    guidance; pass_fn(U, G, lam, direction) runs one pass of a whole
    (sub-)image.  Returns this rank's (C, H, w) strip of the result."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    squeeze = g_strip.dim() == 2
    g3 = g_strip.unsqueeze(0) if squeeze else g_strip
    start = _rect_owned(0, rank, H, W, world)
    if tuple(f_strip.shape[1:]) != (start[1] - start[0], start[3] - start[2]):
        raise ValueError(f"rank {rank} must hold columns [{start[2]}, {start[3]}) of every row")
    # the guidance of each direction's widened strips (fixed for all passes)
    gneed = {d: redistribute(g3, start, lambda k, d=d: _rect_needed(d, k, H, W, world, r), group)
             for d in (0, 1)}
    held, x = start, f_strip
    for t in range(2 * iters):
        d = axis_order if t % 2 == 0 else 1 - axis_order
        need = _rect_needed(d, rank, H, W, world, r)
        xin = redistribute(x, held, lambda k, d=d: _rect_needed(d, k, H, W, world, r), group)
        g = gneed[d][0] if squeeze else gneed[d]
        y = pass_fn(xin, g, lam, d)
        held = _rect_owned(d, rank, H, W, world)
        x = _crop(y, need, held).contiguous()
    if held != start:
        x = redistribute(x, held, lambda k: _rect_owned(0, k, H, W, world), group)
    return x


def sgwls_filter_sharded(f_strip: torch.Tensor, g_strip: torch.Tensor, lam: float, H: int, W: int, *,
                         group=None, **kw) -> torch.Tensor:
    """filter_sharded with the library's CUDA pass on every rank (CUDA
    tensors; NCCL or any backend with point-to-point sends; with NCCL each
    rank sets its CUDA device before the process group's first call).
    Every rank of the group takes part in every re-partition.  Keyword
    parameters as ``sgwls_filter``; the sliding step must be 1 (strips of
    a sliding-step pass would not share the whole image's centres)."""
    from . import sgwls_filter_pass
    if int(kw.get("step", 1)) != 1:
        raise ValueError("the sharded filter needs step = 1")
    iters = int(kw.pop("iters", 1))
    axis_order = int(kw.pop("axis_order", 0))
    r = int(kw.get("r", 1))

    def cuda_pass(U, G, lam_, direction):
        return sgwls_filter_pass(U.contiguous(), G.contiguous(), lam_, direction, iters=1, **kw)

    return filter_sharded(f_strip, g_strip, lam, H, W, cuda_pass, r=r, iters=iters, axis_order=axis_order,
                          group=group)
