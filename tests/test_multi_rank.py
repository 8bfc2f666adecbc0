"""The N > 1 host path of bench.py on CPU: two gloo ranks (no GPU).

Every rank filters its own image (weak scaling, no collective on the data
path); the job's time is the slowest rank's and its throughput counts the
work of all ranks; the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK_CODE = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world, _ = bench._dist()
ms = [7.0, 11.5][rank]
total = bench._max_over_ranks(ms, world, "cpu")
value = bench._job_value(world, 2.0, 10, total)
print(json.dumps({{"rank": rank, "world": world, "total": total, "value": value, "seed": bench._rank_seed(rank)}}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_max_time_and_job_value():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_CODE.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for d in outs:
        assert d["world"] == 2
        assert d["total"] == pytest.approx(11.5)                    # the slowest rank
        assert d["value"] == pytest.approx(2 * 2.0 * 10 / 11.5e-3)  # all ranks' work
    assert outs[0]["seed"] != outs[1]["seed"]                        # each rank its own image


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    assert res.stdout.strip() == ""


_SHARD_CODE = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import torch.distributed as dist
import synth
from oracle import COLUMN, ROW, Params, sgwls, sgwls_pass
from paper_1705_01674_gb300.shard import filter_sharded, split
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
H, W, r, T, order = {H}, {W}, {r}, {T}, {order}
F = synth.rgb_scene(H, W, seed=31, n_rect=10, n_disk=2)[:2].astype(np.float64)
G = synth.luminance(synth.rgb_scene(H, W, seed=31, n_rect=10, n_disk=2)).astype(np.float64)
prm = Params(r=r, iters=1, sigma_s=float(r), sigma_r=0.2)

def oracle_pass(U, Gs, lam, d):
    return torch.from_numpy(sgwls_pass(U.numpy(), Gs.numpy(), lam, prm, COLUMN if d == 0 else ROW))

a, b = split(W, world)[rank]
out = filter_sharded(torch.from_numpy(F[:, :, a:b].copy()), torch.from_numpy(G[:, a:b].copy()), 1.7, H, W,
                     oracle_pass, r=r, iters=T, axis_order=order)
ref = sgwls(F, G, 1.7, Params(r=r, iters=T, axis_order=order, sigma_s=float(r), sigma_r=0.2))
err = float(np.abs(out.numpy() - ref[:, :, a:b]).max())
print(json.dumps({{"rank": rank, "err": err, "cols": [a, b]}}))
dist.destroy_process_group()
"""


@pytest.mark.parametrize("world,H,W,r,T,order", [
    (2, 17, 23, 1, 2, 0),
    (3, 14, 19, 2, 1, 1),     # strips narrower than the 2r halo: blocks from two ranks away
    (3, 21, 30, 1, 2, 1),
])
def test_sharded_filter_equals_whole_image(world, H, W, r, T, order):
    """One image split into column strips over gloo ranks: every pass runs
    on each rank's strip plus a 2r halo, the ranks re-partition between
    directions, and the stitched result equals the whole-image filter (the
    oracle's pass is the per-rank compute here, on the CPU)."""
    pytest.importorskip("torch")
    port = _free_port()
    code = _SHARD_CODE.format(root=ROOT, H=H, W=W, r=r, T=T, order=order)
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-3000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    cols = sorted(tuple(d["cols"]) for d in outs)
    assert cols[0][0] == 0 and cols[-1][1] == W and all(cols[i][1] == cols[i + 1][0] for i in range(world - 1))
    for d in outs:
        assert d["err"] < 1e-12, d
