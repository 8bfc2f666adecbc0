"""The work-queue order of the queue-scheduled pass, checked on the host:
tests/sched_check.cpp includes the scheduling header the kernel uses
(paper_1705_01674_gb300/csrc/sgwls_sched.h), is built with the host C++
compiler and verifies, over image widths 3 .. 4099, radii 1 .. 8, chunk
group counts, look-aheads and ring sizes, that every work item is decoded
exactly once, that every wait of the kernel is on an item placed earlier
in the queue (so no wait can be circular), and that the reader counts the
ring relies on match the items that read each band."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_queue_schedule_properties(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "sched_check")
    subprocess.run([cxx, "-O2", "-std=c++17", os.path.join(HERE, "sched_check.cpp"), "-o", exe], check=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-2000:]
    assert res.stdout.startswith("ok")
