"""The multi-rank path of bench.py on the CPU: two ranks over gloo (the GPU
runs use NCCL with the same calls).  The job's time is the slowest rank's,
every rank sees it, and the whole-job rate counts the pixels of all ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_CODE = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"])
dist.init_process_group("gloo")
dist.barrier()
t = bench.slowest_rank(10.0 * (rank + 1) + 0.25, "cpu")
rate = bench.job_rate(1000, 5, dist.get_world_size(), t)
dist.barrier()
print(json.dumps({"rank": rank, "t": t, "rate": rate}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_take_the_slowest_time():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_CODE, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["t"] == 20.25                       # the slower rank's time, on both ranks
        assert o["rate"] == pytest.approx(2 * 1000 * 5 / 0.02025, rel=1e-12)  # both ranks' pixels over that time


def test_single_process_is_unchanged():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank(12.5, "cpu") == 12.5
    assert bench.job_rate(8388608, 50, 1, 506.3) == pytest.approx(8388608 * 50 / 0.5063, rel=1e-12)
