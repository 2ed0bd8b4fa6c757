"""The N > 1 launch of bench.py on the host: ranks are independent solves, so the only
cross-rank steps are the barrier and the max-over-ranks of the timed region, and rank 0 alone
prints. Checked here with two gloo ranks on the CPU (no GPU): the max-over-ranks helper, the
whole-job value, and the reference arm's rank handling."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")

WORKER = r"""
import os, sys
sys.path.insert(0, os.environ["ABG_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
t = bench.max_over_ranks(1.5 + rank, dist, "cpu")   # rank r took 1.5 + r seconds
dist.barrier()
assert t == 1.5 + (world - 1), t
assert bench.job_value(world, 5, t) == world * 5 / t
print(f"rank {rank} ok {t}")
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_two_gloo_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), ABG_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    for r, (p, out) in enumerate(zip(procs, outs)):
        assert p.returncode == 0, out
        assert f"rank {r} ok 2.5" in out


def test_single_process_helpers():
    import importlib
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.job_value(1, 5, 2.0) == 2.5


def test_reference_arm_other_ranks_exit_without_work():
    # under torchrun only rank 0 times and prints the reference arm; rank 1 exits 0 at once
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "0"], env=env,
                         capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""
