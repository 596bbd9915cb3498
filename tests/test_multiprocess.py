"""Multi-process (replica) bookkeeping of bench.py on CPU with the gloo backend.

The Lanczos chains of different GPUs are independent (the paper's parallel
scaling over q is linear): ranks share no data, only the timing reduction.
These tests run two gloo ranks on the CPU: the slowest rank's time is what every
rank sees, the whole-job rate counts every rank's chains, and the reference arm
does its work on rank 0 only.
"""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    wall = 1.0 + 0.5 * rank  # rank 1 is the slow one
    m = bench.max_over_ranks(wall, "cpu")
    rate = bench.whole_job_rate(world, 3, 10, m)
    dist.barrier()
    q.put((rank, m, rate))
    dist.destroy_process_group()


def test_timing_reduction_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [1.5, 1.5]
    assert out[0][2] == pytest.approx(2 * 3 * 10 / 1.5)


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, "cpu") == 2.5
    assert bench.whole_job_rate(1, 3, 10, 2.0) == 15.0


def test_reference_arm_rank1_exits_without_work():
    """Under a launcher the non-zero ranks of the reference arm print nothing and exit 0."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
