"""The multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2) on 127.0.0.1.

The GPU arm times N independent replicas and reports the slowest rank's time; the
reference arm runs on rank 0 only and the other ranks exit 0 without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench.dist_env()
    got = bench.max_over_ranks(1.5 + 2.0 * rank, w, device="cpu")
    out[rank] = (r, w, got)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gives_every_rank_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res == {0: (0, 2, 3.5), 1: (1, 2, 3.5)}


def test_max_over_ranks_single_rank_is_the_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.25, 1) == 0.25


def test_reference_arm_runs_on_rank_zero_only():
    """A rank other than 0 of the reference arm returns at once: exit 0, no JSON line."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert p.returncode == 0 and p.stdout.strip() == ""
