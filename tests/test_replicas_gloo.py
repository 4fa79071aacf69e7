"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the path shards into
independent replicas (no data-path collective), so what N > 1 adds is the seed partition, the
max-over-ranks timing and the reference arm's rank-0-only rule."""

import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    seeds = bench.replica_seeds(rank, 4)
    # per-rank "times": the reduction must return the largest
    t = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out[rank] = (t, gathered)
    dist.destroy_process_group()


def test_seed_partition_and_max_over_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, gathered = res[rank]
        assert t == 11.0
        flat = [s for g in gathered for s in g]
        assert len(flat) == len(set(flat)) == 8
        assert gathered[0] == [3000, 3001, 3002, 3003] and gathered[1] == [3004, 3005, 3006, 3007]


def test_max_over_ranks_without_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
