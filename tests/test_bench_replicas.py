"""CPU test of the multi-process (replica) path of bench.py with two gloo ranks: the job's
time is the slowest rank's and its throughput counts every rank's work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    mx = bench.max_over_ranks([1.0 + rank, 10.0 - rank], dist, "cpu")
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(" ".join(repr(v) for v in mx))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_max_and_throughput(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        vals = [float(v) for v in open(tmp_path / f"r{r}.txt").read().split()]
        assert vals == [2.0, 10.0]           # the slowest rank's times, on every rank
    import bench
    assert bench.job_gflops(2, 1e9, 2.0) == pytest.approx(1000.0)   # 2 ranks x 1 GFLOP in 2 ms
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]           # one process


def test_timed_region_lasts_about_a_second():
    """A short block of products is repeated until the timed region lasts ~1 s (so the 25 ms
    clock samples fall inside it); a block that already lasts that long runs once."""
    import bench
    assert bench.timed_repeats(20, 0.19) == 264          # 20 x 0.19 ms = 3.8 ms per block
    assert bench.timed_repeats(5000, 0.3) == 1           # 1.5 s already
    assert bench.timed_repeats(5000, 0.19) == 2          # 0.95 s: one more block
    assert bench.timed_repeats(0, 0.0) >= 1
    for steps, est in ((1, 0.005), (7, 0.12), (300, 1.1)):
        r = bench.timed_repeats(steps, est)
        assert r * steps * est * 1e-3 >= 1.0 > (r - 1) * steps * est * 1e-3
