"""The benchmark's multi-rank path on CPU: two gloo ranks (replicas), the job time
is the slowest rank's and the throughput counts both ranks' analyses."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_ms = 100.0 if rank == 0 else 250.0
    t_max, value = bench.aggregate_ranks(t_ms, steps=10, world=world, device="cpu")
    q.put((rank, t_max, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, value in out:
        assert t_max == 250.0
        assert value == pytest.approx(2 * 10 / 0.25)


def test_single_rank_is_plain_throughput():
    sys.path.insert(0, ROOT)
    import bench
    t_max, value = bench.aggregate_ranks(50.0, steps=5, world=1)
    assert t_max == 50.0 and value == pytest.approx(100.0)
