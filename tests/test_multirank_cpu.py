"""The benchmark's multi-rank path on CPU: two gloo ranks, one box per rank (or a
round-robin share of independent boxes), no data-path communication; the only
collectives are the max over ranks of the time and the sum of the work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, t_max, pairs = bench.aggregate_over_ranks(1000.0 * (rank + 1), 0.5 + rank, "cpu")
    shards = bench.shard_boxes(list(range(11)), rank, world)
    dist.barrier()
    q.put((rank, value, t_max, pairs, shards))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    world = 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, q), nprocs=world, join=True, start_method="spawn")
    res = sorted(q.get() for _ in range(world))
    for rank, value, t_max, pairs, _ in res:
        assert t_max == pytest.approx(1.5)
        assert pairs == pytest.approx(3000.0)
        assert value == pytest.approx(3000.0 / 1.5)
    a, b = res[0][4], res[1][4]
    assert sorted(a + b) == list(range(11)) and not set(a) & set(b)


def test_single_process_aggregate_is_local():
    import bench
    assert bench.aggregate_over_ranks(10.0, 2.0, "cpu") == (5.0, 2.0, 10.0)
