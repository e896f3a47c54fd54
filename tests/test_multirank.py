"""The multi-rank host logic on CPU with two gloo ranks: max-over-ranks timing, the
barrier, and the sharding of independent instances (no GPU, no NCCL)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    from paper_1211_6932_gb300.sharding import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        m = bench.max_over_ranks(1.5 + rank, world)
        weights = [(7 * i) % 13 + 1 for i in range(40)]
        mine = shard(weights, world, rank)
        q.put((rank, m, mine, sum(weights[i] for i in mine)))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r, m, mine, w = q.get(timeout=120)
        out[r] = (m, mine, w)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 2.5  # the slower rank's time, on every rank
    allidx = sorted(out[0][1] + out[1][1])
    assert allidx == list(range(40))  # every instance exactly once
    assert out[0][1] == list(range(len(out[0][1])))  # contiguous
    assert abs(out[0][2] - out[1][2]) <= 13  # within one instance's weight


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_partitions_and_balances(world):
    from paper_1211_6932_gb300.sharding import shard
    weights = [64 * 64, 512 * 300, 100 * 77, 480 * 480, 70 * 500] * 20
    parts = [shard(weights, world, r) for r in range(world)]
    assert sorted(i for p in parts for i in p) == list(range(len(weights)))
    loads = [sum(weights[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(weights)
    with pytest.raises(ValueError):
        shard(weights, world, world)
