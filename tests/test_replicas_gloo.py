"""The N > 1 path (independent replicas) on CPU: two gloo ranks on 127.0.0.1."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_1411_3769_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = list(range(11))
        mine = replicas.shard(items, rank, world)
        everyone = replicas.gather(mine, dist)
        slowest = replicas.max_over_ranks(1.0 + rank, dist)          # rank 1 is the slowest
        thr = replicas.weak_throughput(10.0, 1.0 + rank, dist)       # 2 ranks x 10 units / 2 s
        q.put((rank, mine, everyone, slowest, thr))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    all_items = sorted(x for r in res.values() for x in r[1])
    assert all_items == list(range(11))                 # every instance exactly once
    for r in res.values():
        assert r[2] == [res[0][1], res[1][1]]            # gather in rank order
        assert r[3] == 2.0                               # max over ranks
        assert r[4] == pytest.approx(10.0)               # 20 units / 2 s


def test_single_process_fallbacks():
    from paper_1411_3769_gb300 import replicas
    assert replicas.shard(range(5), 0, 1) == [0, 1, 2, 3, 4]
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.weak_throughput(4.0, 2.0) == 2.0
    assert replicas.gather("x") == ["x"]
    with pytest.raises(ValueError):
        replicas.shard(range(5), 2, 2)
