"""The N > 1 placement path on the CPU: two gloo ranks shard a set of
independent networks round robin (no collective on the data path), contract
their shards with the CPU oracle, and reduce the elapsed time with a max."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2501_00227_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import graphgen as g
        import oracle as O
        mine = shard.shard(10, rank, world)
        results = {}
        for i in mine:
            n, e = g.random_regular3(12 + 2 * (i % 3), 100 + i)
            o = O.greedy_order(n, e, nrepeat=1, seed=1)
            results[i] = O.mis_count(n, e, o)
        t = shard.max_over_ranks(float(rank + 1), dist)
        gathered = [None] * world
        dist.all_gather_object(gathered, results)
        out.put((rank, t, gathered))
    finally:
        dist.destroy_process_group()


def test_shard_round_robin():
    assert shard.shard(10, 0, 2) == [0, 2, 4, 6, 8]
    assert shard.shard(10, 1, 2) == [1, 3, 5, 7, 9]
    assert sorted(sum((shard.shard(7, r, 3) for r in range(3)), [])) == list(range(7))
    with pytest.raises(ValueError):
        shard.shard(4, 2, 2)
    assert shard.max_over_ranks(3.5) == 3.5


def test_two_gloo_ranks_shard_and_reduce():
    import oracle as O
    import graphgen as g
    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, gathered in got:
        assert t == 2.0                            # max over ranks of rank + 1
        merged = {}
        for part in gathered:
            merged.update(part)
        assert sorted(merged) == list(range(10))   # every unit exactly once
        for i, (size, cnt) in merged.items():
            n, e = g.random_regular3(12 + 2 * (i % 3), 100 + i)
            poly = O.bruteforce_poly(n, e)
            alpha = max(k for k, c in enumerate(poly) if c)
            assert (size, cnt) == (alpha, poly[alpha])
