"""The multi-process path on CPU (gloo, world size 2): sharding of an uneven
batch, max-over-ranks timing and summed work."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2001_07557_gb300 import dist as lqdist


def test_shard_by_cost_balances_and_covers():
    sizes = [8 ** 4, 12 ** 4, 16 ** 4, 20 ** 4]
    parts = lqdist.shard_by_cost(sizes, 2)
    assert sorted(i for p in parts for i in p) == [0, 1, 2, 3]
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) == 20 ** 4  # the largest lattice alone; the other three share the second rank
    assert lqdist.shard_by_cost(sizes, 1) == [[0, 1, 2, 3]]
    assert lqdist.shard_by_cost([1, 1, 1], 4)[3] == []
    with pytest.raises(ValueError):
        lqdist.shard_by_cost(sizes, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = lqdist.shard_by_cost([8 ** 4, 12 ** 4, 16 ** 4, 20 ** 4], world)
        mine = parts[rank]
        t = lqdist.job_time(1.0 + rank)            # rank 1 is the slowest
        w = lqdist.job_work(float(len(mine)))       # every lattice counted once
        q.put((rank, mine, t, w))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_job_accounting():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(i for _, mine, _, _ in res for i in mine) == [0, 1, 2, 3]
    assert all(t == 2.0 for _, _, t, _ in res)
    assert all(w == 4.0 for _, _, _, w in res)
