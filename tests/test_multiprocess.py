"""The multi-rank host logic (problem sharding, max-over-ranks timing) with two
gloo processes on the CPU."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

from paper_2203_10477_gb300 import inputs
from paper_2203_10477_gb300.shard import max_over_ranks, shard_problems, sum_over_ranks


def test_shard_covers_every_problem_once_and_balances():
    tab = inputs.c3_table(4096)
    sizes = tab["nx"]
    for world in (1, 2, 3, 4, 8):
        parts = [shard_problems(sizes, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [int(np.sum(sizes[p])) for p in parts]
        assert max(loads) - min(loads) <= int(sizes.max())
    with pytest.raises(ValueError):
        shard_problems(sizes, 2, 2)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = inputs.c3_table(64)["nx"]
        mine = shard_problems(sizes, rank, world)
        work = float(np.sum(sizes[mine]))
        tmax = max_over_ranks([1.0 + rank, 10.0 - rank], dist)
        tot = sum_over_ranks([work, len(mine)], dist)
        q.put((rank, tmax, tot, mine))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    sizes = inputs.c3_table(64)["nx"]
    for rank, tmax, tot, mine in res:
        assert tmax == [2.0, 10.0]
        assert tot[0] == float(np.sum(sizes)) and tot[1] == 64.0
    assert sorted(res[0][3] + res[1][3]) == list(range(64))
