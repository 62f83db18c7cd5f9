"""The replica path of multi-GPU runs, on CPU: two gloo ranks shard a request
stream, take the max of their timings and pool their latencies."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2005_12764_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = list(range(11))
        mine = replicas.shard(items, rank, world)
        t = replicas.max_over_ranks(1.5 + rank, dist)
        s = replicas.sum_over_ranks(len(mine), dist)
        lat = replicas.gather_lists([rank * 100 + k for k in mine], dist)
        q.put((rank, mine, t, s, lat))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, s0, l0), (r1, m1, t1, s1, l1) = out
    assert sorted(m0 + m1) == list(range(11)) and not set(m0) & set(m1)
    assert t0 == t1 == 2.5                     # max over ranks
    assert s0 == s1 == 11                      # every item taken once
    assert l0 == l1 and sorted(l0) == sorted([k for k in m0] + [100 + k for k in m1])


def test_single_process_fallbacks():
    from paper_2005_12764_gb300 import replicas
    assert replicas.shard(range(5), 0, 1) == [0, 1, 2, 3, 4]
    assert replicas.max_over_ranks(3.0) == 3.0 and replicas.gather_lists([1, 2]) == [1, 2]
