"""The multi-rank benchmark path on CPU: two gloo ranks, each with its own batch of
independent problems (seed 2007 + rank), exchange only the elapsed time (max) and the
point-update count (sum) -- the weak-scaling aggregation bench.py uses under torchrun."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        members = bench._members(rank)
        info = bench._batch_points(members)
        local_upd = sum(n for _, n in info) * 100  # pretend every member took 100 steps
        local_ms = 1000.0 + 250.0 * rank
        q.put((rank, bench.aggregate(local_ms, local_upd, dist, "cpu"), local_upd,
               [(m.nr, m.nl, m.a) for m in members[:3]]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_weak_scaling():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (_, (ms0, upd0), l0, m0), (_, (ms1, upd1), l1, m1) = out
    assert ms0 == ms1 == 1250.0            # max over ranks
    assert upd0 == upd1 == float(l0 + l1)  # sum over ranks
    assert m0 != m1                        # each rank draws its own members
