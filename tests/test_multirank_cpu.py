"""Host-side multi-rank logic of bench.py on CPU: two gloo ranks, barrier,
max-over-ranks timing and whole-job throughput (replicas, no data collective)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    assert bench.dist_env() == (rank, world, rank)
    d = bench.init_dist(world, "gloo")
    bench.barrier(d)
    t_local = 1.0 + rank          # rank 1 is the slow one
    tmax = bench.max_over_ranks(d, t_local)
    out[rank] = (tmax, bench.aggregate_throughput(100.0, tmax, world))
    bench.barrier(d)
    d.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    for r in range(2):
        tmax, thr = res[r]
        assert tmax == 2.0                    # the slowest rank sets the time
        assert thr == pytest.approx(100.0 * 2 / 2.0)


def test_single_rank_is_identity():
    import bench
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.aggregate_throughput(10.0, 2.0, 1) == 5.0
