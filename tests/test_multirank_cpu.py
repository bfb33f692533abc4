"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

Each rank is an independent replica; the job time is the slowest rank and
the job throughput counts every rank's units.  No GPU is used."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    r = bench.Ranks(world, "gloo", None)
    r.barrier()
    t = r.max(1.0 + rank)  # rank 1 is slower
    rate = r.job_rate(100.0, t)
    info = bench.dist_info()
    r.close()
    out.put((rank, t, rate, info))


def test_two_rank_replicas_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate, info in res:
        assert t == 2.0  # max over ranks
        assert rate == pytest.approx(100.0 * 2 / 2.0)  # whole-job units / slowest time
        assert info == (rank, 2, rank)


def test_single_rank_is_plain():
    import bench

    r = bench.Ranks(1)
    assert r.max(3.5) == 3.5
    assert r.job_rate(10.0, 2.0) == 5.0
    r.barrier()
    r.close()
