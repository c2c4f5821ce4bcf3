"""The benchmark's multi-rank framing on CPU: two gloo ranks, each rendering its own view,
combine their timings (max over ranks) and their query counts (sum over ranks).  The
data path has no collective; only these reductions frame the measurement."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), RPNN_BENCH_BACKEND="gloo")
    import bench
    ws, r, local = bench.dist_init()
    assert (ws, r, local) == (world, rank, rank)
    t = bench.max_over_ranks(10.0 * (rank + 1), ws, "cpu")
    q = bench.sum_over_ranks(1000.0 + rank, ws, "cpu")
    bench.barrier(ws)
    out[rank] = (t, q)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_ranks_reduce_time_and_queries():
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(world):
            assert out[r] == (20.0, 2001.0)


def test_single_rank_is_identity(monkeypatch):
    import bench
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    ws, r, local = bench.dist_init()
    assert (ws, r, local) == (1, 0, 0)
    assert bench.max_over_ranks(3.5, ws, "cpu") == 3.5
    assert bench.sum_over_ranks(7.0, ws, "cpu") == 7.0
