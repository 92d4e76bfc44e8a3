"""The multi-rank path of bench.py on CPU (gloo, world size 2): ranks run independent
replicas, the only collectives are the timing barrier and the max/sum reductions, and the
whole-job value is all ranks' units divided by the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    d = bench.Dist(backend="gloo")
    d.barrier()
    units = 1000.0 * (rank + 1)          # uneven work per rank
    seconds = 2.0 if rank == 0 else 5.0  # rank 1 is the slowest
    value, tmax = bench.aggregate(units, seconds, d)
    out.put((rank, value, tmax, d.world, d.rank))
    d.close()


def test_two_rank_aggregate_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tmax, world, r in res:
        assert world == 2 and r == rank
        assert tmax == 5.0                       # max over ranks
        assert abs(value - 3000.0 / 5.0) < 1e-9  # all ranks' units / slowest time


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    d = bench.Dist()
    assert d.world == 1 and d.pg is None
    value, t = bench.aggregate(10.0, 2.0, d)
    assert value == 5.0 and t == 2.0
