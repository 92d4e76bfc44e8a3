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


def _sweep_worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    from paper_1308_0692_gb300 import sweep
    dist.init_process_group(backend="gloo")
    idx = sweep.shard(10, rank, world)
    # a stand-in for one rank's sweep report over its share (no GPU work here)
    rep = {"seed": 1, "unknowns": 100 * len(idx), "schedule": {"rank": rank},
           "tune_seconds": 1.0 + rank, "batch_seconds": 10.0 * (rank + 1), "refine_seconds": 2.0,
           "reference_seconds": 3.0,
           "per_instance": [{"index": i, "steps": 100 + i, **({"err": {"u": 1e-7 * i, "wall_shear": 1e-8}} if i % 3 else {})}
                            for i in idx]}
    reps = [None] * world
    dist.all_gather_object(reps, rep)
    merged = sweep.merge_reports(reps)
    dist.destroy_process_group()
    out.put((rank, idx, merged["count"], [r["index"] for r in merged["per_instance"]], merged["batch_seconds"],
             merged["unknowns"], merged["instances_checked"], merged["max_velocity_error"]))


def test_sweep_shards_round_robin_and_rank0_gathers():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sweep_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(2)])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, idx0, n0, order0, t0, u0, c0, e0), (r1, idx1, n1, order1, t1, u1, c1, e1) = res
    assert idx0 == [0, 2, 4, 6, 8] and idx1 == [1, 3, 5, 7, 9]     # disjoint, same size mix
    assert n0 == n1 == 10 and order0 == order1 == list(range(10))
    assert t0 == t1 == 20.0                                         # slowest rank's time
    assert u0 == 1000 and c0 == 6 and abs(e0 - 8e-7) < 1e-20
