"""The benchmark's multi-rank aggregation on CPU with gloo, world size 2: the whole-job time
is the slowest rank's, the walker-moves are summed over ranks (one independent inversion per
rank, no data-path collective); a rank that dies between steps makes the survivor's next
collective end with an error within the process group's time-out instead of hanging."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [1200.0, 1500.0][rank]
    moves = [4.096e9, 3.0e9][rank]
    q.put((rank, bench.aggregate(ms, moves, dist, "cpu")))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, total, value = out[r]
        assert ms == 1500.0
        assert total == pytest.approx(7.096e9)
        assert value == pytest.approx(7.096e9 / 1.5)


def test_aggregate_single_rank():
    import bench
    ms, total, value = bench.aggregate(2000.0, 1e9)
    assert (ms, total) == (2000.0, 1e9) and value == pytest.approx(5e8)


def _rank_dies(rank, world, port, q):
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)            # a rank that fails between steps, with no collective in flight
    import bench
    try:
        bench.aggregate(1200.0, 4.096e9, dist, "cpu")
        q.put("returned")
    except Exception as e:     # the survivor's next collective ends with an error, not a hang
        q.put("error: " + type(e).__name__)


def test_a_dead_rank_ends_the_next_collective_with_an_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_dies, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    msg = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert msg.startswith("error"), msg
    assert procs[1].exitcode == 3
