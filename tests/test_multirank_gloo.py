"""The replica path of bench.py on two CPU ranks (gloo): the slowest rank's time is
taken, the whole-job value counts every rank's work over that time, and each rank
draws its own catalogues.  No GPU: the aggregation is host logic."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(100.0 + 25.0 * rank, world, torch.device("cpu"))
    v = bench.replica_value(512.0 ** 3, 240, 10, t, world)
    q.put((rank, t, v, bench.rank_seeds(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        rank, t, v, seeds = q.get(timeout=120)
        got[rank] = (t, v, seeds)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0][0] == got[1][0] == 125.0                      # max over ranks
    expect = 2 * 512.0 ** 3 * 240 * 10 / 0.125
    assert got[0][1] == pytest.approx(expect) and got[1][1] == pytest.approx(expect)
    assert all(got[0][2][k] != got[1][2][k] for k in got[0][2])  # independent catalogues per rank


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.replica_value(8.0, 2, 3, 1000.0, 1) == 48.0
