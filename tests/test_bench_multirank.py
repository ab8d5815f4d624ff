"""bench.py's multi-GPU form is N independent replicas (the path has no
exchange step): each rank times its own replica, the job time is the maximum
over ranks, and the whole-job rate counts every rank's work.  Checked here
with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank 1 is the slow one on the device clock, rank 0 on the wall clock
    mine = [1.0 + rank, 3.0 - rank]
    got = bench.max_over_ranks(mine, world, device="cpu")
    out[rank] = (got, bench.whole_job_rate(4.0e9, world, got[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_with_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        got, rate = res[r]
        assert got == [2.0, 3.0]
        assert rate == pytest.approx(2 * 4.0e9 / (2.0 * 1e9))


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.whole_job_rate(1e9, 1, 1.0) == 1.0
