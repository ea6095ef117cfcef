"""The replica timing path of bench.py across processes (gloo, CPU): every
rank reports its own step time and the job takes the maximum, so the
whole-job value is ranks x triangles / slowest rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    r, ws, local = bench.dist_setup(world)
    assert (r, ws, local) == (rank, world, rank)
    bench.dist_barrier(ws)
    ms = 1.0 + 2.5 * rank                      # rank 1 is the slow one
    out[rank] = bench.dist_max(ms, ws)
    import torch.distributed as dist

    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(90)
            assert p.exitcode == 0
        assert dict(out) == {0: 3.5, 1: 3.5}
