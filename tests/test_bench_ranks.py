"""The bench's multi-rank aggregation (one process per GPU, weak scaling):
whole-job rate = units of all ranks / the slowest rank's time.  Run as two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed (r + 1) * 100 units in (r + 1) * 2 seconds
        rate, max_s, units = bench.whole_job_rate((rank + 1) * 100.0, (rank + 1) * 2.0, dist, "cpu")
        q.put((rank, rate, max_s, units))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, max_s, units in res:
        assert units == 300.0 and max_s == 4.0 and rate == pytest.approx(75.0)


def test_whole_job_rate_without_a_process_group():
    assert bench.whole_job_rate(10.0, 4.0) == (2.5, 4.0, 10.0)
