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


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the CPU oracle on the benchmark's
    workload) prints exactly one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_roofline_fields_name_the_binding_floor():
    peak, _ = bench._measured_peak()
    # memory-bound case: 1 GB, few FP64 instructions
    f = bench._roofline_fields(1e9, 1e9 / (peak * 1e9) * 1e6 / 0.8, 1e6)
    assert f["bound"] == "hbm" and f["frac_of_bound"] == pytest.approx(0.8, rel=1e-3)
    # FP64-bound case: the instructions need longer than the bytes
    t_f64 = 1e9 / bench.FP64_PIPE_PER_S * 1e6
    f = bench._roofline_fields(1e6, t_f64 / 0.5, 1e9)
    assert f["bound"] == "fp64" and f["frac_of_bound"] == pytest.approx(0.5, rel=1e-3)
