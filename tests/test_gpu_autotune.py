"""The autotuner's choice against pinned geometries.

The autotuner (jac_opts.autotune) times every candidate kernel geometry on the
matrix and keeps the fastest, with a cost-model prior that another candidate
must beat by more than 5 %.  Its choice must be stable: on the FE-like
27-point 128^3 system in mixed precision (the case whose choice swung between
geometries 2.6x apart when each candidate was timed once), the autotuned solve
to 1e-10 must run within 10 % of the fastest of the best pinned geometries.
JAC_AUTOTUNE_LOG=1 makes the library print each candidate's timing, from
which the three fastest candidates are taken and set up pinned.
"""
import re
import statistics

import numpy as np
import pytest

from paper_2112_02377_gb300 import jacobi as J
from paper_2112_02377_gb300 import workloads as W

pytestmark = pytest.mark.gpu

_LINE = re.compile(r"autotune: variant (\d+) rows (\d+) ctas/SM (\d+) lanes (\d+) sync (\d+) stages (\d+): "
                   r"([0-9.]+) us/sweep")


def _solve_ms(ctx, reps=3):
    ms = []
    for _ in range(reps):
        J.jac_set_x(ctx, None)
        k, rel, st = J.jac_solve(ctx, 1e-10, 200000)
        assert st == J.JAC_OK and rel <= 1e-10
        ms.append(J.jac_stats(ctx)["last_ms"])
    return statistics.median(ms)


def test_fe27_mixed_autotuned_geometry_is_within_10_percent_of_the_best_pinned(monkeypatch, capfd):
    monkeypatch.setenv("JAC_AUTOTUNE_LOG", "1")
    A = W.fe27_deleted(128, seed=0)
    xs, b = W.solution_and_rhs(A, 0)
    common = dict(precision=J.JAC_MIXED, inner_sweeps=128, sweeps_per_graph=256)
    capfd.readouterr()
    ctx = J.jac_setup(A, b, J.JAC_BANDROW_NNZ, 64, J.opts(autotune=1, **common))
    try:
        log = capfd.readouterr().err
        auto_ms = _solve_ms(ctx)
    finally:
        J.jac_free(ctx)
    cands = []
    for m in _LINE.finditer(log):
        v, rows, cps, lanes, sync, stages = (int(g) for g in m.groups()[:6])
        cands.append((float(m.group(7)), v, rows, cps, lanes, stages))
    assert len(cands) >= 5, log
    cands.sort()
    pinned = []
    for us, v, rows, cps, lanes, stages in cands[:3]:
        o = dict(variant=v, tile_rows=rows, **common)
        if v == 2 and rows == 256:
            o.update(ctas_per_sm=cps, lanes_per_row=lanes, stages=stages if cps == 2 else 0)
        c = J.jac_setup(A, b, J.JAC_BANDROW_NNZ, 64, J.opts(**o))
        try:
            pinned.append(_solve_ms(c))
        finally:
            J.jac_free(c)
    assert auto_ms <= 1.10 * min(pinned), (auto_ms, pinned)
