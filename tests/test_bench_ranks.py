"""The N > 1 path of bench.py on CPU (two gloo ranks): every rank times its
own independent particle set, the job's time is the slowest rank's (max over
ranks), throughput counts the units of all ranks, and the reference arm runs
on rank 0 only.  The GPU step itself is one process per GPU with no data-path
collective (replicas), so only this host logic is shared between ranks."""
import io
import os
import socket
import sys
import types
from contextlib import redirect_stdout

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], world, dist, "cpu")
        out[rank] = t
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world, port = 2, _free_port()
    times = [3.5, 7.25]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, times, out), nprocs=world, join=True)
        got = [out[r] for r in range(world)]
    assert got == [7.25, 7.25]
    # whole-job rate: both ranks' particles over the slowest rank's time
    assert bench.job_rate(bench.N_PART, world, 7.25e-3) == pytest.approx(2 * bench.N_PART / 7.25e-3)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(4.0, 1, None, "cpu") == 4.0
    assert bench.job_rate(100, 1, 2.0) == 50.0


def test_ranks_draw_independent_sets():
    from paper_1811_06332_gb300 import inputs
    a = inputs.uniform_cube(1024, bench.rank_seed(0))
    b = inputs.uniform_cube(1024, bench.rank_seed(1))
    assert bench.rank_seed(0) != bench.rank_seed(1)
    assert not np.array_equal(a[0], b[0])


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    args = types.SimpleNamespace(steps=1, warmup=0, gpus=2)
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    assert buf.getvalue() == ""
