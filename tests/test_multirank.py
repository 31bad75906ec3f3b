"""The multi-process path of bench.py on CPU: two gloo ranks (127.0.0.1), each with its own
problem, the job time taken as the maximum over ranks and the throughput counting the
systems of every rank (weak scaling, no collective on the data path)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from paper_2203_11154_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.rank_seed("paradiag-511", rank)
        f, u0 = inputs.paradiag_problem(7, 4, seed=seed)
        ms_local = 10.0 + 5.0 * rank  # this rank's time for its steps
        ms = bench.max_over_ranks(ms_local, world, "cpu")
        value = bench.job_throughput(4, 3, world, ms)
        out[rank] = (seed, float(f[0, 0, 0]), ms, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    (s0, f0, ms0, v0), (s1, f1, ms1, v1) = res[0], res[1]
    assert s1 == s0 + 1 and f0 != f1          # independent problems per rank
    assert ms0 == ms1 == 15.0                 # the slowest rank's time, on every rank
    assert v0 == v1 == pytest.approx(4 * 3 * 2 / 0.015)  # systems of all ranks


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_throughput(64, 5, 1, 1000.0) == pytest.approx(320.0)
