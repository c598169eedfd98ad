"""The N > 1 path of bench.py on CPU: two gloo ranks, one graph each (replicas, no
data-path collective); the job's time is the slowest rank's and its work both graphs."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        import bench
        ws, r, local = bench.dist_info()
        g = bench.make_graph("sbm2k", r)
        ms, e_job = bench.reduce_over_ranks(10.0 + 5.0 * r, g.E, "cpu")
        q.put((r, ws, local, ms, e_job, g.E, int(g.src[:64].sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (r0, ws0, l0, ms0, ej0, e0, h0), (r1, ws1, l1, ms1, ej1, e1, h1) = out
    assert (r0, r1, ws0, ws1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert ms0 == ms1 == 15.0                 # the slowest rank's time
    assert ej0 == ej1 == e0 + e1              # both ranks' edges
    assert h0 != h1                           # each rank embeds its own graph


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload, steps, warmup, gpus = "sbm2k", 1, 0, 2
    assert bench.reference_arm(A()) == 0
    assert capsys.readouterr().out == ""       # rank 1 prints nothing and does no work
