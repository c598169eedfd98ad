"""Row-sharded embedding of one graph, host side (CPU only).

* row_ranges (the partition the library's multi-GPU driver uses): contiguous, covering,
  balanced by edge count.
* The row-range form of the FP64 oracle, stitched over ranks, equals the whole-graph
  oracle: rows are independent once the class sizes and the node table are known.
* Two gloo ranks run the driver's exchange (all-reduce of n_k, all-gather of the node
  table, then each rank's rows) with the oracle's row-range form, and the stitched Z
  equals the whole-graph oracle.
"""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from oracle import shard as oshard
from synth import chung_lu, random_tiny, sbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2406_03726_gb300.shard import edges_of_rows, row_ranges  # noqa: E402


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_row_ranges_cover_and_balance(world):
    g = chung_lu(5000, 40000, seed=71, K=5)
    counts = np.bincount(g.src, minlength=g.N)
    rr = row_ranges(counts, world)
    assert len(rr) == world and rr[0][0] == 0 and rr[-1][1] == g.N
    assert all(a[1] == b[0] for a, b in zip(rr, rr[1:])) and all(r0 <= r1 for r0, r1 in rr)
    loads = [int(counts[r0:r1].sum()) for r0, r1 in rr]
    assert sum(loads) == g.E
    # each range ends at the first row that reaches its share: at most one row over it
    assert max(loads) <= g.E / world + counts.max()


def test_row_ranges_degenerate():
    assert row_ranges(np.zeros(0, np.int64), 3) == [(0, 0), (0, 0), (0, 0)]
    assert row_ranges(np.array([0, 0, 5]), 2)[-1][1] == 3
    with pytest.raises(ValueError):
        row_ranges(np.ones(4), 0)


def _stitched(g, flags, world):
    counts = np.bincount(g.src, minlength=g.N)
    rr = row_ranges(counts, world)
    parts = [edges_of_rows(g.src, r0, r1) for r0, r1 in rr]
    nk = sum(oshard.partial_label_counts(g.labels[r0:r1], g.K) for r0, r1 in rr)
    degs = [oshard.row_degrees(g.src[e], None if g.w is None else g.w[e], r0, r1, flags) for (r0, r1), e in
            zip(rr, parts)]
    tabs = [oshard.node_table(g.labels[r0:r1], d, nk, flags) for (r0, r1), d in zip(rr, degs)]
    y_all = np.concatenate([t[0] for t in tabs])
    s_all = np.concatenate([t[1] for t in tabs])
    Zs = [oshard.rows(g.src[e], g.dst[e], None if g.w is None else g.w[e], r0, r1, y_all, s_all, d, g.K, flags)
          for (r0, r1), e, d in zip(rr, parts, degs)]
    return np.concatenate(Zs) if Zs else np.zeros((0, g.K))


@pytest.mark.parametrize("seed", range(8))
def test_oracle_rows_stitch_to_the_whole(seed):
    g = random_tiny(seed, n_max=60, e_max=400)
    for flags in range(8):
        Z = oracle.embed_graph(g, flags)
        for world in (1, 2, 3):
            Zs = _stitched(g, flags, world)
            scale = max(1.0, float(np.abs(Z).max(initial=0.0)))
            assert np.abs(Zs - Z).max(initial=0.0) <= 1e-12 * scale, (flags, world)
            assert np.array_equal(Zs == 0, Z == 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import shard as osh
    from paper_2406_03726_gb300.shard import edges_of_rows, row_ranges
    from synth import sbm as make
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = make(900, seed=72, weighted=True)        # every rank draws the same graph ...
        flags = 7
        # ... and takes its rows [r0, r1) of the edge-balanced ranges, and their edges
        counts = torch.from_numpy(np.bincount(g.src[edges_of_rows(g.src, 0, g.N)], minlength=g.N))
        rr = row_ranges(counts.numpy(), world)
        r0, r1 = rr[rank]
        e = edges_of_rows(g.src, r0, r1)
        src, dst, w = g.src[e], g.dst[e], g.w[e]
        # 1. partial class sizes, summed over the ranks
        nk = torch.from_numpy(osh.partial_label_counts(g.labels[r0:r1], g.K))
        dist.all_reduce(nk, op=dist.ReduceOp.SUM)
        # 2. this rank's node table entries, gathered in rank (= row) order
        deg = osh.row_degrees(src, w, r0, r1, flags)
        y, s = osh.node_table(g.labels[r0:r1], deg, nk.numpy(), flags)
        cap = max(r1_ - r0_ for r0_, r1_ in rr)
        mine = torch.zeros((cap, 2), dtype=torch.float64)
        mine[:r1 - r0, 0] = torch.from_numpy(y.astype(np.float64))
        mine[:r1 - r0, 1] = torch.from_numpy(s)
        allt = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(allt, mine)
        tab = torch.cat([allt[r][: rr[r][1] - rr[r][0]] for r in range(world)]).numpy()
        # 3. this rank's rows of Z, then all of them at rank 0
        Z = osh.rows(src, dst, w, r0, r1, tab[:, 0].astype(np.int64), tab[:, 1], deg, g.K, flags)
        Zp = torch.zeros((cap, g.K), dtype=torch.float64)
        Zp[:r1 - r0] = torch.from_numpy(Z)
        allz = [torch.zeros_like(Zp) for _ in range(world)]
        dist.all_gather(allz, Zp)
        if rank == 0:
            Zall = torch.cat([allz[r][: rr[r][1] - rr[r][0]] for r in range(world)]).numpy()
            q.put((rank, Zall, rr))
        else:
            q.put((rank, None, rr))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_stitch_to_the_whole_oracle():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in range(world)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    Zall, rr = out[0][1], out[0][2]
    assert rr == out[1][2] and rr[0][1] > 0 and rr[1][1] - rr[1][0] > 0   # both ranks hold rows
    g = sbm(900, seed=72, weighted=True)
    Z = oracle.embed_graph(g, 7)
    assert np.abs(Zall - Z).max() <= 1e-12
