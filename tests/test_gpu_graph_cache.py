"""gee_embed's launch-graph cache: a repeated call replays a captured CUDA graph.  The
replay must give the bits of a direct launch and must read the inputs afresh."""
import numpy as np
import pytest

import oracle

from synth import chung_lu, sbm

from gpu_util import assert_z_matches, dev_graph

pytestmark = pytest.mark.gpu


def _call(gee, args, flags, Z, ws, status):
    src, dst, w, y, N, K = args
    opts = gee.make_opts(flags)
    rc = gee.gee_embed(src, dst, w, int(src.numel()), N, y, K, opts, Z, ws, ws.numel(), None, status)
    assert rc == 0, gee.gee_strerror(rc)


@pytest.mark.parametrize("make", [lambda: sbm(3000, seed=31, weighted=True),
                                  lambda: chung_lu(20000, 150000, seed=32, K=20)])
def test_replay_matches_direct_launch(make):
    import torch
    import paper_2406_03726_gb300 as gee
    g = make()
    src, dst, w, y = dev_graph(g)
    args = (src, dst, w, y, g.N, g.K)
    opts = gee.make_opts(gee.ALL_OPTIONS)
    n = gee.gee_workspace_size(g.E, g.N, g.K, g.weighted, opts)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    Zd = torch.empty((g.N, g.K), dtype=torch.float32, device="cuda")
    _call(gee, args, gee.ALL_OPTIONS | gee.NO_GRAPH_CACHE, Zd, ws, status)
    Zc = torch.empty_like(Zd)
    for _ in range(4):  # seen, captured, replayed twice
        Zc.fill_(float("nan"))
        status.fill_(-1)
        _call(gee, args, gee.ALL_OPTIONS, Zc, ws, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(Zc, Zd)
    assert_z_matches(Zc.cpu().numpy(), oracle.embed_graph(g, gee.ALL_OPTIONS), what="graph replay")
    assert gee.gee_graph_cache_clear() == 0


def test_replay_reads_new_inputs():
    import torch
    import paper_2406_03726_gb300 as gee
    g = sbm(2500, seed=33, weighted=True)
    src, dst, w, y = dev_graph(g)
    args = (src, dst, w, y, g.N, g.K)
    opts = gee.make_opts(gee.ALL_OPTIONS)
    ws = torch.empty(gee.gee_workspace_size(g.E, g.N, g.K, True, opts), dtype=torch.uint8, device="cuda")
    Z = torch.empty((g.N, g.K), dtype=torch.float32, device="cuda")
    for _ in range(3):
        _call(gee, args, gee.ALL_OPTIONS, Z, ws, None)
    torch.cuda.synchronize()
    assert_z_matches(Z.cpu().numpy(), oracle.embed_graph(g, gee.ALL_OPTIONS), what="before")
    # new contents at the same addresses: the next (replayed) call must see them
    rng = np.random.default_rng(34)
    g2_labels = rng.permutation(g.labels)
    g2_w = (rng.random(g.E) + 0.5).astype(np.float32)
    y.copy_(torch.from_numpy(g2_labels))
    w.copy_(torch.from_numpy(g2_w))
    _call(gee, args, gee.ALL_OPTIONS, Z, ws, None)
    torch.cuda.synchronize()
    g.labels, g.w = g2_labels, g2_w
    assert_z_matches(Z.cpu().numpy(), oracle.embed_graph(g, gee.ALL_OPTIONS), what="after new inputs")
    assert gee.gee_graph_cache_clear() == 0


def test_timed_replay_reports_phases():
    import torch
    import paper_2406_03726_gb300 as gee
    g = sbm(4000, seed=35, weighted=True)
    src, dst, w, y = dev_graph(g)
    opts = gee.make_opts(gee.ALL_OPTIONS)
    n = gee.gee_workspace_size(g.E, g.N, g.K, True, opts)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    Z = torch.empty((g.N, g.K), dtype=torch.float32, device="cuda")
    Zd = torch.empty_like(Z)
    gee.embed(src, dst, w, g.N, y, g.K, gee.ALL_OPTIONS | gee.NO_GRAPH_CACHE, Z=Zd)
    ran = None
    for it in range(4):  # direct, captured, replayed twice
        ph = np.full(len(gee.PHASES), -2.0, np.float32)
        Z.zero_()
        rc = gee.gee_embed_timed(src, dst, w, g.E, g.N, y, g.K, opts, Z, ws, n, None, None, ph)
        assert rc == 0
        assert torch.equal(Z, Zd)
        assert np.all((ph == -1.0) | (ph >= 0.0))
        if ran is None:
            ran = ph >= 0.0
        assert np.array_equal(ph >= 0.0, ran), f"call {it}: phases {ph}"
    assert ran[gee.PHASES.index("k_scatter_final")] and ran[gee.PHASES.index("k_spmm")]
    assert gee.gee_graph_cache_clear() == 0


def test_rows_per_item_is_part_of_the_cache_key():
    # the same buffers with a different rows_per_item must run (and cache) a new launch
    # plan, not replay the graph captured for the first value
    import torch
    import paper_2406_03726_gb300 as gee
    g = chung_lu(30000, 200000, seed=36, K=12)
    src, dst, w, y = dev_graph(g)
    assert gee.gee_graph_cache_clear() == 0
    n = max(gee.gee_workspace_size(g.E, g.N, g.K, False, gee.make_opts(gee.ALL_OPTIONS, 0, 0, r)) for r in (1, 8))
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    Z = {r: torch.empty((g.N, g.K), dtype=torch.float32, device="cuda") for r in (1, 8)}
    for r in (1, 8):
        opts = gee.make_opts(gee.ALL_OPTIONS, 0, 0, r)
        for _ in range(3):  # seen, captured, replayed
            rc = gee.gee_embed(src, dst, None, g.E, g.N, y, g.K, opts, Z[r], ws, n, None, None)
            assert rc == 0, gee.gee_strerror(rc)
    torch.cuda.synchronize()
    assert gee.gee_graph_cache_size() == (2, 2)
    # rows_per_item only groups rows into work items: the bits do not change
    assert torch.equal(Z[1], Z[8])
    assert_z_matches(Z[8].cpu().numpy(), oracle.embed_graph(g, gee.ALL_OPTIONS), what="rows_per_item 8")
    assert gee.gee_graph_cache_clear() == 0
    assert gee.gee_graph_cache_size() == (0, 0)
