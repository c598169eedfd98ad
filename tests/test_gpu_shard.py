"""Row shards of one graph through the library (gee_shard_build / _table / _embed).

The ranks run one after another in this process; their exchange (the sum of the class
sizes, the concatenation of the node-table slices) is done here on the host between the
library calls, exactly where a multi-GPU run puts its all-reduce and all-gather.  No
kernel waits on another rank.  The stitched rows must match the oracle and gee_embed of
the whole graph within the tolerance (not bit for bit: a row that several lanes share is
split among them by its entries' positions in the CSR, and a shard's CSR places the row
elsewhere than the whole graph's)."""
import numpy as np
import pytest

import oracle
from paper_2406_03726_gb300.shard import edges_of_rows, row_ranges
from synth import chung_lu, sbm

from gpu_util import assert_z_matches

pytestmark = pytest.mark.gpu

ALL = 7


def _sharded(gee, g, world, opts):
    import torch
    counts = np.bincount(g.src, minlength=g.N)
    rr = row_ranges(counts, world)
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ranks = []
    nk = torch.zeros(g.K, dtype=torch.int32, device="cuda")
    for (r0, r1) in rr:                               # 1. build, partial n_k
        e = edges_of_rows(g.src, r0, r1)
        d = dict(r0=r0, r1=r1, src=t(g.src[e]), dst=t(g.dst[e]), w=None if g.w is None else t(g.w[e]),
                 y=t(g.labels[r0:r1]), E=len(e))
        n = gee.gee_shard_workspace_size(d["E"], g.N, r0, r1, g.K, g.weighted, opts)
        assert n > 0
        d["ws"], d["n"] = torch.empty(n, dtype=torch.uint8, device="cuda"), n
        part = torch.zeros(g.K, dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc = gee.gee_shard_build(d["src"], d["dst"], d["w"], d["E"], g.N, r0, r1, d["y"], g.K, opts, part, d["ws"],
                                 n, None, st)
        assert rc == 0, gee.gee_strerror(rc)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        nk += part                                    # 2. the all-reduce
        ranks.append(d)
    tabs = []
    for d in ranks:                                   # 3. node-table slices
        tb = torch.zeros((max(d["r1"] - d["r0"], 1), 2), dtype=torch.int32, device="cuda")
        rc = gee.gee_shard_table(d["E"], g.N, d["r0"], d["r1"], d["y"], g.K, g.weighted, opts, nk, tb, d["ws"],
                                 d["n"], None)
        assert rc == 0, gee.gee_strerror(rc)
        tabs.append(tb[: d["r1"] - d["r0"]])
    tab = torch.cat(tabs).contiguous()                # 4. the all-gather
    assert tab.shape[0] == g.N
    Zs = []
    for d in ranks:                                   # 5. each rank's rows
        Z = torch.full((d["r1"] - d["r0"], g.K), float("nan"), dtype=torch.float32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc = gee.gee_shard_embed(d["E"], g.N, d["r0"], d["r1"], d["y"], g.K, g.weighted, opts, tab, Z, d["ws"],
                                 d["n"], None, st)
        assert rc == 0, gee.gee_strerror(rc)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        Zs.append(Z)
    return torch.cat(Zs), rr


@pytest.mark.parametrize("make,world,hub", [
    (lambda: sbm(3000, seed=81, weighted=True), 3, 2048),                      # K = 3, weighted
    (lambda: chung_lu(60000, 500000, d_max=20000, seed=82, K=24), 4, 1024),    # K > 8, split hub rows
    (lambda: chung_lu(20000, 150000, seed=83, K=7, weighted=True), 2, 512),    # K <= 8, weighted hubs
])
def test_shards_stitch_to_the_whole_graph(make, world, hub):
    import torch
    import paper_2406_03726_gb300 as gee
    g = make()
    opts = gee.make_opts(ALL, hub, 0, 8, 4, 64)       # every tuning field explicit
    Zs, rr = _sharded(gee, g, world, opts)
    assert sum(1 for r0, r1 in rr if r1 > r0) >= 2
    assert_z_matches(Zs.cpu().numpy(), oracle.embed_graph(g, ALL), what=f"{world} shards")
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    whole = gee.embed(t(g.src), t(g.dst), t(g.w), g.N, t(g.labels), g.K, opts=gee.make_opts(
        ALL | gee.NO_GRAPH_CACHE, hub, 0, 8, 4, 64))
    torch.cuda.synchronize()
    assert_z_matches(Zs.cpu().numpy(), whole.double().cpu().numpy(), rtol=2e-6, what="shards vs whole graph")


def test_shard_embed_reports_a_workspace_without_its_build():
    import torch
    import paper_2406_03726_gb300 as gee
    g = chung_lu(20000, 120000, seed=84, K=12)
    opts = gee.make_opts(ALL)
    r0, r1 = 0, g.N // 2
    e = edges_of_rows(g.src, r0, r1)
    n = gee.gee_shard_workspace_size(len(e), g.N, r0, r1, g.K, False, opts)
    ws = torch.zeros(n, dtype=torch.uint8, device="cuda")    # never built
    y = torch.from_numpy(g.labels[r0:r1]).cuda()
    tab = torch.zeros((g.N, 2), dtype=torch.int32, device="cuda")
    Z = torch.empty((r1 - r0, g.K), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert gee.gee_shard_embed(len(e), g.N, r0, r1, y, g.K, False, opts, tab, Z, ws, n, None, st) == 0
    torch.cuda.synchronize()
    assert int(st.item()) & gee.STATUS_STALE
