"""gee_reembed: Z for new labels on the CSR, degrees and plans a previous gee_embed left in
its workspace (Section 2: W is built from known or predicted labels, so iterative use
embeds one graph with updated labels).  The result must equal, bit for bit, gee_embed
with the new labels, and match the oracle; a workspace that does not hold such a build
is reported with GEE_STATUS_STALE."""
import numpy as np
import pytest

import oracle
from synth import chung_lu, sbm

from gpu_util import assert_z_matches, dev_graph

pytestmark = pytest.mark.gpu

ALL = 7


def _new_labels(g, seed):
    rng = np.random.default_rng(seed)
    y = rng.permutation(g.labels).astype(np.int32)
    y[rng.random(g.N) < 0.05] = -1            # some nodes lose their label
    return y


@pytest.mark.parametrize("make,hub", [(lambda: sbm(3000, seed=61, weighted=True), 0),
                                      (lambda: chung_lu(40000, 300000, d_max=12000, seed=62, K=20), 1024),
                                      (lambda: chung_lu(20000, 150000, seed=63, K=6, weighted=True), 512)])
def test_reembed_equals_embed_with_new_labels(make, hub):
    import torch
    import paper_2406_03726_gb300 as gee
    g = make()
    src, dst, w, y = dev_graph(g)
    opts = gee.make_opts(ALL, hub)
    n = gee.gee_workspace_size(g.E, g.N, g.K, g.weighted, opts)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    Z = torch.empty((g.N, g.K), dtype=torch.float32, device="cuda")
    assert gee.gee_embed(src, dst, w, g.E, g.N, y, g.K, opts, Z, ws, n, None, st) == 0
    for rep in range(4):  # seen, captured, replayed twice (labels changed in place each time)
        y2 = _new_labels(g, 100 + rep)
        y.copy_(torch.from_numpy(y2))
        Zr = torch.full_like(Z, float("nan"))
        rc = gee.gee_reembed(y, g.E, g.N, g.K, g.weighted, opts, Zr, ws, n, None, st)
        assert rc == 0, gee.gee_strerror(rc)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        # the same graph embedded from scratch with the new labels, in a fresh workspace
        ref = gee.embed(src, dst, w, g.N, y, g.K, ALL | gee.NO_GRAPH_CACHE, hub_threshold=hub)
        torch.cuda.synchronize()
        assert torch.equal(Zr, ref), f"rep {rep}"
        g2 = type(g)(g.src, g.dst, g.w, y2, g.N, g.K)
        assert_z_matches(Zr.cpu().numpy(), oracle.embed_graph(g2, ALL), what=f"reembed rep {rep}")
    gee.gee_graph_cache_clear()


def test_reembed_reports_a_stale_workspace():
    import torch
    import paper_2406_03726_gb300 as gee
    a = chung_lu(30000, 200000, seed=64, K=16)
    b = chung_lu(31000, 200000, seed=65, K=16)
    src, dst, w, y = dev_graph(a)
    opts = gee.make_opts(ALL)
    n = max(gee.gee_workspace_size(x.E, x.N, x.K, False, opts) for x in (a, b))
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    Z = torch.empty((b.N, b.K), dtype=torch.float32, device="cuda")
    assert gee.gee_embed(src, dst, w, a.E, a.N, y, a.K, opts, Z, ws, n, None, st) == 0
    yb = torch.from_numpy(b.labels).cuda()
    # other sizes than the build that the workspace holds: reported, nothing read out of range
    rc = gee.gee_reembed(yb, b.E, b.N, b.K, False, gee.make_opts(ALL | gee.NO_GRAPH_CACHE), Z, ws, n, None, st)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) & gee.STATUS_STALE
    # a zeroed workspace holds no build either
    ws.zero_()
    rc = gee.gee_reembed(y, a.E, a.N, a.K, False, gee.make_opts(ALL | gee.NO_GRAPH_CACHE), Z, ws, n, None, st)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) & gee.STATUS_STALE
