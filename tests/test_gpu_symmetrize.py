"""GEE_SYMMETRIZE: an undirected edge list given once per edge.  The reverse copies are
made inside the CSR build; the CSR must equal, bit for bit, the oracle's CSR of the
expanded list (every edge in input order, each followed by its reverse unless it is a
self-loop), and Z must match the oracle on that list."""
import numpy as np
import pytest

import oracle
from synth import chung_lu, random_tiny, sbm

from gpu_util import assert_z_matches, dev_graph

pytestmark = pytest.mark.gpu

ALL = 7


def _one_direction(g):
    keep = g.src <= g.dst                       # each undirected edge once (self-loops once)
    return type(g)(g.src[keep], g.dst[keep], None if g.w is None else g.w[keep], g.labels, g.N, g.K)


def _check(gee, g, flags_list, hub=0):
    import torch
    sym = oracle.symmetrize(g.src, g.dst, g.w)
    gs = type(g)(sym[0], sym[1], sym[2], g.labels, g.N, g.K)
    src, dst, w, y = dev_graph(g)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rowptr, col, val, nk, deg = gee.build_csr(src, dst, w, g.N, y, g.K, ALL | gee.SYMMETRIZE, hub, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    rp, cl, vl = oracle.csr(gs.src, gs.dst, gs.w, g.N)
    assert np.array_equal(rowptr.cpu().numpy(), rp)
    assert np.array_equal(col.cpu().numpy(), cl)
    assert np.array_equal(val.cpu().numpy(), vl)
    for f in flags_list:
        Z = gee.embed(src, dst, w, g.N, y, g.K, f | gee.SYMMETRIZE, hub_threshold=hub, status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert_z_matches(Z.cpu().numpy(), oracle.embed_graph(gs, f), what=f"{g.name} flags {f}")


@pytest.mark.parametrize("seed", range(10))
def test_symmetrize_tiny(seed):
    import paper_2406_03726_gb300 as gee
    g = random_tiny(seed, n_max=300, e_max=3000)       # self-loops, duplicates, unlabelled nodes
    _check(gee, g, range(8))


@pytest.mark.parametrize("make,hub", [(lambda: sbm(2000, seed=1), 0),
                                      (lambda: chung_lu(60000, 500000, d_max=20000, seed=92, K=20), 1024),
                                      (lambda: chung_lu(30000, 200000, seed=93, K=5, weighted=True), 512)])
def test_symmetrize_one_direction_of_undirected_graphs(make, hub):
    import paper_2406_03726_gb300 as gee
    g = _one_direction(make())
    _check(gee, g, (0, ALL), hub)


def test_symmetrize_in_a_batch_equals_alone():
    import torch
    import paper_2406_03726_gb300 as gee
    gs = [_one_direction(x) for x in (sbm(1500, seed=94, weighted=True), chung_lu(20000, 150000, seed=95, K=30),
                                       random_tiny(96, n_max=200, e_max=2000))]
    dev = [dev_graph(g) for g in gs]
    plan = gee.BatchPlan([(s, d, w, y, g.N, g.K) for (s, d, w, y), g in zip(dev, gs)], ALL | gee.SYMMETRIZE)
    Zb = plan.launch()
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum().item()) == 0
    for (s, d, w, y), g, Z in zip(dev, gs, Zb):
        solo = gee.embed(s, d, w, g.N, y, g.K, ALL | gee.SYMMETRIZE | gee.NO_GRAPH_CACHE)
        torch.cuda.synchronize()
        assert torch.equal(Z, solo)
    plan.close()


def test_symmetrize_reports_a_bad_target_read_as_a_source():
    import torch
    import paper_2406_03726_gb300 as gee
    g = random_tiny(97, n_max=100, e_max=500)
    bad = g.dst.copy()
    bad[len(bad) // 2] = g.N + 3                      # read as a source by the reverse copies
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gee.embed(t(g.src), t(bad), None if g.w is None else t(g.w), g.N, t(g.labels), g.K, ALL | gee.SYMMETRIZE,
              status=st)
    torch.cuda.synchronize()
    assert int(st.item()) & gee.STATUS_INDEX


@pytest.mark.slow
def test_symmetrize_chung_lu_600k_given_once():
    """The Chung-Lu N=600,000 graph (10M undirected edges, K=50) given once per edge: the
    CSR of its 20M entries bit for bit, and Z with every option against the oracle."""
    import paper_2406_03726_gb300 as gee
    g = _one_direction(chung_lu(600_000, 10_000_000, seed=3))
    assert g.E == 10_000_000
    _check(gee, g, (ALL,))


def test_symmetrize_through_host_buffers():
    """gee_embed_host with GEE_SYMMETRIZE: the host copies carry the edges once."""
    import torch
    import paper_2406_03726_gb300 as gee
    g = _one_direction(sbm(3000, seed=7, weighted=True))
    gs = type(g)(*oracle.symmetrize(g.src, g.dst, g.w), g.labels, g.N, g.K)
    opts = gee.make_opts(ALL | gee.SYMMETRIZE)
    n = gee.gee_host_workspace_size(g.E, g.N, g.K, True, opts)
    assert n > gee.gee_host_workspace_size(g.E, g.N, g.K, True, gee.make_opts(ALL))   # room for 2E entries
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    Z = torch.empty((g.N, g.K), dtype=torch.float32).pin_memory()
    st = np.zeros(1, np.uint32)
    rc = gee.gee_embed_host(pin(g.src), pin(g.dst), pin(g.w), g.E, g.N, pin(g.labels), g.K, opts, Z, ws, n, None, st)
    assert rc == 0 and st[0] == 0
    assert_z_matches(Z.double().numpy(), oracle.embed_graph(gs, ALL), what="host entry point, symmetrized")
