"""Batched embedding: many graphs of different N, E, K in one launch sequence.

Each graph's Z must match the FP64 oracle (1e-5 relative, exact zeros) and be
bit-identical to the single-graph entry point's Z for the same graph; a CUDA-graph
replay must give the same bits again; a bad graph must only flag its own status."""
import numpy as np
import pytest

import oracle
from synth import batch_graph, batch_specs, sbm

from gpu_util import assert_z_matches, dev_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ALL = 7


@pytest.fixture(scope="module")
def gee():
    import paper_2406_03726_gb300 as gee
    gee.lib()
    return gee


def small_mix(G, seed, n_range=(100, 6000), d_range=(5.0, 60.0)):
    specs = batch_specs(G, seed=seed, n_range=n_range, d_range=d_range)
    return [batch_graph(s) for s in specs]


def test_batch_matches_oracle_and_solo_bits(gee):
    graphs = small_mix(40, seed=41)
    graphs.append(sbm(2500, seed=5, weighted=True))          # a 2-pass SBM
    dg = [dev_graph(g) for g in graphs]
    plan = gee.BatchPlan([(s, d, w, y, g.N, g.K) for (s, d, w, y), g in zip(dg, graphs)], ALL)
    Zs = plan.launch(use_graph=False)
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum().item()) == 0
    for g, (s, d, w, y), Zb in zip(graphs, dg, Zs):
        zb = Zb.double().cpu().numpy()
        assert_z_matches(zb, oracle.embed_graph(g, ALL), what=g.name)
        solo = gee.embed(s, d, w, g.N, y, g.K, ALL)
        torch.cuda.synchronize()
        assert np.array_equal(solo.double().cpu().numpy(), zb), g.name
    # replay through a captured CUDA graph, twice: same bits
    before = [z.clone() for z in Zs]
    for _ in range(2):
        for z in Zs:
            z.fill_(float("nan"))
        plan.launch(use_graph=True)
        torch.cuda.synchronize()
        for a, b in zip(before, Zs):
            assert torch.equal(a, b)
    plan.close()


def test_batch_options_and_unweighted_mix(gee):
    graphs = small_mix(12, seed=42)
    for g in graphs[::2]:
        g.w = None
    dg = [dev_graph(g) for g in graphs]
    for flags in (0, 1, 2, 4, 6):
        plan = gee.BatchPlan([(s, d, w, y, g.N, g.K) for (s, d, w, y), g in zip(dg, graphs)], flags)
        Zs = plan.launch(use_graph=False)
        torch.cuda.synchronize()
        for g, Zb in zip(graphs, Zs):
            assert_z_matches(Zb.double().cpu().numpy(), oracle.embed_graph(g, flags), what=f"{g.name} f{flags}")
        plan.close()


def test_batch_with_empty_and_tiny_graphs(gee):
    from synth.graphs import Graph
    graphs = small_mix(6, seed=43)
    graphs.insert(2, Graph(np.zeros(0, np.int32), np.zeros(0, np.int32), None, np.array([0, 1, -1], np.int32), 3, 2))
    graphs.insert(4, Graph(np.array([0], np.int32), np.array([0], np.int32), None, np.array([0], np.int32), 1, 1))
    dg = [dev_graph(g) for g in graphs]
    plan = gee.BatchPlan([(s, d, w, y, g.N, g.K) for (s, d, w, y), g in zip(dg, graphs)], ALL)
    Zs = plan.launch(use_graph=True)
    torch.cuda.synchronize()
    for g, Zb in zip(graphs, Zs):
        assert_z_matches(Zb.double().cpu().numpy(), oracle.embed_graph(g, ALL), what=g.name)
    plan.close()


def test_batch_status_is_per_graph(gee):
    graphs = small_mix(5, seed=44)
    bad = graphs[3]
    bad.src = bad.src.copy()
    bad.src[7] = bad.N + 3
    dg = [dev_graph(g) for g in graphs]
    plan = gee.BatchPlan([(s, d, w, y, g.N, g.K) for (s, d, w, y), g in zip(dg, graphs)], ALL)
    plan.launch(use_graph=False)
    torch.cuda.synchronize()
    st = plan.status.cpu().numpy()
    assert st[3] & 1 and np.all(np.delete(st, 3) == 0)
    plan.close()


def test_embed_batch_one_shot_entry_point(gee):
    graphs = small_mix(8, seed=45)
    dg = [dev_graph(g) for g in graphs]
    Zs = [torch.empty((g.N, g.K), device="cuda") for g in graphs]
    arr = gee.make_graphs([(s, d, w, y, Z, g.E, g.N, g.K) for (s, d, w, y), g, Z in zip(dg, graphs, Zs)])
    opts = gee.make_opts(ALL)
    n = gee.gee_batch_workspace_size(arr, len(graphs), opts)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    st = torch.zeros(len(graphs), dtype=torch.int32, device="cuda")
    assert gee.gee_embed_batch(arr, len(graphs), opts, ws, n, None, st) == 0
    torch.cuda.synchronize()
    assert int(st.abs().sum().item()) == 0
    for g, Zb in zip(graphs, Zs):
        assert_z_matches(Zb.double().cpu().numpy(), oracle.embed_graph(g, ALL), what=g.name)


def test_batch_of_one_graph(gee):
    g = small_mix(1, seed=46)[0]
    s, d, w, y = dev_graph(g)
    plan = gee.BatchPlan([(s, d, w, y, g.N, g.K)], ALL)
    for use_graph in (False, True):
        Zb = plan.launch(use_graph=use_graph)[0]
        torch.cuda.synchronize()
        assert np.array_equal(Zb.cpu().numpy(), gee.embed(s, d, w, g.N, y, g.K, ALL).cpu().numpy())
    plan.close()
