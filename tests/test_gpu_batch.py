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


def test_batch_with_split_hub_rows_in_many_graphs(gee):
    """A low split threshold makes hub rows in most graphs of the batch, so the hub chunks of
    different graphs share the k_wdeg / k_spmm hub phase (chunk -> hub -> graph mapping)."""
    from synth import chung_lu
    graphs = [chung_lu(n, n * d, seed=110 + i, K=k, weighted=(i % 2 == 0), d_max=n // 2)
              for i, (n, d, k) in enumerate([(3000, 20, 5), (8000, 12, 24), (5000, 30, 3), (12000, 10, 40),
                                             (2000, 40, 8), (6000, 16, 64)])]
    dg = [dev_graph(g) for g in graphs]
    hub = 512
    assert all(int((np.bincount(g.src, minlength=g.N) > hub).sum()) > 0 for g in graphs)
    plan = gee.BatchPlan([(s, d, w, y, g.N, g.K) for (s, d, w, y), g in zip(dg, graphs)], ALL, hub_threshold=hub)
    Zs = plan.launch(use_graph=False)
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum().item()) == 0
    for g, (s, d, w, y), Zb in zip(graphs, dg, Zs):
        assert_z_matches(Zb.double().cpu().numpy(), oracle.embed_graph(g, ALL), what=g.name)
        solo = gee.embed(s, d, w, g.N, y, g.K, ALL | gee.NO_GRAPH_CACHE, hub_threshold=hub)
        torch.cuda.synchronize()
        assert torch.equal(solo, Zb), g.name
    plan.close()


@pytest.mark.slow
def test_full_4096_graph_batch_on_a_seeded_sample(gee):
    """The whole 4,096-graph mix (about 3.5e9 directed edges) in one launch sequence, with
    the batch tuner's options as the benchmark runs it; every 64th graph, the largest and
    the most skewed are checked against the oracle."""
    from synth.torch_batch import batch_graph_torch
    specs = batch_specs(4096, seed=4)
    graphs = [batch_graph_torch(sp, "cuda") for sp in specs]
    torch.cuda.synchronize()
    items = [(s, d, w, y, sp["N"], sp["K"]) for (s, d, w, y), sp in zip(graphs, specs)]
    best, _ = gee.batch_autotune(items, ALL)          # the launch configuration the benchmark times
    torch.cuda.empty_cache()
    plan = gee.BatchPlan(items, opts=best)
    Zs = plan.launch(use_graph=True)
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum().item()) == 0
    largest = max(range(len(specs)), key=lambda i: specs[i]["E"])
    skew = []
    for i, (s, d, w, y) in enumerate(graphs):
        deg = torch.bincount(s.long(), minlength=specs[i]["N"])
        skew.append(float(deg.max().item()) / max(1.0, float(deg.float().mean().item())))
    skewed = int(np.argmax(skew))
    sample = sorted(set(list(range(0, len(specs), 64)) + [largest, skewed]))
    from synth.graphs import Graph
    for i in sample:
        s, d, w, y = (t.cpu().numpy() for t in graphs[i])
        g = Graph(s, d, w, y, specs[i]["N"], specs[i]["K"])
        assert_z_matches(Zs[i].double().cpu().numpy(), oracle.embed_graph(g, ALL), what=f"graph {i}")
    plan.close()
    del graphs, Zs, items
    torch.cuda.empty_cache()


def test_batch_tuner_picks_candidates_that_keep_parity(gee):
    """gee_batch_autotune: the chosen fields come from its candidate lists (a field set by
    the caller stays fixed), and the tuned plan still matches the oracle graph by graph."""
    graphs = small_mix(24, seed=45)
    assert any(g.K > 8 for g in graphs) and any(g.K <= 8 for g in graphs)
    dg = [dev_graph(g) for g in graphs]
    items = [(s, d, w, y, g.N, g.K) for (s, d, w, y), g in zip(dg, graphs)]
    best, ms = gee.batch_autotune(items, ALL)
    assert ms > 0.0 and best.flags == ALL
    assert best.vec_width in (2, 4, 8) and best.short_len in (64, 128, 256)
    assert best.rows_per_item in (0, 4, 16, 32) and best.hub_threshold == 0
    plan = gee.BatchPlan(items, opts=best)
    Zs = plan.launch(use_graph=True)
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum().item()) == 0
    for g, Zb in zip(graphs, Zs):
        assert_z_matches(Zb.double().cpu().numpy(), oracle.embed_graph(g, ALL), what=g.name)
    plan.close()
    # a field given by the caller is not searched
    fixed = gee.make_opts(ALL, 0, 0, 0, 2, 0)
    import ctypes
    from paper_2406_03726_gb300 import _native as nat
    Zkeep = [torch.empty((g.N, g.K), device="cuda") for g in graphs]   # outlive the tuner's launches
    arr = nat.make_graphs([(s, d, w, y, Z, g.E, g.N, g.K) for (s, d, w, y), g, Z in zip(dg, graphs, Zkeep)])
    n = gee.gee_batch_autotune_workspace_size(arr, len(graphs), fixed)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    out, t = gee.make_opts(ALL), ctypes.c_float(0.0)
    assert gee.gee_batch_autotune(arr, len(graphs), fixed, ws, n, None, out, t) == 0
    assert out.vec_width == 2
