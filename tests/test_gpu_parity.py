"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer outputs (CSR rowptr/col, n_k, unweighted degrees, class counts) must be
bit-exact; Z must be within 1e-5 relative error of the oracle on every non-zero entry and
exactly zero where the oracle is zero.  Sizes run from tiny adversarial graphs to the
full paper-shaped workloads (SBM N=2,000 and N=10,000, Chung-Lu N=600,000)."""
import numpy as np
import pytest

import oracle
from synth import batch_graph, batch_specs, chung_lu, random_tiny, sbm

from gpu_util import RTOL, assert_z_matches, dev_graph, z_error_report, z_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL = 7


@pytest.fixture(scope="module")
def gee():
    import paper_2406_03726_gb300 as gee
    gee.lib()
    return gee


def run(gee, g, flags, **kw):
    src, dst, w, y = dev_graph(g)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    Z = gee.embed(src, dst, w, g.N, y, g.K, flags, status=status, **kw)
    torch.cuda.synchronize()
    return Z.double().cpu().numpy(), int(status.item())


# ---------------------------------------------------------------------------- small

@pytest.mark.parametrize("seed", range(48))
def test_tiny_all_option_settings(gee, seed):
    g = random_tiny(seed)
    for f in range(8):
        Zg, st = run(gee, g, f)
        assert st == 0
        assert_z_matches(Zg, oracle.embed_graph(g, f), what=f"seed {seed} flags {f}")


@pytest.mark.parametrize("seed", range(24))
def test_tiny_csr_bit_exact(gee, seed):
    g = random_tiny(seed, n_max=300, e_max=3000)
    src, dst, w, y = dev_graph(g)
    for f in (0, ALL):
        rowptr, col, val, nk, deg = gee.build_csr(src, dst, w, g.N, y, g.K, f)
        torch.cuda.synchronize()
        r_o, c_o, v_o = oracle.csr(g.src, g.dst, g.w, g.N)
        assert np.array_equal(rowptr.cpu().numpy(), r_o)
        assert np.array_equal(col.cpu().numpy(), c_o)
        assert np.array_equal(val.cpu().numpy(), v_o)
        assert np.array_equal(nk.cpu().numpy(), oracle.label_counts(g.labels, g.K))
        d_o = oracle.degrees(g.src, g.w, g.N, f)
        if g.w is None:
            assert np.array_equal(deg.cpu().numpy().astype(np.float64), d_o)
        else:
            assert np.allclose(deg.cpu().numpy(), d_o, rtol=1e-6, atol=0)


@pytest.mark.parametrize("seed", range(8))
def test_class_counts_and_counts_invariant(gee, seed):
    g = random_tiny(100 + seed, n_max=400, e_max=5000, weighted=False)
    src, dst, w, y = dev_graph(g)
    rowptr, col, _, nk, _ = gee.build_csr(src, dst, None, g.N, y, g.K, 0)
    C = gee.class_counts(rowptr, col, g.N, y, g.K)
    torch.cuda.synchronize()
    C_o = oracle.class_counts(g.src, g.dst, g.N, g.labels, g.K)
    assert np.array_equal(C.cpu().numpy(), C_o)
    # unweighted, no options: Z n_k reproduces the integer counts
    Zg, _ = run(gee, g, 0)
    n = oracle.label_counts(g.labels, g.K).astype(np.float64)
    assert np.allclose(Zg * n[None, :], C_o, rtol=1e-5, atol=0)


# ----------------------------------------------------------------- paper workloads

def test_sbm_2000_options_off_and_all(gee):
    g = sbm(2000, seed=1)
    for f in (0, ALL):
        Zg, st = run(gee, g, f)
        assert st == 0
        Zo = oracle.embed_graph(g, f)
        assert_z_matches(Zg, Zo, what=f"sbm2000 flags {f}")
        z_error_report(Zg, Zo, f"SBM N=2,000 flags {f}")
    src, dst, w, y = dev_graph(g)
    rowptr, col, _, nk, deg = gee.build_csr(src, dst, None, g.N, y, g.K, ALL)
    r_o, c_o, _ = oracle.csr(g.src, g.dst, None, g.N)
    assert np.array_equal(rowptr.cpu().numpy(), r_o) and np.array_equal(col.cpu().numpy(), c_o)


def test_sbm_10000_weighted_all_options(gee):
    g = sbm(10_000, seed=2, weighted=True)
    Zg, st = run(gee, g, ALL)
    assert st == 0
    Zo = oracle.embed_graph(g, ALL)
    assert_z_matches(Zg, Zo, what="sbm10000")
    z_error_report(Zg, Zo, "SBM N=10,000 weighted, all options")
    src, dst, w, y = dev_graph(g)
    rowptr, col, val, _, _ = gee.build_csr(src, dst, w, g.N, y, g.K, ALL)
    r_o, c_o, v_o = oracle.csr(g.src, g.dst, g.w, g.N)
    assert np.array_equal(rowptr.cpu().numpy(), r_o)
    assert np.array_equal(col.cpu().numpy(), c_o)
    assert np.array_equal(val.cpu().numpy(), v_o)


@pytest.fixture(scope="module")
def cl600k():
    return chung_lu(600_000, 10_000_000, seed=3)


def test_chung_lu_600k_all_options(gee, cl600k):
    g = cl600k
    Zg, st = run(gee, g, ALL)
    assert st == 0
    Zo = oracle.embed_graph(g, ALL)
    assert_z_matches(Zg, Zo, what="chung-lu 600k")
    z_error_report(Zg, Zo, "Chung-Lu N=600,000, all options")
    r = np.linalg.norm(Zg, axis=1)
    assert np.all((np.abs(r - 1) < 1e-5) | (r == 0))


def _tuned(gee, g):
    """The options bench.py times: the autotuner's choice for this graph, all options."""
    src, dst, w, y = dev_graph(g)
    opts, ms = gee.autotune(src, dst, w, g.N, y, g.K, ALL)
    assert ms > 0.0
    return opts


@pytest.mark.parametrize("name", ["sbm2k", "sbm10k", "cl600k"])
def test_bench_workloads_in_the_tuned_launch_configuration(gee, cl600k, name):
    """Each single-graph workload of the benchmark, embedded with the tuning fields the
    benchmark times (the split threshold and the short-row bound move rows between paths,
    so they change the rounding), against the oracle entry by entry."""
    g = {"sbm2k": lambda: sbm(2000, seed=1), "sbm10k": lambda: sbm(10000, seed=2, weighted=True),
         "cl600k": lambda: cl600k}[name]()
    opts = _tuned(gee, g)
    Zg, st = run(gee, g, ALL, opts=opts)
    assert st == 0
    assert_z_matches(Zg, oracle.embed_graph(g, ALL), what=f"{name} tuned {opts.hub_threshold},"
                                                           f"{opts.vec_width},{opts.short_len}")


def test_chung_lu_600k_csr_and_degrees(gee, cl600k):
    g = cl600k
    src, dst, w, y = dev_graph(g)
    rowptr, col, _, nk, deg = gee.build_csr(src, dst, None, g.N, y, g.K, ALL)
    r_o, c_o, _ = oracle.csr(g.src, g.dst, None, g.N)
    assert np.array_equal(rowptr.cpu().numpy(), r_o)
    assert np.array_equal(col.cpu().numpy(), c_o)
    assert np.array_equal(nk.cpu().numpy(), oracle.label_counts(g.labels, g.K))
    assert np.array_equal(deg.cpu().numpy().astype(np.float64), oracle.degrees(g.src, None, g.N, 1))


# ------------------------------------------------------------------ structure edges

@pytest.mark.parametrize("N", [1, 2, 2047, 2048, 2049, 4097, 65536, 65537, (1 << 21)])
def test_radix_pass_boundaries(gee, N):
    rng = np.random.default_rng(N)
    E = 50_000
    src = rng.integers(0, N, E).astype(np.int32)
    dst = rng.integers(0, N, E).astype(np.int32)
    src[:10] = N - 1
    dst[10:20] = N - 1
    w = (1.0 - rng.random(E, dtype=np.float32)).astype(np.float32)
    K = 5
    y = rng.integers(-1, K, N).astype(np.int32)
    from synth.graphs import Graph
    g = Graph(src, dst, w, y, N, K)
    Zg, st = run(gee, g, ALL)
    assert st == 0
    assert_z_matches(Zg, oracle.embed_graph(g, ALL), what=f"N={N}")
    s_, d_, w_, y_ = dev_graph(g)
    rowptr, col, val, _, _ = gee.build_csr(s_, d_, w_, N, y_, K, 0)
    r_o, c_o, v_o = oracle.csr(src, dst, w, N)
    assert np.array_equal(rowptr.cpu().numpy(), r_o) and np.array_equal(col.cpu().numpy(), c_o)
    assert np.array_equal(val.cpu().numpy(), v_o)


@pytest.mark.parametrize("m,lap", [(100_000, False), (100_000, True), (1_000_000, True)])
def test_star_hub_closed_form(gee, m, lap):
    N = m + 1
    y = np.ones(N, np.int32)
    y[0] = 0
    leaves = np.arange(1, N, dtype=np.int32)
    src = np.concatenate([np.zeros(m, np.int32), leaves])
    dst = np.concatenate([leaves, np.zeros(m, np.int32)])
    perm = np.random.default_rng(m).permutation(2 * m)
    from synth.graphs import Graph
    g = Graph(src[perm].copy(), dst[perm].copy(), None, y, N, 2)
    f = 2 if lap else 0
    Zg, st = run(gee, g, f, hub_threshold=4096)
    assert st == 0
    r = 1.0 / np.sqrt(m) if lap else 1.0
    assert abs(Zg[0, 0]) == 0.0 and abs(Zg[0, 1] - r) <= RTOL * r
    assert np.all(Zg[1:, 1] == 0.0) and np.max(np.abs(Zg[1:, 0] - r)) <= RTOL * r


def test_split_threshold_and_lanes_sweep(gee):
    g = chung_lu(60_000, 600_000, d_max=20_000, seed=21, K=7, weighted=True)
    Zo = oracle.embed_graph(g, ALL)
    ref = None
    for hub in (64, 1000, 4096, 1 << 29):
        for lpr in (0, 1, 4, 32):
            Zg, st = run(gee, g, ALL, hub_threshold=hub, lanes_per_row=lpr)
            assert st == 0
            assert_z_matches(Zg, Zo, what=f"hub={hub} lpr={lpr}")
            if ref is None:
                ref = Zg
            else:
                assert np.allclose(Zg, ref, rtol=2e-5, atol=0)


def test_deterministic_bits(gee):
    g = chung_lu(60_000, 600_000, d_max=20_000, seed=22, K=20, weighted=True)
    a, _ = run(gee, g, ALL, hub_threshold=512)
    b, _ = run(gee, g, ALL, hub_threshold=512)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("K", [1, 2, 3, 8, 9, 33, 64])
def test_class_count_range(gee, K):
    g = batch_graph({"index": K, "N": 3000, "m": 60_000, "E": 120_000, "K": K, "kind": "chung_lu",
                     "seed": 1234 + K})
    for f in (0, ALL):
        Zg, st = run(gee, g, f, hub_threshold=512)
        assert st == 0
        assert_z_matches(Zg, oracle.embed_graph(g, f), what=f"K={K} flags={f}")


def test_batch_mix_graphs_individually(gee):
    for spec in batch_specs(12, seed=4):
        g = batch_graph(spec)
        Zg, st = run(gee, g, ALL)
        assert st == 0
        assert_z_matches(Zg, oracle.embed_graph(g, ALL), what=f"batch graph {spec['index']}")


# --------------------------------------------------------------------- degenerate

def test_empty_edge_list(gee):
    from synth.graphs import Graph
    y = np.array([0, 1, -1, 1], np.int32)
    g = Graph(np.zeros(0, np.int32), np.zeros(0, np.int32), None, y, 4, 2)
    for f in range(8):
        Zg, st = run(gee, g, f)
        assert st == 0
        assert_z_matches(Zg, oracle.embed_graph(g, f), what=f"E=0 flags {f}")


def test_unlabelled_and_empty_classes(gee):
    g = random_tiny(5, n_max=200, e_max=2000)
    y = np.full(g.N, -1, np.int32)
    g.labels = y
    for f in (0, ALL):
        Zg, st = run(gee, g, f)
        assert st == 0 and np.all(Zg == 0)
    g.labels = np.zeros(g.N, np.int32)          # only class 0 is used
    Zg, _ = run(gee, g, ALL)
    assert np.all(Zg[:, 1:] == 0)


def test_zero_nodes(gee):
    status = torch.ones(1, dtype=torch.int32, device="cuda")
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    Z = gee.embed(e, e, None, 0, e, 3, ALL, status=status)
    torch.cuda.synchronize()
    assert Z.shape == (0, 3) and int(status.item()) == 0


@pytest.mark.parametrize("case", ["src", "dst", "label_hi", "label_lo", "nan", "neg_lap"])
def test_invalid_inputs_reported(gee, case):
    g = random_tiny(9, n_max=100, e_max=500, weighted=True)
    g.src, g.dst, g.w, g.labels = g.src.copy(), g.dst.copy(), g.w.copy(), g.labels.copy()
    flags = ALL
    if case == "src":
        g.src[3] = g.N
        want = 1
    elif case == "dst":
        g.dst[0] = -5
        want = 1
    elif case == "label_hi":
        g.labels[0] = g.K
        want = 2
    elif case == "label_lo":
        g.labels[0] = -2
        want = 2
    elif case == "nan":
        g.w[1] = np.nan
        want = 4
    else:
        g.w[2] = -0.5
        want = 4
    if g.E < 4 and case in ("src", "dst", "nan", "neg_lap"):
        pytest.skip("graph too small")
    _, st = run(gee, g, flags)
    assert st & want
    if case == "neg_lap":   # negative weights are fine without the Laplacian
        _, st = run(gee, g, 1)
        assert st == 0


def test_host_buffer_entry_point(gee):
    g = sbm(3000, seed=7, weighted=True)
    E, N, K = g.E, g.N, g.K
    opts = gee.make_opts(ALL)
    n = gee.gee_host_workspace_size(E, N, K, True, opts)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    pin = lambda a: torch.from_numpy(a).pin_memory()
    src, dst, w, y = pin(g.src), pin(g.dst), pin(g.w), pin(g.labels)
    Z = torch.empty((N, K), dtype=torch.float32).pin_memory()
    st = np.zeros(1, np.uint32)
    rc = gee.gee_embed_host(src, dst, w, E, N, y, K, opts, Z, ws, n, None, st)
    assert rc == 0 and st[0] == 0
    assert_z_matches(Z.double().numpy(), oracle.embed_graph(g, ALL), what="host entry point")


@pytest.mark.slow
def test_serving_large_graph_sampled_rows(gee):
    """The large serving graph: Chung-Lu, N = 2M, 100M undirected edges (200M directed),
    K = 16, weighted.  index_pointers bit-exact, unweighted-equivalent row lengths exact,
    weighted degrees within 1e-6, and 10,000 sampled rows of Z against the oracle."""
    from synth.torch_batch import batch_graph_torch
    spec = {"index": -1, "N": 2_000_000, "m": 100_000_000, "E": 200_000_000, "K": 16, "kind": "chung_lu",
            "seed": 77}
    src, dst, w, y = batch_graph_torch(spec, "cuda")
    N, K = spec["N"], spec["K"]
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rowptr, col, val, nk, deg = gee.build_csr(src, dst, w, N, y, K, ALL, status=st)
    Z = gee.embed(src, dst, w, N, y, K, ALL, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    s, d, wv, yv = (t.cpu().numpy() for t in (src, dst, w, y))
    del col, val
    torch.cuda.empty_cache()
    rp = np.concatenate([[0], np.cumsum(np.bincount(s, minlength=N))])
    assert np.array_equal(rowptr.cpu().numpy().astype(np.int64), rp)
    assert np.array_equal(nk.cpu().numpy(), oracle.label_counts(yv, K))
    dref = oracle.degrees(s, wv, N, oracle.DIAG_AUG)
    dg = deg.double().cpu().numpy()
    assert np.max(np.abs(dg - dref) / dref) <= 1e-6
    Zo = oracle.embed(s, d, wv, N, yv, K, ALL)
    rows = np.random.default_rng(5).choice(N, 10_000, replace=False)
    hubs = np.argsort(np.diff(rp))[-50:]                  # the longest rows (split across CTAs)
    pick = np.unique(np.concatenate([rows, hubs]))
    assert_z_matches(Z.double().cpu().numpy()[pick], Zo[pick], what="N=2M sampled rows")
