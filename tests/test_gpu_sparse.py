"""Sparse Z (gee_embed_sparse) against the oracle's sparse form.

The structure (index pointers and classes) must equal the oracle's bit for bit; every
value must match within the tolerance, with exact zeros where the oracle's are zero.
Rows are placed in windows of 1024 CSR positions and rows longer than that go through
the chunk-merge path, so the cases cover short rows, rows of several chunks, empty rows,
unlabelled neighbours and class counts from 1 to far above the dense limit."""
import numpy as np
import pytest

import oracle
from synth import chung_lu, random_tiny, sbm
from synth.graphs import Graph

from gpu_util import RTOL, dev_graph, z_errors

pytestmark = pytest.mark.gpu

ALL = 7


def _relabel(g, K, seed):
    """The same graph with labels drawn from K classes (every fifth node unlabelled)."""
    rng = np.random.default_rng(seed)
    y = rng.integers(0, K, g.N).astype(np.int32)
    y[::5] = -1
    return Graph(g.src, g.dst, g.w, y, g.N, K, name=f"{g.name} K={K}")


def _check(gee, g, flags, what=""):
    import torch
    src, dst, w, y = dev_graph(g)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    zr, zc, zv = gee.embed_sparse(src, dst, w, g.N, y, g.K, flags, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0, (what, int(st.item()))
    rp_o, zc_o, zv_o = oracle.embed_sparse_graph(g, flags)
    assert np.array_equal(zr.cpu().numpy(), rp_o), what
    assert np.array_equal(zc.cpu().numpy(), zc_o), what
    err, bad = z_errors(zv.double().cpu().numpy(), zv_o)
    assert bad == 0 and err <= RTOL, f"{what} flags {flags}: rel err {err:.2e}, {bad} false non-zeros"
    return zr, zc, zv


@pytest.mark.parametrize("seed", range(6))
def test_sparse_tiny_all_options(seed):
    import paper_2406_03726_gb300 as gee
    g = random_tiny(seed, n_max=300, e_max=3000, weighted=(seed % 2 == 1))
    for K in (1, g.K, 70, 1000):
        h = _relabel(g, K, seed) if K != g.K else g
        for flags in range(8):
            _check(gee, h, flags, f"tiny seed {seed} K={K}")


@pytest.mark.parametrize("K", [3, 64, 5000, 200000])
def test_sparse_long_rows_split_in_chunks(K):
    """Hub rows of up to ~27,000 entries: the window path, single-chunk long rows (1024 to
    4096 entries) and the chunk-merge path (rows of up to seven 4096-entry chunks)."""
    import paper_2406_03726_gb300 as gee
    g = _relabel(chung_lu(100000, 1500000, d_max=60000, seed=131, weighted=True), K, 132)
    deg = np.bincount(g.src, minlength=g.N)
    assert int((deg > 1024).sum()) >= 100 and int((deg > 4096).sum()) >= 10 and int(deg.max()) > 3 * 4096
    for flags in (0, ALL, 2, 5):
        _check(gee, g, flags, f"chung-lu K={K}")


def test_sparse_matches_dense_for_few_classes():
    """K <= 64: the sparse values are the dense path's entries at the structure (to
    rounding: the two sum in different orders), and the dense Z is zero elsewhere."""
    import torch
    import paper_2406_03726_gb300 as gee
    g = sbm(3000, seed=133, weighted=True)
    src, dst, w, y = dev_graph(g)
    zr, zc, zv = gee.embed_sparse(src, dst, w, g.N, y, g.K, ALL)
    Z = gee.embed(src, dst, w, g.N, y, g.K, ALL)
    torch.cuda.synchronize()
    zr, zc, zv, Z = zr.cpu().numpy(), zc.cpu().numpy(), zv.double().cpu().numpy(), Z.double().cpu().numpy()
    rows = np.repeat(np.arange(g.N), np.diff(zr))
    assert np.allclose(zv, Z[rows, zc], rtol=2e-5, atol=0)
    mask = np.zeros_like(Z, bool)
    mask[rows, zc] = True
    assert np.all(Z[~mask] == 0)


def test_sparse_edge_cases():
    import torch
    import paper_2406_03726_gb300 as gee
    # no edges: with augmentation every labelled node has its own class, scaled to 1
    N, K = 5000, 300
    y = torch.from_numpy((np.arange(N) % K).astype(np.int32)).cuda()
    y[7] = -1
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    zr, zc, zv = gee.embed_sparse(e, e, None, N, y, K, ALL)
    torch.cuda.synchronize()
    counts = np.diff(zr.cpu().numpy())
    assert counts[7] == 0 and counts.sum() == N - 1
    assert np.allclose(zv.cpu().numpy(), 1.0, rtol=1e-6, atol=0)
    # every neighbour unlabelled: rows are empty (without augmentation)
    g = sbm(800, seed=134)
    yy = np.full(g.N, -1, np.int32)
    h = Graph(g.src, g.dst, None, yy, g.N, 4, name="unlabelled")
    zr, zc, zv = _check(gee, h, 0, "unlabelled")
    assert int(zr[-1].item()) == 0
    # zero nodes
    zr, zc, zv = gee.embed_sparse(e, e, None, 0, torch.zeros(0, dtype=torch.int32, device="cuda"), 3, ALL)
    assert zr.numel() == 1 and int(zr[0].item()) == 0
    # too little room for the entries is refused on the host
    g = random_tiny(3, n_max=50, e_max=200)
    src, dst, w, y = dev_graph(g)
    o = gee.make_opts(ALL)
    n = gee.gee_sparse_workspace_size(g.E, g.N, g.K, False, o)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    out = torch.empty(g.E + g.N, dtype=torch.int32, device="cuda")
    rp = torch.empty(g.N + 1, dtype=torch.int32, device="cuda")
    assert gee.gee_embed_sparse(src, dst, None, g.E, g.N, y, g.K, o, rp, out, out, g.E + g.N - 1, ws, n) == 1


def test_sparse_symmetrize_and_determinism():
    import torch
    import paper_2406_03726_gb300 as gee
    g = _relabel(chung_lu(30000, 200000, d_max=8000, seed=135), 2000, 136)
    one = g.src <= g.dst
    h = Graph(g.src[one], g.dst[one], None, g.labels, g.N, g.K, name="once")
    sym = oracle.symmetrize(h.src, h.dst, None)
    hs = Graph(sym[0], sym[1], None, g.labels, g.N, g.K, name="expanded")
    src, dst, w, y = dev_graph(h)
    a = gee.embed_sparse(src, dst, None, h.N, y, h.K, ALL | gee.SYMMETRIZE)
    b = gee.embed_sparse(src, dst, None, h.N, y, h.K, ALL | gee.SYMMETRIZE)
    torch.cuda.synchronize()
    for x, z in zip(a, b):
        assert torch.equal(x, z)                     # the same bits on every call
    rp_o, zc_o, zv_o = oracle.embed_sparse_graph(hs, ALL)
    assert np.array_equal(a[0].cpu().numpy(), rp_o) and np.array_equal(a[1].cpu().numpy(), zc_o)
    err, bad = z_errors(a[2].double().cpu().numpy(), zv_o)
    assert bad == 0 and err <= RTOL


@pytest.mark.slow
def test_sparse_chung_lu_600k_many_classes():
    """The Chung-Lu N=600,000 graph (20M entries, hub rows up to ~10^5 entries) with
    K = 100,000 classes: dense Z would be 240 GB."""
    import paper_2406_03726_gb300 as gee
    g = _relabel(chung_lu(600_000, 10_000_000, seed=3), 100_000, 137)
    _check(gee, g, ALL, "chung-lu 600k K=100000")
