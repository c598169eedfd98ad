"""Pins for the FP64 oracle (CPU only).

The oracle is checked against things other than itself: the CSR example printed in
Section 3, a library stable sort, brute-force dense matrices (Table 1 / Eq. 1), closed
forms on graphs whose embedding follows from the definitions by hand, and invariants of
the mathematics.  None of these checks touches the CUDA path.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dense
from synth import random_tiny, sbm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALL_FLAGS = list(range(8))


def _flags_name(f):
    return "".join(c for c, b in (("A", 1), ("L", 2), ("C", 4)) if f & b) or "none"


# ------------------------------------------------------------------ CSR (Section 3)

def test_csr_fig1_fragment():
    fx = json.load(open(os.path.join(GOLDEN, "csr_fig1_fragment.json")))
    # any matrix consistent with the fragment: rows 0-1 hold 3 non-zeros, row 2 holds
    # 2 at column 1 and 3 at column 5, and there are rows after it
    src = np.array([3, 2, 0, 1, 0, 2, 3], np.int32)
    dst = np.array([0, 1, 4, 2, 6, 5, 3], np.int32)
    w = np.array([7, 2, 1, 5, 4, 3, 9], np.float32)
    rowptr, col, val = oracle.csr(src, dst, w, 7)
    r = fx["row"]
    assert list(rowptr[r:r + 2]) == fx["index_pointers_2_3"]
    assert list(col[3:5]) == fx["col_indices_3_5"]
    assert list(val[3:5]) == fx["data_3_5"]
    assert rowptr[-1] == src.size


@pytest.mark.parametrize("seed", range(12))
def test_csr_equals_library_stable_sort(seed):
    g = random_tiny(seed, n_max=60, e_max=400)
    rowptr, col, val = oracle.csr(g.src, g.dst, g.w, g.N)
    perm = np.argsort(g.src, kind="stable")
    assert np.array_equal(col, g.dst[perm])
    wv = np.ones(g.E, np.float32) if g.w is None else g.w
    assert np.array_equal(val, wv[perm])
    expect = np.concatenate([[0], np.cumsum(np.bincount(g.src, minlength=g.N))])
    assert np.array_equal(rowptr, expect)


# ------------------------------------------------------------ brute force (Table 1)

def _brute_class_counts(src, dst, N, y, K):
    C = np.zeros((N, K), np.int64)
    for s, d in zip(src.tolist(), dst.tolist()):
        if y[d] >= 0:
            C[s, y[d]] += 1
    return C


@pytest.mark.parametrize("seed", range(40))
def test_edge_list_oracle_equals_dense_table1(seed):
    g = random_tiny(seed)
    for f in ALL_FLAGS:
        Z1 = oracle.embed_graph(g, f)
        Z2 = dense.embed_dense(g.src, g.dst, g.w, g.N, g.labels, g.K, f)
        scale = max(1.0, float(np.abs(Z2).max(initial=0.0)))
        assert np.abs(Z1 - Z2).max(initial=0.0) <= 1e-12 * scale, _flags_name(f)
        # zero pattern is structural: both forms agree exactly
        assert np.array_equal(Z1 == 0, Z2 == 0), _flags_name(f)


def test_edge_list_oracle_equals_dense_hypothesis():
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=150, deadline=None)
    @hyp.given(seed=st.integers(0, 2 ** 31), flags=st.integers(0, 7))
    def check(seed, flags):
        g = random_tiny(seed, n_max=24, e_max=80)
        Z1 = oracle.embed_graph(g, flags)
        Z2 = dense.embed_dense(g.src, g.dst, g.w, g.N, g.labels, g.K, flags)
        assert np.allclose(Z1, Z2, rtol=1e-12, atol=1e-14)

    check()


@pytest.mark.parametrize("seed", range(10))
def test_class_counts_brute_force(seed):
    g = random_tiny(seed, weighted=False)
    C = oracle.class_counts(g.src, g.dst, g.N, g.labels, g.K)
    assert np.array_equal(C, _brute_class_counts(g.src, g.dst, g.N, g.labels, g.K))


def test_label_counts_and_degrees_brute_force():
    g = random_tiny(7, weighted=True)
    nk = oracle.label_counts(g.labels, g.K)
    assert np.array_equal(nk, [sum(1 for y in g.labels if y == k) for k in range(g.K)])
    for f in (0, oracle.DIAG_AUG):
        deg = oracle.degrees(g.src, g.w, g.N, f)
        ref = [math.fsum(float(w) for s, w in zip(g.src, g.w) if s == i) + (1.0 if f else 0.0)
               for i in range(g.N)]
        assert np.allclose(deg, ref, rtol=1e-15, atol=0)


# ------------------------------------------------------------------ closed forms

def _undirected(pairs, N):
    u = np.array([p[0] for p in pairs], np.int32)
    v = np.array([p[1] for p in pairs], np.int32)
    return np.concatenate([u, v]), np.concatenate([v, u])


def test_complete_graph():
    n = 9
    y = np.array([0, 0, 1, 1, 1, 2, 2, 2, 2], np.int32)
    K = 3
    src, dst = _undirected([(i, j) for i in range(n) for j in range(i + 1, n)], n)
    nk = np.bincount(y, minlength=K)
    Z = oracle.embed(src, dst, None, n, y, K, 0)
    expect = (nk[None, :] - (y[:, None] == np.arange(K)[None, :])) / nk[None, :]
    assert np.allclose(Z, expect, rtol=1e-15, atol=0)
    # with A + I every node reaches every node of every class exactly once
    Z = oracle.embed(src, dst, None, n, y, K, oracle.DIAG_AUG)
    assert np.allclose(Z, 1.0, rtol=1e-15, atol=0)


@pytest.mark.parametrize("d", [2, 4, 6])
def test_regular_ring_lattice_laplacian(d):
    # circulant graph: node i joined to i +- 1 .. i +- d/2 (mod n), every degree is d
    n, K = 23, 4
    y = (np.arange(n) * 7 % K).astype(np.int32)
    pairs = [(i, (i + s) % n) for i in range(n) for s in range(1, d // 2 + 1)]
    src, dst = _undirected(pairs, n)
    nk = np.bincount(y, minlength=K).astype(np.float64)
    counts = np.zeros((n, K))
    for i in range(n):
        for s in range(1, d // 2 + 1):
            counts[i, y[(i + s) % n]] += 1
            counts[i, y[(i - s) % n]] += 1
    Z = oracle.embed(src, dst, None, n, y, K, oracle.LAPLACIAN)
    assert np.allclose(Z, counts / nk / d, rtol=1e-14, atol=0)          # A W / d
    Z = oracle.embed(src, dst, None, n, y, K, oracle.LAPLACIAN | oracle.DIAG_AUG)
    self_term = (y[:, None] == np.arange(K)[None, :]) / nk
    assert np.allclose(Z, (counts / nk + self_term) / (d + 1), rtol=1e-14, atol=0)


@pytest.mark.parametrize("m", [1, 5, 1000])
def test_star_graph(m):
    N = m + 1
    y = np.ones(N, np.int32)
    y[0] = 0
    src, dst = _undirected([(0, i) for i in range(1, N)], N)
    Z = oracle.embed(src, dst, None, N, y, 2, 0)
    # m terms of 1/m: exact up to the m roundings of the running sum
    assert np.allclose(Z[0], [0.0, 1.0], rtol=m * 1.2e-16, atol=0) and np.all(Z[1:] == [1.0, 0.0])
    Z = oracle.embed(src, dst, None, N, y, 2, oracle.LAPLACIAN)
    r = 1.0 / math.sqrt(m)
    assert np.allclose(Z[0], [0.0, r], rtol=m * 1.2e-16 + 1e-15, atol=0)
    assert np.allclose(Z[1:], [r, 0.0], rtol=1e-15, atol=0)
    Z = oracle.embed(src, dst, None, N, y, 2, oracle.CORRELATION | oracle.LAPLACIAN)
    assert np.allclose(Z[0], [0.0, 1.0], rtol=1e-15) and np.allclose(Z[1:], [1.0, 0.0], rtol=1e-15)


def test_single_class_is_degree_over_n():
    g = random_tiny(3, n_max=50, e_max=300, weighted=True)
    y = np.zeros(g.N, np.int32)
    Z = oracle.embed(g.src, g.dst, g.w, g.N, y, 1, 0)
    deg = np.zeros(g.N)
    np.add.at(deg, g.src, g.w.astype(np.float64))
    assert np.allclose(Z[:, 0], deg / g.N, rtol=1e-14, atol=0)


def test_isolated_and_unlabelled_nodes():
    # nodes 0-1 joined, node 2 isolated, node 3 unlabelled and joined to node 0
    src, dst = _undirected([(0, 1), (0, 3)], 4)
    y = np.array([0, 1, 1, -1], np.int32)
    Z = oracle.embed(src, dst, None, 4, y, 2, oracle.LAPLACIAN | oracle.DIAG_AUG)
    # isolated node: D = 1 after augmentation, Z_2 = e_{y_2} / n_{y_2}
    assert np.allclose(Z[2], [0.0, 0.5], rtol=1e-15)
    # the unlabelled neighbour contributes nothing to node 0
    deg = np.array([3.0, 2.0, 1.0, 2.0])
    assert np.allclose(Z[0], [1 / deg[0] / 1.0, 1 / math.sqrt(deg[0] * deg[1]) / 2.0], rtol=1e-15)
    # without augmentation an isolated node has D = 0 and a zero row
    Z = oracle.embed(src, dst, None, 4, y, 2, oracle.LAPLACIAN | oracle.CORRELATION)
    assert np.all(Z[2] == 0.0)


def test_empty_class_column_is_zero():
    g = random_tiny(11, n_max=30, e_max=200)
    y = np.minimum(g.labels, 0).astype(np.int32)    # only class 0 (and -1) used
    for f in ALL_FLAGS:
        Z = oracle.embed(g.src, g.dst, g.w, g.N, y, 3, f)
        assert np.all(Z[:, 1:] == 0.0)


# ------------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", range(8))
def test_counts_times_class_sizes(seed):
    g = random_tiny(seed, weighted=False)
    Z = oracle.embed_graph(g, 0)
    nk = oracle.label_counts(g.labels, g.K)
    C = oracle.class_counts(g.src, g.dst, g.N, g.labels, g.K)
    assert np.allclose(Z * nk[None, :], C, rtol=1e-14, atol=0)


@pytest.mark.parametrize("seed", range(8))
def test_correlation_rows_unit_or_zero(seed):
    g = random_tiny(seed)
    for f in (4, 5, 6, 7):
        Z = oracle.embed_graph(g, f)
        r = np.linalg.norm(Z, axis=1)
        assert np.all((np.abs(r - 1.0) < 1e-14) | (r == 0.0))


@pytest.mark.parametrize("seed", range(6))
def test_weight_scaling(seed):
    g = random_tiny(seed, weighted=True)
    w3 = (g.w * np.float32(3.0)).astype(np.float32)
    # without the Laplacian, A W is linear in w
    Z = oracle.embed_graph(g, 0)
    Zs = oracle.embed(g.src, g.dst, w3, g.N, g.labels, g.K, 0)
    assert np.allclose(Zs, 3.0 * Z, rtol=1e-6, atol=0)
    # augmentation adds the unscaled self term S = I W (S[i, y_i] = 1 / n_{y_i}), so
    # Z(3w) = 3 (Z(w) - S) + S
    nk = np.bincount(g.labels[g.labels >= 0], minlength=g.K).astype(np.float64)
    S = np.zeros((g.N, g.K))
    lab = np.nonzero(g.labels >= 0)[0]
    S[lab, g.labels[lab]] = 1.0 / nk[g.labels[lab]]
    Z = oracle.embed_graph(g, oracle.DIAG_AUG)
    Zs = oracle.embed(g.src, g.dst, w3, g.N, g.labels, g.K, oracle.DIAG_AUG)
    assert np.allclose(Zs, 3.0 * (Z - S) + S, rtol=1e-6, atol=1e-12)
    assert not np.allclose(Zs, 3.0 * Z, rtol=1e-6, atol=1e-12) or not lab.size
    # with the Laplacian and no augmentation, Z does not depend on the scale of w
    Z = oracle.embed_graph(g, oracle.LAPLACIAN)
    Zs = oracle.embed(g.src, g.dst, w3, g.N, g.labels, g.K, oracle.LAPLACIAN)
    assert np.allclose(Zs, Z, rtol=1e-6, atol=1e-300)


@pytest.mark.parametrize("seed", range(6))
def test_node_relabel_permutes_rows_and_edge_order_is_irrelevant(seed):
    g = random_tiny(seed)
    rng = np.random.default_rng(seed)
    pi = rng.permutation(g.N).astype(np.int32)            # new id of old node i
    y2 = np.empty_like(g.labels)
    y2[pi] = g.labels
    order = rng.permutation(g.E)
    w2 = None if g.w is None else g.w[order]
    for f in ALL_FLAGS:
        Z = oracle.embed_graph(g, f)
        Z2 = oracle.embed(pi[g.src[order]], pi[g.dst[order]], w2, g.N, y2, g.K, f)
        assert np.allclose(Z2[pi], Z, rtol=1e-13, atol=1e-300)


def test_class_relabel_permutes_columns():
    g = random_tiny(5, k_max=5)
    perm = np.random.default_rng(0).permutation(g.K)
    y2 = np.where(g.labels >= 0, perm[np.maximum(g.labels, 0)], -1).astype(np.int32)
    for f in ALL_FLAGS:
        Z = oracle.embed_graph(g, f)
        Z2 = oracle.embed(g.src, g.dst, g.w, g.N, y2, g.K, f)
        assert np.allclose(Z2[:, perm], Z, rtol=1e-14, atol=0)


# ------------------------------------------------------------------- validation

def test_validation_errors():
    src = np.array([0, 1], np.int32)
    dst = np.array([1, 0], np.int32)
    y = np.array([0, 1], np.int32)
    assert oracle.validate(src, dst, None, 2, y, 2) == 0
    assert oracle.validate(src, np.array([1, 2], np.int32), None, 2, y, 2) & oracle.ERR_INDEX
    assert oracle.validate(src, dst, None, 2, np.array([0, 2], np.int32), 2) & oracle.ERR_LABEL
    assert oracle.validate(src, dst, None, 2, np.array([0, -2], np.int32), 2) & oracle.ERR_LABEL
    bad = np.array([1.0, np.nan], np.float32)
    assert oracle.validate(src, dst, bad, 2, y, 2) & oracle.ERR_WEIGHT
    neg = np.array([1.0, -1.0], np.float32)
    assert oracle.validate(src, dst, neg, 2, y, 2, 0) == 0
    assert oracle.validate(src, dst, neg, 2, y, 2, oracle.LAPLACIAN) & oracle.ERR_WEIGHT
    with pytest.raises(ValueError):
        oracle.embed(src, dst, neg, 2, y, 2, oracle.LAPLACIAN)


def test_oracle_on_paper_sbm_small():
    # the smallest SBM of Section 4 (N = 100), all options on, against the dense form
    g = sbm(100, seed=9)
    Z1 = oracle.embed_graph(g, oracle.ALL_OPTIONS)
    Z2 = dense.embed_dense(g.src, g.dst, g.w, g.N, g.labels, g.K, oracle.ALL_OPTIONS)
    assert np.allclose(Z1, Z2, rtol=1e-13, atol=0)


@pytest.mark.parametrize("seed", range(30))
def test_row_parallel_oracle_is_bit_identical(seed):
    # the all-core CPU baseline restates the edge-list oracle row by row: each row's sums
    # keep the edge-list order, so every bit of Z must agree, for any thread count
    g = random_tiny(seed, n_max=80, e_max=600)
    for f in ALL_FLAGS:
        Z = oracle.embed_graph(g, f)
        for threads in (1, 2, 7):
            assert np.array_equal(oracle.embed_rows_graph(g, f, threads), Z)


def test_row_parallel_oracle_larger_graphs_and_errors():
    from synth import chung_lu
    for g in (chung_lu(20000, 150000, seed=41, K=9, weighted=True), sbm(1200, seed=42)):
        for f in (0, oracle.ALL_OPTIONS, oracle.DIAG_AUG | oracle.LAPLACIAN):
            assert np.array_equal(oracle.embed_rows_graph(g, f, 6), oracle.embed_graph(g, f))
    g = sbm(300, seed=43, weighted=True)
    bad = g.dst.copy()
    bad[5] = g.N
    with pytest.raises(ValueError):
        oracle.embed_rows(g.src, bad, g.w, g.N, g.labels, g.K, 7, 4)


@pytest.mark.parametrize("seed", range(10))
def test_symmetrize_interleaves_both_directions(seed):
    # the undirected reading: every listed edge followed by its reverse, except for self-loops
    g = random_tiny(seed, n_max=50, e_max=300, weighted=True)
    src, dst = np.append(g.src, [0, 0]).astype(np.int32), np.append(g.dst, [0, 1]).astype(np.int32)
    wt = np.append(g.w, [0.5, 0.25]).astype(np.float32)   # a self-loop and an edge, last
    s, d, w = oracle.symmetrize(src, dst, wt)
    keep = np.stack([np.ones(src.size, bool), src != dst], 1).reshape(-1)
    assert np.array_equal(s, np.stack([src, dst], 1).reshape(-1)[keep])
    assert np.array_equal(d, np.stack([dst, src], 1).reshape(-1)[keep])
    assert np.array_equal(w, np.stack([wt, wt], 1).reshape(-1)[keep])
    assert list(s[-3:]) == [0, 0, 1] and list(d[-3:]) == [0, 1, 0]
    s2, d2, w2 = oracle.symmetrize(src, dst, None)
    assert np.array_equal(s2, s) and np.array_equal(d2, d) and w2 is None


def test_symmetrized_one_direction_reproduces_the_undirected_graph():
    # an SBM graph stores both directions; listing each undirected edge once (src < dst) and
    # symmetrizing gives the same A, so the same Z up to summation order
    g = sbm(400, seed=91, weighted=True)
    one = g.src < g.dst
    s, d, w = oracle.symmetrize(g.src[one], g.dst[one], g.w[one])
    assert s.size == g.E
    for f in ALL_FLAGS:
        Z = oracle.embed_graph(g, f)
        Zs = oracle.embed(s, d, w, g.N, g.labels, g.K, f)
        assert np.allclose(Zs, Z, rtol=1e-12, atol=1e-15), f


def _sparse_structure(g, flags):
    """Brute force: the classes of each row's labelled neighbours, plus its own class with
    augmentation when it is labelled."""
    rows = [set() for _ in range(g.N)]
    for s, d in zip(g.src, g.dst):
        if g.labels[d] >= 0:
            rows[s].add(int(g.labels[d]))
    if flags & 1:
        for i in range(g.N):
            if g.labels[i] >= 0:
                rows[i].add(int(g.labels[i]))
    return [sorted(r) for r in rows]


@pytest.mark.parametrize("seed", range(12))
def test_sparse_z_is_the_dense_z_on_its_structure(seed):
    # Section 3 keeps Z sparse: the structure is that of (A (+I)) W, the values the dense
    # oracle's, bit for bit; every entry outside the structure is an exact zero
    g = random_tiny(seed, n_max=80, e_max=600, weighted=(seed % 2 == 0))
    for flags in ALL_FLAGS:
        rp, zc, zv = oracle.embed_sparse_graph(g, flags)
        Z = oracle.embed_graph(g, flags)
        struct = _sparse_structure(g, flags)
        assert rp[0] == 0 and np.all(np.diff(rp) >= 0)
        dense_from_sparse = np.zeros_like(Z)
        for i in range(g.N):
            cols = zc[rp[i]:rp[i + 1]]
            assert list(cols) == struct[i], (seed, flags, i)
            dense_from_sparse[i, cols] = zv[rp[i]:rp[i + 1]]
        assert np.array_equal(dense_from_sparse, Z), (seed, flags)


def test_sparse_z_with_many_classes():
    # K far above the dense limit: a star whose leaves carry distinct classes, plus a ring
    N, K = 3001, 50000
    hub = 0
    src = np.concatenate([np.zeros(N - 1, np.int32), np.arange(1, N, dtype=np.int32)])
    dst = np.concatenate([np.arange(1, N, dtype=np.int32), np.zeros(N - 1, np.int32)])
    y = (np.arange(N, dtype=np.int32) * 7) % K
    rp, zc, zv = oracle.embed_sparse(src, dst, None, N, y, K, 0)
    # the hub's row: one entry per leaf class, each 1 / n_k = 1 (every class holds one node)
    hub_cols = zc[rp[hub]:rp[hub + 1]]
    assert np.array_equal(hub_cols, np.sort(y[1:]))
    assert np.all(zv[rp[hub]:rp[hub + 1]] == 1.0)
    # a leaf's row: the hub's class only
    assert rp[2] - rp[1] == 1 and zc[rp[1]] == y[hub]
    # with augmentation and correlation every row is unit-norm
    rp, zc, zv = oracle.embed_sparse(src, dst, None, N, y, K, 5)
    for i in (0, 1, 1500):
        v = zv[rp[i]:rp[i + 1]]
        assert abs(np.sqrt(np.sum(v * v)) - 1.0) < 1e-12
