"""Statistics of the seeded generators against what the paper prints (CPU only)."""
import json
import os

import numpy as np
import pytest

from synth import (batch_graph, batch_specs, chung_lu, edge_density, expected_sbm_edges,
                   random_tiny, sbm)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_table2_density_eq2():
    fx = json.load(open(os.path.join(GOLDEN, "table2_density.json")))
    for d in fx["datasets"]:
        assert abs(edge_density(d["edges"], d["nodes"]) - d["density"]) <= 1e-5, d["name"]


def test_section4_sbm_edge_range():
    fx = json.load(open(os.path.join(GOLDEN, "sbm_section4.json")))
    small, _ = expected_sbm_edges(fx["sizes"][0], fx["priors"], fx["p_in"], fx["p_out"])
    large, _ = expected_sbm_edges(fx["sizes"][-1], fx["priors"], fx["p_in"], fx["p_out"])
    assert round(small / 1e3, 1) == fx["edges_smallest_thousands"]
    assert round(large / 1e6, 1) == fx["edges_largest_millions"]


@pytest.mark.parametrize("N,seed", [(100, 1), (1000, 2), (3000, 3)])
def test_sbm_edge_count_and_symmetry(N, seed):
    g = sbm(N, seed=seed, weighted=True)
    m = g.meta["undirected_edges"]
    mean, std = expected_sbm_edges(N, labels=g.labels)
    assert abs(m - mean) <= 5 * std + 1
    assert g.E == 2 * m
    a = np.stack([g.src, g.dst, g.w.view(np.int32)], 1)
    b = np.stack([g.dst, g.src, g.w.view(np.int32)], 1)
    a = a[np.lexsort(a.T[::-1])]
    b = b[np.lexsort(b.T[::-1])]
    assert np.array_equal(a, b)
    assert np.all(g.src != g.dst)
    assert g.w.min() > 0 and g.w.max() <= 1


def test_sbm_within_between_ratio():
    g = sbm(3000, seed=5)
    same = g.labels[g.src] == g.labels[g.dst]
    n = np.bincount(g.labels, minlength=3).astype(np.float64)
    within_pairs = np.sum(n * (n - 1)) / 2
    between_pairs = 3000 * 2999 / 2 - within_pairs
    p_in = same.sum() / 2 / within_pairs
    p_out = (~same).sum() / 2 / between_pairs
    assert abs(p_in - 0.13) < 0.005 and abs(p_out - 0.10) < 0.005


def test_chung_lu_small_properties():
    g = chung_lu(20_000, 200_000, d_max=5_000, seed=7, K=10)
    assert g.E == 400_000
    assert np.all(g.src != g.dst)
    key = np.minimum(g.src, g.dst).astype(np.int64) * g.N + np.maximum(g.src, g.dst)
    assert np.unique(key).size == 200_000          # deduplicated
    deg = np.bincount(g.src, minlength=g.N)
    assert deg.max() > 20 * deg.mean()             # heavy tail
    sizes = np.bincount(g.labels, minlength=10)
    assert np.all(np.diff(sizes) <= 0) and sizes.min() >= 1   # Zipf class sizes


def test_batch_specs_ranges():
    sp = batch_specs(512, seed=4)
    N = np.array([s["N"] for s in sp])
    K = np.array([s["K"] for s in sp])
    assert N.min() >= 100 and N.max() <= 50_000
    assert K.min() >= 2 and K.max() <= 64
    d = np.array([s["E"] / s["N"] for s in sp])
    assert d.min() >= 4.9 and d.max() <= 200.1
    g = batch_graph(sp[0])
    assert g.E == sp[0]["E"] and g.N == sp[0]["N"] and np.all(g.src != g.dst)


def test_generators_are_seeded():
    a, b = random_tiny(3), random_tiny(3)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.labels, b.labels)
    a, b = sbm(500, seed=4), sbm(500, seed=4)
    assert np.array_equal(a.dst, b.dst)
