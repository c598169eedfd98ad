"""The autotuner: it picks valid tuning fields, every candidate it runs computes Z within
the oracle tolerance, and a repeated call is answered from its cache."""
import ctypes

import numpy as np
import pytest

import oracle
from synth import chung_lu, sbm

from gpu_util import assert_z_matches, dev_graph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make", [lambda: sbm(3000, seed=51, weighted=True),
                                  lambda: chung_lu(30000, 200000, seed=52, K=24)])
def test_autotune_picks_valid_opts(make):
    import torch
    import paper_2406_03726_gb300 as gee
    g = make()
    src, dst, w, y = dev_graph(g)
    best, ms = gee.autotune(src, dst, w, g.N, y, g.K, gee.ALL_OPTIONS)
    assert best.flags == gee.ALL_OPTIONS and ms > 0.0
    assert best.hub_threshold > 0
    assert 1 <= best.rows_per_item <= 32 and best.rows_per_item & (best.rows_per_item - 1) == 0
    assert best.vec_width in (2, 4, 8) and best.short_len in (32, 64, 128, 256)
    Z = gee.embed(src, dst, w, g.N, y, g.K, opts=best)
    torch.cuda.synchronize()
    assert_z_matches(Z.cpu().numpy(), oracle.embed_graph(g, gee.ALL_OPTIONS), what="tuned opts")
    # the cache answers the second call with the same choice and time
    best2, ms2 = gee.autotune(src, dst, w, g.N, y, g.K, gee.ALL_OPTIONS)
    assert (best2.hub_threshold, best2.rows_per_item, best2.vec_width, best2.short_len, ms2) == \
        (best.hub_threshold, best.rows_per_item, best.vec_width, best.short_len, ms)


def test_every_row_block_size_gives_the_same_bits():
    """Rows per work item only changes how rows are grouped into blocks: a row's lanes
    and its sum order depend on its length alone, so Z keeps its bits."""
    import torch
    import paper_2406_03726_gb300 as gee
    g = chung_lu(20000, 120000, seed=53, K=40, weighted=True)
    src, dst, w, y = dev_graph(g)
    ref = None
    for rpi in (1, 2, 8, 32):
        Z = gee.embed(src, dst, w, g.N, y, g.K, gee.ALL_OPTIONS | gee.NO_GRAPH_CACHE, rows_per_item=rpi)
        torch.cuda.synchronize()
        if ref is None:
            ref = Z
            assert_z_matches(Z.cpu().numpy(), oracle.embed_graph(g, gee.ALL_OPTIONS), what="rpi 1")
        else:
            assert torch.equal(Z, ref), f"rows_per_item {rpi}"


@pytest.mark.parametrize("vec", [2, 4, 8])
def test_every_vector_width_gives_the_same_bits(vec):
    """The ring depth only changes how far ahead a lane's vectors are requested: every
    entry is added in the same order, so Z keeps its bits."""
    import torch
    import paper_2406_03726_gb300 as gee
    for g in (chung_lu(20000, 150000, seed=54, K=30, weighted=True), sbm(2500, seed=55, weighted=True)):
        src, dst, w, y = dev_graph(g)
        ref = gee.embed(src, dst, w, g.N, y, g.K, gee.ALL_OPTIONS | gee.NO_GRAPH_CACHE, vec_width=2)
        Z = gee.embed(src, dst, w, g.N, y, g.K, gee.ALL_OPTIONS | gee.NO_GRAPH_CACHE, vec_width=vec)
        torch.cuda.synchronize()
        assert torch.equal(Z, ref), f"{g.name} vec_width {vec}"
        assert_z_matches(Z.cpu().numpy(), oracle.embed_graph(g, gee.ALL_OPTIONS), what=f"vec {vec}")


@pytest.mark.parametrize("short_len", [16, 64, 256])
def test_short_row_bound_keeps_parity(short_len):
    import torch
    import paper_2406_03726_gb300 as gee
    g = chung_lu(30000, 250000, seed=56, K=40)
    src, dst, w, y = dev_graph(g)
    Z = gee.embed(src, dst, w, g.N, y, g.K, gee.ALL_OPTIONS | gee.NO_GRAPH_CACHE, short_len=short_len)
    torch.cuda.synchronize()
    assert_z_matches(Z.cpu().numpy(), oracle.embed_graph(g, gee.ALL_OPTIONS), what=f"short_len {short_len}")


def test_tuning_cache_persists_through_a_file(tmp_path):
    import json
    import torch
    import paper_2406_03726_gb300 as gee
    g = chung_lu(25000, 180000, seed=57, K=12)
    src, dst, w, y = dev_graph(g)
    assert gee.gee_tune_cache_clear() == 0
    best, ms = gee.autotune(src, dst, w, g.N, y, g.K, gee.ALL_OPTIONS)
    p = tmp_path / "tune.json"
    assert gee.gee_tune_cache_save(p) == 0
    entries = json.loads(p.read_text())["entries"]
    assert len(entries) == 1 and entries[0]["gpu"] == torch.cuda.get_device_name()
    assert entries[0]["best"] == [best.flags, best.hub_threshold, best.lanes_per_row, best.rows_per_item,
                                  best.vec_width, best.short_len]
    assert gee.gee_tune_cache_clear() == 0
    assert gee.gee_tune_cache_load(p) == (0, 1)
    best2, ms2 = gee.autotune(src, dst, w, g.N, y, g.K, gee.ALL_OPTIONS)   # answered from the file
    assert (best2.hub_threshold, best2.rows_per_item, best2.vec_width, best2.short_len) == \
        (best.hub_threshold, best.rows_per_item, best.vec_width, best.short_len)
    assert abs(ms2 - ms) <= 1e-6 * max(ms, 1.0)
    assert gee.gee_tune_cache_load(p) == (0, 0)                            # already cached: no duplicate
