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
    Z = gee.embed(src, dst, w, g.N, y, g.K, gee.ALL_OPTIONS, hub_threshold=best.hub_threshold,
                  rows_per_item=best.rows_per_item)
    torch.cuda.synchronize()
    assert_z_matches(Z.cpu().numpy(), oracle.embed_graph(g, gee.ALL_OPTIONS), what="tuned opts")
    # the cache answers the second call with the same choice and time
    best2, ms2 = gee.autotune(src, dst, w, g.N, y, g.K, gee.ALL_OPTIONS)
    assert (best2.hub_threshold, best2.rows_per_item, ms2) == (best.hub_threshold, best.rows_per_item, ms)


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
