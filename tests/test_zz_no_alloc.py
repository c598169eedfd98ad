"""gee_embed_static -- the entry point for callers that cannot allocate device memory.

Such callers (code that only receives device pointers from another framework, or a
latency-critical loop that must not call cudaMalloc) get a variant of gee_embed whose
scratch is an array built into the library instead of a caller workspace.  These tests
call it through the C ABI and check its Z against gee_embed's on the same inputs, for
two calls in a row on different graphs (so the second call runs on the scratch the first
one left behind), check that repeated calls on the same buffers keep giving that Z while
the device's free memory (cudaMemGetInfo) stays the same and no launch graph is cached,
and check that an oversized graph is refused without any launch.

This file is collected last on purpose: it is the only test that touches the library's
built-in scratch array.
"""
import numpy as np
import pytest

from gpu_util import assert_z_matches, dev_graph
from synth import chung_lu, sbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL = 7


@pytest.fixture(scope="module")
def gee():
    import paper_2406_03726_gb300 as gee
    gee.lib()
    return gee


def _with_workspace(gee, g, flags):
    src, dst, w, y = dev_graph(g)
    Z = gee.embed(src, dst, w, g.N, y, g.K, flags)
    torch.cuda.synchronize()
    return Z.double().cpu().numpy()


def _static(gee, g, flags):
    src, dst, w, y = dev_graph(g)
    Z = torch.full((g.N, g.K), float("nan"), dtype=torch.float32, device="cuda")
    status = torch.full((1,), 123, dtype=torch.int32, device="cuda")
    rc = gee.gee_embed_static(src, dst, w, g.E, g.N, y, g.K, gee.make_opts(flags), Z, None, status)
    assert rc == 0, gee.gee_strerror(rc)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return Z.double().cpu().numpy()


def test_static_scratch_matches_workspace_entry_point(gee):
    # a 2-pass graph with split hub rows, then a 1-pass weighted graph, then the first again
    g1 = chung_lu(40_000, 400_000, d_max=15_000, seed=31, K=12, weighted=True)
    g2 = sbm(1500, seed=32, weighted=True)
    for g, flags in ((g1, ALL), (g2, ALL), (g1, 3)):
        ref = _with_workspace(gee, g, flags)
        got = _static(gee, g, flags)
        assert_z_matches(got, ref, what=f"{g.name} flags {flags}")


def test_static_repeated_calls_allocate_nothing(gee):
    # the latency-loop case: the same buffers and options again and again
    g = sbm(2000, seed=33, weighted=True)
    src, dst, w, y = dev_graph(g)
    ref = _with_workspace(gee, g, ALL)
    Z = torch.empty((g.N, g.K), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    opts = gee.make_opts(ALL)
    assert gee.gee_graph_cache_clear() == 0

    def call():
        Z.fill_(float("nan"))
        rc = gee.gee_embed_static(src, dst, w, g.E, g.N, y, g.K, opts, Z, None, status)
        assert rc == 0, gee.gee_strerror(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert_z_matches(Z.cpu().double().numpy(), ref, what="static repeated call")  # no device copy

    call()  # the first call on the device may load the library's device code
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(4):
        call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    assert gee.gee_graph_cache_size() == (0, 0)


def test_static_scratch_refuses_oversized_graph(gee):
    # the scratch need of this shape exceeds GEE_STATIC_WORKSPACE_BYTES: refused up front
    E, N, K = 20_000_000, 10_000, 3
    assert gee.gee_workspace_size(E, N, K, True) > (64 << 20)
    one = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = gee.gee_embed_static(one, one, one, E, N, one, K, None, one, None, None)
    assert rc == 2   # GEE_ERR_TOO_LARGE
