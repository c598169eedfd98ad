"""The C-ABI library builds, loads and exports every entry point declared in include/gee.h
(CPU only: no call here touches a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(gee_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_03726_gb300.build import build_library
    build_library()
    import paper_2406_03726_gb300 as gee
    return gee.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("gee_embed", "gee_workspace_size", "gee_build_csr", "gee_class_counts", "gee_embed_host",
                 "gee_strerror", "gee_version"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_2406_03726_gb300._native as nat
    for n in declared_functions():
        assert hasattr(nat, n), n


def test_host_only_calls(lib):
    import paper_2406_03726_gb300 as gee
    assert gee.gee_version() >= 100
    assert "workspace" in gee.gee_strerror(3)
    # sizing is pure host arithmetic
    n1 = gee.gee_workspace_size(11_124_844, 10_000, 3, True)
    n0 = gee.gee_workspace_size(11_124_844, 10_000, 3, False)
    assert n1 > n0 > 11_124_844 * 4
    assert gee.gee_workspace_size(10, 1 << 22, 3, False) == 0     # beyond the N limit
    assert gee.gee_workspace_size(10, 100, 65, False) == 0         # beyond the K limit
    assert gee.gee_host_workspace_size(100, 10, 3, True) > gee.gee_workspace_size(100, 10, 3, True)


def test_argument_errors_need_no_gpu(lib):
    import paper_2406_03726_gb300 as gee
    # rejected before any CUDA call
    assert gee.gee_embed(None, None, None, 10, 5, None, 3, None, None, None, 0) == 1          # NULL inputs
    assert gee.gee_embed(None, None, None, 0, 5, 1, 0, None, 1, None, 0) == 1                 # K = 0
    assert gee.gee_embed(None, None, None, 0, 1 << 22, 1, 3, None, 1, None, 0) == 2           # N too large
    assert gee.gee_class_counts(None, None, 5, None, 3, None) == 1


def test_tuning_fields_checked_on_host(lib):
    import paper_2406_03726_gb300 as gee
    # rows_per_item and lanes_per_row must be powers of two up to 32
    for bad in (gee.make_opts(7, 0, 0, 3), gee.make_opts(7, 0, 0, 64), gee.make_opts(7, 0, 5, 0),
                gee.make_opts(7, -1, 0, 0)):
        assert gee.gee_embed(1, 1, None, 4, 5, 1, 3, bad, 1, 1, 1 << 20) == 1
    # the autotuner's workspace covers every candidate, so it is at least the plain one
    for E, N, K, w in ((11_124_844, 10_000, 3, True), (20_000_000, 600_000, 50, False), (100, 10, 2, True)):
        assert gee.gee_autotune_workspace_size(E, N, K, w) >= gee.gee_workspace_size(E, N, K, w)
    assert gee.gee_autotune_workspace_size(10, 1 << 22, 3, False) == 0
    best = gee.make_opts(7)
    assert gee.gee_autotune(None, None, None, 10, 5, None, 3, None, None, None, 0, None, None) == 1  # no best
    assert gee.gee_autotune(None, None, None, 0, 1 << 22, 1, 3, None, 1, 1, 0, None, best) == 2     # N too large
