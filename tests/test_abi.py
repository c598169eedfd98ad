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
    # row shards: the range must lie in [0, N], and undirected-once input is refused
    assert gee.gee_shard_workspace_size(100, 50, 0, 20, 3, False, gee.make_opts(7)) > 0
    assert gee.gee_shard_workspace_size(100, 50, 30, 20, 3, False, gee.make_opts(7)) == 0
    assert gee.gee_shard_workspace_size(100, 50, 0, 51, 3, False, gee.make_opts(7)) == 0
    assert gee.gee_shard_workspace_size(100, 50, 0, 20, 3, False, gee.make_opts(7 | gee.SYMMETRIZE)) == 0


def test_sparse_and_batch_tuner_host_checks(lib):
    import paper_2406_03726_gb300 as gee
    from paper_2406_03726_gb300 import _native as nat
    o = gee.make_opts(7)
    # sparse Z: K up to 2^20 classes, the usual N and E limits
    assert gee.gee_sparse_workspace_size(1000, 100, 1 << 20, False, o) > 0
    assert gee.gee_sparse_workspace_size(1000, 100, (1 << 20) + 1, False, o) == 0
    assert gee.gee_sparse_workspace_size(1000, (1 << 21) + 1, 5, False, o) == 0
    assert gee.gee_sparse_workspace_size(1000, 100, 0, False, o) == 0
    # the workspace holds the CSR build plus two run buffers of E + N entries
    assert gee.gee_sparse_workspace_size(10_000, 500, 7, True, o) > gee.gee_workspace_size(10_000, 500, 7, True, o)
    # too little room for Z's entries (E + N) is refused before any CUDA call
    assert gee.gee_embed_sparse(1, 1, None, 40, 10, 1, 3, o, 1, 1, 1, 49, 1, 1 << 20) == 1
    assert gee.gee_embed_sparse(1, 1, None, 40, 10, 1, 3, gee.make_opts(7 | gee.SYMMETRIZE), 1, 1, 1, 89, 1,
                                1 << 20) == 1
    # the batch tuner's workspace covers every candidate plan
    graphs = (nat.gee_graph * 2)()
    graphs[0] = nat.gee_graph(1, 1, 1, 1, 1, 5000, 300, 20)
    graphs[1] = nat.gee_graph(1, 1, None, 1, 1, 800, 90, 4)
    base = gee.gee_batch_workspace_size(graphs, 2, o)
    assert base > 0 and gee.gee_batch_autotune_workspace_size(graphs, 2, o) >= base


def test_tuning_fields_checked_on_host(lib):
    import paper_2406_03726_gb300 as gee
    # rows_per_item and lanes_per_row must be powers of two up to 32
    for bad in (gee.make_opts(7, 0, 0, 3), gee.make_opts(7, 0, 0, 64), gee.make_opts(7, 0, 5, 0),
                gee.make_opts(7, -1, 0, 0)):
        assert gee.gee_embed(1, 1, None, 4, 5, 1, 3, bad, 1, 1, 1 << 20) == 1
    # ring depth 2, 4 or 8; short-row bound a power of two from 8 to 256 (0: automatic)
    for bad in (gee.make_opts(7, 0, 0, 0, 3), gee.make_opts(7, 0, 0, 0, 16), gee.make_opts(7, 0, 0, 0, 0, 48),
                gee.make_opts(7, 0, 0, 0, 0, 4), gee.make_opts(7, 0, 0, 0, 0, 512)):
        assert gee.gee_embed(1, 1, None, 4, 5, 1, 3, bad, 1, 1, 1 << 20) == 1
    # the autotuner's workspace covers every candidate, so it is at least the plain one
    for E, N, K, w in ((11_124_844, 10_000, 3, True), (20_000_000, 600_000, 50, False), (100, 10, 2, True)):
        assert gee.gee_autotune_workspace_size(E, N, K, w) >= gee.gee_workspace_size(E, N, K, w)
    assert gee.gee_autotune_workspace_size(10, 1 << 22, 3, False) == 0
    best = gee.make_opts(7)
    assert gee.gee_autotune(None, None, None, 10, 5, None, 3, None, None, None, 0, None, None) == 1  # no best
    assert gee.gee_autotune(None, None, None, 0, 1 << 22, 1, 3, None, 1, 1, 0, None, best) == 2     # N too large


def _c_layout(tmp_path, body):
    """Compile and run a C program including gee.h (plain C, no CUDA); returns its stdout."""
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not found")
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "gee.h"\nint main(void) {\n'
                   + body + "return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    return subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout


def test_binding_structs_match_header(tmp_path):
    import ctypes
    import paper_2406_03726_gb300._native as nat
    structs = {"gee_opts": nat.gee_opts, "gee_graph": nat.gee_graph, "gee_server_config": nat.gee_server_config,
               "gee_request": nat.gee_request, "gee_server_stats": nat.gee_server_stats}
    body = ""
    for name, cls in structs.items():
        body += f'printf("{name} size %zu\\n", sizeof({name}));\n'
        for f, _ in cls._fields_:
            body += f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));\n'
    got = {}
    for line in _c_layout(tmp_path, body).splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


def test_python_constants_match_header(tmp_path):
    import paper_2406_03726_gb300 as gee
    pairs = {"GEE_DIAG_AUG": gee.DIAG_AUG, "GEE_LAPLACIAN": gee.LAPLACIAN, "GEE_CORRELATION": gee.CORRELATION,
             "GEE_ALL_OPTIONS": gee.ALL_OPTIONS, "GEE_NO_GRAPH_CACHE": gee.NO_GRAPH_CACHE,
             "GEE_SYMMETRIZE": gee.SYMMETRIZE,
             "GEE_STATUS_INDEX": gee.STATUS_INDEX, "GEE_STATUS_LABEL": gee.STATUS_LABEL,
             "GEE_STATUS_WEIGHT": gee.STATUS_WEIGHT, "GEE_STATUS_TIMEOUT": gee.STATUS_TIMEOUT,
             "GEE_STATUS_INTERNAL": gee.STATUS_INTERNAL, "GEE_STATUS_STALE": gee.STATUS_STALE,
             "GEE_ERR_NOMEM": gee.ERR_NOMEM, "GEE_PENDING": gee.PENDING, "GEE_ERR_STATE": gee.ERR_STATE,
             "GEE_MAX_N": gee.MAX_N, "GEE_MAX_E": gee.MAX_E, "GEE_MAX_K": gee.MAX_K,
             "GEE_MAX_K_SPARSE": gee.MAX_K_SPARSE,
             "GEE_NUM_PHASES": len(gee.PHASES)}
    body = "".join(f'printf("{k} %lld\\n", (long long)({k}));\n' for k in pairs)
    got = dict((k, int(v)) for k, v in (line.split() for line in _c_layout(tmp_path, body).splitlines()))
    for k, v in pairs.items():
        assert got[k] == v, k


def test_kernel_constants_match_header(tmp_path):
    # the kernels carry their own copies of the status bits, option bits and K limit
    hdr = open(os.path.join(ROOT, "paper_2406_03726_gb300", "csrc", "gee_internal.cuh")).read()
    consts = {m[0]: int(m[1]) for m in re.findall(r"\b(k\w+) = (\d+)u?\b", hdr)}
    body = "".join(f'printf("{k} %lld\\n", (long long)({k}));\n' for k in
                   ("GEE_STATUS_INDEX", "GEE_STATUS_LABEL", "GEE_STATUS_WEIGHT", "GEE_STATUS_TIMEOUT",
                    "GEE_STATUS_INTERNAL", "GEE_STATUS_STALE", "GEE_DIAG_AUG", "GEE_LAPLACIAN", "GEE_CORRELATION", "GEE_MAX_K"))
    c = dict((k, int(v)) for k, v in (line.split() for line in _c_layout(tmp_path, body).splitlines()))
    assert (consts["kStIndex"], consts["kStLabel"], consts["kStWeight"], consts["kStTimeout"],
            consts["kStInternal"], consts["kStStale"]) == (c["GEE_STATUS_INDEX"], c["GEE_STATUS_LABEL"],
                                                         c["GEE_STATUS_WEIGHT"], c["GEE_STATUS_TIMEOUT"],
                                                         c["GEE_STATUS_INTERNAL"], c["GEE_STATUS_STALE"])
    assert (consts["kOptAug"], consts["kOptLap"], consts["kOptCor"]) == \
        (c["GEE_DIAG_AUG"], c["GEE_LAPLACIAN"], c["GEE_CORRELATION"])
    assert consts["kMaxK"] == c["GEE_MAX_K"]


def test_tune_cache_file_roundtrip_on_the_host(lib, tmp_path):
    # the file format needs no GPU: an empty cache saves as valid JSON; a file with entries of
    # another GPU loads nothing (they stay in the file); malformed or missing files are refused
    import json
    import paper_2406_03726_gb300 as gee
    assert gee.gee_tune_cache_clear() == 0
    p = tmp_path / "tune.json"
    assert gee.gee_tune_cache_save(p) == 0
    assert json.loads(p.read_text()) == {"format": "gee-tune-1", "entries": []}
    entry = ('{"gpu": "Some Other GPU", "E": 1000, "N": 100, "K": 3, "weighted": 1, '
             '"fixed": [7, 0, 0, 0, 0, 0], "best": [7, 2048, 0, 4, 8, 64], "ms": 0.125}')
    p.write_text('{"format": "gee-tune-1", "entries": [\n' + entry + '\n]}\n')
    assert json.loads(p.read_text())["entries"][0]["best"] == [7, 2048, 0, 4, 8, 64]
    assert gee.gee_tune_cache_load(p) == (0, 0)
    bad = tmp_path / "bad.json"
    bad.write_text('{"format": "gee-tune-1", "entries": [\n{"gpu": "X", "E": oops}\n]}\n')
    assert gee.gee_tune_cache_load(bad)[0] == 1
    assert gee.gee_tune_cache_load(tmp_path / "missing.json")[0] == 1
    nohead = tmp_path / "nohead.json"
    nohead.write_text(entry + "\n")
    assert gee.gee_tune_cache_load(nohead)[0] == 1
