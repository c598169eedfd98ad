"""Host-side pieces of bench.py that decide what the JSON line claims (CPU only): the
algorithmic bytes of each kernel, and the rule that an ncu traffic figure is reported
only for the kernel source it was measured on."""
import hashlib
import json
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def shape(E, N, K, weighted):
    return SimpleNamespace(E=E, N=N, K=K, w=object() if weighted else None)


def test_kernel_bytes_two_pass_weighted():
    # SBM N=10,000, K=3, weighted: ids of 14 bits take two radix passes
    E, N, K = 11_124_844, 10_000, 3
    b = bench.kernel_bytes(shape(E, N, K, True))
    assert set(b) == {"k_prep", "k_scatter_first", "k_count", "k_scatter_final", "k_rowscan", "k_wdeg",
                      "k_spmm"}
    assert b["k_prep"] == 4 * E + 4 * N
    assert b["k_scatter_first"] == 12 * E + 8 * E      # src, dst, w in; packed key, w out
    assert b["k_count"] == 4 * E + 4 * N
    assert b["k_scatter_final"] == 8 * E + 8 * E       # packed key, w in; col, val out
    assert b["k_wdeg"] == 4 * E + 4 * (N + 1) + 20 * N
    # the product: col + val, index pointers, node table, D^-1/2 and Z, read or written once
    assert b["k_spmm"] == 8 * E + 4 * (N + 1) + 8 * N + 4 * N + 4 * N * K
    assert abs(b["k_spmm"] - 89.3e6) < 0.2e6           # the figure the ncu summary compares with


def test_kernel_bytes_one_pass_unweighted():
    E, N, K = 5_000, 200, 4                           # ids of 8 bits: one pass
    b = bench.kernel_bytes(shape(E, N, K, False))
    assert "k_scatter_first" not in b and "k_count" not in b
    assert b["k_scatter_final"] == 8 * E + 4 * E       # src, dst in; col out
    assert b["k_wdeg"] == 0                            # degrees come from the row lengths
    assert b["k_rowscan"] == 4 * N + 4 * (N + 1) + 20 * N
    assert b["k_spmm"] == 4 * E + 4 * (N + 1) + 12 * N + 4 * N * K


def test_one_pass_limit_matches_the_library():
    hdr = open(os.path.join(ROOT, "paper_2406_03726_gb300", "csrc", "gee_internal.cuh")).read()
    assert f"constexpr int kOnePassBits = {bench.ONE_PASS_BITS};" in hdr


@pytest.fixture()
def fake_root(tmp_path, monkeypatch):
    src = tmp_path / "paper_2406_03726_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "gee_kernels.cu").write_text("// kernels, version A\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _write_traffic(root, sha):
    (root / "profiles" / "traffic.json").write_text(json.dumps(
        {"source_sha1": sha, "sbm10k": {"k_spmm": 91373568}}))


def test_traffic_reported_for_the_profiled_source(fake_root):
    sha = hashlib.sha1((fake_root / "paper_2406_03726_gb300" / "csrc" / "gee_kernels.cu").read_bytes()).hexdigest()
    _write_traffic(fake_root, sha)
    assert bench.traffic_for("k_spmm", "sbm10k") == 91373568
    assert bench.traffic_for("k_scatter_first", "sbm10k") is None   # not captured
    assert bench.traffic_for("k_spmm", "cl600k") is None            # other workload


def test_traffic_null_once_the_kernels_change(fake_root):
    k = fake_root / "paper_2406_03726_gb300" / "csrc" / "gee_kernels.cu"
    _write_traffic(fake_root, hashlib.sha1(k.read_bytes()).hexdigest())
    k.write_text("// kernels, version B\n")
    assert bench.traffic_for("k_spmm", "sbm10k") is None


def test_traffic_null_without_a_summary(fake_root):
    assert bench.traffic_for("k_spmm", "sbm10k") is None
