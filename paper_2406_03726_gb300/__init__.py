"""GB300-native sparse Graph Encoder Embedding (Qin & Shen, arXiv 2406.03726).

``Z = A W`` (Eq. 1) with diagonal augmentation, Laplacian normalisation and correlation
(Section 2, Table 1), computed by hand-written sm_103a CUDA kernels behind the C ABI of
``include/gee.h``.  ``_native`` holds the one-to-one ctypes binding; the helpers below
only allocate device memory with PyTorch and call it.
"""
from __future__ import annotations

from ._native import (  # noqa: F401
    gee_request,
    gee_server_cancel,
    gee_server_config,
    gee_server_create,
    gee_server_destroy,
    gee_server_fetch,
    gee_server_get_stats,
    gee_server_poll,
    gee_server_release,
    gee_server_submit,
    gee_batch_autotune,
    gee_batch_autotune_workspace_size,
    gee_batch_plan_create,
    gee_batch_plan_destroy,
    gee_batch_plan_launch,
    gee_batch_plan_launch_timed,
    gee_batch_workspace_size,
    gee_embed_batch,
    gee_graph,
    make_graphs,
    gee_build_csr,
    gee_class_counts,
    gee_embed_sparse,
    gee_sparse_workspace_size,
    gee_embed,
    gee_embed_host,
    gee_embed_static,
    gee_graph_cache_clear,
    gee_graph_cache_size,
    gee_reembed,
    gee_tune_cache_clear,
    gee_tune_cache_load,
    gee_tune_cache_save,
    gee_shard_build,
    gee_shard_embed,
    gee_shard_table,
    gee_shard_workspace_size,
    gee_autotune,
    gee_autotune_workspace_size,
    gee_embed_timed,
    gee_host_workspace_size,
    gee_opts,
    gee_strerror,
    gee_version,
    gee_workspace_size,
    lib,
    make_opts,
)

DIAG_AUG = 1
LAPLACIAN = 2
CORRELATION = 4
ALL_OPTIONS = 7
NO_GRAPH_CACHE = 0x100
SYMMETRIZE = 0x200

STATUS_INDEX = 1
STATUS_LABEL = 2
STATUS_WEIGHT = 4
STATUS_TIMEOUT = 8
STATUS_INTERNAL = 16
STATUS_STALE = 32

ERR_NOMEM = 6
PENDING = 7
ERR_STATE = 8

PHASES = ("memset", "k_prep", "k_offsets_first", "k_scatter_first", "k_count", "k_offsets_final",
          "k_scatter_final", "k_rowscan", "k_wdeg", "k_spmm")

MAX_N = 1 << 21
MAX_E = 1 << 30
MAX_K = 64
MAX_K_SPARSE = 1 << 20


class GeeError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__(f"{what}: {gee_strerror(code)} (code {code})" if what else gee_strerror(code))
        self.code = code


def _check(rc, what):
    if rc != 0:
        raise GeeError(rc, what)


def workspace(E, N, K, weighted, opts=None, device=None):
    """A device byte tensor large enough for ``gee_embed`` on this shape."""
    import torch
    n = gee_workspace_size(E, N, K, weighted, opts)
    return torch.empty(max(n, 256), dtype=torch.uint8, device=device or "cuda")


def embed(src, dst, w, N, labels, K, flags=0, hub_threshold=0, lanes_per_row=0, ws=None, Z=None,
          status=None, stream=None, rows_per_item=0, vec_width=0, short_len=0, opts=None):
    """Z (float32 [N, K], on the device of ``src``) from device tensors.  ``status`` may be a
    uint32 device tensor of one element receiving the GEE_STATUS_* bits."""
    import torch
    E = int(src.numel())
    if opts is None:
        opts = make_opts(flags, hub_threshold, lanes_per_row, rows_per_item, vec_width, short_len)
    dev = labels.device
    if Z is None:
        Z = torch.empty((N, K), dtype=torch.float32, device=dev)
    if ws is None:
        ws = workspace(E, N, K, w is not None, opts, dev)
    rc = gee_embed(src, dst, w, E, N, labels, K, opts, Z, ws, ws.numel(), stream, status)
    _check(rc, "gee_embed")
    return Z


def autotune(src, dst, w, N, labels, K, flags=0, stream=None):
    """(opts, ms): the split threshold and rows per work item gee_autotune picks for this
    graph (a gee_opts with ``flags``), and the mean call time it measured."""
    import ctypes
    import torch
    E = int(src.numel())
    opts = make_opts(flags)
    n = gee_autotune_workspace_size(E, N, K, w is not None, opts)
    if n == 0:
        raise GeeError(1, "gee_autotune_workspace_size")
    ws = torch.empty(n, dtype=torch.uint8, device=labels.device)
    Z = torch.empty((N, K), dtype=torch.float32, device=labels.device)
    best = make_opts(flags)
    ms = ctypes.c_float(0.0)
    _check(gee_autotune(src, dst, w, E, N, labels, K, opts, Z, ws, n, stream, best, ms), "gee_autotune")
    return best, float(ms.value)


def build_csr(src, dst, w, N, labels, K, flags=0, hub_threshold=0, lanes_per_row=0, status=None, stream=None):
    """(rowptr int32 [N+1], col int32 [E], val float32 [E], n_k int32 [K], deg float32 [N])."""
    import torch
    E = int(src.numel())
    dev = labels.device
    opts = make_opts(flags, hub_threshold, lanes_per_row)
    n = gee_workspace_size(E, N, K, w is not None, opts)
    ws = torch.empty(max(n, 256), dtype=torch.uint8, device=dev)
    cap = 2 * E if flags & SYMMETRIZE else E      # both copies of every undirected edge
    rowptr = torch.empty(N + 1, dtype=torch.int32, device=dev)
    col = torch.empty(cap, dtype=torch.int32, device=dev)
    val = torch.empty(cap, dtype=torch.float32, device=dev)
    nk = torch.empty(K, dtype=torch.int32, device=dev)
    deg = torch.empty(N, dtype=torch.float32, device=dev)
    rc = gee_build_csr(src, dst, w, E, N, labels, K, opts, rowptr, col, val, nk, deg, ws, ws.numel(), stream,
                       status)
    _check(rc, "gee_build_csr")
    if flags & SYMMETRIZE:
        used = int(rowptr[N].item())
        col, val = col[:used], val[:used]
    return rowptr, col, val, nk, deg


def embed_sparse(src, dst, w, N, labels, K, flags=0, status=None, stream=None, opts=None):
    """Sparse Z (CSR over classes): (zrowptr int32 [N+1], zcol int32 [nnz], zval float32 [nnz]),
    for any K up to MAX_K_SPARSE.  Row i lists the classes of its labelled neighbours (and
    its own class with DIAG_AUG), ascending."""
    import torch
    E = int(src.numel()) if src is not None else 0
    dev = labels.device
    o = opts if opts is not None else make_opts(flags)
    n = gee_sparse_workspace_size(E, N, K, w is not None, o)
    if n == 0:
        raise GeeError(1, "gee_sparse_workspace_size")
    ws = torch.empty(max(n, 256), dtype=torch.uint8, device=dev)
    cap = (2 * E if o.flags & SYMMETRIZE else E) + N
    zrowptr = torch.empty(N + 1, dtype=torch.int32, device=dev)
    zcol = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    zval = torch.empty(max(cap, 1), dtype=torch.float32, device=dev)
    rc = gee_embed_sparse(src, dst, w, E, N, labels, K, o, zrowptr, zcol, zval, cap, ws, ws.numel(), stream, status)
    _check(rc, "gee_embed_sparse")
    nnz = int(zrowptr[N].item())
    return zrowptr, zcol[:nnz], zval[:nnz]


def class_counts(rowptr, col, N, labels, K, stream=None):
    import torch
    C = torch.empty((N, K), dtype=torch.int32, device=labels.device)
    _check(gee_class_counts(rowptr, col, N, labels, K, C, stream), "gee_class_counts")
    return C


def batch_autotune(graphs, flags=0, stream=None):
    """Tuning fields for a batch, by timing whole batch launches (gee_batch_autotune).
    graphs: (src, dst, w, labels, N, K) device tensors as for BatchPlan; their Z is
    scratch here.  Returns (gee_opts, ms per launch)."""
    import ctypes
    import torch
    items, Zs = [], []
    for (src, dst, w, labels, N, K) in graphs:
        Z = torch.empty((N, K), dtype=torch.float32, device=labels.device)
        Zs.append(Z)
        items.append((src, dst, w, labels, Z, int(src.numel()), N, K))
    arr = make_graphs(items)
    o = make_opts(flags)
    n = gee_batch_autotune_workspace_size(arr, len(items), o)
    if n == 0:
        raise GeeError(1, "gee_batch_autotune_workspace_size")
    ws = torch.empty(n, dtype=torch.uint8, device=graphs[0][3].device)
    best = make_opts(flags)
    ms = ctypes.c_float(0.0)
    _check(gee_batch_autotune(arr, len(items), o, ws, n, stream, best, ms), "gee_batch_autotune")
    del ws, Zs
    return best, float(ms.value)


class BatchPlan:
    """A reusable plan for many graphs (device tensors), launched as one kernel sequence
    (replayed as a CUDA graph with use_graph=True)."""

    def __init__(self, graphs, flags=0, hub_threshold=0, lanes_per_row=0, device=None, stream=None, opts=None):
        import torch
        self.opts = opts if opts is not None else make_opts(flags, hub_threshold, lanes_per_row)
        self.items = []
        self.Z = []
        for (src, dst, w, labels, N, K) in graphs:
            Z = torch.empty((N, K), dtype=torch.float32, device=labels.device)
            self.Z.append(Z)
            self.items.append((src, dst, w, labels, Z, int(src.numel()), N, K))
        self.G = len(self.items)
        self.arr = make_graphs(self.items)
        n = gee_batch_workspace_size(self.arr, self.G, self.opts)
        if n == 0:
            raise GeeError(1, "gee_batch_workspace_size")
        self.ws = torch.empty(n, dtype=torch.uint8, device=device or graphs[0][3].device)
        self.status = torch.zeros(self.G, dtype=torch.int32, device=self.ws.device)
        rc, self.handle = gee_batch_plan_create(self.arr, self.G, self.opts, self.ws, n, stream)
        _check(rc, "gee_batch_plan_create")

    def launch(self, stream=None, use_graph=True, status=True):
        rc = gee_batch_plan_launch(self.handle, stream, self.status if status else None, use_graph)
        _check(rc, "gee_batch_plan_launch")
        return self.Z

    def launch_timed(self, phase_ms, stream=None):
        """Launch with per-phase CUDA-event times written into the float32 array phase_ms."""
        _check(gee_batch_plan_launch_timed(self.handle, stream, phase_ms), "gee_batch_plan_launch_timed")
        return self.Z

    def close(self):
        if getattr(self, "handle", None) is not None:
            gee_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (one device memory pool of `budget` bytes).  Requests are
    NumPy host arrays (pinned memory is used when given torch pinned tensors); the caller
    keeps them alive until the request completes."""

    def __init__(self, budget, flags=0, max_batch=0, streams=0):
        cfg = gee_server_config(int(budget), max_batch, streams, flags, 0)
        rc, self.handle = gee_server_create(cfg)
        _check(rc, "gee_server_create")
        self._keep = {}

    def submit(self, src, dst, w, labels, N, K):
        E = int(len(src))
        req = gee_request(_ptr(src), _ptr(dst), _ptr(w), _ptr(labels), E, N, K)
        rc, ticket = gee_server_submit(self.handle, req)
        if rc:
            raise GeeError(rc, "gee_server_submit")
        self._keep[ticket] = (src, dst, w, labels, N, K)
        return ticket

    def poll(self, ticket, wait=False):
        """None while pending, else (device Z address, status bits, latency ms)."""
        rc, z, st, lat = gee_server_poll(self.handle, ticket, wait)
        if rc == PENDING:
            return None
        _check(rc, "gee_server_poll")
        return z, st, lat

    def fetch(self, ticket):
        import numpy as np
        _, _, _, _, N, K = self._keep[ticket]
        Z = np.empty((N, K), np.float32)
        _check(gee_server_fetch(self.handle, ticket, Z), "gee_server_fetch")
        return Z

    def cancel(self, ticket):
        rc = gee_server_cancel(self.handle, ticket)
        if rc == 0:
            self._keep.pop(ticket, None)
        return rc

    def release(self, ticket):
        _check(gee_server_release(self.handle, ticket), "gee_server_release")
        self._keep.pop(ticket, None)

    def stats(self):
        rc, st = gee_server_get_stats(self.handle)
        _check(rc, "gee_server_get_stats")
        return {f: getattr(st, f) for f, _ in st._fields_ if f != "reserved"}

    def close(self):
        if getattr(self, "handle", None) is not None:
            gee_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(a):
    from ._native import ptr
    return ptr(a)
