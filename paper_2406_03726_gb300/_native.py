"""ctypes binding of libgee.so: one Python function per C entry point, same names, same
arguments.  Arguments are marshalled only (tensors / ints -> pointers); every step of
the computation runs in the CUDA library.  There is no fallback: if the library is not
built, every call raises."""
from __future__ import annotations

import ctypes
import os

from .build import LIB_PATH

_P = ctypes.c_void_p
_I32, _I64, _U32, _SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t


class gee_opts(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("hub_threshold", ctypes.c_int32),
                ("lanes_per_row", ctypes.c_int32), ("rows_per_item", ctypes.c_int32),
                ("vec_width", ctypes.c_int32), ("short_len", ctypes.c_int32)]


class gee_graph(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("Z", ctypes.c_void_p), ("E", ctypes.c_int64),
                ("N", ctypes.c_int32), ("K", ctypes.c_int32)]


class gee_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_batch", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


class gee_request(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("E", ctypes.c_int64), ("N", ctypes.c_int32), ("K", ctypes.c_int32)]


class gee_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("running", ctypes.c_int64), ("launches", ctypes.c_int64), ("edges_done", ctypes.c_int64),
                ("pool_bytes", ctypes.c_uint64), ("bytes_in_use", ctypes.c_uint64),
                ("peak_bytes_in_use", ctypes.c_uint64), ("last_error", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_SIGNATURES = {
    "gee_version": ([], ctypes.c_int),
    "gee_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "gee_workspace_size": ([_I64, _I32, _I32, ctypes.c_int, _P], _SZ),
    "gee_host_workspace_size": ([_I64, _I32, _I32, ctypes.c_int, _P], _SZ),
    "gee_embed": ([_P, _P, _P, _I64, _I32, _P, _I32, _P, _P, _P, _SZ, _P, _P], ctypes.c_int),
    "gee_embed_timed": ([_P, _P, _P, _I64, _I32, _P, _I32, _P, _P, _P, _SZ, _P, _P, _P], ctypes.c_int),
    "gee_build_csr": ([_P, _P, _P, _I64, _I32, _P, _I32, _P, _P, _P, _P, _P, _P, _P, _SZ, _P, _P],
                      ctypes.c_int),
    "gee_class_counts": ([_P, _P, _I32, _P, _I32, _P, _P], ctypes.c_int),
    "gee_embed_static": ([_P, _P, _P, _I64, _I32, _P, _I32, _P, _P, _P, _P], ctypes.c_int),
    "gee_graph_cache_clear": ([], ctypes.c_int),
    "gee_graph_cache_size": ([_P], ctypes.c_int),
    "gee_tune_cache_save": ([ctypes.c_char_p], ctypes.c_int),
    "gee_tune_cache_load": ([ctypes.c_char_p, _P], ctypes.c_int),
    "gee_tune_cache_clear": ([], ctypes.c_int),
    "gee_reembed": ([_P, _I64, _I32, _I32, ctypes.c_int, _P, _P, _P, _SZ, _P, _P], ctypes.c_int),
    "gee_shard_workspace_size": ([_I64, _I32, _I32, _I32, _I32, ctypes.c_int, _P], _SZ),
    "gee_sparse_workspace_size": ([_I64, _I32, _I32, ctypes.c_int, _P], _SZ),
    "gee_embed_sparse": ([_P, _P, _P, _I64, _I32, _P, _I32, _P, _P, _P, _P, _I64, _P, _SZ, _P, _P], ctypes.c_int),
    "gee_shard_build": ([_P, _P, _P, _I64, _I32, _I32, _I32, _P, _I32, _P, _P, _P, _SZ, _P, _P], ctypes.c_int),
    "gee_shard_table": ([_I64, _I32, _I32, _I32, _P, _I32, ctypes.c_int, _P, _P, _P, _P, _SZ, _P], ctypes.c_int),
    "gee_shard_embed": ([_I64, _I32, _I32, _I32, _P, _I32, ctypes.c_int, _P, _P, _P, _P, _SZ, _P, _P],
                        ctypes.c_int),
    "gee_autotune_workspace_size": ([_I64, _I32, _I32, ctypes.c_int, _P], _SZ),
    "gee_autotune": ([_P, _P, _P, _I64, _I32, _P, _I32, _P, _P, _P, _SZ, _P, _P, _P], ctypes.c_int),
    "gee_batch_workspace_size": ([_P, _I32, _P], _SZ),
    "gee_embed_batch": ([_P, _I32, _P, _P, _SZ, _P, _P], ctypes.c_int),
    "gee_batch_plan_create": ([_P, _I32, _P, _P, _SZ, _P, _P], ctypes.c_int),
    "gee_batch_plan_launch": ([_P, _P, _P, ctypes.c_int], ctypes.c_int),
    "gee_batch_plan_launch_timed": ([_P, _P, _P], ctypes.c_int),
    "gee_batch_plan_destroy": ([_P], None),
    "gee_batch_autotune_workspace_size": ([_P, _I32, _P], _SZ),
    "gee_batch_autotune": ([_P, _I32, _P, _P, _SZ, _P, _P, _P], ctypes.c_int),
    "gee_server_create": ([_P, _P], ctypes.c_int),
    "gee_server_submit": ([_P, _P, _P], ctypes.c_int),
    "gee_server_poll": ([_P, _I64, ctypes.c_int, _P, _P, _P], ctypes.c_int),
    "gee_server_fetch": ([_P, _I64, _P], ctypes.c_int),
    "gee_server_cancel": ([_P, _I64], ctypes.c_int),
    "gee_server_release": ([_P, _I64], ctypes.c_int),
    "gee_server_get_stats": ([_P, _P], ctypes.c_int),
    "gee_server_destroy": ([_P], None),
    "gee_embed_host": ([_P, _P, _P, _I64, _I32, _P, _I32, _P, _P, _P, _SZ, _P, _P], ctypes.c_int),
}

_lib = None


def library_path() -> str:
    return LIB_PATH


def lib():
    """The loaded libgee.so.  Raises RuntimeError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgee.so is not built ({LIB_PATH}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def ptr(x):
    """Device/host address of a tensor, ndarray, int or None (-> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_opts(flags=0, hub_threshold=0, lanes_per_row=0, rows_per_item=0, vec_width=0, short_len=0):
    return gee_opts(flags, hub_threshold, lanes_per_row, rows_per_item, vec_width, short_len)


def _opts_ref(opts):
    if opts is None:
        return None
    if isinstance(opts, int):
        opts = make_opts(opts)
    return ctypes.byref(opts)


# ---- one function per C entry point ----------------------------------------------------

def gee_version() -> int:
    return lib().gee_version()


def gee_strerror(code: int) -> str:
    return lib().gee_strerror(code).decode()


def gee_workspace_size(E, N, K, weighted, opts=None) -> int:
    return lib().gee_workspace_size(E, N, K, 1 if weighted else 0, _opts_ref(opts))


def gee_host_workspace_size(E, N, K, weighted, opts=None) -> int:
    return lib().gee_host_workspace_size(E, N, K, 1 if weighted else 0, _opts_ref(opts))


def gee_embed(src, dst, w, E, N, labels, K, opts, Z, workspace, workspace_bytes, stream=None, d_status=None) -> int:
    return lib().gee_embed(ptr(src), ptr(dst), ptr(w), E, N, ptr(labels), K, _opts_ref(opts), ptr(Z),
                           ptr(workspace), workspace_bytes, stream_handle(stream), ptr(d_status))


def gee_embed_timed(src, dst, w, E, N, labels, K, opts, Z, workspace, workspace_bytes, stream=None,
                    d_status=None, phase_ms=None) -> int:
    return lib().gee_embed_timed(ptr(src), ptr(dst), ptr(w), E, N, ptr(labels), K, _opts_ref(opts), ptr(Z),
                                 ptr(workspace), workspace_bytes, stream_handle(stream), ptr(d_status),
                                 ptr(phase_ms))


def gee_build_csr(src, dst, w, E, N, labels, K, opts, rowptr, col, val, nk, deg, workspace, workspace_bytes,
                  stream=None, d_status=None) -> int:
    return lib().gee_build_csr(ptr(src), ptr(dst), ptr(w), E, N, ptr(labels), K, _opts_ref(opts), ptr(rowptr),
                               ptr(col), ptr(val), ptr(nk), ptr(deg), ptr(workspace), workspace_bytes,
                               stream_handle(stream), ptr(d_status))


def gee_class_counts(rowptr, col, N, labels, K, C, stream=None) -> int:
    return lib().gee_class_counts(ptr(rowptr), ptr(col), N, ptr(labels), K, ptr(C), stream_handle(stream))


def gee_embed_host(src, dst, w, E, N, labels, K, opts, Z, workspace, workspace_bytes, stream=None,
                   status=None) -> int:
    return lib().gee_embed_host(ptr(src), ptr(dst), ptr(w), E, N, ptr(labels), K, _opts_ref(opts), ptr(Z),
                                ptr(workspace), workspace_bytes, stream_handle(stream), ptr(status))


def gee_embed_static(src, dst, w, E, N, labels, K, opts, Z, stream=None, d_status=None) -> int:
    return lib().gee_embed_static(ptr(src), ptr(dst), ptr(w), E, N, ptr(labels), K, _opts_ref(opts), ptr(Z),
                                  stream_handle(stream), ptr(d_status))


def gee_autotune_workspace_size(E, N, K, weighted, opts=None) -> int:
    return lib().gee_autotune_workspace_size(E, N, K, 1 if weighted else 0, _opts_ref(opts))


def gee_autotune(src, dst, w, E, N, labels, K, opts, Z, workspace, workspace_bytes, stream=None, best=None,
                 best_ms=None) -> int:
    """best: a gee_opts to fill; best_ms: a ctypes.c_float or None."""
    return lib().gee_autotune(ptr(src), ptr(dst), ptr(w), E, N, ptr(labels), K, _opts_ref(opts), ptr(Z),
                              ptr(workspace), workspace_bytes, stream_handle(stream),
                              ctypes.byref(best) if best is not None else None,
                              ctypes.byref(best_ms) if best_ms is not None else None)


def gee_graph_cache_clear() -> int:
    return lib().gee_graph_cache_clear()


def gee_reembed(labels, E, N, K, weighted, opts, Z, workspace, workspace_bytes, stream=None, d_status=None) -> int:
    return lib().gee_reembed(ptr(labels), E, N, K, int(bool(weighted)), _opts_ref(opts), ptr(Z), ptr(workspace),
                             workspace_bytes, stream_handle(stream), ptr(d_status))


def gee_sparse_workspace_size(E, N, K, weighted, opts=None) -> int:
    return lib().gee_sparse_workspace_size(E, N, K, int(bool(weighted)), _opts_ref(opts))


def gee_embed_sparse(src, dst, w, E, N, labels, K, opts, zrowptr, zcol, zval, zcap, workspace, workspace_bytes,
                     stream=None, d_status=None) -> int:
    return lib().gee_embed_sparse(ptr(src), ptr(dst), ptr(w), E, N, ptr(labels), K, _opts_ref(opts), ptr(zrowptr),
                                  ptr(zcol), ptr(zval), zcap, ptr(workspace), workspace_bytes, stream_handle(stream),
                                  ptr(d_status))


def gee_shard_workspace_size(E, N, r0, r1, K, weighted, opts=None) -> int:
    return lib().gee_shard_workspace_size(E, N, r0, r1, K, int(bool(weighted)), _opts_ref(opts))


def gee_shard_build(src, dst, w, E, N, r0, r1, labels, K, opts, nk, workspace, workspace_bytes, stream=None,
                    d_status=None) -> int:
    return lib().gee_shard_build(ptr(src), ptr(dst), ptr(w), E, N, r0, r1, ptr(labels), K, _opts_ref(opts), ptr(nk),
                                 ptr(workspace), workspace_bytes, stream_handle(stream), ptr(d_status))


def gee_shard_table(E, N, r0, r1, labels, K, weighted, opts, nk, tab, workspace, workspace_bytes, stream=None) -> int:
    return lib().gee_shard_table(E, N, r0, r1, ptr(labels), K, int(bool(weighted)), _opts_ref(opts), ptr(nk), ptr(tab),
                                 ptr(workspace), workspace_bytes, stream_handle(stream))


def gee_shard_embed(E, N, r0, r1, labels, K, weighted, opts, tab, Z, workspace, workspace_bytes, stream=None,
                    d_status=None) -> int:
    return lib().gee_shard_embed(E, N, r0, r1, ptr(labels), K, int(bool(weighted)), _opts_ref(opts), ptr(tab), ptr(Z),
                                 ptr(workspace), workspace_bytes, stream_handle(stream), ptr(d_status))


def gee_tune_cache_save(path) -> int:
    return lib().gee_tune_cache_save(str(path).encode())


def gee_tune_cache_load(path):
    """(rc, entries loaded)."""
    n = ctypes.c_int(0)
    rc = lib().gee_tune_cache_load(str(path).encode(), ctypes.byref(n))
    return rc, n.value


def gee_tune_cache_clear() -> int:
    return lib().gee_tune_cache_clear()


def gee_graph_cache_size():
    """(remembered argument sets, of which captured as CUDA graphs)."""
    cap = ctypes.c_int(0)
    n = lib().gee_graph_cache_size(ctypes.byref(cap))
    return n, cap.value


def make_graphs(items):
    """ctypes array of gee_graph from (src, dst, w, labels, Z, E, N, K) tuples."""
    arr = (gee_graph * len(items))()
    for i, (src, dst, w, labels, Z, E, N, K) in enumerate(items):
        arr[i] = gee_graph(ptr(src), ptr(dst), ptr(w), ptr(labels), ptr(Z), E, N, K)
    return arr


def gee_batch_workspace_size(graphs, G, opts=None) -> int:
    return lib().gee_batch_workspace_size(graphs, G, _opts_ref(opts))


def gee_batch_autotune_workspace_size(graphs, G, opts=None) -> int:
    return lib().gee_batch_autotune_workspace_size(graphs, G, _opts_ref(opts))


def gee_batch_autotune(graphs, G, opts, workspace, workspace_bytes, stream=None, best=None, best_ms=None) -> int:
    return lib().gee_batch_autotune(graphs, G, _opts_ref(opts), ptr(workspace), workspace_bytes,
                                    stream_handle(stream), ctypes.byref(best), ctypes.byref(best_ms))


def gee_embed_batch(graphs, G, opts, workspace, workspace_bytes, stream=None, d_status=None) -> int:
    return lib().gee_embed_batch(graphs, G, _opts_ref(opts), ptr(workspace), workspace_bytes,
                                 stream_handle(stream), ptr(d_status))


def gee_batch_plan_create(graphs, G, opts, workspace, workspace_bytes, stream=None):
    """(return code, plan handle)."""
    h = ctypes.c_void_p()
    rc = lib().gee_batch_plan_create(graphs, G, _opts_ref(opts), ptr(workspace), workspace_bytes,
                                     stream_handle(stream), ctypes.byref(h))
    return rc, h


def gee_batch_plan_launch(plan, stream=None, d_status=None, use_graph=True) -> int:
    return lib().gee_batch_plan_launch(plan, stream_handle(stream), ptr(d_status), 1 if use_graph else 0)


def gee_batch_plan_destroy(plan) -> None:
    lib().gee_batch_plan_destroy(plan)


def gee_batch_plan_launch_timed(plan, stream=None, phase_ms=None) -> int:
    return lib().gee_batch_plan_launch_timed(plan, stream_handle(stream), ptr(phase_ms))


def gee_server_create(config):
    """(return code, server handle)."""
    h = ctypes.c_void_p()
    rc = lib().gee_server_create(ctypes.byref(config), ctypes.byref(h))
    return rc, h


def gee_server_submit(server, request):
    """(return code, ticket)."""
    t = ctypes.c_int64()
    rc = lib().gee_server_submit(server, ctypes.byref(request), ctypes.byref(t))
    return rc, t.value


def gee_server_poll(server, ticket, wait=False):
    """(return code, device Z address, status bits, latency in ms)."""
    z = ctypes.c_void_p()
    st = ctypes.c_uint32()
    lat = ctypes.c_double()
    rc = lib().gee_server_poll(server, ticket, 1 if wait else 0, ctypes.byref(z), ctypes.byref(st), ctypes.byref(lat))
    return rc, z.value, st.value, lat.value


def gee_server_fetch(server, ticket, Z_host) -> int:
    return lib().gee_server_fetch(server, ticket, ptr(Z_host))


def gee_server_cancel(server, ticket) -> int:
    return lib().gee_server_cancel(server, ticket)


def gee_server_release(server, ticket) -> int:
    return lib().gee_server_release(server, ticket)


def gee_server_get_stats(server):
    st = gee_server_stats()
    rc = lib().gee_server_get_stats(server, ctypes.byref(st))
    return rc, st


def gee_server_destroy(server) -> None:
    lib().gee_server_destroy(server)
