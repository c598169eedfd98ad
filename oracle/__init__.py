"""FP64 CPU oracle for sparse GEE -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, the smoke check in ``__graft_entry__.py`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under ``paper_2406_03726_gb300``
never imports it, and it imports nothing from the library.

Two independent forms of the same definitions:

* ``embed`` / ``csr`` / ``degrees`` / ``label_counts`` / ``class_counts`` call the plain C
  edge-list oracle in ``gee_oracle.c`` (Section 2 edge-list GEE, Section 3 CSR).
* ``dense.embed_dense`` evaluates Table 1 literally with dense NumPy matrices (small N).
* ``embed_rows`` is the same edge-list oracle restated row by row on several host threads
  (``gee_oracle_rows.c``): it is the all-core CPU baseline, bit-identical to ``embed``
  because each row's sums keep the edge-list order.
* ``embed_sparse`` keeps Z sparse (Section 3): per row the classes of its labelled
  neighbours (+ its own with augmentation), each value equal to ``embed``'s bit for bit.

Parity pinning: every function here is checked in ``tests/test_oracle.py`` against
closed forms, invariants, a library stable sort, brute force on tiny inputs and the
CSR example of Section 3 -- never against the CUDA path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import build_oracle, library_path, sources

DIAG_AUG = 1
LAPLACIAN = 2
CORRELATION = 4
ALL_OPTIONS = DIAG_AUG | LAPLACIAN | CORRELATION

ERR_INDEX = 1
ERR_LABEL = 2
ERR_WEIGHT = 4
ERR_ARG = 8

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path) or any(os.path.getmtime(path) < os.path.getmtime(s) for s in sources()):
            build_oracle()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        lib.oracle_validate.argtypes = [P, P, P, i64, i32, P, i32, u32]
        lib.oracle_validate.restype = ctypes.c_int
        lib.oracle_label_counts.argtypes = [P, i32, i32, P]
        lib.oracle_label_counts.restype = None
        lib.oracle_csr.argtypes = [P, P, P, i64, i32, P, P, P]
        lib.oracle_csr.restype = None
        lib.oracle_degrees.argtypes = [P, P, i64, i32, u32, P]
        lib.oracle_degrees.restype = None
        lib.oracle_class_counts.argtypes = [P, P, i64, i32, P, i32, P]
        lib.oracle_class_counts.restype = None
        lib.oracle_embed.argtypes = [P, P, P, i64, i32, P, i32, u32, P]
        lib.oracle_embed.restype = ctypes.c_int
        lib.oracle_symmetrize.argtypes = [P, P, P, i64, P, P, P]
        lib.oracle_symmetrize.restype = i64
        lib.oracle_embed_rows.argtypes = [P, P, P, i64, i32, P, i32, u32, ctypes.c_int, P]
        lib.oracle_embed_rows.restype = ctypes.c_int
        lib.oracle_embed_sparse.argtypes = [P, P, P, i64, i32, P, i32, u32, P, P, P]
        lib.oracle_embed_sparse.restype = ctypes.c_int
        _lib = lib
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def symmetrize(src, dst, w=None):
    """(src, dst, w) of the directed list of an undirected edge list given once per edge:
    for every edge in input order, the edge and then (unless it is a self-loop) its reverse."""
    src, dst, w = _i32(src), _i32(dst), _f32(w)
    E = src.size
    os_, od = np.zeros(2 * E, np.int32), np.zeros(2 * E, np.int32)
    ow = None if w is None else np.zeros(2 * E, np.float32)
    n = _load().oracle_symmetrize(_ptr(src), _ptr(dst), _ptr(w), E, _ptr(os_), _ptr(od), _ptr(ow))
    return os_[:n], od[:n], None if ow is None else ow[:n]


def validate(src, dst, w, N, labels, K, flags=0) -> int:
    src, dst, w, y = _i32(src), _i32(dst), _f32(w), _i32(labels)
    return _load().oracle_validate(_ptr(src), _ptr(dst), _ptr(w), src.size, N, _ptr(y), K, flags)


def label_counts(labels, K) -> np.ndarray:
    y = _i32(labels)
    nk = np.zeros(K, np.int64)
    _load().oracle_label_counts(_ptr(y), y.size, K, _ptr(nk))
    return nk


def csr(src, dst, w, N):
    """(rowptr int64 [N+1], col int32 [E], val float32 [E]) -- stable by input order."""
    src, dst, w = _i32(src), _i32(dst), _f32(w)
    E = src.size
    rowptr = np.zeros(N + 1, np.int64)
    col = np.zeros(E, np.int32)
    val = np.zeros(E, np.float32)
    _load().oracle_csr(_ptr(src), _ptr(dst), _ptr(w), E, N, _ptr(rowptr), _ptr(col), _ptr(val))
    return rowptr, col, val


def degrees(src, w, N, flags=0) -> np.ndarray:
    src, w = _i32(src), _f32(w)
    deg = np.zeros(N, np.float64)
    _load().oracle_degrees(_ptr(src), _ptr(w), src.size, N, flags, _ptr(deg))
    return deg


def class_counts(src, dst, N, labels, K) -> np.ndarray:
    src, dst, y = _i32(src), _i32(dst), _i32(labels)
    C = np.zeros((N, K), np.int64)
    _load().oracle_class_counts(_ptr(src), _ptr(dst), src.size, N, _ptr(y), K, _ptr(C))
    return C


def embed(src, dst, w, N, labels, K, flags=0) -> np.ndarray:
    """Z (N x K, float64).  Raises ValueError with the error bits on invalid input."""
    src, dst, w, y = _i32(src), _i32(dst), _f32(w), _i32(labels)
    Z = np.zeros((N, K), np.float64)
    err = _load().oracle_embed(_ptr(src), _ptr(dst), _ptr(w), src.size, N, _ptr(y), K, flags, _ptr(Z))
    if err:
        raise ValueError(f"oracle: invalid input (error bits {err})")
    return Z


def embed_sparse(src, dst, w, N, labels, K, flags=0):
    """Sparse Z (Section 3): (zrowptr int64 [N+1], zcol int32, zval float64) with, per row,
    the classes of its labelled neighbours (+ its own with augmentation) ascending."""
    src, dst, w, y = _i32(src), _i32(dst), _f32(w), _i32(labels)
    E = src.size
    zrowptr = np.zeros(N + 1, np.int64)
    zcol = np.zeros(E + N + 1, np.int32)
    zval = np.zeros(E + N + 1, np.float64)
    err = _load().oracle_embed_sparse(_ptr(src), _ptr(dst), _ptr(w), E, N, _ptr(y), K, flags, _ptr(zrowptr),
                                      _ptr(zcol), _ptr(zval))
    if err:
        raise ValueError(f"invalid input (oracle error bits {err})")
    n = int(zrowptr[N])
    return zrowptr, zcol[:n], zval[:n]


def embed_sparse_graph(g, flags=0):
    return embed_sparse(g.src, g.dst, g.w, g.N, g.labels, g.K, flags)


def embed_graph(g, flags=0) -> np.ndarray:
    return embed(g.src, g.dst, g.w, g.N, g.labels, g.K, flags)


def embed_rows(src, dst, w, N, labels, K, flags=0, threads=None) -> np.ndarray:
    """Z of ``embed``, computed row-parallel on ``threads`` host threads (default: all
    cores); bit-identical to ``embed``."""
    src, dst, w, y = _i32(src), _i32(dst), _f32(w), _i32(labels)
    if threads is None:
        threads = os.cpu_count() or 1
    Z = np.zeros((N, K), np.float64)
    err = _load().oracle_embed_rows(_ptr(src), _ptr(dst), _ptr(w), src.size, N, _ptr(y), K, flags,
                                    int(threads), _ptr(Z))
    if err:
        raise ValueError(f"oracle: invalid input (error bits {err})")
    return Z


def embed_rows_graph(g, flags=0, threads=None) -> np.ndarray:
    return embed_rows(g.src, g.dst, g.w, g.N, g.labels, g.K, flags, threads)
