"""Dense restatement of Table 1 -- TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Builds the N x N adjacency matrix A, the N x K weight matrix W and the diagonal degree
matrix D explicitly in float64 and evaluates the formulas of Table 1 (Section 3) as
matrix products, combining the options in the order D^-1/2 (A + I) D^-1/2 W, then the
row 2-norm.  Meant for N up to a few thousand; it shares nothing with the C oracle
except the reading of the paper.
"""
from __future__ import annotations

import numpy as np

from . import CORRELATION, DIAG_AUG, LAPLACIAN


def adjacency(src, dst, w, N) -> np.ndarray:
    """A_ij = sum of the weights of the edge-list entries (i, j) (weight 1 if absent)."""
    A = np.zeros((N, N), np.float64)
    vals = np.ones(len(src), np.float64) if w is None else np.asarray(w, np.float64)
    np.add.at(A, (np.asarray(src, np.int64), np.asarray(dst, np.int64)), vals)
    return A


def weight_matrix(labels, K) -> np.ndarray:
    """W: row j is the one-hot of y_j scaled by 1/n_{y_j} (Section 2); unlabelled rows are 0."""
    y = np.asarray(labels, np.int64)
    N = y.size
    W = np.zeros((N, K), np.float64)
    lab = y >= 0
    nk = np.bincount(y[lab], minlength=K).astype(np.float64)
    W[np.nonzero(lab)[0], y[lab]] = 1.0 / nk[y[lab]]
    return W


def embed_dense(src, dst, w, N, labels, K, flags=0) -> np.ndarray:
    A = adjacency(src, dst, w, N)
    if flags & DIAG_AUG:
        A = A + np.eye(N)                                  # Table 1: (A_S + I_S)
    if flags & LAPLACIAN:
        d = A.sum(axis=1)                                  # D = diag(row sums)
        dm = np.zeros(N)
        dm[d > 0] = d[d > 0] ** -0.5
        Dm = np.diag(dm)
        A = Dm @ A @ Dm                                    # Table 1: D^-0.5 A D^-0.5
    Z = A @ weight_matrix(labels, K)                       # Eq. 1: Z = A W
    if flags & CORRELATION:
        r = np.linalg.norm(Z, axis=1)                      # Table 1: row 2-norm
        nz = r > 0
        Z[nz] = Z[nz] / r[nz, None]
    return Z
