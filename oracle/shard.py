"""FP64 oracle of GEE split by source rows -- TEST INFRASTRUCTURE ONLY.

The same definitions as the edge-list oracle (Section 2: n_k from the labels, W_j^k =
1/n_{y_j}, Z_i^k = sum over row i's entries of e_ij W_j^k; Table 1 options with D taken
after A + I; row 2-norm last), evaluated for the rows [r0, r1) of one rank from that
rank's edges, its rows' labels, the class sizes summed over all ranks and the node table
{y_j, s_j = D_jj^-1/2 / n_{y_j}} of every node.  The multi-rank tests stitch the ranks'
rows and check them against the whole-graph oracle.  Plain NumPy loops in float64.
"""
from __future__ import annotations

import numpy as np

DIAG_AUG, LAPLACIAN, CORRELATION = 1, 2, 4


def partial_label_counts(labels_local, K):
    """n_k over this rank's rows (labels -1 count nowhere)."""
    y = np.asarray(labels_local)
    return np.bincount(y[y >= 0], minlength=K).astype(np.int64)[:K]


def row_degrees(src, w, r0, r1, flags):
    """D_ii of the rows [r0, r1): the row sums of A (+1 with A + I), in edge order."""
    deg = np.zeros(r1 - r0, np.float64)
    for e in range(len(src)):
        deg[src[e] - r0] += float(w[e]) if w is not None else 1.0
    if flags & DIAG_AUG:
        deg += 1.0
    return deg


def node_table(labels_local, deg, nk, flags):
    """{y_j, s_j} of the rank's rows: s_j = D_jj^-1/2 / n_{y_j} (Laplacian) or 1 / n_{y_j};
    unlabelled nodes and empty classes give s_j = 0."""
    y = np.asarray(labels_local).astype(np.int64)
    s = np.zeros(len(y), np.float64)
    for j in range(len(y)):
        if y[j] < 0 or nk[y[j]] == 0:
            continue
        d = 1.0
        if flags & LAPLACIAN:
            d = 1.0 / np.sqrt(deg[j]) if deg[j] > 0 else 0.0
        s[j] = d / float(nk[y[j]])
    return y, s


def rows(src, dst, w, r0, r1, y_all, s_all, deg, K, flags):
    """Z of the rows [r0, r1) (float64 [r1 - r0, K]) from the rank's edges and the node
    table of all nodes (y_all, s_all)."""
    n = r1 - r0
    Z = np.zeros((n, K), np.float64)
    dinv = np.ones(n)
    if flags & LAPLACIAN:
        dinv = np.array([1.0 / np.sqrt(d) if d > 0 else 0.0 for d in deg])
    for e in range(len(src)):
        i, j = src[e] - r0, dst[e]
        k = y_all[j]
        if k < 0:
            continue
        a = float(w[e]) if w is not None else 1.0
        Z[i, k] += dinv[i] * a * s_all[j]
    if flags & DIAG_AUG:
        for i in range(n):
            k = y_all[r0 + i]
            if k >= 0:
                Z[i, k] += dinv[i] * s_all[r0 + i]
    if flags & CORRELATION:
        for i in range(n):
            r = np.sqrt(np.sum(Z[i] * Z[i]))
            if r > 0:
                Z[i] /= r
    return Z
