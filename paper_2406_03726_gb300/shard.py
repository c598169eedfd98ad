"""One graph embedded across several GPUs by source rows (one process per GPU).

Rows of Z are independent once every node's table entry {y_j, s_j = D_jj^-1/2 / n_{y_j}}
is known (Section 2, per-entry form of Eq. 1), so rank r owns the rows [r0, r1) and only
the edges whose source lies there.  The exchange is two collectives: an all-reduce of the
K class sizes and an all-gather of the 8-byte node-table entries.  Every computation runs
in the CUDA library (gee_shard_build / gee_shard_table / gee_shard_embed); this module only
chooses the row ranges, marshals arguments and moves data with torch.distributed.
"""
from __future__ import annotations

import numpy as np

from ._native import (gee_shard_build, gee_shard_embed, gee_shard_table, gee_shard_workspace_size,
                      gee_strerror, make_opts)


def row_ranges(row_counts, world: int):
    """Split rows 0..N-1 into `world` contiguous ranges [r0, r1) of about equal edge count
    (hub rows make equal row counts uneven in work).  row_counts: out-degree of every row.
    Returns a list of (r0, r1); ranges cover [0, N) in order and may be empty."""
    counts = np.asarray(row_counts, dtype=np.int64)
    N = counts.size
    if world < 1:
        raise ValueError("world must be >= 1")
    csum = np.concatenate([[0], np.cumsum(counts)])
    total = int(csum[-1])
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        # first row whose prefix reaches the target, never before the previous bound
        b = int(np.searchsorted(csum, target, side="left"))
        bounds.append(min(max(b, bounds[-1]), N))
    bounds.append(N)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def edges_of_rows(src, r0, r1):
    """Indices of the edges whose source lies in [r0, r1) (host arrays), in input order."""
    src = np.asarray(src)
    return np.nonzero((src >= r0) & (src < r1))[0]


class ShardError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise ShardError(f"{what}: {gee_strerror(rc)} (code {rc})")


def embed_rows(src, dst, w, N, labels, K, r0, r1, flags=0, opts=None, group=None, stream=None):
    """Z of rows [r0, r1) of a graph of N nodes on this rank's GPU.

    src/dst/w: this rank's edges (device tensors; every src in [r0, r1), dst global);
    labels: device int32 [r1 - r0], the labels of this rank's rows.  Every rank of `group`
    (torch.distributed, NCCL) calls this with its own range; the ranges cover [0, N).
    Returns (Z float32 [r1 - r0, K], status int32 [1]) on the device."""
    import torch
    import torch.distributed as dist
    dev = labels.device
    E = int(src.numel())
    rows = r1 - r0
    o = opts if opts is not None else make_opts(flags)
    weighted = w is not None
    n = gee_shard_workspace_size(E, N, r0, r1, K, weighted, o)
    if n == 0:
        raise ShardError("gee_shard_workspace_size: invalid shape")
    ws = torch.empty(n, dtype=torch.uint8, device=dev)
    nk = torch.zeros(K, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    _check(gee_shard_build(src, dst, w, E, N, r0, r1, labels, K, o, nk, ws, n, stream, status), "gee_shard_build")
    dist.all_reduce(nk, op=dist.ReduceOp.SUM, group=group)            # the K class sizes
    world = dist.get_world_size(group)
    # every rank's row count, then the table entries gathered in row order
    sizes = torch.tensor([rows], dtype=torch.int64, device=dev)
    all_sizes = [torch.zeros_like(sizes) for _ in range(world)]
    dist.all_gather(all_sizes, sizes, group=group)
    all_sizes = [int(t.item()) for t in all_sizes]
    cap = max(all_sizes)
    mine = torch.zeros((max(cap, 1), 2), dtype=torch.int32, device=dev)
    _check(gee_shard_table(E, N, r0, r1, labels, K, weighted, o, nk, mine, ws, n, stream), "gee_shard_table")
    gathered = torch.empty((world * max(cap, 1), 2), dtype=torch.int32, device=dev)
    dist.all_gather_into_tensor(gathered, mine, group=group)          # 8 bytes per node
    tab = torch.cat([gathered[r * max(cap, 1): r * max(cap, 1) + all_sizes[r]] for r in range(world)])
    if tab.shape[0] != N:
        raise ShardError(f"the ranges cover {tab.shape[0]} rows, not N = {N}")
    Z = torch.empty((rows, K), dtype=torch.float32, device=dev)
    _check(gee_shard_embed(E, N, r0, r1, labels, K, weighted, o, tab.contiguous(), Z, ws, n, stream, status),
           "gee_shard_embed")
    return Z, status
