"""Device-side (PyTorch) drawing of the many-graph mix, for batches too large to draw
with NumPy on the host.  Same recipe as ``graphs.batch_graph`` (see its docstring) with
PyTorch's CUDA random generator seeded per graph, so results differ bitwise from the
NumPy version but follow the same law.  Draws graphs only; no embedding arithmetic."""
from __future__ import annotations

import math

import numpy as np

from .graphs import _chung_lu_theta


def batch_graph_torch(spec: dict, device, weighted: bool = True):
    """(src int32 [E], dst int32 [E], w float32 [E] or None, labels int32 [N]) on `device`."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(spec["seed"]) % (2 ** 63 - 1))
    N, m, K = int(spec["N"]), int(spec["m"]), int(spec["K"])
    labels = torch.randint(0, K, (N,), generator=gen, device=device, dtype=torch.int64)
    if spec["kind"] == "sbm":
        q = 1.3 / (1.3 + (K - 1))
        u = torch.randint(0, N, (m,), generator=gen, device=device)
        same = torch.rand(m, generator=gen, device=device) < q
        order = torch.argsort(labels, stable=True)
        counts = torch.bincount(labels, minlength=K)
        starts = torch.cumsum(counts, 0) - counts
        lu = labels[u]
        pick = starts[lu] + torch.floor(torch.rand(m, generator=gen, device=device) * counts[lu]).long()
        v_same = order[torch.clamp(pick, max=N - 1)]
        v_any = torch.randint(0, N, (m,), generator=gen, device=device)
        v = torch.where(same, v_same, v_any)
    else:
        d = 2.0 * m / N
        p = _chung_lu_theta(N, 1.0 / 1.1, m, min(N / 3.0, 40.0 * d))
        cdf = torch.from_numpy(np.cumsum(p)).to(device)
        cdf[-1] = 1.0
        u = torch.clamp(torch.searchsorted(cdf, torch.rand(m, generator=gen, device=device, dtype=torch.float64),
                                           right=True), max=N - 1)
        v = torch.clamp(torch.searchsorted(cdf, torch.rand(m, generator=gen, device=device, dtype=torch.float64),
                                           right=True), max=N - 1)
        relabel = torch.randperm(N, generator=gen, device=device)
        u, v = relabel[u], relabel[v]
    v = torch.where(u == v, (v + 1) % N, v)
    src = torch.cat([u, v])
    dst = torch.cat([v, u])
    perm = torch.randperm(2 * m, generator=gen, device=device)
    src = src[perm].to(torch.int32).contiguous()
    dst = dst[perm].to(torch.int32).contiguous()
    w = None
    if weighted:
        w_und = 1.0 - torch.rand(m, generator=gen, device=device, dtype=torch.float32)
        w = torch.cat([w_und, w_und])[perm].contiguous()
    return src, dst, w, labels.to(torch.int32).contiguous()
