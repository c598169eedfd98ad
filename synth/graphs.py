"""Seeded synthetic graphs with the shapes of the paper's workloads.

* ``sbm``      -- the stochastic block model of Section 4 (3 classes, priors [0.2, 0.3, 0.5],
                  within-class probability 0.13, between-class probability 0.10).
* ``chung_lu`` -- a power-law (Chung-Lu) graph standing in for the CL-100K-1d8 graphs of
                  Table 2, whose files are not available here.
* ``batch_specs`` / ``batch_graph`` -- the many-graph mix (log-uniform N, uniform mean
                  degree, SBM or Chung-Lu per graph, 2..64 classes, weights in (0, 1]).
* ``random_tiny`` -- small adversarial graphs (duplicates, self-loops, isolated and
                  unlabelled nodes, empty classes) for exhaustive checks.

Every graph is returned as a directed edge list in which each undirected edge is stored
in both directions with the same weight, in a shuffled order, with int32 node ids,
int32 labels (-1 = unlabelled) and optional float32 weights drawn as ``1 - U[0, 1)``,
i.e. uniform on (0, 1].  Randomness comes from NumPy's PCG64 seeded by the caller.

Nothing here computes any part of the embedding.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PAPER_SBM_PRIORS = (0.2, 0.3, 0.5)
PAPER_SBM_P_IN = 0.13
PAPER_SBM_P_OUT = 0.10


@dataclass
class Graph:
    src: np.ndarray            # int32 [E]   edge source i
    dst: np.ndarray            # int32 [E]   edge target j
    w: np.ndarray | None       # float32 [E] edge weight e_ij, None = unweighted (all ones)
    labels: np.ndarray         # int32 [N]   class of each node, -1 = unlabelled
    N: int
    K: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def E(self) -> int:
        return int(self.src.shape[0])

    @property
    def weighted(self) -> bool:
        return self.w is not None


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _bernoulli_positions(rng: np.random.Generator, M: int, p: float) -> np.ndarray:
    """Indices of [0, M) each kept independently with probability p.

    Uses geometric gaps between successive kept indices, which is exactly the law of
    M independent Bernoulli(p) trials."""
    if M <= 0 or p <= 0.0:
        return np.empty(0, np.int64)
    if p >= 1.0:
        return np.arange(M, dtype=np.int64)
    chunks = []
    pos = -1
    while True:
        mean = (M - 1 - pos) * p
        n = int(mean + 6.0 * math.sqrt(mean + 1.0) + 64)
        cand = pos + np.cumsum(rng.geometric(p, size=n), dtype=np.int64)
        keep = cand[cand < M]
        chunks.append(keep)
        if keep.size < cand.size:
            break
        pos = int(cand[-1])
    return np.concatenate(chunks)


def _tri_unrank(k: np.ndarray):
    """Map k in [0, n(n-1)/2) to the pair (i, j), 0 <= j < i, in row-major order."""
    k = k.astype(np.int64)
    i = np.floor((1.0 + np.sqrt(1.0 + 8.0 * k.astype(np.float64))) / 2.0).astype(np.int64)
    # correct possible off-by-one from floating point
    i = np.where(i * (i - 1) // 2 > k, i - 1, i)
    i = np.where((i + 1) * i // 2 <= k, i + 1, i)
    j = k - i * (i - 1) // 2
    return i, j


def _finish(rng, u, v, labels, K, N, weighted, name, meta=None) -> Graph:
    """Store each undirected edge (u, v) in both directions, draw weights, shuffle."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    m = u.size
    src = np.concatenate([u, v]).astype(np.int32)
    dst = np.concatenate([v, u]).astype(np.int32)
    w = None
    if weighted:
        w_und = (np.float32(1.0) - rng.random(m, dtype=np.float32)).astype(np.float32)
        w = np.concatenate([w_und, w_und])
    perm = rng.permutation(src.size)
    src = np.ascontiguousarray(src[perm])
    dst = np.ascontiguousarray(dst[perm])
    if w is not None:
        w = np.ascontiguousarray(w[perm])
    meta = dict(meta or {})
    meta["undirected_edges"] = int(m)
    return Graph(src, dst, w, np.ascontiguousarray(labels, dtype=np.int32), int(N), int(K), name, meta)


def sbm(N: int, priors=PAPER_SBM_PRIORS, p_in: float = PAPER_SBM_P_IN,
        p_out: float = PAPER_SBM_P_OUT, seed: int = 1, weighted: bool = False,
        name: str = "sbm") -> Graph:
    """Stochastic block model (Section 4): labels i.i.d. categorical(priors); each
    unordered pair {i, j}, i != j, is an edge with probability p_in when y_i == y_j and
    p_out otherwise."""
    rng = _rng(seed)
    K = len(priors)
    labels = rng.choice(K, size=N, p=np.asarray(priors, dtype=np.float64)).astype(np.int32)
    members = [np.nonzero(labels == k)[0].astype(np.int64) for k in range(K)]
    us, vs = [], []
    for a in range(K):
        for b in range(a, K):
            ma, mb = members[a], members[b]
            if a == b:
                n = ma.size
                idx = _bernoulli_positions(rng, n * (n - 1) // 2, p_in)
                i, j = _tri_unrank(idx)
                us.append(ma[i])
                vs.append(ma[j])
            else:
                idx = _bernoulli_positions(rng, ma.size * mb.size, p_out)
                us.append(ma[idx // mb.size])
                vs.append(mb[idx % mb.size])
    u = np.concatenate(us) if us else np.empty(0, np.int64)
    v = np.concatenate(vs) if vs else np.empty(0, np.int64)
    return _finish(rng, u, v, labels, K, N, weighted, name,
                   {"kind": "sbm", "seed": seed, "priors": list(priors), "p_in": p_in, "p_out": p_out})


def expected_sbm_edges(N: int, priors=PAPER_SBM_PRIORS, p_in=PAPER_SBM_P_IN, p_out=PAPER_SBM_P_OUT,
                       labels: np.ndarray | None = None):
    """Expected undirected edge count of ``sbm`` and its standard deviation.

    Without ``labels`` the mean is over the label draw too:
    C(N, 2) * (sum(pi_k^2) p_in + (1 - sum(pi_k^2)) p_out) (std None).  With the realised
    ``labels`` the count is a sum of independent Bernoulli trials, whose exact mean and
    standard deviation are returned."""
    if labels is None:
        q = float(np.sum(np.square(priors)))
        return N * (N - 1) / 2.0 * (q * p_in + (1.0 - q) * p_out), None
    n = np.bincount(labels, minlength=len(priors)).astype(np.float64)
    within = float(np.sum(n * (n - 1) / 2.0))
    between = N * (N - 1) / 2.0 - within
    mean = within * p_in + between * p_out
    var = within * p_in * (1 - p_in) + between * p_out * (1 - p_out)
    return mean, math.sqrt(var)


def edge_density(undirected_edges: int, N: int) -> float:
    """Edge density of Eq. 2: d = 2|E| / (|V| (|V| - 1))."""
    return 2.0 * undirected_edges / (N * (N - 1.0))


def zipf_labels(rng: np.random.Generator, N: int, K: int, s: float = 1.2) -> np.ndarray:
    """Class sizes proportional to (k + 1)^-s, each at least 1, assigned by a random
    permutation of the nodes."""
    p = (np.arange(K, dtype=np.float64) + 1.0) ** (-s)
    p /= p.sum()
    sizes = np.maximum(1, np.floor(p * N).astype(np.int64))
    sizes[0] += N - sizes.sum()
    labels = np.repeat(np.arange(K, dtype=np.int32), sizes)
    return labels[rng.permutation(N)]


def _chung_lu_theta(N: int, a: float, m: float, d_max: float) -> np.ndarray:
    """Weights (i + i0)^-a with i0 chosen by bisection so the largest expected degree
    2 m theta_0 / sum(theta) is close to d_max."""
    idx = np.arange(N, dtype=np.float64)

    def top(i0):
        t = (idx + i0) ** (-a)
        return 2.0 * m * t[0] / t.sum()

    lo, hi = math.log(1e-6), math.log(1e9)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if top(math.exp(mid)) > d_max:
            lo = mid
        else:
            hi = mid
    theta = (idx + math.exp(hi)) ** (-a)
    return theta / theta.sum()


def chung_lu(N: int, m_target: int, gamma: float = 2.1, d_max: float = 3.0e5, seed: int = 3,
             K: int = 50, zipf_s: float = 1.2, weighted: bool = False, dedup: bool = True,
             name: str = "chung_lu") -> Graph:
    """Chung-Lu power-law graph: endpoints drawn independently with probability
    proportional to (i + i0)^(-1/(gamma-1)); self-loops dropped; with ``dedup`` the
    unordered pairs are made unique and the draw is topped up until exactly m_target
    distinct undirected edges remain.  Node ids are randomly permuted (hubs are spread
    over the id range) and labels follow ``zipf_labels``."""
    rng = _rng(seed)
    p = _chung_lu_theta(N, 1.0 / (gamma - 1.0), m_target, d_max)
    cdf = np.cumsum(p)
    cdf[-1] = 1.0

    def draw(n):
        u = np.searchsorted(cdf, rng.random(n), side="right")
        v = np.searchsorted(cdf, rng.random(n), side="right")
        return np.minimum(u, N - 1), np.minimum(v, N - 1)

    if dedup:
        keys = np.empty(0, np.int64)
        for _ in range(64):
            need = m_target - keys.size
            if need <= 0:
                break
            u, v = draw(int(need * 1.25) + 1024)
            keep = u != v
            lo = np.minimum(u, v)[keep].astype(np.int64)
            hi = np.maximum(u, v)[keep].astype(np.int64)
            keys = np.unique(np.concatenate([keys, lo * N + hi]))
        if keys.size > m_target:
            keys = keys[rng.permutation(keys.size)[:m_target]]
        u, v = keys // N, keys % N
    else:
        u, v = draw(m_target)
        v = np.where(u == v, (v + 1) % N, v)
    relabel = rng.permutation(N).astype(np.int64)
    u, v = relabel[u], relabel[v]
    labels = zipf_labels(rng, N, K, zipf_s)
    return _finish(rng, u, v, labels, K, N, weighted, name,
                   {"kind": "chung_lu", "seed": seed, "gamma": gamma, "d_max": d_max})


# ----------------------------------------------------------------------------------------
# many-graph mix


def batch_specs(G: int, seed: int = 4, n_range=(100, 50_000), d_range=(5.0, 200.0),
                k_range=(2, 64)) -> list[dict]:
    """Per-graph parameters of the many-graph workload: N log-uniform in n_range, mean
    degree uniform in d_range (capped at N - 1), E = N * d directed edges, SBM or
    Chung-Lu by coin flip, K uniform in k_range (at most N), weights in (0, 1]."""
    rng = _rng(seed)
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    Ns = np.rint(np.exp(rng.uniform(lo, hi, G))).astype(np.int64)
    ds = np.minimum(rng.uniform(d_range[0], d_range[1], G), Ns - 1)
    kinds = rng.integers(0, 2, G)
    Ks = np.minimum(rng.integers(k_range[0], k_range[1] + 1, G), Ns)
    seeds = rng.integers(0, 2 ** 62, G)
    specs = []
    for g in range(G):
        N = int(Ns[g])
        m = max(1, int(round(N * ds[g] / 2.0)))
        specs.append({"index": g, "N": N, "m": m, "E": 2 * m, "K": int(Ks[g]),
                      "kind": "sbm" if kinds[g] == 0 else "chung_lu", "seed": int(seeds[g])})
    return specs


def batch_graph(spec: dict, weighted: bool = True) -> Graph:
    """One graph of the mix, drawn with NumPy.  SBM graphs: labels uniform over K, each
    edge joins a uniform node u to a node of u's own class with the probability that a
    within/between ratio of 1.3 (0.13 / 0.10 as in Section 4) gives, else to a uniform
    node.  Chung-Lu graphs: both endpoints drawn with probability (i + i0)^(-1/1.1) (the
    largest expected degree about min(N/3, 40 d)).  Self-loops are moved to the next node
    id and multi-edges are kept, so E is exact."""
    rng = _rng(spec["seed"])
    N, m, K = spec["N"], spec["m"], spec["K"]
    labels = rng.integers(0, K, N).astype(np.int32)
    if spec["kind"] == "sbm":
        q = 1.3 / (1.3 + (K - 1))
        u = rng.integers(0, N, m)
        same = rng.random(m) < q
        order = np.argsort(labels, kind="stable")
        counts = np.bincount(labels, minlength=K)
        starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
        lu = labels[u]
        pick = starts[lu] + np.floor(rng.random(m) * counts[lu]).astype(np.int64)
        v_same = order[np.minimum(pick, N - 1)]
        v_any = rng.integers(0, N, m)
        v = np.where(same, v_same, v_any)
    else:
        d = 2.0 * m / N
        p = _chung_lu_theta(N, 1.0 / 1.1, m, min(N / 3.0, 40.0 * d))
        cdf = np.cumsum(p)
        cdf[-1] = 1.0
        u = np.minimum(np.searchsorted(cdf, rng.random(m), side="right"), N - 1)
        v = np.minimum(np.searchsorted(cdf, rng.random(m), side="right"), N - 1)
        relabel = rng.permutation(N)
        u, v = relabel[u], relabel[v]
    v = np.where(u == v, (v + 1) % N, v)
    return _finish(rng, u, v, labels, K, N, weighted, f"batch{spec['index']}", dict(spec))


# ----------------------------------------------------------------------------------------
# small adversarial graphs


def random_tiny(seed: int, n_max: int = 40, e_max: int = 200, k_max: int = 6,
                weighted: bool | None = None, directed: bool | None = None) -> Graph:
    """A small random graph meant to hit corner cases: duplicate edges, self-loops,
    isolated nodes, unlabelled nodes (-1) and empty classes.  Directed (edges not
    mirrored) half of the time."""
    rng = _rng(seed)
    N = int(rng.integers(1, n_max + 1))
    K = int(rng.integers(1, k_max + 1))
    E = int(rng.integers(0, e_max + 1))
    if weighted is None:
        weighted = bool(rng.integers(0, 2))
    if directed is None:
        directed = bool(rng.integers(0, 2))
    labels = rng.integers(-1, K, N).astype(np.int32) if rng.random() < 0.5 else \
        rng.integers(0, K, N).astype(np.int32)
    # occasionally leave the top classes empty
    if K > 1 and rng.random() < 0.3:
        labels = np.minimum(labels, K - 2).astype(np.int32)
    hub = int(rng.integers(0, N))
    u = rng.integers(0, N, E)
    v = rng.integers(0, N, E)
    if E and rng.random() < 0.3:       # a hub
        u[: E // 3] = hub
    if E and rng.random() < 0.3:       # duplicates
        k = E // 4
        u[E - k:] = u[:k]
        v[E - k:] = v[:k]
    if directed:
        src, dst = u.astype(np.int32), v.astype(np.int32)
        w = (np.float32(1.0) - rng.random(E, dtype=np.float32)) if weighted else None
        return Graph(src, dst, w, labels, N, K, f"tiny{seed}", {"directed": True})
    return _finish(rng, u, v, labels, K, N, weighted, f"tiny{seed}", {"directed": False})
