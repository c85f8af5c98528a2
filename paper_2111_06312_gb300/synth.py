"""Seeded synthetic inputs: graphs, feature matrices and labels.

This module only builds *inputs* (sparsity patterns, feature values, labels).
It holds none of the method's arithmetic (no normalisation, no products, no
SVD), so both the FP64 oracle and the CUDA path may consume what it returns.

The paper measures on Cora, Pubmed, ogbn-arxiv and SNAP graphs (Sec. 6,
Table 1).  None of those datasets is used: seeded stand-ins with the same node
and edge counts and a power-law degree profile take their place.

Graphs are returned as undirected CSR (both directions stored), int32
``rowptr``/``colidx``, rows sorted by column, no duplicate entries.  Node
labels are randomly permuted so that hubs are scattered over the index range
as in a real dataset (no accidental degree ordering).
"""
from __future__ import annotations

import dataclasses
import numpy as np

BASE_SEED = 20211106312


@dataclasses.dataclass
class Graph:
    n: int
    rowptr: np.ndarray  # int32 [n+1]
    colidx: np.ndarray  # int32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr).astype(np.int64)


@dataclasses.dataclass
class SparseFeatures:
    n: int
    d: int
    rowptr: np.ndarray  # int32 [n+1]
    colidx: np.ndarray  # int32 [nnz]
    values: np.ndarray  # float32 [nnz]


def _pairs_to_csr(n: int, a: np.ndarray, b: np.ndarray, self_loops: np.ndarray | None = None) -> Graph:
    """Undirected pair list (a_t, b_t), a_t != b_t, unique -> symmetric CSR."""
    rows = np.concatenate([a, b])
    cols = np.concatenate([b, a])
    if self_loops is not None and len(self_loops):
        rows = np.concatenate([rows, self_loops])
        cols = np.concatenate([cols, self_loops])
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order]
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    assert rowptr[-1] < 2**31
    return Graph(n, rowptr.astype(np.int32), cols.astype(np.int32))


def _unique_pairs(n: int, n_pairs: int, draw, rng: np.random.Generator):
    """Draw endpoint pairs with ``draw(size)`` until ``n_pairs`` distinct
    unordered non-self pairs exist; keeps first occurrences in draw order."""
    keys = np.empty(0, dtype=np.int64)
    while True:
        need = n_pairs - len(keys)
        if need <= 0:
            break
        batch = int(need * 1.15) + 1024
        a = draw(batch)
        b = draw(batch)
        keep = a != b
        a, b = a[keep], b[keep]
        lo = np.minimum(a, b).astype(np.int64)
        hi = np.maximum(a, b).astype(np.int64)
        keys = np.concatenate([keys, lo * n + hi])
        _, first = np.unique(keys, return_index=True)
        keys = keys[np.sort(first)]
    keys = keys[:n_pairs]
    return (keys // n).astype(np.int64), (keys % n).astype(np.int64)


def chung_lu(n: int, m_directed: int, seed: int, gamma: float = 2.5,
             max_degree: float | None = None, isolated_self_loops: bool = True,
             permute: bool = True) -> Graph:
    """Chung-Lu power-law graph.

    Expected degrees w_i = w0 (i + i0)^(-1/(gamma-1)); w0 makes sum(w) = m and
    i0 is solved so that max(w) = ``max_degree`` (default i0 = 1).  m/2
    unordered pairs are drawn with endpoint probability proportional to w,
    self pairs and duplicates are rejected and redrawn.  Isolated nodes get a
    self-loop when ``isolated_self_loops`` (the configs' rule for T = D^-1 A,
    whose rows need a nonzero degree).
    """
    rng = np.random.default_rng(seed)
    a = 1.0 / (gamma - 1.0)
    idx = np.arange(n, dtype=np.float64)
    if max_degree is None:
        i0 = 1.0
    else:
        target = m_directed / float(max_degree)

        def f(i0):
            return float(np.sum((i0 / (idx + i0)) ** a))

        lo, hi = 1e-9, 1e12
        for _ in range(200):
            mid = np.sqrt(lo * hi)
            if f(mid) < target:
                lo = mid
            else:
                hi = mid
        i0 = np.sqrt(lo * hi)
    w = (idx + i0) ** (-a)
    w *= m_directed / w.sum()
    cdf = np.cumsum(w)
    cdf /= cdf[-1]

    def draw(size):
        return np.minimum(np.searchsorted(cdf, rng.random(size), side="right"), n - 1)

    pa, pb = _unique_pairs(n, m_directed // 2, draw, rng)
    if permute:
        perm = rng.permutation(n)
        pa, pb = perm[pa], perm[pb]
    loops = None
    if isolated_self_loops:
        deg = np.bincount(pa, minlength=n) + np.bincount(pb, minlength=n)
        loops = np.nonzero(deg == 0)[0].astype(np.int64)
    return _pairs_to_csr(n, pa, pb, loops)


def erdos_renyi(n: int, mean_degree: float, seed: int, isolated_self_loops: bool = True) -> Graph:
    """G(n, p) with p = mean_degree / (n - 1): a binomial number of distinct
    uniform pairs."""
    rng = np.random.default_rng(seed)
    p = mean_degree / (n - 1)
    n_pairs = int(rng.binomial(n * (n - 1) // 2, p))

    def draw(size):
        return rng.integers(0, n, size=size)

    pa, pb = _unique_pairs(n, n_pairs, draw, rng)
    loops = None
    if isolated_self_loops:
        deg = np.bincount(pa, minlength=n) + np.bincount(pb, minlength=n)
        loops = np.nonzero(deg == 0)[0].astype(np.int64)
    return _pairs_to_csr(n, pa, pb, loops)


def tfidf_features(n: int, d: int, density: float, seed: int) -> SparseFeatures:
    """Sparse nonnegative TF-IDF-like features: each entry is nonzero with
    probability ``density`` (at least one per row), lognormal(0, 1) values,
    rows scaled to unit L2 norm."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n, d)) < density
    empty = ~mask.any(axis=1)
    mask[np.nonzero(empty)[0], rng.integers(0, d, size=int(empty.sum()))] = True
    rows, cols = np.nonzero(mask)
    vals = rng.lognormal(0.0, 1.0, size=len(rows))
    norms = np.sqrt(np.bincount(rows, weights=vals * vals, minlength=n))
    vals = vals / norms[rows]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return SparseFeatures(n, d, rowptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float32))


def dense_features(n: int, d: int, seed: int) -> np.ndarray:
    """Dense i.i.d. N(0, 1) FP32 features, row-major n x d."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, d), dtype=np.float32)


def labels(n: int, classes: int, train_frac: float, seed: int):
    """Uniform class labels and a random training mask."""
    rng = np.random.default_rng(seed)
    y = rng.integers(0, classes, size=n).astype(np.int64)
    train = np.zeros(n, dtype=bool)
    train[rng.choice(n, size=int(round(train_frac * n)), replace=False)] = True
    return y, train


# ---- small structured graphs (closed-form spectra) --------------------------

def cycle(n: int) -> Graph:
    i = np.arange(n)
    return _pairs_to_csr(n, i, (i + 1) % n)


def complete(n: int) -> Graph:
    a, b = np.triu_indices(n, 1)
    return _pairs_to_csr(n, a, b)


def from_edges(n: int, edges, self_loops=()) -> Graph:
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return _pairs_to_csr(n, e[:, 0], e[:, 1], np.asarray(list(self_loops), dtype=np.int64))


def induced_subgraph(g: Graph, nodes: np.ndarray, isolated_self_loops: bool = True) -> Graph:
    """Subgraph induced by ``nodes`` (relabelled 0..len-1); isolated nodes of
    the result get a self-loop when requested."""
    nodes = np.asarray(nodes, dtype=np.int64)
    remap = -np.ones(g.n, dtype=np.int64)
    remap[nodes] = np.arange(len(nodes))
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    cols = g.colidx.astype(np.int64)
    keep = (remap[rows] >= 0) & (remap[cols] >= 0) & (rows < cols)
    a, b = remap[rows[keep]], remap[cols[keep]]
    loops = None
    if isolated_self_loops:
        deg = np.bincount(a, minlength=len(nodes)) + np.bincount(b, minlength=len(nodes))
        loops = np.nonzero(deg == 0)[0]
    return _pairs_to_csr(len(nodes), a, b, loops)


def bfs_ball(g: Graph, size: int, root: int | None = None) -> np.ndarray:
    """The first ``size`` nodes reached by breadth-first search from ``root``
    (default: a node of median degree), continuing from the next unvisited
    node when a component is exhausted."""
    deg = np.diff(g.rowptr)
    start = int(np.argsort(deg, kind="stable")[g.n // 2]) if root is None else int(root)
    seen = np.zeros(g.n, dtype=bool)
    order = []
    nxt = 0
    frontier = [start]
    seen[start] = True
    while len(order) < size:
        if not frontier:
            while seen[nxt]:
                nxt += 1
            seen[nxt] = True
            frontier = [nxt]
        new = []
        for v in frontier:
            order.append(v)
            if len(order) == size:
                break
            nb = g.colidx[g.rowptr[v]:g.rowptr[v + 1]]
            nb = nb[~seen[nb]]
            seen[nb] = True
            new.extend(nb.tolist())
        frontier = new
    return np.asarray(order[:size], dtype=np.int64)


# ---- the five workload recipes ------------------------------------------------

def workload_ne_small(seed_offset: int = 0) -> Graph:
    """Cora-sized NE graph: n = 2,708, ~10,556 directed edges, gamma 2.5."""
    return chung_lu(2708, 10556, BASE_SEED + 0 + seed_offset)


def workload_concat_graph() -> tuple[Graph, SparseFeatures]:
    """Pubmed-sized: n = 19,717, ~88,648 directed edges; X 19,717 x 500 at 1%."""
    g = chung_lu(19717, 88648, BASE_SEED + 1, isolated_self_loops=False)
    x = tfidf_features(19717, 500, 0.01, BASE_SEED + 1 + 1000)
    return g, x


def workload_ne_large(n: int = 1_000_000, m: int = 20_000_000, max_degree: float = 50_000.0) -> Graph:
    """Large NE graph: n = 10^6, 2x10^7 directed edges, max degree ~5x10^4."""
    return chung_lu(n, m, BASE_SEED + 2, max_degree=max_degree)


def cached(name: str) -> Graph:
    """``workload_<name>`` graph, cached as .npz in the temp directory (the
    10^6-node graph takes ~20 s to draw)."""
    import os
    import tempfile

    path = os.path.join(tempfile.gettempdir(), f"isvd_synth_{name}_v1.npz")
    if os.path.exists(path):
        z = np.load(path)
        return Graph(int(z["n"]), z["rowptr"], z["colidx"])
    g = {"ne_large": workload_ne_large, "ne_small": workload_ne_small}[name]()
    try:
        tmp = path + f".{os.getpid()}.npz"
        np.savez(tmp, n=g.n, rowptr=g.rowptr, colidx=g.colidx)
        os.replace(tmp, path)
    except OSError:
        pass
    return g


def workload_batched(count: int = 256, n_lo: int = 500, n_hi: int = 50_000, mean_degree: float = 8.0):
    """Many uneven graphs: n ~ U[n_lo, n_hi]; even index Erdos-Renyi, odd index
    Chung-Lu; rank drawn from {16, 32, 64}."""
    rng = np.random.default_rng(BASE_SEED + 3)
    sizes = rng.integers(n_lo, n_hi + 1, size=count)
    ranks = rng.choice(np.array([16, 32, 64]), size=count)
    graphs = []
    for g_i, n in enumerate(sizes):
        s = BASE_SEED + 3 + 1 + g_i
        if g_i % 2 == 0:
            graphs.append(erdos_renyi(int(n), mean_degree, s))
        else:
            graphs.append(chung_lu(int(n), int(round(mean_degree * n)) // 2 * 2, s))
    return graphs, [int(r) for r in ranks]


def workload_finetune(n: int = 169_343, m: int = 1_166_243, d: int = 128, classes: int = 40):
    """ogbn-arxiv-sized: n = 169,343, ~1.17M directed edges; dense X n x 128;
    40 classes with a 10% training mask."""
    g = chung_lu(n, m // 2 * 2, BASE_SEED + 4, isolated_self_loops=False)
    x = dense_features(n, d, BASE_SEED + 4 + 1000)
    y, train = labels(n, classes, 0.10, BASE_SEED + 4 + 2000)
    return g, x, y, train


def workload_finetune_sub(size: int = 2000):
    """Induced subgraph of the ogbn-arxiv-sized graph on a ``size``-node BFS
    ball, with the matching feature rows and labels."""
    g, x, y, train = workload_finetune()
    nodes = bfs_ball(g, size)
    return induced_subgraph(g, nodes, isolated_self_loops=False), x[nodes], y[nodes], train[nodes]
