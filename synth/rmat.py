"""R-MAT graphs and the link-prediction split (input preparation only).

Recipe (applied identically for every workload):
  1. ef * 2^scale directed draws; each draw descends `scale` levels of the
     adjacency quadtree picking quadrant (0,0),(0,1),(1,0),(1,1) with
     probabilities a, b, c, 1-a-b-c (default 0.57/0.19/0.19/0.05).
  2. A seeded random relabelling of the 2^scale ids, so that hubs are not
     clustered at small ids.
  3. Symmetrise, drop self-loops, deduplicate.
  4. Drop isolated vertices and compact ids (ascending order kept).
  5. CSR: int64 row pointer, int32 neighbour ids ascending within each row.
The link-prediction split follows Sec. 6.1: 20% of the undirected edges, by
a seeded shuffle, are held out; isolated vertices of the remaining graph are
dropped (ids compacted again) together with held-out edges that touch them;
an equal number of negative pairs (u != v, not an edge of the full graph) is
drawn uniformly by seeded rejection.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Graph:
    rowptr: np.ndarray  # int64 [n+1]
    col: np.ndarray     # int32 [nnz]

    @property
    def n(self) -> int:
        return len(self.rowptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


@dataclass
class LinkSplit:
    train: Graph
    test_pos: np.ndarray  # int32 [m, 2] in train ids
    test_neg: np.ndarray  # int32 [m, 2] in train ids


def rmat_edges(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19,
               chunk: int = 1 << 24) -> tuple[np.ndarray, np.ndarray]:
    """Directed R-MAT draws (step 1 and 2 of the recipe)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = edge_factor << scale
    src = np.zeros(m, dtype=np.uint32)
    dst = np.zeros(m, dtype=np.uint32)
    ab, abc = a + b, a + b + c
    for s0 in range(0, m, chunk):
        s1 = min(m, s0 + chunk)
        u = np.zeros(s1 - s0, dtype=np.uint32)
        v = np.zeros(s1 - s0, dtype=np.uint32)
        for _ in range(scale):
            r = rng.random(s1 - s0, dtype=np.float32)
            u = (u << 1) | (r >= ab).astype(np.uint32)
            v = (v << 1) | (((r >= a) & (r < ab)) | (r >= abc)).astype(np.uint32)
        src[s0:s1] = u
        dst[s0:s1] = v
    perm = rng.permutation(1 << scale).astype(np.uint32)
    return perm[src], perm[dst]


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, compact: bool = True) -> Graph:
    """Steps 3-5: symmetrise, drop self-loops, dedup, optionally drop isolated
    vertices, build CSR."""
    src = np.asarray(src, dtype=np.uint64)
    dst = np.asarray(dst, dtype=np.uint64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    keys = np.concatenate([(src << np.uint64(32)) | dst, (dst << np.uint64(32)) | src])
    keys = np.unique(keys)
    u = (keys >> np.uint64(32)).astype(np.int64)
    v = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    if compact:
        present = np.zeros(n, dtype=bool)
        present[u] = True
        newid = np.cumsum(present, dtype=np.int64) - 1
        u, v = newid[u], newid[v]
        n = int(present.sum())
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(u, minlength=n), out=rowptr[1:])
    return Graph(rowptr, v.astype(np.int32))


def to_csr(n, src, dst, compact=True) -> Graph:
    return csr_from_edges(n, src, dst, compact)


def rmat_graph(scale: int, edge_factor: int, seed: int, **kw) -> Graph:
    s, d = rmat_edges(scale, edge_factor, seed, **kw)
    return csr_from_edges(1 << scale, s, d)


def random_graph(n: int, p: float, seed: int, compact: bool = False) -> Graph:
    """Erdos-Renyi G(n, p) (small test graphs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    return csr_from_edges(n, iu[keep], ju[keep], compact=compact)


def link_split(g: Graph, seed: int, test_frac: float = 0.2) -> LinkSplit:
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED))
    n = g.n
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.rowptr))
    dst = g.col.astype(np.int64)
    und = src < dst
    eu, ev = src[und], dst[und]
    order = rng.permutation(len(eu))
    ntest = int(round(test_frac * len(eu)))
    test_idx, train_idx = order[:ntest], order[ntest:]
    tr = csr_from_edges(n, eu[train_idx], ev[train_idx], compact=False)
    deg = np.diff(tr.rowptr)
    present = deg > 0
    newid = np.cumsum(present, dtype=np.int64) - 1
    # compact the training graph
    tsrc = np.repeat(np.arange(n, dtype=np.int64), deg)
    keep_rows = present[tsrc]
    rowptr = np.zeros(int(present.sum()) + 1, dtype=np.int64)
    np.cumsum(deg[present], out=rowptr[1:])
    train = Graph(rowptr, newid[tr.col.astype(np.int64)][keep_rows].astype(np.int32))
    tu, tv = eu[test_idx], ev[test_idx]
    ok = present[tu] & present[tv]
    test_pos = np.stack([newid[tu[ok]], newid[tv[ok]]], axis=1).astype(np.int32)
    # negatives: uniform pairs over V_train, not an edge of the full graph
    nt = train.n
    full_keys = set()
    if nt > 0:
        fk = (newid[src[present[src] & present[dst]]] * nt + newid[dst[present[src] & present[dst]]])
        full_keys = np.unique(fk)
    negs = []
    need = len(test_pos)
    while need > 0 and nt > 1:
        cu = rng.integers(0, nt, size=2 * need + 16)
        cv = rng.integers(0, nt, size=2 * need + 16)
        ok = cu != cv
        cu, cv = cu[ok], cv[ok]
        hit = np.isin(cu * nt + cv, full_keys)
        cu, cv = cu[~hit], cv[~hit]
        take = min(need, len(cu))
        negs.append(np.stack([cu[:take], cv[:take]], axis=1))
        need -= take
    test_neg = (np.concatenate(negs).astype(np.int32) if negs
                else np.zeros((0, 2), dtype=np.int32))
    return LinkSplit(train, test_pos, test_neg)


# Named workloads: R-MAT parameters of the benchmark configurations.
_WORKLOADS = {
    "rmat12": dict(scale=12, edge_factor=8, seed=20211020),
    "rmat20": dict(scale=20, edge_factor=16, seed=20211021),
    "rmat22": dict(scale=22, edge_factor=16, seed=20211022),
}


def workload(name: str, split: bool = True):
    """The graph of a named workload (and its link split unless split=False)."""
    cfg = _WORKLOADS[name]
    g = rmat_graph(cfg["scale"], cfg["edge_factor"], cfg["seed"])
    return link_split(g, cfg["seed"]) if split else g
