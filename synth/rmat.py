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


_LIB = None


def _clib():
    """Builds and loads synth/librmatgen.so (gcc, OpenMP)."""
    global _LIB
    if _LIB is None:
        import ctypes as C
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        src, so = os.path.join(here, "rmatgen.c"), os.path.join(here, "librmatgen.so")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            tmp = so + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src])
            os.replace(tmp, so)
        L = C.CDLL(so)
        vp, i64, u64, f64, i32 = C.c_void_p, C.c_int64, C.c_uint64, C.c_double, C.c_int
        L.rmat_edges.argtypes = [i32, i64, u64, f64, f64, f64, vp, vp]
        L.rmat_edges.restype = None
        L.csr_build.argtypes = [i64, i64, vp, vp, i32, vp, vp, vp, vp, vp]
        L.csr_build.restype = i64
        L.link_split.argtypes = [i64, vp, vp, u64, f64, vp, vp, vp, vp, vp, vp, vp]
        L.link_split.restype = i64
        L.csr_large_count.argtypes = [i64, i64, vp, vp, i32, vp, vp]
        L.csr_large_count.restype = vp
        L.csr_large_fill.argtypes = [vp, vp, vp]
        L.csr_large_fill.restype = None
        _LIB = L
    return _LIB


def _p(a):
    import ctypes as C
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def rmat_edges(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19):
    """Directed R-MAT draws followed by a seeded relabelling (steps 1-2)."""
    m = edge_factor << scale
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    _clib().rmat_edges(scale, m, seed, a, b, c, _p(src), _p(dst))
    return src, dst


def _csr_c(n: int, src: np.ndarray, dst: np.ndarray, compact: bool) -> Graph:
    import ctypes as C
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    m = len(src)
    work = np.empty(max(4 * m, 2), dtype=np.uint64)
    nn = C.c_int64()
    nnz = _clib().csr_build(n, m, _p(src), _p(dst), int(compact), _p(work), C.byref(nn), None, None, None)
    rowptr = np.zeros(nn.value + 1, dtype=np.int64)
    col = np.empty(max(nnz, 1), dtype=np.int32)
    _clib().csr_build(n, m, _p(src), _p(dst), int(compact), _p(work), C.byref(nn), _p(rowptr), _p(col), None)
    return Graph(rowptr, col[:nnz])


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
    return _csr_c(1 << scale, s, d, compact=True)


def rmat_graph_large(scale: int, edge_factor: int, seed: int, **kw) -> Graph:
    """rmat_graph built on all threads in about a third of its memory (a
    counting sort by row, then each row sorted and deduplicated): the same
    CSR, for graphs of billions of entries."""
    import ctypes as C
    s, d = rmat_edges(scale, edge_factor, seed, **kw)
    nn, nnz = C.c_int64(), C.c_int64()
    h = _clib().csr_large_count(1 << scale, len(s), _p(s), _p(d), 1, C.byref(nn), C.byref(nnz))
    del s, d
    rowptr = np.empty(nn.value + 1, dtype=np.int64)
    col = np.empty(max(nnz.value, 1), dtype=np.int32)
    _clib().csr_large_fill(h, _p(rowptr), _p(col))
    return Graph(rowptr, col[:nnz.value])


def random_graph(n: int, p: float, seed: int, compact: bool = False) -> Graph:
    """Erdos-Renyi G(n, p) (small test graphs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    return csr_from_edges(n, iu[keep], ju[keep], compact=compact)


def link_split(g: Graph, seed: int, test_frac: float = 0.2) -> LinkSplit:
    import ctypes as C
    n, nnz = g.n, g.nnz
    ne = nnz // 2
    work = np.empty(ne + (4 * n + ne) // 8 + 2, dtype=np.uint64)
    ntr, nte = C.c_int64(), C.c_int64()
    rp, co = np.ascontiguousarray(g.rowptr, np.int64), np.ascontiguousarray(g.col, np.int32)
    if co.size == 0:
        co = np.zeros(1, dtype=np.int32)
    m2 = _clib().link_split(n, _p(rp), _p(co), seed, test_frac, _p(work), C.byref(ntr), C.byref(nte),
                            None, None, None, None)
    trp = np.zeros(ntr.value + 1, dtype=np.int64)
    tco = np.empty(max(m2, 1), dtype=np.int32)
    pos = np.empty((max(nte.value, 1), 2), dtype=np.int32)
    neg = np.empty((max(nte.value, 1), 2), dtype=np.int32)
    _clib().link_split(n, _p(rp), _p(co), seed, test_frac, _p(work), C.byref(ntr), C.byref(nte),
                       _p(trp), _p(tco), _p(pos), _p(neg))
    return LinkSplit(Graph(trp, tco[:m2]), pos[:nte.value], neg[:nte.value])


def fit_pairs(g: Graph, count: int = 400000, seed: int = 5):
    """Pairs of a training-edge AUC: training edges (u < v; a seeded sample of
    `count` of them, drawn with replacement, when there are more) and as many
    uniform vertex pairs (u != v).  Returns (pos, neg), int32 [m, 2] each."""
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    keep = src < g.col
    pos = np.stack([src[keep], g.col[keep]], 1)
    rng = np.random.default_rng(seed)
    if len(pos) > count:
        pos = pos[rng.integers(0, len(pos), count)]
    neg = rng.integers(0, g.n, size=(len(pos), 2))
    neg = neg[neg[:, 0] != neg[:, 1]]
    return pos.astype(np.int32), neg.astype(np.int32)


# Named workloads: R-MAT parameters of the benchmark configurations, and the
# degree-corrected planted partitions of the same sizes on which held-out
# link prediction is informative (synth/sbm.py).
_WORKLOADS = {
    "rmat12": dict(scale=12, edge_factor=8, seed=20211020),
    "rmat20": dict(scale=20, edge_factor=16, seed=20211021),
    "rmat22": dict(scale=22, edge_factor=16, seed=20211022),
    "sbm12": dict(scale=12, edge_factor=8, seed=20211030, communities=32, mu=0.8),
    "sbm20": dict(scale=20, edge_factor=16, seed=20211031, communities=1024, mu=0.8),
}


def workload(name: str, split: bool = True):
    """The graph of a named workload (and its link split unless split=False)."""
    cfg = _WORKLOADS[name]
    if "communities" in cfg:
        from .sbm import sbm_graph
        g = sbm_graph(1 << cfg["scale"], cfg["communities"], cfg["edge_factor"], cfg["mu"], cfg["seed"])
    else:
        g = rmat_graph(cfg["scale"], cfg["edge_factor"], cfg["seed"])
    return link_split(g, cfg["seed"]) if split else g
