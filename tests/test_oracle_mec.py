"""Pins for MULTIEDGECOLLAPSE (Alg. 4, Sec. 4) in the oracle.

1. Structural invariants of every level of the R-MAT hierarchy.
2. An independent second definition of the mapping, written here: the hubs
   are the lexicographically-first maximal independent set, in degree order,
   of the graph of eligible edges (hub^2: deg(u) <= delta or deg(v) <= delta),
   and every other vertex joins its earliest-ranked eligible hub neighbour.
   Checked exhaustively on all graphs with up to 6 vertices and on random
   graphs with 8-16 vertices.
3. The density reading (delta counts both directions of every edge) pinned by
   the paper's coarsening table (tests/golden/coarsening_density.txt) and by a
   star graph on which the two readings give different results.
"""
import itertools
import os

import numpy as np
import pytest

import synth


def lf_mis_mapping(n, rowptr, col):
    """Second definition of one MEC level (no greedy walk)."""
    deg = np.diff(rowptr)
    nnz = int(rowptr[-1])
    rank = np.empty(n, dtype=np.int64)
    order = sorted(range(n), key=lambda v: (-deg[v], v))
    for r, v in enumerate(order):
        rank[v] = r
    small = [deg[v] * n <= nnz for v in range(n)]
    elig = [[int(u) for u in col[rowptr[v]:rowptr[v + 1]] if small[v] or small[u]] for v in range(n)]
    hub = [False] * n
    for v in order:  # lexicographically-first MIS in rank order
        hub[v] = not any(hub[u] and rank[u] < rank[v] for u in elig[v])
    cid = {}
    for v in order:
        if hub[v]:
            cid[v] = len(cid)
    mp = np.empty(n, dtype=np.int32)
    for v in range(n):
        if hub[v]:
            mp[v] = cid[v]
        else:
            h = min((u for u in elig[v] if hub[u]), key=lambda u: rank[u])
            mp[v] = cid[h]
    return mp, len(cid)


def image_edges(rowptr, col, mp):
    s = set()
    for v in range(len(rowptr) - 1):
        for u in col[rowptr[v]:rowptr[v + 1]]:
            if mp[v] != mp[u]:
                s.add((int(mp[v]), int(mp[u])))
    return s


def check_invariants(rowptr, col, mp, nc, rp2, co2):
    n = len(rowptr) - 1
    deg = np.diff(rowptr)
    nnz = int(rowptr[-1])
    # map is total and onto [0, nc)
    assert mp.min(initial=0) >= 0 and (n == 0 or mp.max() == nc - 1)
    assert len(np.unique(mp)) == nc
    # cluster ids appear in discovery order: first member in degree order
    order = sorted(range(n), key=lambda v: (-deg[v], v))
    seen = []
    for v in order:
        if mp[v] not in seen:
            seen.append(mp[v])
    assert seen == list(range(nc))
    # coarse edges == image of fine edges minus self loops, dedup, symmetric
    coarse = set()
    for c in range(nc):
        row = co2[rp2[c]:rp2[c + 1]]
        assert np.all(np.diff(row) > 0)
        coarse.update((c, int(x)) for x in row)
    assert coarse == image_edges(rowptr, col, mp)
    assert all((b, a) in coarse for a, b in coarse)
    # each cluster is a star around its hub (the first member in order);
    # at most one member has degree above delta, and if so it is the hub
    hub_of = {}
    for v in order:
        hub_of.setdefault(int(mp[v]), v)
    adj = [set(col[rowptr[v]:rowptr[v + 1]].tolist()) for v in range(n)]
    big = lambda x: deg[x] * n > nnz
    for v in range(n):
        h = hub_of[int(mp[v])]
        if v != h:
            assert h in adj[v]
            assert not (big(v) and big(h))
            assert not big(v)


def test_rmat_hierarchy_invariants(orc):
    g = synth.rmat_graph(10, 8, 4)
    graphs, maps = orc.mec_hierarchy(g.rowptr, g.col)
    assert len(graphs) >= 3
    for i, mp in enumerate(maps):
        rp, co = graphs[i]
        rp2, co2 = graphs[i + 1]
        check_invariants(rp, co, mp, len(rp2) - 1, rp2, co2)
        mp2, nc2 = lf_mis_mapping(len(rp) - 1, rp, co)
        np.testing.assert_array_equal(mp, mp2)


def all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        e = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        s = np.array([a for a, b in e], dtype=np.int64)
        t = np.array([b for a, b in e], dtype=np.int64)
        yield synth.csr_from_edges(n, s, t, compact=False)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_exhaustive_small_graphs(orc, n):
    for g in all_graphs(n):
        mp, nc = orc.mec_map(g.rowptr, g.col)
        mp2, nc2 = lf_mis_mapping(n, g.rowptr, g.col)
        assert nc == nc2
        np.testing.assert_array_equal(mp, mp2)
        rp2, co2 = orc.coarsen(g.rowptr, g.col, mp, nc)
        check_invariants(g.rowptr, g.col, mp, nc, rp2, co2)


def test_random_graphs_8_to_16(orc):
    rng = np.random.default_rng(12345)
    for trial in range(20000):
        n = int(rng.integers(8, 17))
        p = float(rng.uniform(0.05, 0.7))
        g = synth.random_graph(n, p, int(rng.integers(1 << 31)))
        mp, nc = orc.mec_map(g.rowptr, g.col)
        mp2, nc2 = lf_mis_mapping(n, g.rowptr, g.col)
        assert nc == nc2
        np.testing.assert_array_equal(mp, mp2)
        rp2, co2 = orc.coarsen(g.rowptr, g.col, mp, nc)
        check_invariants(g.rowptr, g.col, mp, nc, rp2, co2)


def test_density_reading_from_paper_table():
    path = os.path.join(os.path.dirname(__file__), "golden", "coarsening_density.txt")
    e, frac, v1, printed = np.loadtxt(path)
    assert round(frac * 2 * e / v1, 1) == printed
    assert round(frac * e / v1, 1) != printed


def test_density_counts_directed_entries(orc):
    # star K_{1,4}: avg degree (directed entries / |V|) = 8/5 = 1.6, so leaves
    # (deg 1) are below delta and the centre absorbs them all: one cluster.
    # Counting undirected edges (4/5 = 0.8) would block every merge.
    g = synth.csr_from_edges(5, np.zeros(4, dtype=np.int64), np.arange(1, 5), compact=False)
    mp, nc = orc.mec_map(g.rowptr, g.col)
    assert nc == 1 and np.all(mp == 0)


def test_hub2_blocks_two_hubs(orc):
    # two hubs (deg 5 each) joined by an edge, each with 4 leaves; delta =
    # 2*9/10 = 1.8 so hub-hub is ineligible: two clusters, not one.
    s = [0, 0, 0, 0, 0, 5, 5, 5, 5]
    t = [5, 1, 2, 3, 4, 6, 7, 8, 9]
    g = synth.csr_from_edges(10, np.array(s), np.array(t), compact=False)
    mp, nc = orc.mec_map(g.rowptr, g.col)
    assert nc == 2
    assert mp[0] != mp[5]


def test_degree_order_stable_descending(orc):
    g = synth.rmat_graph(9, 4, 2)
    deg = np.diff(g.rowptr)
    order = orc.degree_order(g.rowptr)
    np.testing.assert_array_equal(order, np.lexsort((np.arange(g.n), -deg)))


def test_stop_condition(orc):
    assert orc.continue_coarsening(80, 100, 50, 0.8)
    assert not orc.continue_coarsening(81, 100, 50, 0.8)   # shrank < 20%
    assert not orc.continue_coarsening(100, 1000, 100, 0.8)  # not above threshold
    assert orc.continue_coarsening(101, 1000, 100, 0.8)
    # a graph at or below the threshold is still coarsened once (do-while)
    g = synth.random_graph(30, 0.2, 3)
    graphs, maps = orc.mec_hierarchy(g.rowptr, g.col, threshold=100)
    assert len(graphs) == 2 and len(maps) == 1
