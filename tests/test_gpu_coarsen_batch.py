"""Batched coarsening (many graphs coarsened level by level as one union).

The union's degree order sorts by graph first, so each graph keeps its own
rank order and hub numbering: every hierarchy must equal, bit for bit, the one
gosh_coarsen builds for the graph alone (maps, row pointers, entries, level
count), and the oracle's MULTIEDGECOLLAPSE hierarchy (Alg. 4).  Cases mix
graph sizes and densities (so graphs stop at different levels), graphs without
edges, single vertices, a forced sorted path and a level cap.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gosh, needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]


def mixed_graphs(seed):
    rng = np.random.default_rng(seed)
    gs = []
    for i in range(12):
        gs.append(synth.rmat_graph(int(rng.integers(6, 13)), int(rng.integers(2, 24)), int(rng.integers(1 << 30))))
    for i in range(12):
        n = int(rng.integers(2, 300))
        gs.append(synth.random_graph(n, float(rng.uniform(0.0, 0.3)), int(rng.integers(1 << 30))))
    # no edges; a single vertex; a star with a path
    gs.append(synth.csr_from_edges(7, np.zeros(0, np.int64), np.zeros(0, np.int64), compact=False))
    gs.append(synth.csr_from_edges(1, np.zeros(0, np.int64), np.zeros(0, np.int64), compact=False))
    gs.append(synth.csr_from_edges(12, np.array([0, 0, 0, 0, 5, 6, 7]), np.array([1, 2, 3, 4, 6, 7, 8]),
                                   compact=False))
    order = rng.permutation(len(gs))
    return [gs[i] for i in order]


def assert_same(g, hb, hs, gr, threshold, shrink, max_levels=64):
    assert len(hb) == len(hs)
    for i in range(len(hs)):
        rb, cb, mb = hb.level_arrays(i)
        rs, cs, ms = hs.level_arrays(i)
        np.testing.assert_array_equal(rb, rs)
        np.testing.assert_array_equal(cb, cs)
        if ms is not None:
            np.testing.assert_array_equal(mb, ms)
    graphs, maps = oracle.mec_hierarchy(gr.rowptr, gr.col, threshold, shrink, max_levels)
    assert len(graphs) == len(hb)
    for i in range(len(graphs)):
        rb, cb, mb = hb.level_arrays(i)
        np.testing.assert_array_equal(rb, graphs[i][0])
        np.testing.assert_array_equal(cb, graphs[i][1])
        if i < len(maps):
            np.testing.assert_array_equal(mb, maps[i])


@pytest.mark.parametrize("seed,threshold", [(1, 100), (2, 4), (3, 30)])
def test_batch_coarsening_equals_single(seed, threshold):
    g = gosh()
    grs = mixed_graphs(seed)
    csrs = [g.to_device_csr(gr.rowptr, gr.col) for gr in grs]
    hb = g.gosh_coarsen_batch(csrs, threshold, 0.8)
    for i, gr in enumerate(grs):
        hs = g.gosh_coarsen(csrs[i], threshold, 0.8)
        assert_same(g, hb[i], hs, gr, threshold, 0.8)
        hs.close()
    for h in hb:
        h.close()


@pytest.mark.parametrize("bitmap_max", ["0", "40"])
def test_batch_coarsening_sorted_path(monkeypatch, bitmap_max):
    # coarse graphs wider than the bitmap limit are built by a radix sort of
    # packed (map v, map u) keys over the whole union
    monkeypatch.setenv("GOSH_COARSEN_BITMAP_MAX", bitmap_max)
    g = gosh()
    grs = mixed_graphs(4)[:10]
    csrs = [g.to_device_csr(gr.rowptr, gr.col) for gr in grs]
    hb = g.gosh_coarsen_batch(csrs, 10, 0.8)
    for i, gr in enumerate(grs):
        hs = g.gosh_coarsen(csrs[i], 10, 0.8)
        assert_same(g, hb[i], hs, gr, 10, 0.8)


def test_batch_coarsening_level_cap_and_handles_outlive_each_other():
    g = gosh()
    grs = [synth.rmat_graph(11, 8, s) for s in range(5)]
    csrs = [g.to_device_csr(gr.rowptr, gr.col) for gr in grs]
    hb = g.gosh_coarsen_batch(csrs, 1, 1.0, 3)
    assert all(len(h) == 3 for h in hb)
    # levels coarsened together share buffers: freeing some handles leaves
    # the others intact
    for h in hb[:3]:
        h.close()
    for i in (3, 4):
        hs = g.gosh_coarsen(csrs[i], 1, 1.0, 3)
        assert_same(g, hb[i], hs, grs[i], 1, 1.0, 3)
