"""The library's host side of random-walk sampling (Sec. 3.2) against the
oracle, on the CPU (no device involved): the pair table the walk entry point
sends to the device and the order in which the device visits it are the
oracle's, bit for bit, for graphs with isolated vertices, dead ends, stars
and R-MAT hubs, several walk lengths and windows, and position counts on
both sides of the Feistel cycle-walking boundary."""
import numpy as np
import pytest

import oracle
import synth
from paper_2110_10049_gb300 import build, gosh as g


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()


def graphs():
    return [synth.rmat_graph(9, 8, 2), synth.random_graph(40, 0.1, 5),
            synth.csr_from_edges(7, np.array([0, 0, 0, 4]), np.array([1, 2, 3, 5]), compact=False),
            synth.csr_from_edges(3, np.zeros(0, np.int64), np.zeros(0, np.int64), compact=False)]


@pytest.mark.parametrize("l,w", [(2, 1), (4, 2), (8, 3), (11, 5)])
def test_walk_pairs_equal_oracle(l, w):
    for gi, gr in enumerate(graphs()):
        for epoch in (0, 3):
            got = g.gosh_walk_pairs(gr.rowptr, gr.col, l, w, 2, epoch, 77 + gi, 5)
            ref = oracle.walk_pairs(gr.rowptr, gr.col, l, w, 2, epoch, 77 + gi, 5)
            np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 16, 17, 255, 256, 257, 1000, 65536, 65537])
def test_walk_order_equals_oracle(P):
    for level, epoch, seed, graph in ((0, 0, 1, 0), (3, 7, 2 ** 40 + 5, 9)):
        np.testing.assert_array_equal(g.gosh_walk_order(P, level, epoch, seed, graph),
                                      oracle.walk_perm(P, seed, graph, level, epoch))
